"""GB300 (sm_103a) implementation of one pcSIR / SIR particle-filter step.

The compute path lives in the C-ABI library ``libpcsir.so`` (CUDA kernels in
``csrc/``); ``paper_1310_5541_gb300.pcsir`` is its thin ctypes binding and
``paper_1310_5541_gb300.synth`` draws the seeded synthetic inputs.
"""

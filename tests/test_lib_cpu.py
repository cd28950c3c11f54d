"""Host-side checks of the C-ABI library that need no GPU: it loads, exports
every entry point the headers in include/ declare, its structs have the
headers' layout, and argument errors are rejected on the host."""
import ctypes
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = sorted(glob.glob(os.path.join(ROOT, "include", "*.h")))


@pytest.fixture(scope="module")
def binding():
    import __graft_entry__

    __graft_entry__.build()
    from paper_1310_5541_gb300 import pcsir

    return pcsir


def _declared_functions():
    src = "\n".join(open(h).read() for h in HEADERS)
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*([a-z_0-9]+)\s*\(", src, flags=re.M)))


def test_exports_every_declared_entry_point(binding):
    names = _declared_functions()
    assert "pcsir_step" in names and "sir_step" in names and "pcsir_surrogate_train" in names and len(names) >= 30
    lib = ctypes.CDLL(binding.LIB_PATH)
    for n in names:
        assert hasattr(lib, n), n


def test_struct_layout_matches_header(binding, tmp_path):
    prog = tmp_path / "layout.c"
    fields = {
        "pcsir_config": [f[0] for f in binding.pcsir_config._fields_],
        "pcsir_result": [f[0] for f in binding.pcsir_result._fields_],
        "pcsir_outputs": [f[0] for f in binding.pcsir_outputs._fields_],
        "pcsir_target": [f[0] for f in binding.pcsir_target._fields_],
        "pcsir_surrogate_config": [f[0] for f in binding.pcsir_surrogate_config._fields_],
        "pcsir_surrogate_check": [f[0] for f in binding.pcsir_surrogate_check._fields_],
        "pcsir3_config": [f[0] for f in binding.pcsir3_config._fields_],
        "pcsir3_result": [f[0] for f in binding.pcsir3_result._fields_],
        "pcsir3_outputs": [f[0] for f in binding.pcsir3_outputs._fields_],
        "pcsir3_target": [f[0] for f in binding.pcsir3_target._fields_],
        "pcsir3_batch_outputs": [f[0] for f in binding.pcsir3_batch_outputs._fields_],
    }
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "pcsir.h"', '#include "pcsir_surrogate.h"', '#include "pcsir3.h"',
             "int main(void){", 'printf("NPARAMS %d\\n", PCSIR_SUR_NPARAMS);']
    for s, fs in fields.items():
        lines.append('printf("%s %%zu\\n", sizeof(%s));' % (s, s))
        for f in fs:
            lines.append('printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (s, f, s, f))
    lines.append("return 0;}")
    prog.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)], check=True)
    out = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                 check=True).stdout.splitlines())
    assert int(out["NPARAMS"]) == binding.SUR_NPARAMS
    for s, fs in fields.items():
        cls = getattr(binding, s)
        assert int(out[s]) == ctypes.sizeof(cls), s
        for f in fs:
            assert int(out["%s.%s" % (s, f)]) == getattr(cls, f).offset, (s, f)


def test_invalid_configs_rejected_on_host(binding):
    lib = binding.lib
    base = dict(state_dtype=0, lik_kind=0, patch=9, keep=0, psf_sigma=1.5, bg=10.0, sigma_xi=20.0,
                max_particles=1000, dummy=0, reserved=0)
    bad = [dict(patch=8), dict(patch=0), dict(patch=129), dict(state_dtype=2), dict(lik_kind=5),
           dict(psf_sigma=0.0), dict(bg=0.0), dict(max_particles=0), dict(max_particles=(1 << 26) + 1),
           dict(keep=64), dict(keep=32), dict(lik_kind=1, sigma_xi=0.0), dict(dummy=2), dict(reserved=1)]
    for upd in bad:
        cfg = binding.pcsir_config(**{**base, **upd})
        h = ctypes.c_void_p(123)
        assert lib.pcsir_create(ctypes.byref(cfg), ctypes.byref(h)) == binding.EINVAL, upd
        assert not h.value
    assert lib.pcsir_create(None, None) == binding.EINVAL
    assert lib.pcsir_step(None, None, 1, None, 1, 1, 0.5, None, 0.5, None, None) == binding.EINVAL
    assert lib.sir_step(None, None, 1, None, 1, 1, None, 0.5, None, None) == binding.EINVAL
    assert lib.pcsir_destroy(None) == binding.OK
    assert b"pcsir" in lib.pcsir_version()
    assert lib.pcsir_save(None, b"x.ck") == binding.EINVAL
    assert lib.pcsir_load(None, b"x.ck") == binding.EINVAL
    assert lib.pcsir_batch_set_wait(None, 100, -1) == binding.EINVAL
    assert lib.pcsir_batch_keep(None, 1) == binding.EINVAL
    assert lib.pcsir_batch_kept(None, None, None) == binding.EINVAL


def test_invalid_batched3_targets_rejected_on_host(binding):
    lib = binding.lib
    good = dict(n_particles=100, hx=0.5, hy=0.5, hz=1.0, psf_sigma_xy=1.5, psf_sigma_z=3.0, bg=10.0,
                patch_xy=11, patch_z=7)
    for upd in [dict(n_particles=0), dict(hx=0.0), dict(hz=9.0), dict(psf_sigma_z=0.0), dict(bg=0.0),
                dict(patch_xy=10), dict(patch_z=65)]:
        arr = (binding.pcsir3_target * 1)(binding.pcsir3_target(**{**good, **upd}))
        h = ctypes.c_void_p(123)
        assert lib.pcsir3_batch_create(arr, 1, 0, ctypes.byref(h)) == binding.EINVAL, upd
        assert not h.value
    arr = (binding.pcsir3_target * 1)(binding.pcsir3_target(**good))
    h = ctypes.c_void_p()
    assert lib.pcsir3_batch_create(arr, 0, 0, ctypes.byref(h)) == binding.EINVAL
    assert lib.pcsir3_batch_create(arr, 1, 2, ctypes.byref(h)) == binding.EINVAL  # weights are not kept
    assert lib.pcsir3_batch_destroy(None) == binding.OK


def test_noalloc_binding_rejects_operands_it_cannot_use(binding):
    """The allocation-free resampling takes its scratch from the current device: the binding refuses,
    on the host, operands that are not CUDA tensors of the current device (here: host tensors)."""
    import torch

    lw = torch.zeros(8, dtype=torch.float64)
    with pytest.raises(ValueError):
        binding.pcsir_resample_noalloc(lw, 0.5)
    with pytest.raises(ValueError):
        binding.pcsir_resample_noalloc(lw, 0.5, out=torch.zeros(8, dtype=torch.int32))


def test_invalid_surrogate_configs_rejected_on_host(binding):
    lib = binding.lib
    base = dict(capacity=1000, batch=256, geometry=0, i0_ref=128.0, sigma_ref=1.5, max_pixels=4096)
    for upd in [dict(capacity=0), dict(batch=100), dict(batch=0), dict(batch=65536 + 128), dict(geometry=1),
                dict(i0_ref=0.0), dict(sigma_ref=-1.0), dict(i0_ref=float("nan")), dict(max_pixels=0)]:
        cfg = binding.pcsir_surrogate_config(**{**base, **upd})
        h = ctypes.c_void_p(123)
        assert lib.pcsir_surrogate_create(ctypes.byref(cfg), ctypes.byref(h)) == binding.EINVAL, upd
        assert not h.value
    assert lib.pcsir_surrogate_create(None, None) == binding.EINVAL
    assert lib.pcsir_surrogate_destroy(None) == binding.OK
    assert lib.pcsir_attach_surrogate(None, None, 0.02, 32, 30.0, 1.0) == binding.EINVAL
    assert lib.pcsir_surrogate_train(None, 0, 1, 1, 1e-3, 1, None, None) == binding.EINVAL


def test_autotune_defaults_without_cache(tmp_path, monkeypatch):
    import numpy as np

    from paper_1310_5541_gb300 import autotune

    monkeypatch.setenv("PCSIR_AUTOTUNE_CACHE", str(tmp_path / "absent.json"))
    assert autotune.load() == {}
    np.testing.assert_allclose(autotune.cell_edges([1.5, 3.0]), [0.5, 1.0])

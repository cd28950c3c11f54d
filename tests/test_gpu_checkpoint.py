"""Checkpoint and resume of a context between steps (pcsir_save / pcsir_load, through the C ABI).

A surrogate-assisted pcSIR run carries state in its context: the surrogate's parameters and the
count of surrogate-assisted steps, which salts each step's held-out selection.  Ten steps are run
without interruption; a second run saves after step 5, and a fresh context with a freshly
initialised surrogate loads the file and runs steps 5-9 from the caller's saved particle states.
The resumed steps equal the uninterrupted ones bit for bit (states, held-out selection and its
statistics); the same fresh context without the load does not.
"""
import numpy as np
import pytest
import torch

from paper_1310_5541_gb300 import synth

pytestmark = pytest.mark.gpu
SEED = 1310554900


@pytest.fixture(scope="module")
def pc():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import __graft_entry__

    __graft_entry__.build()
    from paper_1310_5541_gb300 import pcsir

    return pcsir


N, H_CELL, FRAMES, SAVE_AT = 40_000, 0.1, 10, 5
HOLDOUT = dict(holdout_frac=0.2, min_holdout=16, window=25.0, max_err=1e9)


def _setup(pc, m, seed):
    sur = pc.Surrogate(capacity=1, batch=128)
    sur.init(seed)
    p, _, _ = sur.get_params()
    sur.set_params(p, -60.0, 15.0)
    ctx = pc.Context(N, torch.float32, patch=21, psf_sigma=m.sigma_psf, bg=m.bg)
    pc.attach_surrogate(ctx, sur, **HOLDOUT)
    return ctx, sur


def _steps(pc, ctx, seq, st, frames, m):
    """Run the given frames in place on the device state; per frame: new state, estimate, check."""
    out = []
    for k in frames:
        nz = torch.from_numpy(synth.make_noise(N, m.q, SEED + 1, k, np.float32)).cuda()
        pc.pcsir_step(ctx, st, torch.from_numpy(seq.images[k]).cuda(), H_CELL, nz, synth.make_u0(SEED + 1, k))
        torch.cuda.synchronize()
        out.append((st.cpu().numpy(), np.array(ctx.last_result()["estimate"]), pc.surrogate_last_check(ctx)))
    return out


def _same(a, b):
    for (sa, ea, ca), (sb, eb, cb) in zip(a, b):
        np.testing.assert_array_equal(sa, sb)
        # the weight sums meet in FP64 atomics, whose order may vary between launches
        np.testing.assert_allclose(ea, eb, rtol=1e-12, atol=0)
        for key in ("n_dummies", "n_exact", "n_holdout", "n_significant", "n_clipped", "fallback", "max_abs_err"):
            assert ca[key] == cb[key], (key, ca[key], cb[key])
        assert ca["rms_err"] == pytest.approx(cb["rms_err"], rel=1e-12, abs=0.0)


def test_resume_from_checkpoint_is_bit_identical(pc, tmp_path):
    m = synth.Model(patch=21)
    seq = synth.make_sequence(96, 80, FRAMES, m, seed=SEED, vmax=0.5, margin=12)
    st0 = synth.initial_state(seq.gt[0], N, np.float32)

    ctx, sur = _setup(pc, m, 7)
    ref = _steps(pc, ctx, seq, torch.from_numpy(st0.copy()).cuda(), range(FRAMES), m)
    ctx.close()
    sur.close()
    assert any(c["n_holdout"] > 0 for _, _, c in ref) and not any(c["fallback"] for _, _, c in ref)

    ctx, sur = _setup(pc, m, 7)
    st = torch.from_numpy(st0.copy()).cuda()
    first = _steps(pc, ctx, seq, st, range(SAVE_AT), m)
    _same(first, ref[:SAVE_AT])
    path = str(tmp_path / "ctx.pcsirck")
    ctx.save(path)
    saved_state = st.cpu().numpy()  # the particles are the caller's to save
    ctx.close()
    sur.close()

    # a fresh context and a surrogate with other parameters: the load restores both
    ctx2, sur2 = _setup(pc, m, 99)
    ctx2.load(path)
    resumed = _steps(pc, ctx2, seq, torch.from_numpy(saved_state).cuda(), range(SAVE_AT, FRAMES), m)
    _same(resumed, ref[SAVE_AT:])
    ctx2.close()
    sur2.close()

    # without the load the same fresh pair gives other steps (other parameters, other held-out cells)
    ctx3, sur3 = _setup(pc, m, 99)
    other = _steps(pc, ctx3, seq, torch.from_numpy(saved_state).cuda(), range(SAVE_AT, FRAMES), m)
    assert any(not np.array_equal(a[0], b[0]) for a, b in zip(other, ref[SAVE_AT:]))
    ctx3.close()
    sur3.close()


def test_load_rejects_foreign_or_corrupt_files(pc, tmp_path):
    m = synth.Model(patch=21)
    ctx, sur = _setup(pc, m, 3)
    path = tmp_path / "a.pcsirck"
    ctx.save(str(path))
    # another model (patch 9): refused, the context stays usable
    other = pc.Context(1000, torch.float32, patch=9, psf_sigma=m.sigma_psf, bg=m.bg)
    with pytest.raises(pc.PcsirError) as e:
        other.load(str(path))
    assert e.value.status == pc.EINVAL
    # a surrogate record but no surrogate attached
    plain = pc.Context(1000, torch.float32, patch=21, psf_sigma=m.sigma_psf, bg=m.bg)
    with pytest.raises(pc.PcsirError) as e:
        plain.load(str(path))
    assert e.value.status == pc.ESTATE
    # one flipped byte, a truncated file, a missing file
    raw = bytearray(path.read_bytes())
    raw[len(raw) // 2] ^= 0x10
    bad = tmp_path / "bad.pcsirck"
    bad.write_bytes(bytes(raw))
    short = tmp_path / "short.pcsirck"
    short.write_bytes(path.read_bytes()[:-9])
    for p in (bad, short, tmp_path / "missing.pcsirck"):
        with pytest.raises(pc.PcsirError) as e:
            ctx.load(str(p))
        assert e.value.status == pc.EINVAL
    ctx.load(str(path))  # the good file still loads
    for c in (ctx, other, plain):
        c.close()
    sur.close()

"""pcv_evaluate_exact_noalloc: the entry point for callers that cannot allocate device
memory (their MD engine owns the device memory pool, or an allocation would stall them).
It must give the same s, z and MSDs as the regular exact-mode entry point, call after
call, although every call reuses one fixed scratch array.  Kept in its own file so that
it runs after every other test."""
import ctypes

import numpy as np
import pytest

import oracle
from _util import TOL, d_err, problem, s_err, s_kappa, z_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def pcv():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1801_02362_gb300 import build_lib
    from paper_1801_02362_gb300 import pcv as mod

    build_lib.build()
    mod.load()
    return mod


def noalloc(pcv, fr, lm, lam, stream):
    F, N = fr.shape[0], fr.shape[1]
    M = lm.shape[0]
    frames = torch.tensor(fr, dtype=torch.float32, device="cuda")
    land = torch.tensor(lm, dtype=torch.float32, device="cuda")
    s = torch.empty(F, dtype=torch.float64, device="cuda")
    z = torch.empty(F, dtype=torch.float64, device="cuda")
    msd = torch.empty((F, M), dtype=torch.float64, device="cuda")
    err = ctypes.create_string_buffer(256)
    P = lambda t: ctypes.c_void_p(t.data_ptr())
    st = pcv.load().pcv_evaluate_exact_noalloc(F, M, N, P(frames), P(land), None, lam, P(s), P(z), P(msd),
                                                stream, err, 256)
    assert st == pcv.PCV_OK, err.value
    return s.cpu().numpy(), z.cpu().numpy(), msd.cpu().numpy()


def test_noalloc_matches_regular_entry_point_twice(pcv):
    """96 and then 80 frames.  The regular entry point may split the atom sums of a batch
    this small over several CTAs per tile, so its distances carry a different rounding
    (both within the distance tolerance); s amplifies a distance change by its condition
    number, so s is compared with the tolerance scaled by it, as for any two evaluations
    whose distances differ within tolerance."""
    lm, fr_a, lam = problem(41, 300, 200, 96)
    _, fr_b, _ = problem(42, 300, 200, 80)
    stream = torch.cuda.current_stream().cuda_stream
    ctx = pcv.PathCV(lm, lam, eps=-1.0, precision="fp32")
    for fr in (fr_a, fr_b):  # two calls in a row share the fixed scratch
        s, z, msd = noalloc(pcv, fr, lm, lam, stream)
        ref = ctx.evaluate(torch.tensor(fr, dtype=torch.float32, device="cuda"), msd=True)
        torch.cuda.synchronize()
        rs, rz, rmsd = (ref[k].cpu().numpy() for k in ("s", "z", "msd"))
        r = oracle.exact(fr, lm, lam)
        kappa = s_kappa(r["D"], lam, fr, lm)
        assert d_err(msd, rmsd, fr, lm) < TOL["fp32"]
        assert s_err(s, rs, kappa=kappa) < TOL["fp32"]
        assert z_err(z, rz, lam) < TOL["fp32"]
        # and against the oracle
        assert d_err(msd, r["D"], fr, lm) < TOL["fp32"]
        assert s_err(s, r["s"], kappa=kappa) < TOL["fp32"]
        assert z_err(z, r["z"], lam) < TOL["fp32"]
    ctx.close()


@pytest.mark.parametrize("F", [1, 4])
def test_noalloc_few_frames_match_regular_entry_point(pcv, F):
    """One to four frames per call take the call's few-frame branch (one CTA per landmark);
    two calls in a row, each against the regular entry point and the oracle."""
    lm, fr, lam = problem(43, 300, 200, 2 * F)
    stream = torch.cuda.current_stream().cuda_stream
    ctx = pcv.PathCV(lm, lam, eps=-1.0, precision="fp32")
    for part in (fr[:F], fr[F:]):
        s, z, msd = noalloc(pcv, part, lm, lam, stream)
        ref = ctx.evaluate(torch.tensor(part, dtype=torch.float32, device="cuda"), msd=True)
        torch.cuda.synchronize()
        rs, rz, rmsd = (ref[k].cpu().numpy() for k in ("s", "z", "msd"))
        assert d_err(msd, rmsd, part, lm) < TOL["fp32"]
        assert s_err(s, rs) < TOL["fp32"]
        assert z_err(z, rz, lam) < TOL["fp32"]
        r = oracle.exact(part, lm, lam)
        assert d_err(msd, r["D"], part, lm) < TOL["fp32"]
        assert s_err(s, r["s"]) < TOL["fp32"]
        assert z_err(z, r["z"], lam) < TOL["fp32"]
    ctx.close()


def test_noalloc_rejects_problems_beyond_the_fixed_scratch(pcv):
    err = ctypes.create_string_buffer(256)
    big_f = (16 << 20) // (4 * 200) + 1
    st = pcv.load().pcv_evaluate_exact_noalloc(big_f, 200, 300, ctypes.c_void_p(16), ctypes.c_void_p(16), None, 1.0,
                                                ctypes.c_void_p(16), ctypes.c_void_p(16), None, None, err, 256)
    assert st == pcv.PCV_EINVAL
    assert b"scratch" in err.value

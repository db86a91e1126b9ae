"""Few frames per call: the landmark-parallel kernels (one CTA per landmark, the landmark
staged in shared memory) against the oracle -- exact mode with 1..4 frames, close mode fed
one frame per call (the per-MD-step use of Algorithms 1 and 2), and the large
configuration N=5000, M=2000 in FP32 and FP16 storage."""
import numpy as np
import pytest

import oracle
from _util import GRAD_TOL, TOL, d_err, grad_err, problem, s_err, z_err

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


def _eval(ctx, fr, precision, grad=True):
    dt = torch.float64 if precision == "fp64" else torch.float32
    out = ctx.evaluate(torch.tensor(fr, dtype=dt, device="cuda"), grad=grad, msd=True, refreshed=True)
    ctx.sync()
    return {k: v.double().cpu().numpy() if v.dtype != torch.uint8 else v.cpu().numpy() for k, v in out.items()}


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16"])
@pytest.mark.parametrize("n", [61, 140])  # 3N*4 bytes unaligned / aligned to 16
@pytest.mark.parametrize("f", [1, 3, 4])
def test_exact_few_frames(pcv, precision, n, f):
    lm, fr, lam = problem(31, n, 37, f, noise=0.05)
    rng = np.random.default_rng(3)
    w = rng.uniform(0.5, 1.5, n) if n == 61 else None
    r = oracle.exact(fr, lm, lam, w=w, want_grad=True)
    ctx = pcv.PathCV(lm, lam, eps=-1.0, precision=precision, weights=w)
    g = _eval(ctx, fr, precision)
    ctx.close()
    tol = TOL[precision]
    assert d_err(g["msd"], r["D"], fr, lm, w) < tol
    assert s_err(g["s"], r["s"], 37) < tol
    assert z_err(g["z"], r["z"], lam) < tol
    assert grad_err(g["dsdx"], r["dsdx"]) < GRAD_TOL[precision]
    assert grad_err(g["dzdx"], r["dzdx"]) < GRAD_TOL[precision]


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16"])
def test_close_one_frame_per_call(pcv, precision):
    """40 frames fed one per call: refresh decisions carried across calls, approximate and
    refreshed frames from the streaming kernels; identical to the oracle's single run."""
    lm, fr, lam = problem(32, 120, 60, 40, noise=0.03, ou_rho=0.95)
    eps = 0.004
    r = oracle.close(fr, lm, lam, eps, want_grad=True)
    nref = int((r["refreshed"] > 0).sum())
    assert 3 < nref < 37
    ctx = pcv.PathCV(lm, lam, eps=eps, precision=precision)
    parts = [_eval(ctx, fr[t:t + 1], precision) for t in range(fr.shape[0])]
    ctx.close()
    g = {k: np.concatenate([p[k] for p in parts]) for k in parts[0]}
    np.testing.assert_array_equal(g["refreshed"], r["refreshed"])
    tol = TOL[precision]
    assert d_err(g["msd"], r["D"], fr, lm) < tol
    assert s_err(g["s"], r["s"], 60) < tol
    assert z_err(g["z"], r["z"], lam) < tol
    assert grad_err(g["dsdx"], r["dsdx"]) < GRAD_TOL[precision]
    assert grad_err(g["dzdx"], r["dzdx"]) < GRAD_TOL[precision]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("mode", ["exact", "close"])
def test_one_frame_many_landmarks_gradients(pcv, precision, mode):
    """One frame per call against 521 landmarks of 24 atoms (one MD step of a long path):
    the adjoint's landmark sum is split into ranges (ragged last range) whose partial sums
    are added by a second kernel; gradients against the oracle frame by frame."""
    lm, fr, lam = problem(36, 24, 521, 12, noise=0.02, ou_rho=0.9)
    eps = -1.0 if mode == "exact" else 0.01
    r = oracle.exact(fr, lm, lam, want_grad=True) if mode == "exact" else oracle.close(fr, lm, lam, eps,
                                                                                        want_grad=True)
    ctx = pcv.PathCV(lm, lam, eps=eps, precision=precision)
    parts = [_eval(ctx, fr[t:t + 1], precision) for t in range(fr.shape[0])]
    ctx.close()
    g = {k: np.concatenate([p[k] for p in parts]) for k in parts[0]}
    if mode == "close":
        np.testing.assert_array_equal(g["refreshed"], r["refreshed"])
    tol = TOL[precision]
    assert s_err(g["s"], r["s"], 521) < tol
    assert z_err(g["z"], r["z"], lam) < tol
    assert grad_err(g["dsdx"], r["dsdx"]) < GRAD_TOL[precision]
    assert grad_err(g["dzdx"], r["dzdx"]) < GRAD_TOL[precision]


@pytest.mark.parametrize("precision", ["fp32", "fp16"])
def test_large_set_streaming_c5(pcv, precision):
    """N=5000, M=2000 (120 MB FP32 / 60 MB FP16 landmarks), close structure on, one frame
    per call for 8 frames; values against the oracle's run over the same frames."""
    from paper_1801_02362_gb300 import synth

    ldt = np.float16 if precision == "fp16" else np.float32
    lm, fr = synth.make_problem(5, n_atoms=5000, n_landmarks=2000, n_frames=10_000, frame_noise=0.05,
                                landmark_dtype=ldt)
    fr = np.ascontiguousarray(fr[:8])
    lam = 2.3 / oracle.mean_adjacent_msd(lm)
    eps = 0.05
    r = oracle.close(fr, lm, lam, eps, want_grad=False)
    ctx = pcv.PathCV(lm, lam, eps=eps, precision=precision)
    parts = [_eval(ctx, fr[t:t + 1], precision, grad=False) for t in range(fr.shape[0])]
    ctx.close()
    g = {k: np.concatenate([p[k] for p in parts]) for k in ("s", "z", "msd", "refreshed")}
    np.testing.assert_array_equal(g["refreshed"], r["refreshed"])
    tol = TOL[precision]
    assert d_err(g["msd"], r["D"], fr, lm) < tol
    assert s_err(g["s"], r["s"], 2000) < tol
    assert z_err(g["z"], r["z"], lam) < tol

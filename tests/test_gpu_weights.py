"""GPU parity with separate alignment weights w' (pcv_set_landmarks_weighted; Section 3.1
after Eq. der_dist) against the oracle, element by element: exact mode and the close
structure, FP64 / FP32 / FP16 storage, explicit and uniform displacement weights, and with a
neighbour list."""
import numpy as np
import pytest

import oracle
from _util import GRAD_TOL, TOL, grad_err, gsum, problem, s_err, z_err
from test_gpu_nl import assert_clear_gaps

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


def run(pcv, lm, fr, lam, eps, precision, w, wa, nl=None):
    ctx = pcv.PathCV(lm, lam, eps=eps, precision=precision, weights=w, align_weights=wa, neighbor_list=nl)
    dt = torch.float64 if precision == "fp64" else torch.float32
    out = ctx.evaluate(torch.tensor(fr, dtype=dt, device="cuda"), grad=True, msd=True, refreshed=True)
    ctx.sync()
    res = {k: v.double().cpu().numpy() if v.dtype != torch.uint8 else v.cpu().numpy() for k, v in out.items()}
    ctx.close()
    return res


def check(g, r, fr, lm, lam, precision, w):
    tol = TOL[precision]
    fin = np.isfinite(r["D"])
    np.testing.assert_array_equal(np.isfinite(g["msd"]), fin)
    den = np.maximum(r["D"], 1e-3 * (gsum(fr, w)[:, None] + gsum(lm, w)[None, :]))
    assert np.max(np.abs(g["msd"][fin] - r["D"][fin]) / den[fin]) < tol
    assert s_err(g["s"], r["s"], lm.shape[0]) < tol
    assert z_err(g["z"], r["z"], lam) < tol
    assert grad_err(g["dsdx"], r["dsdx"]) < GRAD_TOL[precision]
    assert grad_err(g["dzdx"], r["dzdx"]) < GRAD_TOL[precision]


def weights(seed, n, uniform_w=False):
    rng = np.random.default_rng(seed)
    w = None if uniform_w else rng.uniform(0.3, 3.0, size=n)
    wa = rng.uniform(0.3, 3.0, size=n)
    return w, wa


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16"])
@pytest.mark.parametrize("uniform_w", [False, True])
def test_alignment_weights_exact_mode(pcv, precision, uniform_w):
    """N=57, M=33, F=70, reflecting walk: distances, s, z and both gradients (the centre
    term of Eq. der_dist) against the oracle."""
    lm, fr, lam = problem(91, 57, 33, 70, noise=0.03, schedule="walk", precision=precision)
    w, wa = weights(1, 57, uniform_w)
    r = oracle.exact(fr, lm, lam, w=w, wa=wa, want_grad=True)
    g = run(pcv, lm, fr, lam, -1.0, precision, w, wa)
    check(g, r, fr, lm, lam, precision, w)


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16"])
def test_alignment_weights_close_mode(pcv, precision):
    """N=48, M=40, F=300 drifting frames, several reassignments: the refresh decisions
    exactly, and the approximate frames' gradients with the rotation term's centre part."""
    lm, fr, lam = problem(92, 48, 40, 300, noise=0.01, schedule="drift", precision=precision)
    w, wa = weights(2, 48)
    eps = 0.004
    r = oracle.close(fr, lm, lam, eps, w=w, wa=wa, want_grad=True)
    assert int((r["refreshed"] == 1).sum()) >= 3
    g = run(pcv, lm, fr, lam, eps, precision, w, wa)
    np.testing.assert_array_equal(g["refreshed"], r["refreshed"])
    check(g, r, fr, lm, lam, precision, w)


def test_alignment_weights_with_a_neighbour_list(pcv):
    lm, fr, lam = problem(93, 40, 60, 120, noise=0.03, schedule="walk")
    w, wa = weights(3, 40)
    r = oracle.exact(fr, lm, lam, w=w, wa=wa, want_grad=True, nl=(20, 9))
    assert_clear_gaps(r, 20, fr, lm, TOL["fp32"])
    g = run(pcv, lm, fr, lam, -1.0, "fp32", w, wa, nl=(20, 9))
    check(g, r, fr, lm, lam, "fp32", w)


def test_equal_sets_match_the_single_set(pcv):
    lm, fr, lam = problem(94, 30, 20, 50)
    w, _ = weights(4, 30)
    a = run(pcv, lm, fr, lam, 0.004, "fp32", w, None)
    b = run(pcv, lm, fr, lam, 0.004, "fp32", w, w)
    for key in ("s", "z", "msd", "dsdx", "dzdx", "refreshed"):
        np.testing.assert_array_equal(a[key], b[key])


@pytest.mark.parametrize("precision", ["fp32", "fp16"])
@pytest.mark.parametrize("mode", ["exact", "close"])
def test_alignment_weights_large_structures(pcv, precision, mode):
    """N=4400 atoms, M=16: the structures are too large to stage per warp, so the finish
    runs one block per frame, here with separate alignment weights (the centre terms' block
    sums) and, in close mode, at 80 approximate frames among 79 reassignments (Gamma and Phi
    from the softmax weights and the segments' rotations)."""
    lm, fr, lam = problem(93, 4400, 16, 160 if mode == "close" else 40, noise=0.01, schedule="drift",
                          precision=precision)
    rng = np.random.default_rng(3)
    w, wa = rng.uniform(0.3, 3.0, 4400), rng.uniform(0.3, 3.0, 4400)
    if mode == "close":
        r = oracle.close(fr, lm, lam, 0.004, w=w, wa=wa, want_grad=True)
        assert int((r["refreshed"] == 0).sum()) >= 40
        g = run(pcv, lm, fr, lam, 0.004, precision, w, wa)
        np.testing.assert_array_equal(g["refreshed"], r["refreshed"])
    else:
        r = oracle.exact(fr, lm, lam, w=w, wa=wa, want_grad=True)
        g = run(pcv, lm, fr, lam, -1.0, precision, w, wa)
    check(g, r, fr, lm, lam, precision, w)

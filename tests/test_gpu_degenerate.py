"""Degenerate superpositions on the GPU.  Collinear frames and landmarks make H rank one:
the top eigenvalue of the quaternion matrix is double and the optimal rotation is free about
the line.  With both structures collinear, R a_i is unique, so D, s, z and the gradients are
unique and are compared with the oracle.  Newton on the characteristic quartic converges only
linearly at a double root, so both precisions detect it from P'(l) and take the Jacobi
iteration instead: FP32 inside its eigen-solve, FP64 in a second pass over the pairs the
tiled kernel marked (and inside the one-pair-per-warp FP64 alignments)."""
import numpy as np
import pytest

import oracle
from _util import GRAD_TOL, TOL, d_err, grad_err, s_err, z_err

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


def collinear(rng, n, scale=1.0):
    d = rng.normal(size=3)
    d /= np.linalg.norm(d)
    t = np.sort(rng.normal(size=n)) * scale
    return rng.normal(size=3) + t[:, None] * d[None, :]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_collinear_structures_exact_mode(pcv, precision):
    rng = np.random.default_rng(41)
    n, m, f = 40, 9, 24
    dt = np.float64 if precision == "fp64" else np.float32
    lm = np.stack([collinear(rng, n, scale=1.0 + 0.1 * i) for i in range(m)]).astype(dt).astype(np.float64)
    fr = np.stack([collinear(rng, n, scale=1.05) for _ in range(f)]).astype(dt).astype(np.float64)
    lam = 2.3 / oracle.mean_adjacent_msd(lm)
    r = oracle.exact(fr, lm, lam, want_grad=True)
    ctx = pcv.PathCV(lm, lam, eps=-1.0, precision=precision)
    tdt = torch.float64 if precision == "fp64" else torch.float32
    out = ctx.evaluate(torch.tensor(fr, dtype=tdt, device="cuda"), grad=True, msd=True)
    ctx.sync()
    ctx.close()
    g = {k: v.double().cpu().numpy() for k, v in out.items()}
    tol = TOL[precision]
    assert np.all(np.isfinite(g["msd"]))
    assert d_err(g["msd"], r["D"], fr, lm) < tol
    assert s_err(g["s"], r["s"], m) < tol
    assert z_err(g["z"], r["z"], lam) < tol
    assert grad_err(g["dsdx"], r["dsdx"]) < GRAD_TOL[precision]
    assert grad_err(g["dzdx"], r["dzdx"]) < GRAD_TOL[precision]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_collinear_structures_every_frame_reassigns(pcv, precision):
    """Close-structure mode with a threshold below every frame-to-frame distance: each frame
    is a reassignment, so the frame-to-close-structure alignments (degenerate pairs too) all
    decide "reassign", and every frame's D, s, z and gradients are the exact ones.  Frames are
    evaluated in calls of 1, 3 and 20, so the exact pairs run both as the few-frame path and
    as the tiled kernel over a list of reassignment rows."""
    rng = np.random.default_rng(43)
    n, m, f = 40, 9, 24
    dt = np.float64 if precision == "fp64" else np.float32
    lm = np.stack([collinear(rng, n, scale=1.0 + 0.1 * i) for i in range(m)]).astype(dt).astype(np.float64)
    fr = np.stack([collinear(rng, n, scale=1.05) for _ in range(f)]).astype(dt).astype(np.float64)
    lam = 2.3 / oracle.mean_adjacent_msd(lm)
    eps = 1e-12
    r = oracle.exact(fr, lm, lam, want_grad=True)
    rc = oracle.close(fr, lm, lam, eps, want_grad=True)
    assert np.all(rc["refreshed"][1:] == 1) and rc["refreshed"][0] == 2
    ctx = pcv.PathCV(lm, lam, eps=eps, precision=precision)
    tdt = torch.float64 if precision == "fp64" else torch.float32
    x = torch.tensor(fr, dtype=tdt, device="cuda")
    parts = [ctx.evaluate(x[a:b], grad=True, msd=True, refreshed=True) for a, b in ((0, 1), (1, 4), (4, f))]
    ctx.sync()
    ctx.close()
    g = {k: np.concatenate([o[k].double().cpu().numpy() for o in parts]) for k in parts[0]}
    tol = TOL[precision]
    np.testing.assert_array_equal(g["refreshed"], rc["refreshed"])
    assert d_err(g["msd"], r["D"], fr, lm) < tol
    assert s_err(g["s"], r["s"], m) < tol
    assert z_err(g["z"], r["z"], lam) < tol
    assert grad_err(g["dsdx"], r["dsdx"]) < GRAD_TOL[precision]
    assert grad_err(g["dzdx"], r["dzdx"]) < GRAD_TOL[precision]

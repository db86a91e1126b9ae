"""GPU parity of the neighbour list (pcv_set_neighbor_list) against the oracle's
neighbour-list evaluation, element by element, in exact mode (the original method of
Section 6.2) and with the close structure (end of Section 3.2).

The list is an integer decision taken on floating-point distances.  The tests compare the
list membership exactly (the +inf pattern of the MSD rows) on data whose M_nl-th and
(M_nl+1)-th smallest distances at every update step differ by more than the sum of their
tolerances (checked on the oracle's distances): distances within tolerance cannot order
the two differently, so the choice is the same in any precision."""
import numpy as np
import pytest

import oracle
from _util import GRAD_TOL, TOL, grad_err, gsum, problem, s_err, z_err

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


def evaluate(ctx, fr, precision, grad=True):
    dt = torch.float64 if precision == "fp64" else torch.float32
    frames = torch.tensor(fr, dtype=dt, device="cuda")
    out = ctx.evaluate(frames, grad=grad, msd=True, refreshed=True)
    ctx.sync()
    res = {k: v.double().cpu().numpy() if v.dtype != torch.uint8 else v.cpu().numpy() for k, v in out.items()}
    res["stats"] = ctx.stats()
    return res


def update_rows(r, m_nl):
    """Rows of the oracle's D where every landmark was evaluated (list updates)."""
    return np.where(np.all(np.isfinite(r["D"]), axis=1))[0]


def assert_clear_gaps(r, m_nl, fr, lm, tol):
    """Precondition on the data: at every update the M_nl-th and (M_nl+1)-th smallest
    distances differ by more than the sum of their tolerances (with a margin), so distances
    that pass the D check below cannot order the two differently."""
    ga = gsum(lm)
    for t in update_rows(r, m_nl):
        order = np.argsort(r["D"][t], kind="stable")
        k0, k1 = order[m_nl - 1], order[m_nl]
        gx = float(gsum(fr[t:t + 1])[0])
        den = [max(r["D"][t][k], 1e-3 * (gx + ga[k])) for k in (k0, k1)]
        assert r["D"][t][k1] - r["D"][t][k0] > 1.25 * tol * (den[0] + den[1]), f"near-tie at update frame {t}"


def check(g, r, fr, lm, lam, precision, m_nl, grad=True):
    tol = TOL[precision]
    m = lm.shape[0]
    fin_r = np.isfinite(r["D"])
    np.testing.assert_array_equal(np.isfinite(g["msd"]), fin_r)  # same lists at every frame
    assert np.all(fin_r.sum(axis=1) >= m_nl)
    gx = gsum(fr)[:, None]
    ga = gsum(lm)[None, :]
    den = np.maximum(r["D"], 1e-3 * (gx + ga))
    assert np.max(np.abs(g["msd"][fin_r] - r["D"][fin_r]) / den[fin_r]) < tol
    assert s_err(g["s"], r["s"], m) < tol
    assert z_err(g["z"], r["z"], lam) < tol
    if grad:
        assert grad_err(g["dsdx"], r["dsdx"]) < GRAD_TOL[precision]
        assert grad_err(g["dzdx"], r["dzdx"]) < GRAD_TOL[precision]


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16"])
@pytest.mark.parametrize("m_nl,L", [(12, 7), (34, 40)])
def test_nl_exact_mode(pcv, precision, m_nl, L):
    """Original method: N=40, M=70 (ragged landmark tile), F=300; a list of 12 every 7 steps,
    and of 34 (two landmark columns of the tiled kernels, the second ragged) every 40 steps
    (full 16-frame tiles and a ragged last tile per run)."""
    lm, fr, lam = problem(67, 40, 70, 300, noise=0.03, schedule="walk", precision=precision)
    r = oracle.exact(fr, lm, lam, want_grad=True, nl=(m_nl, L))
    assert_clear_gaps(r, m_nl, fr, lm, TOL[precision])
    ctx = pcv.PathCV(lm, lam, eps=-1.0, precision=precision, neighbor_list=(m_nl, L))
    g = evaluate(ctx, fr, precision)
    check(g, r, fr, lm, lam, precision, m_nl)
    n_upd = len(range(0, fr.shape[0], L))
    assert g["stats"]["landmark_alignments"] == r["state"].counters["landmark_alignments"]
    assert g["stats"]["landmark_alignments"] == n_upd * 70 + (300 - n_upd) * m_nl
    ctx.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16"])
def test_nl_close_mode(pcv, precision):
    """Close structure: N=48, M=90, F=400 drifting frames, several reassignments, a list of 9
    every 10 steps chosen from approximate distances between reassignments."""
    m_nl, L, eps = 9, 10, 0.004
    lm, fr, lam = problem(62, 48, 90, 400, noise=0.01, schedule="drift", precision=precision)
    r = oracle.close(fr, lm, lam, eps, want_grad=True, nl=(m_nl, L))
    assert int((r["refreshed"] == 1).sum()) >= 3
    assert_clear_gaps(r, m_nl, fr, lm, TOL[precision])
    ctx = pcv.PathCV(lm, lam, eps=eps, precision=precision, neighbor_list=(m_nl, L))
    g = evaluate(ctx, fr, precision)
    np.testing.assert_array_equal(g["refreshed"], r["refreshed"])
    check(g, r, fr, lm, lam, precision, m_nl)
    c = r["state"].counters
    for key in ("xy_alignments", "landmark_alignments", "approx_msds", "refreshes_threshold"):
        assert g["stats"][key] == c[key], key
    ctx.close()


def test_nl_split_calls_and_saved_state(pcv):
    """The list and the step count carry over between calls and through save/load."""
    m_nl, L, eps = 10, 9, 0.004
    lm, fr, lam = problem(63, 36, 60, 240, noise=0.01, schedule="drift")
    for mode_eps in (-1.0, eps):
        whole = (oracle.exact(fr, lm, lam, want_grad=True, nl=(m_nl, L)) if mode_eps < 0 else
                 oracle.close(fr, lm, lam, eps, want_grad=True, nl=(m_nl, L)))
        ctx = pcv.PathCV(lm, lam, eps=mode_eps, precision="fp32", neighbor_list=(m_nl, L))
        a = evaluate(ctx, fr[:101], "fp32")
        blob = ctx.save_state()
        ctx.close()
        ctx = pcv.PathCV(lm, lam, eps=mode_eps, precision="fp32", neighbor_list=(m_nl, L))
        ctx.load_state(blob)
        b = evaluate(ctx, fr[101:170], "fp32")
        c = evaluate(ctx, fr[170:], "fp32")
        ctx.close()
        g = {k: np.concatenate([a[k], b[k], c[k]]) for k in ("s", "z", "msd", "dsdx", "dzdx", "refreshed")}
        check(g, whole, fr, lm, lam, "fp32", m_nl)


def test_nl_off_sizes_match_the_full_evaluation(pcv):
    """size 0 or >= M evaluates everything; stride 1 updates at every step."""
    lm, fr, lam = problem(64, 30, 40, 80, noise=0.02, schedule="walk")
    r = oracle.exact(fr, lm, lam, want_grad=True)
    for nl in ((0, 5), (40, 5), (55, 2), (6, 1)):
        ctx = pcv.PathCV(lm, lam, eps=-1.0, precision="fp32", neighbor_list=nl)
        g = evaluate(ctx, fr, "fp32")
        ctx.close()
        check(g, r, fr, lm, lam, "fp32", 40 if nl[1] > 1 else 6)


def test_nl_bad_arguments(pcv):
    lm, fr, lam = problem(65, 10, 8, 4)
    ctx = pcv.PathCV(lm, lam)
    for bad in ((-1, 5), (3, 0)):
        with pytest.raises(pcv.PcvError) as e:
            ctx.set_neighbor_list(*bad)
        assert e.value.status == pcv.PCV_EINVAL
    ctx.close()

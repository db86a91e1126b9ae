"""Pins of the oracle's neighbour list (Section 2; Section 3.1 after Eq. der_dist; the end
of Section 3.2; Section 6.2) against facts that do not come from the neighbour-list code:
the already-pinned full evaluation restricted to a subset chosen by numpy, scipy's
log-sum-exp over that subset, central differences, and the paper's printed cost-model
numbers."""
import json
from pathlib import Path

import numpy as np
import pytest
from scipy.special import logsumexp

import oracle
from paper_1801_02362_gb300 import synth

GOLDEN = Path(__file__).parent / "golden"


def _problem(seed, n, m, f, noise=0.02, schedule="walk"):
    lm, fr = synth.make_problem(seed, n_atoms=n, n_landmarks=m, n_frames=f, frame_noise=noise, schedule=schedule,
                                frame_dtype=np.float64, landmark_dtype=np.float64)
    lam = 2.3 / oracle.mean_adjacent_msd(lm)
    return lm, fr, lam


def _subset_cv(D, S, lam):
    """s and z of Eq. (property_map_cv) over the landmarks S only (q_i = i, 1-based)."""
    d = D[S]
    logw = -lam * d - logsumexp(-lam * d)
    s = float(np.sum((S + 1) * np.exp(logw)))
    z = float(-logsumexp(-lam * d) / lam)
    return s, z


def _first(D, k):
    """numpy's choice of the k smallest (stable sort: ties to the lower index), sorted."""
    return np.sort(np.argsort(D, kind="stable")[:k])


def test_nl_select_order_and_ties():
    rng = np.random.default_rng(3)
    D = rng.integers(0, 6, size=40).astype(np.float64)  # many ties
    for k in (1, 5, 17, 39, 40):
        np.testing.assert_array_equal(oracle.nl_select(D, k), _first(D, k))


def test_nl_exact_is_the_full_evaluation_restricted_to_the_list():
    """Original method (Section 6.2): every L-th step evaluates all landmarks and keeps the
    M_nl closest; the steps in between evaluate only those."""
    lm, fr, lam = _problem(51, n=12, m=30, f=40)
    m_nl, L = 6, 7
    full = oracle.exact(fr, lm, lam)
    r = oracle.exact(fr, lm, lam, nl=(m_nl, L))
    S = None
    for t in range(fr.shape[0]):
        if t % L == 0:
            np.testing.assert_array_equal(r["D"][t], full["D"][t])
            assert r["s"][t] == full["s"][t] and r["z"][t] == full["z"][t]
            S = _first(full["D"][t], m_nl)
            continue
        listed = np.zeros(lm.shape[0], bool)
        listed[S] = True
        np.testing.assert_array_equal(r["D"][t][listed], full["D"][t][listed])
        assert np.all(np.isinf(r["D"][t][~listed]))
        s, z = _subset_cv(full["D"][t], S, lam)
        assert abs(r["s"][t] - s) < 1e-12 * lm.shape[0]
        assert abs(r["z"][t] - z) < 1e-12 * max(abs(z), 1.0 / lam)
        # fewer terms in the sum: z can only grow
        assert r["z"][t] >= full["z"][t] - 1e-15
    c = r["state"].counters
    n_upd = len(range(0, fr.shape[0], L))
    assert c["landmark_alignments"] == n_upd * lm.shape[0] + (fr.shape[0] - n_upd) * m_nl


def test_nl_close_chooses_from_approximate_distances():
    """Close structure with a neighbour list (end of Section 3.2): the decisions of
    Algorithm 2 do not change; reassignments evaluate everything exactly, other update
    steps evaluate every landmark approximately and choose the list from those."""
    lm, fr, lam = _problem(52, n=14, m=24, f=60, noise=0.01, schedule="drift")
    m_nl, L, eps = 5, 6, 0.003
    full = oracle.close(fr, lm, lam, eps)
    r = oracle.close(fr, lm, lam, eps, nl=(m_nl, L))
    np.testing.assert_array_equal(r["refreshed"], full["refreshed"])
    np.testing.assert_array_equal(r["dxy"], full["dxy"])
    assert int((full["refreshed"] == 1).sum()) >= 2
    S = None
    n_upd = 0
    for t in range(fr.shape[0]):
        if full["refreshed"][t] or t % L == 0:
            n_upd += 1
            np.testing.assert_array_equal(r["D"][t], full["D"][t])
            assert r["s"][t] == full["s"][t]
            S = _first(full["D"][t], m_nl)
            continue
        listed = np.zeros(lm.shape[0], bool)
        listed[S] = True
        np.testing.assert_array_equal(r["D"][t][listed], full["D"][t][listed])
        assert np.all(np.isinf(r["D"][t][~listed]))
        s, z = _subset_cv(full["D"][t], S, lam)
        assert abs(r["s"][t] - s) < 1e-12 * lm.shape[0]
        assert abs(r["z"][t] - z) < 1e-12 * max(abs(z), 1.0 / lam)
    c, cf = r["state"].counters, full["state"].counters
    # the list adds no expensive distance computation (cost 1 + N/K of Section 6.2)
    assert c["xy_alignments"] == cf["xy_alignments"]
    assert c["landmark_alignments"] == cf["landmark_alignments"]
    nref = int((full["refreshed"] > 0).sum())
    assert c["approx_msds"] == (n_upd - nref) * lm.shape[0] + (fr.shape[0] - n_upd) * m_nl


@pytest.mark.parametrize("nl", [(0, 5), (30, 5), (45, 3), (7, 1)])
def test_nl_off_cases_equal_the_full_evaluation(nl):
    """No list (M_nl = 0 or >= M) and a list updated every step (L = 1) evaluate every
    landmark at every step."""
    lm, fr, lam = _problem(53, n=10, m=30, f=12)
    a = oracle.exact(fr, lm, lam, want_grad=True)
    b = oracle.exact(fr, lm, lam, want_grad=True, nl=nl)
    for key in ("s", "z", "D", "dsdx", "dzdx"):
        np.testing.assert_array_equal(a[key], b[key])
    a = oracle.close(fr, lm, lam, 0.002, want_grad=True)
    b = oracle.close(fr, lm, lam, 0.002, want_grad=True, nl=nl)
    for key in ("s", "z", "D", "dsdx", "dzdx", "refreshed"):
        np.testing.assert_array_equal(a[key], b[key])


def _fd(fun, x, h=1e-6):
    g = np.zeros_like(x)
    for idx in np.ndindex(x.shape):
        xp = x.copy()
        xm = x.copy()
        xp[idx] += h
        xm[idx] -= h
        g[idx] = (fun(xp) - fun(xm)) / (2 * h)
    return g


def test_nl_gradients_match_central_differences():
    """At a step between list updates the derivatives run over the listed landmarks only;
    the list itself is fixed (it was chosen at an earlier step)."""
    n, m, m_nl = 8, 12, 4
    lm, fr, lam = _problem(54, n=n, m=m, f=3, noise=0.01)
    w = np.random.default_rng(4).uniform(0.5, 1.5, size=n)
    x = fr[1] + 0.02 * np.random.default_rng(5).normal(size=(n, 3))
    # exact mode: frame 0 chooses the list, frame x uses it
    st0 = oracle.CloseState(n, m)
    oracle.exact(fr[:1], lm, lam, w=w, nl=(m_nl, 100), state=st0)
    r = oracle.exact(x[None], lm, lam, w=w, want_grad=True, nl=(m_nl, 100), state=st0.copy())
    assert np.isinf(r["D"][0]).sum() == m - m_nl
    for key in ("s", "z"):
        g = _fd(lambda xx: oracle.exact(xx[None], lm, lam, w=w, nl=(m_nl, 100), state=st0.copy())[key][0], x)
        an = r["dsdx" if key == "s" else "dzdx"][0]
        assert np.max(np.abs(an - g)) < 1e-6 * np.max(np.abs(g)) + 1e-9, key
    # close mode: an approximate step between updates (rotation term included)
    st1 = oracle.CloseState(n, m)
    oracle.close(fr[:1], lm, lam, 10.0, w=w, nl=(m_nl, 100), state=st1)
    r = oracle.close(x[None], lm, lam, 10.0, w=w, want_grad=True, nl=(m_nl, 100), state=st1.copy())
    assert r["refreshed"][0] == 0 and np.isinf(r["D"][0]).sum() == m - m_nl
    for key in ("s", "z"):
        g = _fd(lambda xx: oracle.close(xx[None], lm, lam, 10.0, w=w, nl=(m_nl, 100), state=st1.copy())[key][0], x)
        an = r["dsdx" if key == "s" else "dzdx"][0]
        assert np.max(np.abs(an - g)) < 1e-6 * np.max(np.abs(g)) + 1e-9, key


def test_nl_split_calls_carry_the_list():
    lm, fr, lam = _problem(55, n=10, m=20, f=45, noise=0.02)
    for mode in ("exact", "close"):
        run = (lambda frames, st: oracle.exact(frames, lm, lam, nl=(4, 6), state=st)) if mode == "exact" else (
            lambda frames, st: oracle.close(frames, lm, lam, 0.003, nl=(4, 6), state=st))
        whole = run(fr, oracle.CloseState(10, 20))
        st = oracle.CloseState(10, 20)
        a = run(fr[:17], st)
        b = run(fr[17:], st)
        for key in ("s", "z", "D"):
            np.testing.assert_array_equal(np.concatenate([a[key], b[key]]), whole[key])
        assert st.counters == whole["state"].counters


def test_nl_cost_model_matches_trpcage_numbers():
    """Section 6.3: with 2120 landmarks, a list of 50 updated every 50 steps, the original
    method needs 50 + (2120 - 50)/50 = 91.4 expensive distances per step; the close
    structure keeps 1 + N/K whatever the list (three-atom structures keep this fast)."""
    tc = json.loads((GOLDEN / "cost_model.json").read_text())["trpcage"]
    lm, fr = synth.make_problem(56, n_atoms=3, n_landmarks=tc["n_ref"], n_frames=100, frame_noise=0.02,
                                schedule="walk", frame_dtype=np.float64, landmark_dtype=np.float64)
    r = oracle.exact(fr, lm, 10.0, want_D=False, nl=(tc["m_nl"], tc["l_stride"]))
    c = r["state"].counters
    assert abs(c["landmark_alignments"] / fr.shape[0] - tc["original_per_step"]) < 1e-12
    r = oracle.close(fr, lm, 10.0, 1e6, want_D=False, nl=(tc["m_nl"], tc["l_stride"]))
    c = r["state"].counters
    assert c["refreshes_threshold"] == 0 and c["landmark_alignments"] == tc["n_ref"]
    # 1 + N/K with K = 100 (one assignment in 100 steps), less the first step's x-y alignment
    per_step = (c["xy_alignments"] + c["landmark_alignments"]) / fr.shape[0]
    assert abs(per_step - (oracle.cost_close(tc["n_ref"], fr.shape[0]) - 1.0 / fr.shape[0])) < 1e-12
    assert c["approx_msds"] == tc["n_ref"] + 98 * tc["m_nl"]

"""Pins of the oracle with separate displacement weights w and alignment weights w'
(Section 3.1 after Eq. der_dist: w weighs each atom's displacement in the distance, w' its
contribution to the centre of mass that sets the translation) against facts that do not
come from the oracle's code: an SVD superposition with the same centring, central
differences, translation and rotation invariance, and the w' = w special case."""
import numpy as np

import oracle
from paper_1801_02362_gb300 import synth


def kabsch_wa(x, a, w, wa):
    """SVD fit of a onto x after centring both by their w'-weighted centres, minimising the
    w-weighted distance (Kabsch 1976 with the reflection fix)."""
    w = w / w.sum()
    wa = wa / wa.sum()
    xc = x - wa @ x
    ac = a - wa @ a
    H = (ac * w[:, None]).T @ xc
    U, S, Vt = np.linalg.svd(H)
    d = np.sign(np.linalg.det(Vt.T @ U.T))
    R = Vt.T @ np.diag([1.0, 1.0, d]) @ U.T
    return float(np.sum(w * np.sum((xc - ac @ R.T) ** 2, axis=1)))


def _problem(seed, n, m, f, noise=0.03):
    lm, fr = synth.make_problem(seed, n_atoms=n, n_landmarks=m, n_frames=f, frame_noise=noise, schedule="walk",
                                frame_dtype=np.float64, landmark_dtype=np.float64)
    rng = np.random.default_rng(seed)
    w = rng.uniform(0.3, 3.0, size=n)
    wa = rng.uniform(0.3, 3.0, size=n)
    return lm, fr, w, wa


def test_distances_match_svd_with_the_same_centring():
    lm, fr, w, wa = _problem(81, 11, 7, 4)
    lam = 50.0
    r = oracle.exact(fr, lm, lam, w=w, wa=wa)
    for t in range(fr.shape[0]):
        for i in range(lm.shape[0]):
            d_svd = kabsch_wa(fr[t], lm[i], w, wa)
            assert abs(r["D"][t, i] - d_svd) < 1e-12 * (1.0 + d_svd)
            # the w'-centring is not the distance's optimal translation: never below the
            # distance with w-centring
            assert r["D"][t, i] >= kabsch_wa(fr[t], lm[i], w, w) - 1e-13


def test_equal_weight_sets_reproduce_the_single_set():
    lm, fr, w, _ = _problem(82, 9, 6, 5)
    lam = 2.3 / oracle.mean_adjacent_msd(lm)
    a = oracle.exact(fr, lm, lam, w=w, want_grad=True)
    b = oracle.exact(fr, lm, lam, w=w, wa=w, want_grad=True)
    for key in ("s", "z", "D", "dsdx", "dzdx"):
        np.testing.assert_array_equal(a[key], b[key])
    a = oracle.close(fr, lm, lam, 0.001, w=w, want_grad=True)
    b = oracle.close(fr, lm, lam, 0.001, w=w, wa=w, want_grad=True)
    for key in ("s", "z", "D", "dsdx", "dzdx", "refreshed"):
        np.testing.assert_array_equal(a[key], b[key])


def _fd(fun, x, h=1e-6):
    g = np.zeros_like(x)
    for idx in np.ndindex(x.shape):
        xp, xm = x.copy(), x.copy()
        xp[idx] += h
        xm[idx] -= h
        g[idx] = (fun(xp) - fun(xm)) / (2 * h)
    return g


def test_exact_gradient_with_alignment_weights():
    """Eq. (der_dist) with w' != w: the centre term w'_k sum_j (-2 w_j d_j) no longer
    vanishes; the rotation term still does (R minimises the distance)."""
    lm, fr, w, wa = _problem(83, 8, 6, 3)
    lam = 2.3 / oracle.mean_adjacent_msd(lm)
    r = oracle.exact(fr, lm, lam, w=w, wa=wa, want_grad=True)
    for t in range(fr.shape[0]):
        for key in ("s", "z"):
            g = _fd(lambda x: oracle.exact(x[None], lm, lam, w=w, wa=wa)[key][0], fr[t])
            an = r["dsdx" if key == "s" else "dzdx"][t]
            assert np.max(np.abs(an - g)) < 1e-6 * np.max(np.abs(g)) + 1e-9, (key, t)
            # translation invariance: the gradient sums to zero over the atoms
            assert np.max(np.abs(an.sum(0))) < 1e-10 * np.max(np.abs(an)) * 8
    # the centre term matters: dropping it (w' -> w in the formula) misses the derivative
    t = 0
    g = _fd(lambda x: oracle.exact(x[None], lm, lam, w=w, wa=wa)["z"][0], fr[t])
    wrong = oracle.exact(fr[t:t + 1], lm, lam, w=w, want_grad=True)["dzdx"][0]
    assert np.max(np.abs(wrong - g)) > 1e-3 * np.max(np.abs(g))


def test_close_gradient_with_alignment_weights():
    """Eq. (close_der_dist) with w' != w: the centre term, and dH_xy/dx_k = (w_k y_k -
    w'_k sum_j w_j y_j) e_c^T in the rotation term."""
    n, m = 8, 5
    lm, fr, w, wa = _problem(84, n, m, 3, noise=0.01)
    lam = 2.3 / oracle.mean_adjacent_msd(lm)
    st = oracle.CloseState(n, m)
    oracle.close(fr[:1], lm, lam, eps=10.0, state=st, w=w, wa=wa)
    y, B = fr[0], st.B.copy()
    x = fr[0] + 0.03 * np.random.default_rng(5).normal(size=(n, 3))
    r = oracle.close(x[None], lm, lam, eps=10.0, state=st.copy(), w=w, wa=wa, want_grad=True)
    assert r["refreshed"][0] == 0

    def cvs(xx):
        D = np.array([oracle.close_distance(xx, y, B[i], lm[i], w=w, wa=wa) for i in range(m)])
        s, z, _ = oracle.path_cv(D, lam)
        return s, z

    np.testing.assert_allclose([oracle.close_distance(x, y, B[i], lm[i], w=w, wa=wa) for i in range(m)], r["D"][0],
                               rtol=1e-12, atol=1e-15)
    for k, key in ((0, "dsdx"), (1, "dzdx")):
        g = _fd(lambda xx: cvs(xx)[k], x)
        an = r[key][0]
        assert np.max(np.abs(an - g)) < 1e-6 * np.max(np.abs(g)) + 1e-9, key
        assert np.max(np.abs(an.sum(0))) < 1e-10 * np.max(np.abs(an)) * n

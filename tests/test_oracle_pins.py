"""Pins of the FP64 oracle against facts that do not come from the oracle itself:
SVD-based Kabsch superposition, brute-force rotation search, closed forms, invariants,
finite differences and the worked numbers printed in the paper."""
import json
from pathlib import Path

import numpy as np
import pytest
from scipy.optimize import minimize
from scipy.spatial.transform import Rotation
from scipy.special import logsumexp

import oracle
from _util import problem
from paper_1801_02362_gb300 import synth

GOLDEN = Path(__file__).parent / "golden"


def kabsch(x, a, w=None):
    """Textbook SVD superposition (Kabsch 1976) with the reflection fix."""
    n = x.shape[0]
    w = np.full(n, 1.0 / n) if w is None else w / w.sum()
    xc = x - w @ x
    ac = a - w @ a
    H = (ac * w[:, None]).T @ xc
    U, S, Vt = np.linalg.svd(H)
    d = np.sign(np.linalg.det(Vt.T @ U.T))
    R = Vt.T @ np.diag([1.0, 1.0, d]) @ U.T
    D = float(np.sum(w * np.sum((xc - ac @ R.T) ** 2, axis=1)))
    return D, R


def rand_struct(rng, n, scale=1.0):
    return rng.normal(scale=scale, size=(n, 3))


# ------------------------------------------------------------------------------------
# superposition
@pytest.mark.parametrize("n", [3, 4, 7, 22, 300])
def test_align_matches_kabsch_svd(n):
    rng = np.random.default_rng(100 + n)
    for trial in range(5):
        a = rand_struct(rng, n)
        # x near a rotated copy of a (the interesting regime) or unrelated (trial 0)
        x = rand_struct(rng, n) if trial == 0 else (a @ synth.random_rotation(rng).T + 0.05 * rng.normal(size=(n, 3)) + 3.0)
        w = None if trial % 2 else rng.uniform(0.2, 2.0, size=n)
        r = oracle.align(x, a, w)
        Dk, Rk = kabsch(x, a, w)
        assert abs(r["D"] - Dk) <= 1e-12 * (r["Gx"] + r["Ga"])
        assert abs(r["D_formula"] - r["D"]) <= 1e-12 * (r["Gx"] + r["Ga"])
        gap = (r["evals"][0] - r["evals"][1]) / abs(r["evals"][0])
        if gap > 1e-6:
            assert np.max(np.abs(r["R"] - Rk)) < 1e-9
        assert abs(np.linalg.det(r["R"]) - 1.0) < 1e-12
        assert np.max(np.abs(r["R"] @ r["R"].T - np.eye(3))) < 1e-12


def test_mirror_images_are_not_superimposable():
    """A mirror image (det H < 0) cannot be superimposed by a rotation: the oracle's D is the
    SVD superposition's with the reflection fix, strictly positive for a chiral structure,
    reached by a proper rotation, and never below the (improper) orthogonal Procrustes
    minimum, which is zero."""
    rng = np.random.default_rng(91)
    for n in (4, 7, 30):
        a = rng.normal(size=(n, 3))
        M = np.diag([1.0, 1.0, -1.0])
        x = (a @ M) @ synth.random_rotation(rng).T + 2.0
        r = oracle.align(x, a)
        Dk, Rk = kabsch(x, a)
        scale = r["Gx"] + r["Ga"]
        assert abs(r["D"] - Dk) <= 1e-12 * scale
        assert abs(np.linalg.det(r["R"]) - 1.0) < 1e-12
        assert r["D"] > 1e-3 * scale  # chiral: no rotation maps it onto its mirror image
        # the improper orthogonal fit (reflections allowed) is exact
        w = np.full(n, 1.0 / n)
        xc, ac = x - w @ x, a - w @ a
        U, S, Vt = np.linalg.svd((ac * w[:, None]).T @ xc)
        Q = Vt.T @ U.T
        assert abs(np.linalg.det(Q) + 1.0) < 1e-9
        assert float(w @ np.sum((xc - ac @ Q.T) ** 2, axis=1)) < 1e-20 * scale + 1e-24
        # and the proper rotation's D is the paper's formula G_x + G_a - 2 lambda_max
        assert abs(r["D_formula"] - r["D"]) <= 1e-12 * scale


def collinear(rng, n, scale=1.0):
    """n atoms on a random line through a random point, unevenly spaced."""
    d = rng.normal(size=3)
    d /= np.linalg.norm(d)
    t = np.sort(rng.normal(size=n)) * scale
    return rng.normal(size=3) + t[:, None] * d[None, :]


def test_degenerate_top_eigenvalue_collinear():
    """Collinear structures: H has rank one, the top eigenvalue of K is double and the
    optimal rotation is not unique (any turn about the line).  D is unique: the oracle's
    equals the SVD superposition's and the one-dimensional closed form
    sum w s'^2 + sum w t'^2 - 2 |sum w s' t'| (s', t' the centred positions along each
    line), and the rotation the oracle returns attains it."""
    rng = np.random.default_rng(77)
    for trial in range(12):
        n = 3 + trial
        x, a = collinear(rng, n), collinear(rng, n, scale=1.3)
        w = None if trial % 2 else rng.uniform(0.3, 2.0, size=n)
        r = oracle.align(x, a, w)
        Dk, _ = kabsch(x, a, w)
        ww = np.full(n, 1.0 / n) if w is None else w / w.sum()
        xc, ac = x - ww @ x, a - ww @ a
        s1 = xc @ (xc[-1] - xc[0]) / np.linalg.norm(xc[-1] - xc[0])
        t1 = ac @ (ac[-1] - ac[0]) / np.linalg.norm(ac[-1] - ac[0])
        Dc = float(ww @ s1 ** 2 + ww @ t1 ** 2 - 2.0 * abs(ww @ (s1 * t1)))
        scale = r["Gx"] + r["Ga"]
        assert abs(r["D"] - Dk) <= 1e-12 * scale
        assert abs(r["D"] - Dc) <= 1e-12 * scale
        assert (r["evals"][0] - r["evals"][1]) <= 1e-9 * abs(r["evals"][0])  # degenerate
        Dr = float(ww @ np.sum((xc - ac @ r["R"].T) ** 2, axis=1))
        assert abs(Dr - r["D"]) <= 1e-12 * scale


@pytest.mark.parametrize("n", [3, 4, 5])
def test_align_brute_force_rotation_search(n):
    """The oracle's D is the minimum over SO(3): no rotation of a coarse grid plus local
    refinement does better, and refinement reaches it."""
    rng = np.random.default_rng(7 + n)
    x = rand_struct(rng, n)
    a = rand_struct(rng, n)
    xc = x - x.mean(0)
    ac = a - a.mean(0)

    def dist(rotvec):
        R = Rotation.from_rotvec(rotvec).as_matrix()
        return float(np.mean(np.sum((xc - ac @ R.T) ** 2, axis=1)))

    grid = Rotation.random(4000, random_state=1).as_rotvec()
    vals = np.array([dist(g) for g in grid])
    r = oracle.align(x, a)
    assert vals.min() >= r["D"] - 1e-12
    best = grid[np.argsort(vals)[:5]]
    refined = min(minimize(dist, g0, method="Nelder-Mead", options=dict(xatol=1e-10, fatol=1e-14, maxiter=4000)).fun for g0 in best)
    assert refined >= r["D"] - 1e-12
    assert refined - r["D"] < 1e-8


def test_two_atom_closed_form():
    """Uniform weights, 2 atoms: D = (|u| - |v|)^2 / 4 with u = x1 - x2, v = a1 - a2."""
    rng = np.random.default_rng(3)
    for _ in range(10):
        x = rand_struct(rng, 2)
        a = rand_struct(rng, 2)
        u = np.linalg.norm(x[0] - x[1])
        v = np.linalg.norm(a[0] - a[1])
        assert abs(oracle.align(x, a)["D"] - (u - v) ** 2 / 4) < 1e-13


def test_rigid_motion_symmetry_invariance():
    rng = np.random.default_rng(11)
    n = 40
    x = rand_struct(rng, n)
    a = rand_struct(rng, n)
    Q = synth.random_rotation(rng)
    t = rng.uniform(-5, 5, size=3)
    assert oracle.align(x @ Q.T + t, x)["D"] < 1e-13
    d_xa = oracle.align(x, a)["D"]
    assert abs(d_xa - oracle.align(a, x)["D"]) < 1e-12
    assert abs(d_xa - oracle.align(x @ Q.T + t, a)["D"]) < 1e-12
    assert abs(d_xa - oracle.align(x, a @ Q.T - t)["D"]) < 1e-12


def test_jacobi_matches_library_eigh():
    rng = np.random.default_rng(5)
    for _ in range(50):
        A = rng.normal(size=(4, 4))
        K = A + A.T
        ev, V, sweeps = oracle.jacobi4(K)
        ref = np.linalg.eigh(K)[0][::-1]
        assert sweeps > 0
        assert np.max(np.abs(ev - ref)) < 1e-12 * np.max(np.abs(ref))
        assert np.max(np.abs(K @ V - V * ev)) < 1e-11 * np.max(np.abs(ref))


def test_quaternion_matrix_and_rotation_agree_with_scipy():
    """R(q) is the rotation scipy builds from the same (scalar-first) quaternion, and
    q^T K(H) q = trace(R(q) H) for any H."""
    rng = np.random.default_rng(9)
    for _ in range(20):
        q = rng.normal(size=4)
        q /= np.linalg.norm(q)
        R = oracle.quat_to_rot(q)
        Rs = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
        assert np.max(np.abs(R - Rs)) < 1e-14
        H = rng.normal(size=(3, 3))
        K = oracle.quat_matrix(H)
        assert abs(q @ K @ q - np.trace(R @ H)) < 1e-13


# ------------------------------------------------------------------------------------
# path collective variables
def test_path_cv_logsumexp_and_two_landmark_logistic():
    rng = np.random.default_rng(2)
    for _ in range(20):
        m = int(rng.integers(1, 30))
        D = rng.uniform(0.0, 0.5, size=m)
        lam = float(rng.uniform(1.0, 2000.0))
        s, z, p = oracle.path_cv(D, lam)
        assert abs(z - (-logsumexp(-lam * D) / lam)) < 1e-12 * max(1.0, abs(z))
        qs = np.arange(1, m + 1)
        assert abs(s - np.exp(logsumexp(-lam * D, b=qs) - logsumexp(-lam * D))) < 1e-10 * m
        assert abs(p.sum() - 1.0) < 1e-12
    D = np.array([0.013, 0.021])
    lam = 300.0
    s, _, _ = oracle.path_cv(D, lam)
    assert abs(s - (1.0 + 1.0 / (1.0 + np.exp(lam * (D[1] - D[0]))))) < 1e-14


def test_path_cv_bounds_and_reversal():
    rng = np.random.default_rng(4)
    for _ in range(20):
        m = int(rng.integers(2, 50))
        D = rng.uniform(0.0, 0.2, size=m)
        lam = float(rng.uniform(1.0, 500.0))
        s, z, _ = oracle.path_cv(D, lam)
        assert 1.0 <= s <= m
        assert D.min() - np.log(m) / lam - 1e-15 <= z <= D.min() + 1e-15
        s_rev, z_rev, _ = oracle.path_cv(D[::-1], lam)
        assert abs(s_rev - (m + 1 - s)) < 1e-12 * m
        assert abs(z_rev - z) < 1e-15 + 1e-13 * abs(z)


def test_large_lambda_limit_picks_the_landmark():
    """x a rigid copy of landmark i: s -> i and z -> 0 as lambda -> infinity."""
    lm, _ = synth.make_problem(21, n_atoms=12, n_landmarks=9, n_frames=1, frame_dtype=np.float64,
                               landmark_dtype=np.float64)
    rng = np.random.default_rng(1)
    for i in range(9):
        x = lm[i] @ synth.random_rotation(rng).T + 1.5
        r = oracle.exact(x[None], lm, lam=1e9)
        assert abs(r["s"][0] - (i + 1)) < 1e-9
        assert abs(r["z"][0]) < 1e-12


# ------------------------------------------------------------------------------------
# gradients
def _fd(fun, x, h=1e-6):
    g = np.zeros_like(x)
    for idx in np.ndindex(x.shape):
        xp = x.copy()
        xm = x.copy()
        xp[idx] += h
        xm[idx] -= h
        g[idx] = (fun(xp) - fun(xm)) / (2 * h)
    return g


def test_exact_gradient_matches_central_differences():
    lm, fr = synth.make_problem(31, n_atoms=9, n_landmarks=6, n_frames=3, frame_noise=0.05,
                                frame_dtype=np.float64, landmark_dtype=np.float64)
    lam = 2.3 / oracle.mean_adjacent_msd(lm)
    w = np.random.default_rng(0).uniform(0.5, 1.5, size=9)
    r = oracle.exact(fr, lm, lam, w=w, want_grad=True)
    for t in range(3):
        for key in ("s", "z"):
            g = _fd(lambda x: oracle.exact(x[None], lm, lam, w=w)[key][0], fr[t])
            an = r["dsdx" if key == "s" else "dzdx"][t]
            scale = np.max(np.abs(g))
            assert np.max(np.abs(an - g)) < 1e-6 * scale + 1e-9, (key, t)


def test_exact_gradient_rigid_invariance():
    lm, fr = synth.make_problem(32, n_atoms=15, n_landmarks=8, n_frames=4, frame_dtype=np.float64,
                                landmark_dtype=np.float64)
    lam = 2.3 / oracle.mean_adjacent_msd(lm)
    r = oracle.exact(fr, lm, lam, want_grad=True)
    for key in ("dsdx", "dzdx"):
        for t in range(4):
            g = r[key][t]
            xc = fr[t] - fr[t].mean(0)
            scale = np.max(np.abs(g)) * np.max(np.abs(xc))
            assert np.max(np.abs(g.sum(0))) < 1e-12 * np.max(np.abs(g)) * 15
            assert np.max(np.abs(np.cross(xc, g).sum(0))) < 1e-11 * scale * 15


def test_close_gradient_matches_central_differences():
    """Approximate frames: derivative of D~ through R_xy(x) (Eq. close_der_dist), checked
    against central differences of the oracle's own D~(x) with y and R_{a_i y} fixed."""
    n, m = 8, 5
    lm, fr = synth.make_problem(33, n_atoms=n, n_landmarks=m, n_frames=3, frame_noise=0.01,
                                schedule="walk", frame_dtype=np.float64, landmark_dtype=np.float64)
    lam = 2.3 / oracle.mean_adjacent_msd(lm)
    w = np.random.default_rng(1).uniform(0.5, 1.5, size=n)
    st = oracle.CloseState(n, m)
    r0 = oracle.close(fr[:1], lm, lam, eps=10.0, state=st, w=w)  # initial assignment
    assert r0["refreshed"][0] == 2
    y, B = st.y.copy(), st.B.copy()
    # a frame near y but not a rigid copy of it
    x = fr[0] + 0.03 * np.random.default_rng(2).normal(size=(n, 3))
    r = oracle.close(x[None], lm, lam, eps=10.0, state=st.copy(), w=w, want_grad=True)
    assert r["refreshed"][0] == 0

    def cvs(xx):
        D = np.array([oracle.close_distance(xx, y, B[i], lm[i], w=w) for i in range(m)])
        s, z, _ = oracle.path_cv(D, lam)
        return s, z

    np.testing.assert_allclose([oracle.close_distance(x, y, B[i], lm[i], w=w) for i in range(m)], r["D"][0],
                               rtol=1e-12, atol=1e-15)
    for k, key in ((0, "dsdx"), (1, "dzdx")):
        g = _fd(lambda xx: cvs(xx)[k], x)
        an = r[key][0]
        assert np.max(np.abs(an - g)) < 1e-6 * np.max(np.abs(g)) + 1e-9, key
    # the rotation term matters here: the direct term alone misses the derivative
    g = _fd(lambda xx: cvs(xx)[1], x)
    wn = w / w.sum()
    xc = x - wn @ x
    Rxy = oracle.align(x, y, w)["R"]
    _, _, p = oracle.path_cv(r["D"][0], lam)
    direct = np.zeros_like(x)
    for i in range(m):
        ac = lm[i] - wn @ lm[i]
        dt = xc - ac @ (Rxy @ B[i]).T
        direct += p[i] * 2.0 * wn[:, None] * dt
    assert np.max(np.abs(direct - g)) > 1e-3 * np.max(np.abs(g))


# ------------------------------------------------------------------------------------
# close structure (Algorithm 2)
def _close_problem(seed=41, n=20, m=12, f=60, noise=0.02, schedule="walk"):
    lm, fr = synth.make_problem(seed, n_atoms=n, n_landmarks=m, n_frames=f, frame_noise=noise,
                                schedule=schedule, frame_dtype=np.float64, landmark_dtype=np.float64)
    lam = 2.3 / oracle.mean_adjacent_msd(lm)
    return lm, fr, lam


def test_close_refresh_flags_brute_force():
    """Replay the flags with an independent SVD superposition: frame t refreshes exactly
    when D(x_t, y) > eps for y the last refreshed frame (strict inequality)."""
    lm, fr, lam = _close_problem(noise=0.02)
    for eps in (0.002, 0.004, 0.01):
        r = oracle.close(fr, lm, lam, eps)
        flags = r["refreshed"]
        assert flags[0] == 2
        y = fr[0]
        for t in range(1, fr.shape[0]):
            d, _ = kabsch(fr[t], y)
            assert abs(d - r["dxy"][t]) < 1e-12
            assert bool(flags[t] == 1) == bool(d > eps), (eps, t)
            if flags[t]:
                y = fr[t]


def test_close_distance_matches_an_independent_superposition():
    """Eq. (close_dist) recomputed with SVD superpositions: for an approximate frame x with
    close structure y, D~(x, a_i) = sum_j w_j |R_xy^T (x_j - c_x) - R_{a_i y} (a_ij - c_a)|^2,
    R_xy fitting y onto x and R_{a_i y} fitting a_i onto y."""
    lm, fr, lam = _close_problem(noise=0.02, f=30)
    r = oracle.close(fr, lm, lam, 0.003)
    flags = r["refreshed"]
    assert 0 < int((flags == 0).sum())
    n = fr.shape[1]
    w = np.full(n, 1.0 / n)
    y = fr[0]
    checked = 0
    for t in range(fr.shape[0]):
        if flags[t] != 0:
            y = fr[t]
            continue
        _, Rxy = kabsch(fr[t], y)
        xp = (fr[t] - w @ fr[t]) @ Rxy  # R_xy^T (x - c_x), row-wise
        for i in range(lm.shape[0]):
            _, Ray = kabsch(y, lm[i])
            b = (lm[i] - w @ lm[i]) @ Ray.T
            Dt = float(w @ np.sum((xp - b) ** 2, axis=1))
            assert abs(Dt - r["D"][t, i]) <= 1e-11 * (1.0 + Dt), (t, i)
            checked += 1
    assert checked > 0


def test_close_equals_exact_at_refresh_and_dominates_elsewhere():
    lm, fr, lam = _close_problem(noise=0.02, f=40)
    ex = oracle.exact(fr, lm, lam)
    r = oracle.close(fr, lm, lam, 0.003)
    flags = r["refreshed"]
    assert 0 < int((flags == 1).sum()) < len(flags) - 1
    ref = flags > 0
    np.testing.assert_allclose(r["D"][ref], ex["D"][ref], rtol=0, atol=1e-14)
    np.testing.assert_allclose(r["s"][ref], ex["s"][ref], rtol=0, atol=1e-12)
    # D~ >= D: the approximate rotation is never better than the optimal one
    assert np.all(r["D"][~ref] >= ex["D"][~ref] - 1e-14)
    assert np.any(r["D"][~ref] > ex["D"][~ref] + 1e-8)


def test_close_is_exact_for_rigid_copies_of_y():
    lm, fr, lam = _close_problem(f=1)
    rng = np.random.default_rng(8)
    copies = np.stack([fr[0] @ synth.random_rotation(rng).T + rng.uniform(-3, 3, 3) for _ in range(4)])
    frames = np.concatenate([fr[:1], copies])
    r = oracle.close(frames, lm, lam, 0.01, want_grad=True)
    ex = oracle.exact(frames, lm, lam, want_grad=True)
    assert list(r["refreshed"]) == [2, 0, 0, 0, 0]
    np.testing.assert_allclose(r["D"], ex["D"], rtol=1e-10, atol=1e-14)
    for key in ("dsdx", "dzdx"):
        np.testing.assert_allclose(r[key], ex[key], rtol=0, atol=1e-9 * np.max(np.abs(ex[key])))


def test_close_counters_and_split_calls():
    lm, fr, lam = _close_problem(noise=0.02, f=50)
    m = lm.shape[0]
    r = oracle.close(fr, lm, lam, 0.003)
    c = r["state"].counters
    nref = int((r["refreshed"] == 1).sum())
    napprox = int((r["refreshed"] == 0).sum())
    assert c["refreshes_initial"] == 1 and c["refreshes_threshold"] == nref
    assert c["xy_alignments"] == fr.shape[0] - 1
    assert c["landmark_alignments"] == m * (nref + 1)
    assert c["approx_msds"] == m * napprox
    # expensive distance computations per step match the close-structure cost model
    per_step = (c["xy_alignments"] + c["landmark_alignments"]) / fr.shape[0]
    k = fr.shape[0] / (nref + 1)
    assert abs(per_step - oracle.cost_close(m, k) + 1.0 / fr.shape[0]) < 1e-12
    # a run split in two calls with the state carried over is identical
    st = oracle.CloseState(fr.shape[1], m)
    a = oracle.close(fr[:23], lm, lam, 0.003, state=st)
    b = oracle.close(fr[23:], lm, lam, 0.003, state=st)
    for key in ("s", "z", "D", "refreshed", "dxy"):
        np.testing.assert_array_equal(np.concatenate([a[key], b[key]]), r[key])
    assert st.counters == c


def test_cost_model_matches_paper_worked_numbers():
    g = json.loads((GOLDEN / "cost_model.json").read_text())
    cy, tc = g["cyclooctane"], g["trpcage"]
    assert oracle.cost_original(cy["m_nl"], cy["n_ref"], cy["l_stride"]) == cy["original_per_step"]
    c_close = oracle.cost_close(cy["n_ref"], cy["k_interval"])
    assert round(c_close, cy["close_digits"]) == cy["close_per_step"]
    assert round(cy["original_per_step"] / cy["close_per_step"]) == cy["msd_speedup"]
    assert abs(oracle.cost_original(tc["m_nl"], tc["n_ref"], tc["l_stride"]) - tc["original_per_step"]) < 1e-12
    assert round(oracle.cost_close(tc["n_ref"], tc["k_interval"]), tc["close_digits"]) == tc["close_per_step"]
    assert round(tc["original_per_step"] / tc["close_per_step"]) == tc["msd_speedup"]
    for ds in (cy, tc):
        S = oracle.amdahl(ds["portions"]["MSD"], ds["msd_speedup"])
        assert round(S, ds["S_digits"]) == ds["S_MSD"]
    # Amdahl's law limits: s -> infinity gives 1/(1-p); p = 0.9 caps at 10 (Section 6.2)
    assert abs(oracle.amdahl(0.9, 1e300) - 10.0) < 1e-9


def test_results_do_not_depend_on_the_thread_count():
    """The OpenMP loops share out independent landmarks and atoms only, each output summed in
    the single-thread order: one thread and several give bit-identical results (exact and
    close-structure mode, both weight sets, gradients)."""
    lm, fr, lam = problem(17, 33, 21, 40, noise=0.02, schedule="walk", ou_rho=0.9)
    rng = np.random.default_rng(3)
    w, wa = rng.uniform(0.5, 1.5, 33), rng.uniform(0.5, 1.5, 33)
    n0 = oracle.threads()
    runs = []
    try:
        for t in (1, 4):
            oracle.set_threads(t)
            assert oracle.threads() == t
            runs.append((oracle.exact(fr, lm, lam, w=w, wa=wa, want_grad=True),
                         oracle.close(fr, lm, lam, 0.002, w=w, wa=wa, want_grad=True)))
    finally:
        oracle.set_threads(n0)
    assert int((runs[0][1]["refreshed"] == 1).sum()) >= 2
    for a, b in zip(*runs):
        for k in ("s", "z", "D", "dsdx", "dzdx"):
            np.testing.assert_array_equal(a[k], b[k])


def test_given_distances_enter_the_derivatives_only_through_the_weights():
    """With fixed geometry the derivatives of Eqs. 5-6 are linear in the weights:
    dz/dx = sum_i p_i dD_i/dx and ds/dx = -lambda sum_i p_i (q_i - s) dD_i/dx (softmax
    derivative), with dD_i/dx set by the structures alone.  With two landmarks one set of
    given distances fixes dD_1/dx and dD_2/dx (a 2 x 2 system per coordinate, determinant
    -lambda p_1 p_2 (q_2 - q_1)); a second set must then give exactly the predicted
    gradients, and so must the oracle's own distances.  A derivative that used the computed
    instead of the given distances, or dropped the softmax's mean term, fails this."""
    lm, fr, lam = problem(29, 13, 2, 8, noise=0.02, schedule="walk", ou_rho=0.9)
    eps = 0.002
    q = np.array([1.0, 2.0])
    rng = np.random.default_rng(5)

    def run(D_in):
        r = oracle.close(fr, lm, lam, eps, want_grad=True, D_in=D_in)
        e = np.exp(-lam * (r["D"] - r["D"].min(axis=1, keepdims=True)))
        pw = e / e.sum(axis=1, keepdims=True)
        sv = pw @ q
        return r, pw, -lam * pw * (q[None, :] - sv[:, None])

    def given():
        base = rng.uniform(0.01, 0.02, (fr.shape[0], 1))
        return base + np.concatenate([np.zeros_like(base), rng.uniform(-1.5, 1.5, base.shape) / lam], axis=1)

    rA, pA, gA = run(given())
    assert np.all(rA["refreshed"] == oracle.close(fr, lm, lam, eps)["refreshed"])
    G = np.empty((fr.shape[0], 2, fr.shape[1] * 3))
    for t in range(fr.shape[0]):
        A = np.array([pA[t], gA[t]])
        rhs = np.stack([rA["dzdx"][t].ravel(), rA["dsdx"][t].ravel()])
        G[t] = np.linalg.solve(A, rhs)
    for D_in in (given(), None):
        r, pw, gs = run(D_in)
        np.testing.assert_allclose(r["s"], pw @ q, rtol=1e-13, atol=0)
        for t in range(fr.shape[0]):
            scale = np.abs(G[t]).max()
            np.testing.assert_allclose(r["dzdx"][t].ravel(), pw[t] @ G[t], rtol=0, atol=1e-10 * scale)
            np.testing.assert_allclose(r["dsdx"][t].ravel(), gs[t] @ G[t], rtol=0, atol=1e-10 * lam * scale)


def test_given_distances_enter_only_through_the_weights():
    """The oracle's distance injection (used to separate a derivative's error from that of
    the distances it was evaluated at): the path CVs of Eq. (property_map_cv) are invariant
    to a uniform shift of every distance except z, which moves by the shift; so injecting
    D + c must give the same s and derivatives and z + c, and injecting the oracle's own D
    must change nothing."""
    lm, fr, lam = problem(23, 29, 17, 30, noise=0.02, schedule="walk", ou_rho=0.9)
    eps = 0.002
    r = oracle.close(fr, lm, lam, eps, want_grad=True)
    assert int((r["refreshed"] == 1).sum()) >= 2
    same = oracle.close(fr, lm, lam, eps, want_grad=True, D_in=r["D"])
    for k in ("s", "z", "D", "dsdx", "dzdx"):
        np.testing.assert_array_equal(same[k], r[k])
    c = 0.0123
    shifted = oracle.close(fr, lm, lam, eps, want_grad=True, D_in=r["D"] + c)
    np.testing.assert_allclose(shifted["s"], r["s"], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(shifted["z"], r["z"] + c, rtol=1e-12, atol=1e-12)
    for k in ("dsdx", "dzdx"):
        np.testing.assert_allclose(shifted[k], r[k], rtol=1e-9, atol=1e-12 * np.abs(r[k]).max())
    np.testing.assert_array_equal(shifted["refreshed"], r["refreshed"])  # decisions are not distances
    # NaN entries keep the oracle's own values
    part = r["D"] + c
    part[:, ::2] = np.nan
    mixed = oracle.close(fr, lm, lam, eps, want_grad=True, D_in=part)
    Dm = r["D"].copy()
    Dm[:, 1::2] += c
    np.testing.assert_array_equal(mixed["D"], Dm)

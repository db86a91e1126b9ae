"""The synthetic inputs follow their stated recipe: self-avoiding chains with 0.15 nm bonds and
no non-bonded pair closer than 0.12 nm, uniform proper rotations, the drift and reflecting-walk
schedules on [1, M], landmarks interpolated between two chains, storage rounding, and seeded
determinism.  (Host only; the generators hold none of the method's arithmetic.)"""
import numpy as np

from paper_1801_02362_gb300 import synth


def _dist(a):
    d = a[:, None, :] - a[None, :, :]
    return np.sqrt(np.einsum("ijk,ijk->ij", d, d))


def test_chains_have_fixed_bonds_and_avoid_themselves():
    rng = np.random.default_rng(1)
    for n in (3, 24, 120):
        c = synth.saw_chain(rng, n)
        d = _dist(c)
        assert np.allclose(np.diag(d, 1), synth.BOND_NM, atol=1e-12)
        far = np.abs(np.subtract.outer(np.arange(n), np.arange(n))) >= 2
        assert np.all(d[far] >= synth.MIN_NONBONDED_NM - 1e-12)


def test_rotations_are_proper_and_uniform_in_mean():
    rng = np.random.default_rng(2)
    R = synth.random_rotation(rng, 4000)
    assert np.allclose(np.einsum("nij,nkj->nik", R, R), np.eye(3)[None], atol=1e-12)
    assert np.allclose(np.linalg.det(R), 1.0, atol=1e-12)
    assert np.max(np.abs(R.mean(axis=0))) < 0.05  # E[R] = 0 for the Haar measure


def test_schedules():
    p = synth.positions_drift(11, 6)
    assert p[0] == 1.0 and p[-1] == 6.0 and np.all(np.diff(p) > 0)
    w = synth.positions_reflecting_walk(np.random.default_rng(3), 5000, 9)
    assert np.all((w >= 1.0) & (w <= 9.0))
    steps = np.diff(w)
    assert abs(np.std(steps[np.abs(steps) < 0.5]) - 0.1) < 0.01  # N(0, 0.1) away from the walls


def test_landmarks_interpolate_between_two_chains():
    """Landmark k keeps the geometry of (1 - t_k) A + t_k B up to the N(0, 0.02) noise: its
    internal distances match the interpolation's (rigid motions preserve them)."""
    rng = np.random.default_rng(4)
    n, m = 30, 7
    path = synth.PathModel(rng, n)
    d = _dist(path.A)
    assert np.allclose(np.diag(d, 1), synth.BOND_NM, atol=1e-12)  # the ends are the chains above
    lm = synth.make_landmarks(rng, path, m, noise=0.0)
    t = np.arange(m) / (m - 1)
    ref = path.at(t)
    for k in range(m):
        assert np.allclose(_dist(lm[k]), _dist(ref[k]), atol=1e-10)
    noisy = synth.make_landmarks(np.random.default_rng(5), path, m, noise=0.02)
    dev = np.abs(_dist(noisy[3]) - _dist(ref[3]))
    assert 0.005 < np.mean(dev) < 0.06


def test_rounding_and_seeded_determinism():
    x = np.array([1.0 + 2.0 ** -30, 0.1])
    assert np.array_equal(synth.round_to(x, np.float32), x.astype(np.float32).astype(np.float64))
    a = synth.make_problem(11, n_atoms=20, n_landmarks=5, n_frames=8, frame_noise=0.05)
    b = synth.make_problem(11, n_atoms=20, n_landmarks=5, n_frames=8, frame_noise=0.05)
    c = synth.make_problem(12, n_atoms=20, n_landmarks=5, n_frames=8, frame_noise=0.05)
    assert all(np.array_equal(u, v) for u, v in zip(a, b))
    assert not np.array_equal(a[0], c[0])

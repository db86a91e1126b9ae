"""Pins of the oracle's Gaussian-hill metadynamics bias on the path CVs (Eq. vbias) against
facts that do not come from its code: the Gaussian written out with numpy, central
differences in (s, z) and in the coordinates (through the already-pinned path CVs), the
deposition schedule counted by hand, and split-call invariance."""
import numpy as np
import pytest

import oracle
from paper_1801_02362_gb300 import synth


def _gauss_sum(hills, w, ss, sz, s, z):
    h = np.asarray(hills, dtype=np.float64).reshape(-1, 2)
    return float(np.sum(w * np.exp(-(s - h[:, 0]) ** 2 / (2 * ss ** 2) - (z - h[:, 1]) ** 2 / (2 * sz ** 2))))


def test_hills_value_and_derivatives():
    rng = np.random.default_rng(1)
    hills = rng.normal(size=(17, 2)) * [3.0, 0.02] + [10.0, 0.01]
    w, ss, sz = 1.2, 0.4, 0.005
    for _ in range(20):
        s, z = 10.0 + 3.0 * rng.normal(), 0.01 + 0.02 * rng.normal()
        V, gs, gz = oracle.hills_value(hills, w, ss, sz, s, z)
        assert abs(V - _gauss_sum(hills, w, ss, sz, s, z)) < 1e-13 * max(1.0, V)
        hs, hz = 1e-6 * ss, 1e-6 * sz
        fs = (_gauss_sum(hills, w, ss, sz, s + hs, z) - _gauss_sum(hills, w, ss, sz, s - hs, z)) / (2 * hs)
        fz = (_gauss_sum(hills, w, ss, sz, s, z + hz) - _gauss_sum(hills, w, ss, sz, s, z - hz)) / (2 * hz)
        assert abs(gs - fs) < 1e-6 * (abs(fs) + w / ss)
        assert abs(gz - fz) < 1e-6 * (abs(fz) + w / sz)
    # one hill at the point itself: V = w, zero slope
    V, gs, gz = oracle.hills_value([[2.0, 0.3]], 0.7, 0.1, 0.1, 2.0, 0.3)
    assert V == 0.7 and gs == 0.0 and gz == 0.0


def test_deposition_schedule_and_split_calls():
    """Eq. (vbias) sums over the deposition times t' = tau_G, 2 tau_G, ... with t' < t, the
    hill of time t' sitting at (s(t'), z(t')).  The expected bias below enumerates exactly
    those times, k * tau_G for k = 1, 2, ..., and stops below t; steps are numbered from 0."""
    rng = np.random.default_rng(2)
    f, stride = 50, 7
    s = np.cumsum(rng.normal(size=f)) * 0.3 + 5.0
    z = rng.uniform(0.0, 0.02, size=f)
    w, ss, sz = 0.9, 0.5, 0.004
    r = oracle.metad(s, z, w, ss, sz, stride)
    for t in range(f):
        times = []
        k = 1
        while k * stride < t:
            times.append(k * stride)
            k += 1
        expect = _gauss_sum([[s[u], z[u]] for u in times], w, ss, sz, s[t], z[t]) if times else 0.0
        assert abs(r["V"][t] - expect) < 1e-13 * max(1.0, expect)
    # no hill acts before the first deposition time has passed: V = 0 for t <= tau_G
    assert np.all(r["V"][:stride + 1] == 0.0) and r["V"][stride + 1] > 0.0
    # the run deposits at tau_G, 2 tau_G, ... up to its last step f - 1
    assert r["state"].n_hills == (f - 1) // stride
    np.testing.assert_array_equal(r["state"].hills[:r["state"].n_hills],
                                  np.stack([s[stride::stride], z[stride::stride]], axis=1))
    st = oracle.MetadState()
    a = oracle.metad(s[:23], z[:23], w, ss, sz, stride, state=st)
    b = oracle.metad(s[23:], z[23:], w, ss, sz, stride, state=st)
    np.testing.assert_array_equal(np.concatenate([a["V"], b["V"]]), r["V"])
    np.testing.assert_array_equal(st.hills[:st.n_hills], r["state"].hills[:r["state"].n_hills])


def test_capacity_is_enforced():
    with pytest.raises(RuntimeError):
        oracle.metad(np.zeros(10), np.zeros(10), 1.0, 1.0, 1.0, 1, state=oracle.MetadState(cap=5))


def test_bias_force_is_minus_the_coordinate_gradient():
    """force = -dV(s(x), z(x))/dx: central differences through the path CVs of Eq.
    (property_map_cv) (the oracle's exact evaluation) and the hill sum written out."""
    lm, fr = synth.make_problem(21, n_atoms=7, n_landmarks=6, n_frames=3, frame_noise=0.03,
                                frame_dtype=np.float64, landmark_dtype=np.float64)
    lam = 2.3 / oracle.mean_adjacent_msd(lm)
    ex = oracle.exact(fr, lm, lam, want_grad=True)
    hills = np.stack([ex["s"] + [0.3, -0.2, 0.1], ex["z"] + [0.001, -0.002, 0.0005]], axis=1)
    st = oracle.MetadState()
    st.hills[:3] = hills
    st.state[:] = [3, 1]  # three hills held; the next step (1) deposits nothing with stride 2
    w, ss, sz = 1.5, 0.35, 0.003
    r = oracle.metad(ex["s"], ex["z"], w, ss, sz, 2, state=st, dsdx=ex["dsdx"], dzdx=ex["dzdx"])
    t = 0  # the first frame sees all three hills
    x = fr[t]

    def V_of(xx):
        e = oracle.exact(xx[None], lm, lam)
        return _gauss_sum(hills, w, ss, sz, e["s"][0], e["z"][0])

    g = np.zeros_like(x)
    h = 1e-6
    for idx in np.ndindex(x.shape):
        xp, xm = x.copy(), x.copy()
        xp[idx] += h
        xm[idx] -= h
        g[idx] = (V_of(xp) - V_of(xm)) / (2 * h)
    assert np.max(np.abs(r["force"][t] + g)) < 1e-6 * np.max(np.abs(g)) + 1e-12

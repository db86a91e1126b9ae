"""GPU parity of the metadynamics bias (pcv_metad_*, Eq. vbias) against the oracle's, on the
same seeded inputs (CV values, their derivatives and the hills held before the call), and
the whole chain frames -> path CVs -> bias and force against the oracle's chain.

Tolerance: the Gaussians are evaluated in FP32 from FP64 differences, so every term carries
~1e-6 relative error (argument rounding u |arg| with |arg| < ~20 where a term matters, plus
FP32 lane sums).  V sums positive terms: 5e-6 of max(V, height 1e-3).  dV/ds and dV/dz sum
terms of both signs, so their error is bounded by the sum of the terms' magnitudes,
A_s = sum_k e_k |s - s_k| / sigma_s^2 (A_z likewise), not by |dV/ds|: each force element is
held to 5e-6 (A_s |ds/dx| + A_z |dz/dx|).  Hill positions are copies of s and z:
bit-exact."""
import numpy as np
import pytest

import oracle
from _util import problem

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


def cv_inputs(seed, f, n, m=60):
    rng = np.random.default_rng(seed)
    s = np.clip(1.0 + np.cumsum(rng.normal(scale=0.4, size=f)) % m, 1.0, m)
    z = rng.uniform(-0.002, 0.02, size=f)
    dsdx = rng.normal(size=(f, n, 3))
    dzdx = rng.normal(size=(f, n, 3)) * 0.01
    hills0 = np.stack([rng.uniform(1.0, m, 300), rng.uniform(0.0, 0.02, 300)], axis=1)
    return s, z, dsdx, dzdx, hills0


def term_scales(s, z, hills_all, n_before, height, ss, sz):
    """A_s, A_z of every frame: the magnitudes of the derivative terms summed over the hills
    the frame sees (the first n_before[t] of hills_all)."""
    A_s, A_z = np.zeros(len(s)), np.zeros(len(s))
    for t in range(len(s)):
        h = hills_all[:n_before[t]]
        ds, dz = s[t] - h[:, 0], z[t] - h[:, 1]
        e = abs(height) * np.exp(-ds ** 2 / (2 * ss ** 2) - dz ** 2 / (2 * sz ** 2))
        A_s[t] = np.sum(e * np.abs(ds)) / ss ** 2
        A_z[t] = np.sum(e * np.abs(dz)) / sz ** 2
    return A_s, A_z


def check(gv, gf, rv, rf, height, A=None, dsdx=None, dzdx=None):
    vs = np.maximum(np.abs(rv), 1e-3 * abs(height))
    assert np.max(np.abs(gv - rv) / vs) < 5e-6
    if rf is not None:
        bound = 5e-6 * (A[0][:, None, None] * np.abs(dsdx) + A[1][:, None, None] * np.abs(dzdx)) + 1e-12
        assert np.all(np.abs(gf - rf) <= bound)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_metad_matches_oracle_across_calls(pcv, precision):
    """F=5000 steps in three calls (ragged), 300 hills held before, a hill every 7 steps from
    step 13 on: bias, force and the deposited hills."""
    f, n, height, ss, sz, stride = 5000, 50, 1.2, 0.3, 0.004, 7
    s, z, dsdx, dzdx, hills0 = cv_inputs(1, f, n)
    st = oracle.MetadState(cap=2000)
    st.hills[:300] = hills0
    st.state[:] = [300, 13]
    r = oracle.metad(s, z, height, ss, sz, stride, state=st, dsdx=dsdx, dzdx=dzdx)
    gdt = torch.float64 if precision == "fp64" else torch.float32
    mt = pcv.Metad(height, ss, sz, stride, max_hills=2000)
    mt.set_hills(hills0, 13)
    V, Fo = [], []
    for a, b in ((0, 1234), (1234, 1235), (1235, f)):
        T = lambda x: torch.tensor(x[a:b], dtype=torch.float64, device="cuda")
        out = mt.apply(T(s), T(z), T(dsdx).to(gdt), T(dzdx).to(gdt), precision=precision)
        V.append(out["bias"].cpu().numpy())
        Fo.append(out["force"].double().cpu().numpy())
    torch.cuda.synchronize()
    rf = r["force"]
    if precision == "fp32":  # the GPU combines the FP32-rounded derivatives: the oracle takes the same inputs
        rf = oracle.metad(s, z, height, ss, sz, stride, state=_state(hills0, 13), dsdx=dsdx.astype(np.float32),
                          dzdx=dzdx.astype(np.float32))["force"]
    n_before = 300 + np.array([len([u for u in range(t) if (13 + u) % stride == 0]) for t in range(f)])
    A = term_scales(s, z, st.hills, n_before, height, ss, sz)
    check(np.concatenate(V), np.concatenate(Fo), r["V"], rf, height, A, dsdx, dzdx)
    hills, steps = mt.hills()
    assert steps == 13 + f
    np.testing.assert_array_equal(hills, st.hills[:st.n_hills])
    mt.close()


def _state(hills0, steps):
    st = oracle.MetadState(cap=2000)
    st.hills[:hills0.shape[0]] = hills0
    st.state[:] = [hills0.shape[0], steps]
    return st


def test_metad_capacity_and_arguments(pcv):
    mt = pcv.Metad(1.0, 0.1, 0.1, 1, max_hills=10)
    s = torch.zeros(12, dtype=torch.float64, device="cuda")
    with pytest.raises(pcv.PcvError) as e:
        mt.apply(s, s)  # steps 1..11 would deposit 11 hills
    assert e.value.status == pcv.PCV_EINVAL
    out = mt.apply(s[:11], s[:11])  # steps 1..10 deposit: exactly fills the capacity
    assert mt.hills()[0].shape == (10, 2)
    # no hill before step 1 is evaluated; step t >= 1 sees the hills of steps 1..t-1
    assert float(out["bias"][0]) == 0.0 and float(out["bias"][1]) == 0.0
    assert abs(float(out["bias"][10]) - 9.0) < 1e-6
    mt.close()
    with pytest.raises(pcv.PcvError):
        pcv.Metad(1.0, 0.0, 0.1, 1)


def test_path_cv_to_bias_chain(pcv):
    """Frames -> exact path CVs with derivatives -> bias and force, on the GPU through the C
    ABI, against the oracle's chain.  The GPU's s and z differ from the oracle's within the
    FP32 tolerance; the bias may differ by the first-order effect of that difference."""
    lm, fr, lam = problem(71, 40, 30, 400, noise=0.03, schedule="walk")
    r = oracle.exact(fr, lm, lam, want_grad=True)
    height, ss, sz, stride = 0.8, 0.5, 0.003, 5
    rb = oracle.metad(r["s"], r["z"], height, ss, sz, stride, dsdx=r["dsdx"], dzdx=r["dzdx"])
    ctx = pcv.PathCV(lm, lam, eps=-1.0, precision="fp32")
    out = ctx.evaluate(torch.tensor(fr, dtype=torch.float32, device="cuda"), grad=True)
    mt = pcv.Metad(height, ss, sz, stride, max_hills=1000)
    b = mt.apply(out["s"], out["z"], out["dsdx"], out["dzdx"], precision="fp32")
    torch.cuda.synchronize()
    gs, gz = out["s"].cpu().numpy(), out["z"].cpu().numpy()
    V = b["bias"].cpu().numpy()
    # first-order bound: |dV/ds| |ds| + |dV/dz| |dz| summed over the hills (each moved too)
    bound = np.zeros(len(V))
    hs = gs[stride::stride]
    for t in range(len(V)):
        k = np.arange(stride, t, stride)  # deposition steps t' = tau_G, 2 tau_G, ... below t
        if len(k) == 0:
            continue
        d_s = gs[t] - r["s"][t] - (gs[k] - r["s"][k])
        d_z = gz[t] - r["z"][t] - (gz[k] - r["z"][k])
        e = height * np.exp(-(r["s"][t] - r["s"][k]) ** 2 / (2 * ss ** 2) - (r["z"][t] - r["z"][k]) ** 2 / (2 * sz ** 2))
        bound[t] = np.sum(e * (np.abs(r["s"][t] - r["s"][k]) / ss ** 2 * np.abs(d_s) +
                               np.abs(r["z"][t] - r["z"][k]) / sz ** 2 * np.abs(d_z)))
    assert len(hs) > 10
    assert np.all(np.abs(V - rb["V"]) <= 2 * bound + 5e-6 * np.maximum(np.abs(rb["V"]), 1e-3 * height))
    # the force through the FP32 derivatives: within the gradient tolerance of its scale
    fo = b["force"].double().cpu().numpy()
    scale = np.max(np.abs(rb["force"]).reshape(len(V), -1), axis=1) + 1e-30
    active = scale > 1e-3 * np.max(scale)
    err = np.max(np.abs(fo - rb["force"]).reshape(len(V), -1), axis=1) / scale
    assert np.max(err[active]) < 1e-3
    mt.close()
    ctx.close()

"""Full-size GPU parity in the launch configuration the benchmark times.

The oracle cannot replay 100k frames of Algorithm 2 with gradients in seconds, so the
full-size runs are checked through properties and samples it can compute one by one:
  * every refresh decision: D(x_t, y) > eps with the exact alignment of each frame onto the
    close structure y in force (y tracked through the GPU's own flags, so one wrong flag
    makes the check fail at that frame);
  * sampled frames in full (MSD row, s, z, both gradients): an approximate frame t with close
    structure y is exactly the second frame of the two-frame sequence [y, x_t], a refreshed
    frame is Algorithm 1 on x_t.
"""
import numpy as np
import pytest

import oracle
from _util import GRAD_TOL, TOL, check_grads_at_given_distances, d_err, grad_err, s_err, z_err

S_AT_D = {"fp64": 1e-9, "fp32": 2e-5, "fp16": 2e-5}  # absolute

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


def _sample_refs(res, fr, lm, lam, eps, t):
    """The oracle's evaluation of frame t as the GPU took it (a reassignment: Algorithm 1
    on x_t; else the second frame of [y, x_t]), on its own distances and on the GPU's."""
    flags = res["refreshed"]
    if flags[t]:
        seq, row = fr[t:t + 1], 0
    else:
        y_idx = int(np.nonzero(flags[:t + 1])[0][-1])
        seq, row = np.stack([fr[y_idx], fr[t]]), 1
    r = oracle.close(seq, lm, lam, eps, want_grad=True)
    assert r["refreshed"][row] == (2 if row == 0 else 0)
    D_in = np.full((seq.shape[0], lm.shape[0]), np.nan)
    D_in[row] = res["msd"][t]
    r_at = oracle.close(seq, lm, lam, eps, want_grad=True, D_in=D_in)
    sl = slice(row, row + 1)
    return {k: r[k][sl] for k in ("D", "s", "z", "dsdx", "dzdx")}, {k: r_at[k][sl] for k in ("s", "dsdx", "dzdx")}


def _check_frame_samples(res, fr, lm, lam, eps, ts, precision="fp32"):
    for t in ts:
        r, r_at = _sample_refs(res, fr, lm, lam, eps, t)
        sl = slice(t, t + 1)
        assert d_err(res["msd"][sl], r["D"], fr[sl], lm) < TOL[precision]
        assert s_err(res["s"][sl], r["s"], lm.shape[0]) < TOL[precision]
        assert z_err(res["z"][sl], r["z"], lam) < TOL[precision]
        # at its own distances s is off by the FP32 rounding of the weights times their spread
        # (a few landmarks), not by the rounding of s itself (1e-4 at s ~ 2000)
        assert abs(res["s"][t] - r_at["s"][0]) < S_AT_D[precision], (t, res["s"][t] - r_at["s"][0])
        check_grads_at_given_distances(res["dsdx"][sl], res["dzdx"][sl], r, r_at, precision)


def _check_refresh_sequence(flags, fr, eps):
    """Each frame refreshes iff its exact MSD to the close structure in force exceeds eps."""
    assert flags[0] == 2  # the initial assignment
    y = fr[0]
    for t in range(1, fr.shape[0]):
        d = oracle.align(fr[t], y)["D"]
        if bool(flags[t]) != (d > eps):
            raise AssertionError(f"frame {t}: flag {flags[t]}, exact D(x_t, y) = {d!r} vs eps {eps}")
        if flags[t]:
            y = fr[t]


@pytest.mark.parametrize("eps", [0.01, 0.05, 0.1])
def test_c2_full_size_close_with_gradients(pcv, eps):
    """N=300, M=200, F=100000 FP32, s/z with gradients, at each threshold of the sweep
    (eps = 0.05 nm^2 is the benchmark's step; at 0.01 nearly every frame reassigns, at 0.05
    and 0.1 the segments are long enough for the materialised tensor-core path): every
    refresh decision, the refresh counters, and sampled frames in full."""
    from paper_1801_02362_gb300 import synth

    lm, fr = synth.make_problem(1, n_atoms=300, n_landmarks=200, n_frames=100_000, frame_noise=0.05)
    fr = np.ascontiguousarray(fr, dtype=np.float32)
    lam = 2.3 / oracle.mean_adjacent_msd(lm)
    ctx = pcv.PathCV(lm, lam, eps=eps, precision="fp32")
    out = ctx.evaluate(torch.from_numpy(fr).cuda(), grad=True, msd=True, refreshed=True)
    ctx.sync()
    res = {k: v.cpu().numpy() for k, v in out.items()}
    st = ctx.stats()
    ctx.close()
    flags = res["refreshed"]
    n_ref = int((flags == 1).sum())
    if eps >= 0.05:
        assert 2 <= n_ref < 1000  # long segments: the materialised tensor-core path
    else:
        assert n_ref > 0.9 * fr.shape[0]  # the noise alone exceeds the threshold
    _check_refresh_sequence(flags, fr.astype(np.float64), eps)
    # counters of the cost model (Sec. 6.2): one x-y alignment per frame after the first,
    # M landmark alignments per reassignment and for the initial assignment
    m = lm.shape[0]
    assert st["refreshes_threshold"] == n_ref and st["refreshes_initial"] == 1
    assert st["xy_alignments"] == fr.shape[0] - 1
    assert st["landmark_alignments"] == m * (n_ref + 1)
    assert st["approx_msds"] == m * (fr.shape[0] - 1 - n_ref)
    rng = np.random.default_rng(5)
    refreshed = np.nonzero(flags)[0]
    approx = np.nonzero(flags == 0)[0]
    ts = set(rng.integers(1, fr.shape[0], 10).tolist()) | {int(refreshed[-1]), fr.shape[0] - 1}
    if len(approx):
        ts |= set(rng.choice(approx, min(4, len(approx)), replace=False).tolist())
    _check_frame_samples(res, fr, lm, lam, eps, sorted(ts))


def test_c4_full_size_exact_gradients_sampled(pcv):
    """N=1000, M=500, F=4096 FP32 exact mode with gradients; 6 frames checked in full."""
    from paper_1801_02362_gb300 import synth

    lm, fr = synth.make_problem(4, n_atoms=1000, n_landmarks=500, n_frames=4096, frame_noise=0.05)
    fr = np.ascontiguousarray(fr, dtype=np.float32)
    lam = 2.3 / oracle.mean_adjacent_msd(lm)
    ctx = pcv.PathCV(lm, lam, eps=-1.0, precision="fp32")
    out = ctx.evaluate(torch.from_numpy(fr).cuda(), grad=True, msd=True, refreshed=True)
    ctx.sync()
    res = {k: v.cpu().numpy() for k, v in out.items()}
    ctx.close()
    assert np.all(res["refreshed"] == 1)
    ts = [0, 1, 1777, 2048, 3000, 4095]
    for t in ts:
        r = oracle.exact(fr[t:t + 1], lm, lam, want_grad=True)
        sl = slice(t, t + 1)
        assert d_err(res["msd"][sl], r["D"], fr[sl], lm) < TOL["fp32"]
        assert s_err(res["s"][sl], r["s"], 500) < TOL["fp32"]
        assert z_err(res["z"][sl], r["z"], lam) < TOL["fp32"]
        assert grad_err(res["dsdx"][sl], r["dsdx"]) < GRAD_TOL["fp32"]
        assert grad_err(res["dzdx"][sl], r["dzdx"]) < GRAD_TOL["fp32"]


@pytest.mark.parametrize("precision", ["fp32", "fp16"])
def test_c5_full_size_close_batched_sampled(pcv, precision):
    """N=5000, M=2000 (120 MB FP32 / 64 MB FP16 storage), F=10000 drifting frames, eps=0.05,
    s, z and both gradients (the benchmark's step, FP32 storage): the batched close-structure
    step on materialised deviations (4.2 GB of rotated landmarks for ~35 close structures)
    and the tensor-core segment adjoint; every refresh decision and 6 frames in full."""
    from paper_1801_02362_gb300 import synth

    lm, fr = synth.make_problem(5, n_atoms=5000, n_landmarks=2000, n_frames=10_000, frame_noise=0.05)
    fr = np.ascontiguousarray(fr, dtype=np.float32)
    lm = lm.astype(np.float32).astype(np.float64)
    lam = 2.3 / oracle.mean_adjacent_msd(lm[:50])
    eps = 0.05
    ctx = pcv.PathCV(lm, lam, eps=eps, precision=precision)
    ctx.set_profiling(True)
    out = ctx.evaluate(torch.from_numpy(fr).cuda(), grad=True, msd=True, refreshed=True)
    ctx.sync()
    prof = ctx.profile()
    res = {k: v.cpu().numpy() for k, v in out.items()}
    ctx.close()
    assert "materialize" in prof  # the tiled path on materialised deviations ran
    assert "adjoint_beta_mma" in prof  # and the segment adjoint on the tensor cores
    flags = res["refreshed"]
    assert 10 <= int((flags > 0).sum()) < 200
    _check_refresh_sequence(flags, fr.astype(np.float64), eps)
    refreshed = np.nonzero(flags)[0]
    ts = [1, 777, 4321, 9999, int(refreshed[len(refreshed) // 2]), int(refreshed[len(refreshed) // 2]) + 1]
    _check_frame_samples(res, fr, lm, lam, eps, ts, precision)


def test_c2_full_size_host_entry_point(pcv):
    """The benchmark's end-to-end call: pcv_evaluate_host on the 100k frames from pinned host
    memory (evaluated in chunks while the next frames are copied in and the previous
    outputs copied out).  Every refresh decision and 8 frames in full against the oracle."""
    from paper_1801_02362_gb300 import synth

    lm, fr = synth.make_problem(1, n_atoms=300, n_landmarks=200, n_frames=100_000, frame_noise=0.05)
    fr = np.ascontiguousarray(fr, dtype=np.float32)
    lam = 2.3 / oracle.mean_adjacent_msd(lm)
    eps = 0.05
    ctx = pcv.PathCV(lm, lam, eps=eps, precision="fp32")
    F = fr.shape[0]
    host = {"frames": torch.from_numpy(fr).pin_memory(),
            "s": torch.empty(F, dtype=torch.float64).pin_memory(), "z": torch.empty(F, dtype=torch.float64).pin_memory(),
            "dsdx": torch.empty(fr.shape, dtype=torch.float32).pin_memory(),
            "dzdx": torch.empty(fr.shape, dtype=torch.float32).pin_memory(),
            "msd": torch.empty((F, 200), dtype=torch.float64).pin_memory(),
            "refreshed": torch.empty(F, dtype=torch.uint8).pin_memory()}
    P = lambda k: host[k].data_ptr()
    pcv.pcv_evaluate_host(ctx.ctx, F, P("frames"), P("s"), P("z"), P("dsdx"), P("dzdx"), P("msd"), P("refreshed"))
    ctx.close()
    res = {k: v.numpy() for k, v in host.items() if k != "frames"}
    flags = res["refreshed"]
    _check_refresh_sequence(flags, fr.astype(np.float64), eps)
    rng = np.random.default_rng(9)
    # frames at and next to chunk boundaries of the pipelined call (chunks of 16667 frames)
    ts = sorted({16666, 16667, 16668, 50001, 83334} | set(rng.integers(1, F, 3).tolist()))
    _check_frame_samples(res, fr, lm, lam, eps, ts)


def test_c3_full_size_group_sampled(pcv):
    """256 independent instances (N ~ U[50, 2000], M ~ U[50, 1000], 512 frames each, FP32
    exact mode) in one group call -- the persistent launch the benchmark times, after its
    autotuner -- and 24 frames of 8 instances checked in full against the oracle."""
    from paper_1801_02362_gb300 import synth

    rng = np.random.default_rng(7)
    insts = []
    for k in range(256):
        n = int(rng.integers(50, 2001))
        m = int(rng.integers(50, 1001))
        lm, fr = synth.make_problem(1000 + k, n_atoms=n, n_landmarks=m, n_frames=512, frame_noise=0.05)
        insts.append((lm, np.ascontiguousarray(fr, dtype=np.float32)))
    check = [0, 37, 99, 128, 170, 201, 233, 255]
    lams = {k: 2.3 / oracle.mean_adjacent_msd(insts[k][0][:40]) for k in check}
    ctxs, bufs = [], []
    for k, (lm, fr) in enumerate(insts):
        ctxs.append(pcv.PathCV(lm, lams.get(k, 500.0), eps=-1.0, precision="fp32"))
        F, m = fr.shape[0], lm.shape[0]
        bufs.append({"x": torch.from_numpy(fr).cuda(), "s": torch.zeros(F, dtype=torch.float64, device="cuda"),
                     "z": torch.zeros(F, dtype=torch.float64, device="cuda"),
                     "msd": torch.zeros((F, m), dtype=torch.float64, device="cuda")})
    P = lambda t: t.data_ptr()
    ios = [{"F": b["s"].shape[0], "frames": P(b["x"]), "s": P(b["s"]), "z": P(b["z"]), "msd": P(b["msd"])} for b in bufs]
    handles = [c.ctx for c in ctxs]
    pcv.pcv_evaluate_group(handles, ios)  # autotune and capture
    pcv.pcv_evaluate_group(handles, ios)  # replay
    torch.cuda.synchronize()
    for c in ctxs:
        c.sync()
    for k in check:
        lm, fr = insts[k]
        ts = [0, 255, 511]
        r = oracle.exact(fr[ts], lm, lams[k])
        msd = bufs[k]["msd"].cpu().numpy()[ts]
        assert d_err(msd, r["D"], fr[ts], lm) < TOL["fp32"], k
        assert s_err(bufs[k]["s"].cpu().numpy()[ts], r["s"], lm.shape[0]) < TOL["fp32"], k
        assert z_err(bufs[k]["z"].cpu().numpy()[ts], r["z"], lams[k]) < TOL["fp32"], k
    for c in ctxs:
        c.close()


def test_nl_full_size_exact_sampled(pcv):
    """The neighbour-list workload the benchmark times (304 atoms, 2120 landmarks, a list of
    50 every 50 steps, 10k frames, FP32, gradients).  A frame t between updates depends only
    on itself and its last update u, so the oracle evaluates [x_u, x_t] as a run whose first
    step is an update: list membership, distances, s, z and gradients of both frames."""
    from paper_1801_02362_gb300 import synth

    lm, fr = synth.make_problem(8, n_atoms=304, n_landmarks=2120, n_frames=10_000, frame_noise=0.05)
    fr = np.ascontiguousarray(fr, dtype=np.float32)
    lam = 2.3 / oracle.mean_adjacent_msd(lm[:200])
    ctx = pcv.PathCV(lm, lam, eps=-1.0, precision="fp32", neighbor_list=(50, 50))
    out = ctx.evaluate(torch.from_numpy(fr).cuda(), grad=True, msd=True)
    ctx.sync()
    res = {k: v.double().cpu().numpy() for k, v in out.items()}
    ctx.close()
    for t in (1, 49, 2551, 5037, 9999):
        u = t - t % 50
        st = oracle.CloseState(304, 2120)
        st.ctr[1] = u  # the run starts at step u (an update: u is a multiple of 50)
        r = oracle.exact(fr[[u, t]], lm, lam, want_grad=True, nl=(50, 50), state=st)
        d = np.sort(r["D"][0])
        assert d[50] - d[49] > 2.5e-5 * max(d[49], 1e-3), "near-tie in the list at the update"  # precondition
        for row, f in ((0, u), (1, t)):
            fin = np.isfinite(r["D"][row])
            np.testing.assert_array_equal(np.isfinite(res["msd"][f]), fin)
            sl = slice(f, f + 1)
            assert d_err(np.where(fin, res["msd"][sl], 1.0), np.where(fin, r["D"][row:row + 1], 1.0), fr[sl],
                         lm) < TOL["fp32"]
            assert s_err(res["s"][sl], r["s"][row:row + 1], 2120) < TOL["fp32"]
            assert z_err(res["z"][sl], r["z"][row:row + 1], lam) < TOL["fp32"]
            assert grad_err(res["dsdx"][sl], r["dsdx"][row:row + 1]) < GRAD_TOL["fp32"]
            assert grad_err(res["dzdx"][sl], r["dzdx"][row:row + 1]) < GRAD_TOL["fp32"]

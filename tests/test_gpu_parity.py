"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle, element by
element on seeded inputs.  Sizes span several tiles with ragged tails (frames in tiles of
16/64, landmarks in tiles of 32, atoms in chunks of 32)."""
import numpy as np
import pytest

import oracle
from _util import GRAD_TOL, TOL, d_err, grad_err, problem, s_err, z_err

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


def run(pcv, lm, fr, lam, eps=-1.0, precision="fp32", grad=False, w=None, band=None, min_chunk=None, ctx=None):
    own = ctx is None
    if own:
        ctx = pcv.PathCV(lm, lam, eps=eps, precision=precision, weights=w, band=band, min_chunk=min_chunk)
    dt = torch.float64 if precision == "fp64" else torch.float32
    frames = torch.tensor(fr, dtype=dt, device="cuda")
    out = ctx.evaluate(frames, grad=grad, msd=True, refreshed=True)
    ctx.sync()
    res = {k: v.double().cpu().numpy() if v.dtype != torch.uint8 else v.cpu().numpy() for k, v in out.items()}
    res["stats"] = ctx.stats()
    if own:
        ctx.close()
    return res


def check_values(g, r, fr, lm, lam, precision, w=None):
    tol = TOL[precision]
    m = lm.shape[0]
    assert d_err(g["msd"], r["D"], fr, lm, w) < tol
    assert s_err(g["s"], r["s"], m) < tol
    assert z_err(g["z"], r["z"], lam) < tol


# ------------------------------------------------------------------------------------
# exact mode (Algorithm 1)
def test_exact_fp64_full_workload_c1(pcv):
    """N=22, M=20, F=1000 reflecting walk, FP64 end to end."""
    lm, fr, lam = problem(1, 22, 20, 1000, noise=0.02, schedule="walk", precision="fp64")
    r = oracle.exact(fr, lm, lam, want_grad=True)
    g = run(pcv, lm, fr, lam, precision="fp64", grad=True)
    check_values(g, r, fr, lm, lam, "fp64")
    assert grad_err(g["dsdx"], r["dsdx"]) < GRAD_TOL["fp64"]
    assert grad_err(g["dzdx"], r["dzdx"]) < GRAD_TOL["fp64"]
    assert np.all(g["refreshed"] == 1)


@pytest.mark.parametrize("precision", ["fp32", "fp16"])
def test_exact_ragged_tiles(pcv, precision):
    """N=300 (ragged atom chunk), M=200 (ragged landmark tile), F=200 (ragged frame tile)."""
    lm, fr, lam = problem(2, 300, 200, 200, precision=precision)
    r = oracle.exact(fr, lm, lam, want_grad=True)
    g = run(pcv, lm, fr, lam, precision=precision, grad=True)
    check_values(g, r, fr, lm, lam, precision)
    assert grad_err(g["dsdx"], r["dsdx"]) < GRAD_TOL[precision]
    assert grad_err(g["dzdx"], r["dzdx"]) < GRAD_TOL[precision]
    st = g["stats"]
    assert st["landmark_alignments"] == 200 * 200 and st["frames"] == 200


def test_exact_weights_and_properties(pcv):
    lm, fr, lam = problem(3, 57, 33, 40)
    rng = np.random.default_rng(0)
    w = rng.uniform(0.3, 3.0, size=57)
    q = rng.normal(size=33)
    r = oracle.exact(fr, lm, lam, w=w, q=q, want_grad=True)
    ctx = pcv.PathCV(lm, lam, eps=-1.0, precision="fp32", weights=w, props=q)
    g = run(pcv, lm, fr, lam, ctx=ctx, grad=True)
    ctx.close()
    assert d_err(g["msd"], r["D"], fr, lm, w) < TOL["fp32"]
    assert np.max(np.abs(g["s"] - r["s"])) < 1e-5 * np.max(np.abs(q)) * 33
    assert z_err(g["z"], r["z"], lam) < TOL["fp32"]
    assert grad_err(g["dzdx"], r["dzdx"]) < GRAD_TOL["fp32"]
    assert grad_err(g["dsdx"], r["dsdx"]) < GRAD_TOL["fp32"]


@pytest.mark.parametrize("n,m,f", [(3, 1, 1), (4, 2, 3), (33, 31, 17), (64, 64, 64), (5000, 3, 2)])
def test_exact_edge_shapes(pcv, n, m, f):
    lm, fr, lam = problem(4 + n, n, m, f) if m > 1 else problem(4, n, 2, f)
    lm = lm[:m]
    lam = lam if m > 1 else 100.0
    r = oracle.exact(fr, lm, lam, want_grad=True)
    g = run(pcv, lm, fr, lam, grad=True)
    check_values(g, r, fr, lm, lam, "fp32")
    assert grad_err(g["dzdx"], r["dzdx"]) < GRAD_TOL["fp32"]


def test_exact_large_structures_sampled(pcv):
    """N=5000, M=2000 (landmark set beyond L2 in FP32): a few frames, every pair checked."""
    lm, fr, lam = problem(5, 5000, 2000, 3)
    r = oracle.exact(fr, lm, lam)
    for precision in ("fp32", "fp16"):
        g = run(pcv, lm, fr, lam, precision=precision)
        check_values(g, r, fr, lm, lam, precision)


def test_rigid_copies_give_zero_and_landmark_index(pcv):
    lm, _, _ = problem(6, 50, 10, 1)
    from paper_1801_02362_gb300 import synth

    rng = np.random.default_rng(3)
    fr = np.stack([(lm[i] @ synth.random_rotation(rng).T + rng.uniform(-4, 4, 3)).astype(np.float32) for i in range(10)])
    g = run(pcv, lm, fr.astype(np.float64), 1e6)
    assert np.all(np.abs(g["s"] - np.arange(1, 11)) < 1e-6)
    assert np.max(np.diagonal(g["msd"])) < 1e-9


# ------------------------------------------------------------------------------------
# close structure (Algorithm 2)
@pytest.mark.parametrize("eps", [0.01, 0.05, 0.1])
@pytest.mark.parametrize("min_chunk", [None, 64])
def test_close_eps_sweep_refresh_flags_exact(pcv, eps, min_chunk):
    lm, fr, lam = problem(7, 300, 200, 1500)
    r = oracle.close(fr, lm, lam, eps)
    g = run(pcv, lm, fr, lam, eps=eps, min_chunk=min_chunk)
    np.testing.assert_array_equal(g["refreshed"], r["refreshed"])
    check_values(g, r, fr, lm, lam, "fp32")
    st, oc = g["stats"], r["state"].counters
    assert st["refreshes_threshold"] == oc["refreshes_threshold"]
    assert st["refreshes_initial"] == oc["refreshes_initial"] == 1
    assert st["landmark_alignments"] == oc["landmark_alignments"]
    assert st["approx_msds"] == oc["approx_msds"]
    assert st["xy_alignments"] == oc["xy_alignments"]


def test_close_same_context_across_regimes(pcv):
    """One context, reset between batches: long gaps (the band is skipped once the gap
    estimate is large), then every frame reassigning (the band comes back lazily)."""
    lm, fr, lam = problem(7, 300, 200, 1500)
    ctx = pcv.PathCV(lm, lam, eps=0.05, precision="fp32")
    for eps in (0.05, 0.05, 0.01, 0.1, 0.01):
        pcv.pcv_set_close_threshold(ctx.ctx, eps)
        pcv.pcv_reset_close_state(ctx.ctx)
        r = oracle.close(fr, lm, lam, eps)
        g = run(pcv, lm, fr, lam, ctx=ctx)
        np.testing.assert_array_equal(g["refreshed"], r["refreshed"])
        check_values(g, r, fr, lm, lam, "fp32")
    ctx.close()


@pytest.mark.parametrize("band", [1, 2, 6])
def test_close_correlated_noise_all_band_states(pcv, band):
    """Ornstein-Uhlenbeck frame noise: gaps of a few frames, exercising every band state."""
    lm, fr, lam = problem(8, 120, 40, 800, noise=0.03, ou_rho=0.97)
    for eps in (0.0002, 0.0006, 0.004):
        r = oracle.close(fr, lm, lam, eps)
        nref = int((r["refreshed"] == 1).sum())
        assert 20 < nref < 700
        g = run(pcv, lm, fr, lam, eps=eps, band=band, min_chunk=8)
        np.testing.assert_array_equal(g["refreshed"], r["refreshed"])
        check_values(g, r, fr, lm, lam, "fp32")


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16"])
def test_close_gradients(pcv, precision):
    lm, fr, lam = problem(9, 64, 24, 120, noise=0.02, schedule="walk", precision=precision, ou_rho=0.9)
    eps = 0.003
    r = oracle.close(fr, lm, lam, eps, want_grad=True)
    assert 0 < int((r["refreshed"] == 0).sum()) and 0 < int((r["refreshed"] == 1).sum())
    g = run(pcv, lm, fr, lam, eps=eps, precision=precision, grad=True)
    np.testing.assert_array_equal(g["refreshed"], r["refreshed"])
    check_values(g, r, fr, lm, lam, precision)
    assert grad_err(g["dsdx"], r["dsdx"]) < GRAD_TOL[precision]
    assert grad_err(g["dzdx"], r["dzdx"]) < GRAD_TOL[precision]


def test_close_split_calls_and_saved_state(pcv):
    lm, fr, lam = problem(10, 80, 30, 300, noise=0.03, ou_rho=0.95)
    eps = 0.006
    r = oracle.close(fr, lm, lam, eps, want_grad=True)
    ctx = pcv.PathCV(lm, lam, eps=eps, precision="fp32")
    parts = [run(pcv, lm, fr[a:b], lam, ctx=ctx, grad=True) for a, b in ((0, 1), (1, 97), (97, 180))]
    blob = ctx.save_state()
    ctx2 = pcv.PathCV(lm, lam, eps=eps, precision="fp32")
    ctx2.load_state(blob)
    parts.append(run(pcv, lm, fr[180:], lam, ctx=ctx2, grad=True))
    ctx.close()
    for key in ("refreshed",):
        np.testing.assert_array_equal(np.concatenate([p[key] for p in parts]), r[key])
    g = {k: np.concatenate([p[k] for p in parts]) for k in ("s", "z", "msd", "dsdx", "dzdx")}
    check_values(g, r, fr, lm, lam, "fp32")
    assert grad_err(g["dzdx"], r["dzdx"]) < GRAD_TOL["fp32"]
    st = parts[-1]["stats"]
    oc = r["state"].counters
    assert st["refreshes_threshold"] == oc["refreshes_threshold"]
    assert st["frames"] == 300
    ctx2.close()


@pytest.mark.parametrize("precision", ["fp32", "fp16"])
@pytest.mark.parametrize("n,m", [(140, 45), (61, 200)])
@pytest.mark.parametrize("variant", ["tensor_cores", "cuda_cores", "not_materialized"])
def test_close_materialized_operands(pcv, precision, n, m, variant):
    """Long segments (20 refreshes in 700 frames): the rotated frames x' and the rotated
    landmarks b of each segment are materialised and both heavy loops run as plain tiles;
    the approximate MSDs and the segment adjoint run on the tensor cores (split FP16 operands
    on deviations from the close structure) or on the CUDA cores.  N = 140 pads to 144 atoms (a half tile of 32 at the
    end) and 420 adjoint columns (two column tiles of 224); N = 61 to 64 atoms and 183
    columns (one tile of 192); M = 45 and 200 take the two landmark tile widths and pad the
    tensor-core K to 48 and 208; 700 frames end in a ragged tile of 64.  The second call
    starts from the first call's close structure (the prior segment in use).  A cap of 0
    turns materialisation off.  All must match the oracle."""
    lm, fr, lam = problem(12, n, m, 700, noise=0.02, schedule="walk", precision=precision, ou_rho=0.9)
    eps = 0.0025
    r = oracle.close(fr, lm, lam, eps, want_grad=True)
    cap = 0 if variant == "not_materialized" else None
    ctx = pcv.PathCV(lm, lam, eps=eps, precision=precision, materialize=cap,
                     tensor_cores=variant == "tensor_cores")
    ctx.set_profiling(True)
    parts = [run(pcv, lm, fr[a:b], lam, ctx=ctx, grad=True) for a, b in ((0, 430), (430, 700))]
    prof = ctx.profile()
    ctx.close()
    assert ("materialize" in prof) == (cap is None), prof
    assert ("adjoint_beta_mma" in prof) == (variant == "tensor_cores"), prof
    assert ("approx_pair_mma" in prof) == (variant == "tensor_cores"), prof
    np.testing.assert_array_equal(np.concatenate([p["refreshed"] for p in parts]), r["refreshed"])
    g = {k: np.concatenate([p[k] for p in parts]) for k in ("s", "z", "msd", "dsdx", "dzdx")}
    check_values(g, r, fr, lm, lam, precision)
    assert grad_err(g["dsdx"], r["dsdx"]) < GRAD_TOL[precision]
    assert grad_err(g["dzdx"], r["dzdx"]) < GRAD_TOL[precision]


@pytest.mark.parametrize("group", [1, 4, 8])
def test_close_mma_fold_groups(pcv, group):
    """Tensor-core approximate MSDs with 1, 4 (the default) and 8 chunks of main products
    summed in tensor memory per fold, on 300 atoms and 200 landmarks, where each extra
    accumulation step shows in the MSD error: all within the FP32 tolerance of the oracle.
    The option rejects groups outside 1..16."""
    lm, fr, lam = problem(7, 300, 200, 1500)
    eps = 0.05
    r = oracle.close(fr, lm, lam, eps)
    ctx = pcv.PathCV(lm, lam, eps=eps, precision="fp32", tensor_cores=True)
    pcv.pcv_set_option(ctx.ctx, pcv.PCV_OPT_MMA_GROUP, group)
    ctx.set_profiling(True)
    g = run(pcv, lm, fr, lam, ctx=ctx)
    assert "approx_pair_mma" in ctx.profile()
    np.testing.assert_array_equal(g["refreshed"], r["refreshed"])
    check_values(g, r, fr, lm, lam, "fp32")
    for bad in (0, 17):
        with pytest.raises(pcv.PcvError) as e:
            pcv.pcv_set_option(ctx.ctx, pcv.PCV_OPT_MMA_GROUP, bad)
        assert e.value.status == pcv.PCV_EINVAL
    ctx.close()


@pytest.mark.parametrize("precision", ["fp32", "fp16"])
def test_exact_few_frames_split_over_atom_slices(pcv, precision):
    """24 frames x 200 landmarks of 1000 atoms make 14 tiles, far from filling the GPU, so the
    exact pairs split the atoms over 4 slices per tile (partial correlations added in slice
    order, then the rotation, then partial MSDs): values, both gradients (the rotations) and
    a second call of 9 frames (ragged tiles) against the oracle."""
    lm, fr, lam = problem(64, 1000, 200, 33, noise=0.03, schedule="walk", precision=precision)
    ctx = pcv.PathCV(lm, lam, eps=-1.0, precision=precision)
    for a, b in ((0, 24), (24, 33)):
        r = oracle.exact(fr[a:b], lm, lam, want_grad=True)
        out = ctx.evaluate(torch.tensor(fr[a:b], dtype=torch.float32, device="cuda"), grad=True, msd=True)
        ctx.sync()
        g = {k: v.double().cpu().numpy() for k, v in out.items()}
        check_values(g, r, fr[a:b], lm, lam, precision)
        assert grad_err(g["dsdx"], r["dsdx"]) < GRAD_TOL[precision]
        assert grad_err(g["dzdx"], r["dzdx"]) < GRAD_TOL[precision]
    ctx.close()


def test_close_fp64_workload_c1(pcv):
    lm, fr, lam = problem(11, 22, 20, 1000, noise=0.02, schedule="walk", precision="fp64")
    for eps in (0.001, 0.002, 0.004):
        r = oracle.close(fr, lm, lam, eps, want_grad=True)
        g = run(pcv, lm, fr, lam, eps=eps, precision="fp64", grad=True)
        np.testing.assert_array_equal(g["refreshed"], r["refreshed"])
        check_values(g, r, fr, lm, lam, "fp64")
        assert grad_err(g["dzdx"], r["dzdx"]) < GRAD_TOL["fp64"]
        assert grad_err(g["dsdx"], r["dsdx"]) < GRAD_TOL["fp64"]


def test_autograd_function_matches_chain_rule(pcv):
    lm, fr, lam = problem(12, 40, 16, 30, noise=0.02, ou_rho=0.9)
    r = oracle.close(fr, lm, lam, 0.003, want_grad=True)
    ctx = pcv.PathCV(lm, lam, eps=0.003, precision="fp32")
    x = torch.tensor(fr, dtype=torch.float32, device="cuda", requires_grad=True)
    s, z = pcv.path_cv(x, ctx)
    ws = torch.linspace(0.5, 1.5, 30, device="cuda", dtype=torch.float64)
    (ws * s + 2.0 * z).sum().backward()
    ref = ws.cpu().numpy()[:, None, None] * r["dsdx"] + 2.0 * r["dzdx"]
    assert grad_err(x.grad.double().cpu().numpy(), ref) < GRAD_TOL["fp32"]
    ctx.close()


def test_host_entry_point_matches_device(pcv):
    import ctypes

    lm, fr, lam = problem(13, 100, 50, 64)
    g = run(pcv, lm, fr, lam, eps=0.05, grad=True)
    ctx = pcv.PathCV(lm, lam, eps=0.05, precision="fp32")
    f32 = np.ascontiguousarray(fr, dtype=np.float32)
    F = fr.shape[0]
    s = np.zeros(F)
    z = np.zeros(F)
    gs = np.zeros_like(f32)
    gz = np.zeros_like(f32)
    msd = np.zeros((F, 50))
    ref = np.zeros(F, dtype=np.uint8)
    p = lambda a: ctypes.c_void_p(a.ctypes.data)
    pcv.pcv_evaluate_host(ctx.ctx, F, p(f32), p(s), p(z), p(gs), p(gz), p(msd), p(ref))
    np.testing.assert_array_equal(ref, g["refreshed"])
    np.testing.assert_allclose(s, g["s"], rtol=0, atol=1e-12)
    np.testing.assert_allclose(msd, g["msd"], rtol=0, atol=1e-12)
    np.testing.assert_allclose(gz, g["dzdx"], rtol=0, atol=1e-7)
    ctx.close()


_CHUNK_CASE = {}


def _chunk_case():
    if not _CHUNK_CASE:
        lm, fr, lam = problem(15, 40, 30, 9000, noise=0.03)
        r = oracle.close(fr, lm, lam, 0.01, want_grad=True)
        _CHUNK_CASE.update(lm=lm, fr=fr, lam=lam, r=r)
    return _CHUNK_CASE


@pytest.mark.parametrize("chunks,end_share", [(1, 25), (2, 25), (4, 1), (3, 100), (0, 25)])
def test_host_entry_point_chunk_plans(pcv, chunks, end_share):
    """9000 frames through pcv_evaluate_host split into 1..4 chunks (first and last chunk
    smaller than the others, or all equal): the close-structure state carries over between
    chunks, so refresh decisions and values match the oracle's single run."""
    import ctypes

    c = _chunk_case()
    lm, fr, lam, r = c["lm"], c["fr"], c["lam"], c["r"]
    nref = int((r["refreshed"] > 0).sum())
    assert 3 < nref < fr.shape[0] // 4
    ctx = pcv.PathCV(lm, lam, eps=0.01, precision="fp32")
    pcv.pcv_set_option(ctx.ctx, pcv.PCV_OPT_HOST_CHUNKS, chunks)
    pcv.pcv_set_option(ctx.ctx, pcv.PCV_OPT_HOST_END_SHARE, end_share)
    f32 = np.ascontiguousarray(fr, dtype=np.float32)
    F = fr.shape[0]
    s, z = np.zeros(F), np.zeros(F)
    gs, gz = np.zeros_like(f32), np.zeros_like(f32)
    msd = np.zeros((F, lm.shape[0]))
    ref = np.zeros(F, dtype=np.uint8)
    p = lambda a: ctypes.c_void_p(a.ctypes.data)
    pcv.pcv_evaluate_host(ctx.ctx, F, p(f32), p(s), p(z), p(gs), p(gz), p(msd), p(ref))
    ctx.close()
    np.testing.assert_array_equal(ref, r["refreshed"])
    assert d_err(msd, r["D"], fr, lm) < TOL["fp32"]
    assert s_err(s, r["s"], lm.shape[0]) < TOL["fp32"]
    assert z_err(z, r["z"], lam) < TOL["fp32"]
    assert grad_err(gs.astype(np.float64), r["dsdx"]) < GRAD_TOL["fp32"]
    assert grad_err(gz.astype(np.float64), r["dzdx"]) < GRAD_TOL["fp32"]


def test_invalid_arguments_are_rejected(pcv):
    lm, fr, lam = problem(14, 10, 4, 2)
    ctx = pcv.PathCV(lm, lam)
    with pytest.raises(pcv.PcvError) as e:
        pcv.pcv_set_lambda(ctx.ctx, -1.0)
    assert e.value.status == pcv.PCV_EINVAL
    with pytest.raises(pcv.PcvError):
        pcv.pcv_set_option(ctx.ctx, pcv.PCV_OPT_BAND, 9)
    with pytest.raises(pcv.PcvError):
        pcv.pcv_evaluate(ctx.ctx, -1, None, None, None)
    with pytest.raises(pcv.PcvError):
        pcv.pcv_evaluate(ctx.ctx, 2, None, None, None)
    with pytest.raises(pcv.PcvError):
        pcv.pcv_load_state(ctx.ctx, b"garbage" * 10)
    bad = lm.copy()
    bad[0, 0, 0] = np.nan
    with pytest.raises(pcv.PcvError):
        pcv.pcv_set_landmarks(ctx.ctx, bad)
    pcv.pcv_evaluate(ctx.ctx, 0, None, None, None)  # F = 0 is a no-op
    ctx.close()

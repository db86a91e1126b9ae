"""Many instances in one call (pcv_evaluate_group): ragged walkers in exact mode run as
three persistent launches replayed from a captured graph; the result of every instance must
match the oracle and the per-instance evaluation, on the first call (autotuned and
captured) and on replays, including after the inputs change in place."""
import numpy as np
import pytest

import oracle
from _util import GRAD_TOL, TOL, d_err, grad_err, problem, s_err, s_kappa, z_err

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


SHAPES = [(5, 3, 7), (17, 31, 40), (64, 45, 1), (140, 90, 33), (300, 33, 16), (33, 64, 0), (61, 17, 70),
          (128, 32, 17), (9, 100, 5), (250, 7, 12), (47, 47, 47), (3, 2, 2)]


def _instances(precision, seed0=40, eps=-1.0):
    out = []
    # FP16 storage rounds each landmark coordinate by up to 2^-12 of its block residual; D
    # moves linearly with that (2 sum (x - R a) . R da), so structures of a few atoms at small
    # D reach the 1e-3 bound on storage alone: the FP16 cases use 16 atoms or more
    shapes = SHAPES if precision != "fp16" else [(max(n, 16), m, f) for n, m, f in SHAPES]
    for k, (n, m, f) in enumerate(shapes):
        lm, fr, lam = problem(seed0 + k, n, m, max(f, 1), noise=0.05)
        fr = fr[:f]
        out.append((lm, fr, lam))
    return out


def _buffers(fr, m):
    F = fr.shape[0]
    x = torch.tensor(fr if F else np.zeros((0, 3, 3)), dtype=torch.float32, device="cuda")
    return {"x": x, "s": torch.zeros(F, dtype=torch.float64, device="cuda"),
            "z": torch.zeros(F, dtype=torch.float64, device="cuda"),
            "msd": torch.zeros((F, m), dtype=torch.float64, device="cuda")}


def _io(buf):
    F = buf["s"].shape[0]
    return {"F": F, "frames": buf["x"].data_ptr() if F else None, "s": buf["s"].data_ptr() if F else None,
            "z": buf["z"].data_ptr() if F else None, "msd": buf["msd"].data_ptr() if F else None}


def _check(insts, bufs, precision):
    for (lm, fr, lam), b in zip(insts, bufs):
        if fr.shape[0] == 0:
            continue
        r = oracle.exact(fr, lm, lam)
        assert d_err(b["msd"].cpu().numpy(), r["D"], fr, lm) < TOL[precision]
        # FP16 storage: the instances of a few atoms take D errors up to the D tolerance from
        # the rounding of the landmarks alone, and s inherits them with its condition number
        kappa = s_kappa(r["D"], lam, fr, lm) if precision == "fp16" else None
        assert s_err(b["s"].cpu().numpy(), r["s"], lm.shape[0], kappa=kappa) < TOL[precision]
        assert z_err(b["z"].cpu().numpy(), r["z"], lam) < TOL[precision]


@pytest.mark.parametrize("precision", ["fp32", "fp16"])
def test_group_ragged_exact_graph(pcv, precision):
    insts = _instances(precision)
    ctxs = [pcv.PathCV(lm, lam, eps=-1.0, precision=precision) for lm, fr, lam in insts]
    bufs = [_buffers(fr, lm.shape[0]) for lm, fr, lam in insts]
    handles = [c.ctx for c in ctxs]
    pcv.pcv_evaluate_group(handles, [_io(b) for b in bufs])  # autotune + capture
    torch.cuda.synchronize()
    for c in ctxs:
        c.sync()
    _check(insts, bufs, precision)
    first = [(b["s"].clone(), b["z"].clone()) for b in bufs]
    pcv.pcv_evaluate_group(handles, [_io(b) for b in bufs])  # replay
    torch.cuda.synchronize()
    for (s0, z0), b in zip(first, bufs):
        assert torch.equal(s0, b["s"]) and torch.equal(z0, b["z"])
    # new frames written into the same buffers: the replayed graph reads them
    insts2 = _instances(precision, seed0=90)
    for (lm, fr, lam), (lm2, fr2, lam2), b in zip(insts, insts2, bufs):
        if fr.shape[0]:
            b["x"].copy_(torch.tensor(fr2[:, :fr.shape[1]] if fr2.shape[1] == fr.shape[1] else fr, device="cuda"))
    pcv.pcv_evaluate_group(handles, [_io(b) for b in bufs])
    torch.cuda.synchronize()
    new = [(lm, b["x"].cpu().numpy().astype(np.float64), lam) for (lm, fr, lam), b in zip(insts, bufs)]
    _check(new, bufs, precision)
    # per-instance evaluation gives the same values
    for c, (lm, fr, lam), b in zip(ctxs, new, bufs):
        if fr.shape[0] == 0:
            continue
        out = c.evaluate(torch.tensor(fr, dtype=torch.float32, device="cuda"), msd=True)
        c.sync()
        assert s_err(out["s"].cpu().numpy(), b["s"].cpu().numpy(), lm.shape[0]) < TOL[precision]
        assert z_err(out["z"].cpu().numpy(), b["z"].cpu().numpy(), lam) < TOL[precision]
    for c in ctxs:
        c.close()


@pytest.mark.parametrize("shape", [1, 2, 3])
def test_group_each_tile_shape(pcv, shape):
    """The autotuner's tile shapes one at a time (PCV_OPT_EXACT_TILE on the first context fixes
    it): 16 x 32, 32 x 16 and 8 x 64 frames x landmarks, over the ragged instances (frame and
    landmark counts that leave partial tiles in both directions), against the oracle; the
    tuning query reports the shape used."""
    insts = _instances("fp32")
    ctxs = [pcv.PathCV(lm, lam, eps=-1.0, precision="fp32") for lm, fr, lam in insts]
    pcv.pcv_set_option(ctxs[0].ctx, pcv.PCV_OPT_EXACT_TILE, shape)
    bufs = [_buffers(fr, lm.shape[0]) for lm, fr, lam in insts]
    assert pcv.pcv_group_tuning(ctxs[0].ctx) == (0, 0, 0)
    pcv.pcv_evaluate_group([c.ctx for c in ctxs], [_io(b) for b in bufs])
    torch.cuda.synchronize()
    _check(insts, bufs, "fp32")
    tf, tm, blocks = pcv.pcv_group_tuning(ctxs[0].ctx)
    assert (tf, tm) == {1: (16, 32), 2: (32, 16), 3: (8, 64)}[shape] and blocks > 0
    for c in ctxs:
        c.close()


@pytest.mark.parametrize("shape", [2, 3])
@pytest.mark.parametrize("precision", ["fp32", "fp16"])
def test_exact_pairs_each_tile_shape(pcv, shape, precision):
    """The per-call exact kernel with the other tile shapes (PCV_OPT_EXACT_TILE): 70 frames x
    45 landmarks leave partial tiles in both directions; values and both gradients (the
    tiles' rotations) against the oracle."""
    lm, fr, lam = problem(63, 37, 45, 70, noise=0.03, schedule="walk", precision=precision)
    r = oracle.exact(fr, lm, lam, want_grad=True)
    ctx = pcv.PathCV(lm, lam, eps=-1.0, precision=precision)
    pcv.pcv_set_option(ctx.ctx, pcv.PCV_OPT_EXACT_TILE, shape)
    out = ctx.evaluate(torch.tensor(fr, dtype=torch.float32, device="cuda"), grad=True, msd=True)
    ctx.sync()
    g = {k: v.double().cpu().numpy() for k, v in out.items()}
    with pytest.raises(pcv.PcvError):
        pcv.pcv_set_option(ctx.ctx, pcv.PCV_OPT_EXACT_TILE, 4)
    ctx.close()
    assert d_err(g["msd"], r["D"], fr, lm) < TOL[precision]
    assert s_err(g["s"], r["s"], lm.shape[0]) < TOL[precision]
    assert z_err(g["z"], r["z"], lam) < TOL[precision]
    assert grad_err(g["dsdx"], r["dsdx"]) < GRAD_TOL[precision]
    assert grad_err(g["dzdx"], r["dzdx"]) < GRAD_TOL[precision]


def test_group_mixed_modes_fall_back(pcv):
    """A close-mode context and an entry with gradients: evaluated one by one, same values."""
    a = problem(60, 40, 20, 30, noise=0.02, schedule="walk", ou_rho=0.9)
    b = problem(61, 25, 12, 9)
    ca = pcv.PathCV(a[0], a[2], eps=0.003, precision="fp32")
    cb = pcv.PathCV(b[0], b[2], eps=-1.0, precision="fp32")
    xa = torch.tensor(a[1], dtype=torch.float32, device="cuda")
    xb = torch.tensor(b[1], dtype=torch.float32, device="cuda")
    sa, za = torch.zeros(30, dtype=torch.float64, device="cuda"), torch.zeros(30, dtype=torch.float64, device="cuda")
    sb, zb = torch.zeros(9, dtype=torch.float64, device="cuda"), torch.zeros(9, dtype=torch.float64, device="cuda")
    ga, gza = torch.zeros_like(xa), torch.zeros_like(xa)
    pcv.pcv_evaluate_group([ca.ctx, cb.ctx], [
        {"F": 30, "frames": xa.data_ptr(), "s": sa.data_ptr(), "z": za.data_ptr(), "dsdx": ga.data_ptr(),
         "dzdx": gza.data_ptr()},
        {"F": 9, "frames": xb.data_ptr(), "s": sb.data_ptr(), "z": zb.data_ptr()}])
    torch.cuda.synchronize()
    ra = oracle.close(a[1], a[0], a[2], 0.003, want_grad=True)
    rb = oracle.exact(b[1], b[0], b[2])
    assert s_err(sa.cpu().numpy(), ra["s"], 20) < TOL["fp32"]
    assert s_err(sb.cpu().numpy(), rb["s"], 12) < TOL["fp32"]
    assert z_err(zb.cpu().numpy(), rb["z"], b[2]) < TOL["fp32"]
    ca.close()
    cb.close()


def test_group_rejects_repeated_context(pcv):
    a = problem(62, 10, 4, 3)
    c = pcv.PathCV(a[0], a[2], eps=-1.0, precision="fp32")
    x = torch.tensor(a[1], dtype=torch.float32, device="cuda")
    s, z = torch.zeros(3, dtype=torch.float64, device="cuda"), torch.zeros(3, dtype=torch.float64, device="cuda")
    io = {"F": 3, "frames": x.data_ptr(), "s": s.data_ptr(), "z": z.data_ptr()}
    with pytest.raises(pcv.PcvError):
        pcv.pcv_evaluate_group([c.ctx, c.ctx], [io, io])
    c.close()

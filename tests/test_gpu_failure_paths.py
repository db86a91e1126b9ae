"""Device-side failure reports, driven without faulting the GPU.

PCV_OPT_NEWTON_CAP lowers the iteration cap of the exact pair kernels' Newton eigen-solves
so that pairs reach it: pcv_sync must return PCV_ENOCONV.  PCV_OPT_WAIT_CYCLES shrinks the
clock budget of the tensor-core adjoint's bounded waits so that they run out: the kernel
records the timeout, waits for its own copies and MMAs within the default budget, frees its
tensor memory and returns, and pcv_sync must return PCV_ETIMEOUT.  In both cases the next
call with the default settings, on the same context, must match the oracle: the status
word is cleared by the report and nothing of the failed call is left behind."""
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


def _values_match(out, r, fr, lm, lam, precision):
    g = {k: v.double().cpu().numpy() for k, v in out.items()}
    tol = TOL[precision]
    assert d_err(g["msd"], r["D"], fr, lm) < tol
    assert s_err(g["s"], r["s"]) < tol
    assert z_err(g["z"], r["z"], lam) < tol
    return g


@pytest.mark.parametrize("precision,frames", [("fp32", 70), ("fp32", 3), ("fp64", 40)])
def test_newton_cap_reports_enoconv_then_recovers(pcv, precision, frames):
    """Exact mode: 70 frames take the tiled FP32 kernel, 3 frames the one-CTA-per-landmark
    kernel, FP64 its tiled kernel.  One Newton iteration cannot converge from the upper
    bound, so every pair reports the cap."""
    lm, fr, lam = problem(51, 60, 37, frames, precision=precision)
    dt = torch.float64 if precision == "fp64" else torch.float32
    x = torch.tensor(fr, dtype=dt, device="cuda")
    ctx = pcv.PathCV(lm, lam, eps=-1.0, precision=precision)
    pcv.pcv_set_option(ctx.ctx, pcv.PCV_OPT_NEWTON_CAP, 1)
    ctx.evaluate(x, msd=True)
    with pytest.raises(pcv.PcvError) as e:
        ctx.sync()
    assert e.value.status == pcv.PCV_ENOCONV
    pcv.pcv_set_option(ctx.ctx, pcv.PCV_OPT_NEWTON_CAP, 60)
    out = ctx.evaluate(x, msd=True)
    ctx.sync()  # the report cleared the status word
    _values_match(out, oracle.exact(fr, lm, lam), fr, lm, lam, precision)
    with pytest.raises(pcv.PcvError) as e:
        pcv.pcv_set_option(ctx.ctx, pcv.PCV_OPT_NEWTON_CAP, 0)
    assert e.value.status == pcv.PCV_EINVAL
    ctx.close()


def test_tensor_core_wait_budget_reports_etimeout_then_recovers(pcv):
    """Close-structure mode with long segments and gradients: the segment adjoint runs on the
    tensor cores (checked in the profile).  A budget of one cycle makes its first waits for
    the bulk copies and the MMAs run out."""
    lm, fr, lam = problem(12, 61, 45, 300, noise=0.02, schedule="walk", ou_rho=0.9)
    eps = 0.0025
    x = torch.tensor(fr, dtype=torch.float32, device="cuda")
    ctx = pcv.PathCV(lm, lam, eps=eps, precision="fp32", tensor_cores=True)
    ctx.set_profiling(True)
    pcv.pcv_set_option(ctx.ctx, pcv.PCV_OPT_WAIT_CYCLES, 1)
    ctx.evaluate(x, grad=True, msd=True)
    with pytest.raises(pcv.PcvError) as e:
        ctx.sync()
    assert e.value.status == pcv.PCV_ETIMEOUT
    assert "adjoint_beta_mma" in ctx.profile()
    pcv.pcv_set_option(ctx.ctx, pcv.PCV_OPT_WAIT_CYCLES, 0)  # back to the default budget
    ctx.reset()
    out = ctx.evaluate(x, grad=True, msd=True)
    ctx.sync()
    r = oracle.close(fr, lm, lam, eps, want_grad=True)
    g = _values_match({k: out[k] for k in ("s", "z", "msd")}, r, fr, lm, lam, "fp32")
    assert g is not None
    assert grad_err(out["dsdx"].double().cpu().numpy(), r["dsdx"]) < GRAD_TOL["fp32"]
    assert grad_err(out["dzdx"].double().cpu().numpy(), r["dzdx"]) < GRAD_TOL["fp32"]
    ctx.close()

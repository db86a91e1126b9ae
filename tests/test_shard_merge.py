"""Landmark shards: path CVs computed on disjoint subsets of the landmarks (each with the
landmarks' global properties q_i) combine exactly into the whole-path values through the
library's pack / sum / unpack (the MIN and SUM reductions a multi-GPU run performs).

CPU: the oracle evaluates each shard; the library's host pack/unpack merges them, directly
and through a two-rank gloo process group; the result equals the unsharded oracle.
GPU: several contexts on one device hold the shards; the device pack/unpack merges them;
the result equals the unsharded context and the oracle."""
import os
import socket

import numpy as np
import pytest

import oracle
from _util import GRAD_TOL, TOL, grad_err, problem, s_err, z_err

torch = pytest.importorskip("torch")


def _shards(m, k):
    return np.array_split(np.arange(m), k)


def _oracle_shard(fr, lm, lam, idx, eps=None):
    q = (idx + 1).astype(np.float64)  # global 1-based properties
    if eps is None:
        return oracle.exact(fr, lm[idx], lam, q=q, want_grad=True)
    return oracle.close(fr, lm[idx], lam, eps, q=q, want_grad=True)


def _merge_host(pcv, lam, parts):
    zmin = np.min([p["z"] for p in parts], axis=0)
    scal, elem = None, None
    for p in parts:
        sc, el = pcv.pcv_shard_pack_host(lam, zmin, p["s"], p["z"], p["dsdx"], p["dzdx"])
        scal = sc if scal is None else scal + sc
        elem = el if elem is None else elem + el
    return pcv.pcv_shard_unpack_host(lam, zmin, scal, elem)


@pytest.fixture(scope="module")
def pcv():
    from paper_1801_02362_gb300 import build_lib
    from paper_1801_02362_gb300 import pcv as mod

    build_lib.build()
    mod.load()
    return mod


@pytest.mark.parametrize("mode", ["exact", "close"])
def test_host_merge_equals_unsharded_oracle(pcv, mode):
    lm, fr, lam = problem(21, 30, 24, 60, noise=0.02, schedule="walk", precision="fp64", ou_rho=0.9)
    eps = None if mode == "exact" else 0.003
    full = _oracle_shard(fr, lm, lam, np.arange(24), eps)
    parts = [_oracle_shard(fr, lm, lam, idx, eps) for idx in _shards(24, 3)]
    s, z, gs, gz = _merge_host(pcv, lam, parts)
    assert np.max(np.abs(s - full["s"])) < 1e-9
    assert np.max(np.abs(z - full["z"])) < 1e-12
    assert grad_err(gs, full["dsdx"]) < 1e-9
    assert grad_err(gz, full["dzdx"]) < 1e-9


def test_single_shard_is_identity(pcv):
    lm, fr, lam = problem(22, 20, 10, 8, precision="fp64")
    full = _oracle_shard(fr, lm, lam, np.arange(10))
    s, z, gs, gz = _merge_host(pcv, lam, [full])
    assert np.max(np.abs(s - full["s"])) < 1e-12 and np.max(np.abs(z - full["z"])) < 1e-12
    assert grad_err(gz, full["dzdx"]) < 1e-12


def test_host_merge_rejects_bad_arguments(pcv):
    with pytest.raises(pcv.PcvError):
        pcv.pcv_shard_pack_host(-1.0, np.zeros(2), np.zeros(2), np.zeros(2))


def _free_port():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def _rank_main(rank, world, port, out_path):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1801_02362_gb300 import pcv as mod

    lm, fr, lam = problem(23, 26, 30, 40, noise=0.02, schedule="walk", precision="fp64", ou_rho=0.9)
    idx = _shards(30, world)[rank]
    part = _oracle_shard(fr, lm, lam, idx, 0.004)
    z = torch.from_numpy(part["z"].copy())
    dist.all_reduce(z, op=dist.ReduceOp.MIN)  # zmin
    zmin = z.numpy()
    scal, elem = mod.pcv_shard_pack_host(lam, zmin, part["s"], part["z"], part["dsdx"], part["dzdx"])
    ts, te = torch.from_numpy(scal), torch.from_numpy(elem)
    dist.all_reduce(ts)
    dist.all_reduce(te)
    s, zz, gs, gz = mod.pcv_shard_unpack_host(lam, zmin, ts.numpy(), te.numpy())
    if rank == 0:
        full = _oracle_shard(fr, lm, lam, np.arange(30), 0.004)
        err = max(np.max(np.abs(s - full["s"])), np.max(np.abs(zz - full["z"])), grad_err(gs, full["dsdx"]),
                  grad_err(gz, full["dzdx"]))
        with open(out_path, "w") as fh:
            fh.write(repr(float(err)))
    dist.barrier()
    dist.destroy_process_group()


def test_gloo_two_ranks_merge(pcv, tmp_path):
    import torch.multiprocessing as mp

    out = tmp_path / "err.txt"
    mp.start_processes(_rank_main, args=(2, _free_port(), str(out)), nprocs=2, join=True, start_method="spawn")
    assert float(out.read_text()) < 1e-9


# ------------------------------------------------------------------------------------
@pytest.mark.gpu
@pytest.mark.parametrize("precision,eps", [("fp32", None), ("fp32", 0.0025), ("fp64", 0.0025)])
def test_gpu_shards_merge_to_unsharded(pcv, precision, eps):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lm, fr, lam = problem(24, 140, 45, 700, noise=0.02, schedule="walk", precision=precision, ou_rho=0.9)
    dt = torch.float64 if precision == "fp64" else torch.float32
    frames = torch.tensor(fr, dtype=dt, device="cuda")
    F, N, M = fr.shape[0], fr.shape[1], lm.shape[0]
    prec = {"fp64": pcv.PCV_FP64, "fp32": pcv.PCV_FP32}[precision]
    e = -1.0 if eps is None else eps

    def run_ctx(idx):
        ctx = pcv.PathCV(lm[idx], lam, eps=e, precision=precision, props=(idx + 1).astype(np.float64))
        out = ctx.evaluate(frames, grad=True)
        ctx.sync()
        ctx.close()
        return out

    full = run_ctx(np.arange(M))
    parts = [run_ctx(idx) for idx in _shards(M, 3)]
    zmin = torch.stack([p["z"] for p in parts]).min(dim=0).values.contiguous()
    scal = torch.zeros(F, 2, dtype=torch.float64, device="cuda")
    elem = torch.zeros(F, N, 3, 3, dtype=torch.float64, device="cuda")
    for p in parts:
        sc = torch.empty_like(scal)
        el = torch.empty_like(elem)
        pcv.pcv_shard_pack(prec, F, N, lam, zmin.data_ptr(), p["s"].data_ptr(), p["z"].data_ptr(),
                           p["dsdx"].data_ptr(), p["dzdx"].data_ptr(), sc.data_ptr(), el.data_ptr())
        scal += sc
        elem += el
    s = torch.empty(F, dtype=torch.float64, device="cuda")
    z = torch.empty_like(s)
    gs = torch.empty_like(full["dsdx"])
    gz = torch.empty_like(full["dzdx"])
    pcv.pcv_shard_unpack(prec, F, N, lam, zmin.data_ptr(), scal.data_ptr(), elem.data_ptr(), s.data_ptr(),
                         z.data_ptr(), gs.data_ptr(), gz.data_ptr())
    torch.cuda.synchronize()
    tol, gtol = TOL[precision], GRAD_TOL[precision]
    # against the unsharded context (same arithmetic per landmark) ...
    assert s_err(s.cpu().numpy(), full["s"].cpu().numpy(), M) < tol
    assert z_err(z.cpu().numpy(), full["z"].cpu().numpy(), lam) < tol
    assert grad_err(gs.double().cpu().numpy(), full["dsdx"].double().cpu().numpy()) < gtol
    assert grad_err(gz.double().cpu().numpy(), full["dzdx"].double().cpu().numpy()) < gtol
    # ... and against the oracle
    r = oracle.exact(fr, lm, lam, want_grad=True) if eps is None else oracle.close(fr, lm, lam, eps, want_grad=True)
    assert s_err(s.cpu().numpy(), r["s"], M) < tol
    assert z_err(z.cpu().numpy(), r["z"], lam) < tol
    assert grad_err(gz.double().cpu().numpy(), r["dzdx"]) < gtol
    assert grad_err(gs.double().cpu().numpy(), r["dsdx"]) < gtol

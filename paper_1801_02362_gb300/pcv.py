"""Python binding of the C ABI in include/pcv.h (ctypes; argument marshalling only).

Every computation happens in libpcv.so.  The functions ``pcv_*`` mirror the C entry
points one to one; ``PathCV`` wraps a context for torch device tensors and
``PathCVFunction`` is the autograd.Function whose backward applies the chain rule through
``pcv_combine_grad``.  Loading fails loudly if the library has not been built
(``python -m paper_1801_02362_gb300.build_lib`` or ``__graft_entry__.build()``): there is
no CPU fallback.
"""
from __future__ import annotations

import ctypes
from pathlib import Path

import numpy as np

from . import build_lib

PCV_OK, PCV_EINVAL, PCV_ECUDA, PCV_ENOMEM, PCV_ENOCONV, PCV_ESTATE, PCV_ETIMEOUT = 0, -1, -2, -3, -4, -5, -6
PCV_FP64, PCV_FP32, PCV_FP16_STORAGE = 0, 1, 2
PCV_OPT_BAND, PCV_OPT_CHUNK, PCV_OPT_EXACT_TILE, PCV_OPT_APPROX_TILE, PCV_OPT_PROFILE = 1, 2, 3, 4, 5
PCV_OPT_MATERIALIZE = 6
PCV_OPT_TENSOR_CORES = 7
PCV_OPT_HOST_CHUNKS, PCV_OPT_HOST_END_SHARE = 8, 9
PCV_OPT_NEWTON_CAP, PCV_OPT_WAIT_CYCLES, PCV_OPT_MMA_GROUP = 10, 11, 12
PCV_PROFILE_KERNELS = 25

_STATUS_NAMES = {0: "PCV_OK", -1: "PCV_EINVAL", -2: "PCV_ECUDA", -3: "PCV_ENOMEM", -4: "PCV_ENOCONV",
                 -5: "PCV_ESTATE", -6: "PCV_ETIMEOUT"}


class PcvError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class pcv_batch_io(ctypes.Structure):
    _fields_ = [("F", ctypes.c_int), ("frames", ctypes.c_void_p), ("s", ctypes.c_void_p), ("z", ctypes.c_void_p),
                ("dsdx", ctypes.c_void_p), ("dzdx", ctypes.c_void_p), ("msd", ctypes.c_void_p),
                ("refreshed", ctypes.c_void_p)]


class pcv_stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in ("frames", "xy_alignments", "landmark_alignments", "approx_msds",
                                              "refreshes_threshold", "refreshes_initial", "fp64_rechecks",
                                              "host_syncs", "kernel_launches")]

    def as_dict(self) -> dict:
        return {n: int(getattr(self, n)) for n, _ in self._fields_}


# exported entry points: name -> (restype, argtypes)
_vp, _dp, _i, _d = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int, ctypes.c_double
SIGNATURES = {
    "pcv_create": (_i, [ctypes.POINTER(_vp), _i, _vp, _i]),
    "pcv_destroy": (_i, [_vp]),
    "pcv_set_stream": (_i, [_vp, _vp]),
    "pcv_set_landmarks": (_i, [_vp, _i, _i, _vp, _vp, _vp]),
    "pcv_set_landmarks_weighted": (_i, [_vp, _i, _i, _vp, _vp, _vp, _vp]),
    "pcv_set_lambda": (_i, [_vp, _d]),
    "pcv_set_close_threshold": (_i, [_vp, _d]),
    "pcv_set_neighbor_list": (_i, [_vp, _i, _i]),
    "pcv_evaluate": (_i, [_vp, _i, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "pcv_evaluate_host": (_i, [_vp, _i, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "pcv_host_chunk_plan": (_i, [_i, _i, _i, _vp, _i, _vp]),
    "pcv_combine_grad": (_i, [_vp, _i, _vp, _vp, _vp, _vp, _vp]),
    "pcv_reset_close_state": (_i, [_vp]),
    "pcv_save_state": (_i, [_vp, _vp, ctypes.POINTER(ctypes.c_size_t)]),
    "pcv_load_state": (_i, [_vp, _vp, ctypes.c_size_t]),
    "pcv_get_stats": (_i, [_vp, ctypes.POINTER(pcv_stats)]),
    "pcv_sync": (_i, [_vp]),
    "pcv_set_option": (_i, [_vp, _i, ctypes.c_int64]),
    "pcv_last_error": (ctypes.c_char_p, [_vp]),
    "pcv_get_profile": (_i, [_vp, _i, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)]),
    "pcv_profile_name": (ctypes.c_char_p, [_i]),
    "pcv_evaluate_exact_noalloc": (_i, [_i, _i, _i, _vp, _vp, _vp, _d, _vp, _vp, _vp, _vp, ctypes.c_char_p,
                                       ctypes.c_size_t]),
    "pcv_evaluate_group": (_i, [ctypes.POINTER(_vp), _i, ctypes.POINTER(pcv_batch_io), _vp]),
    "pcv_group_tuning": (_i, [_vp, ctypes.POINTER(_i), ctypes.POINTER(_i), ctypes.POINTER(_i)]),
    "pcv_metad_create": (_i, [ctypes.POINTER(_vp), _i, _vp, _d, _d, _d, _i, _i]),
    "pcv_metad_destroy": (_i, [_vp]),
    "pcv_metad_set_stream": (_i, [_vp, _vp]),
    "pcv_metad_apply": (_i, [_vp, _i, _i, _i, _vp, _vp, _vp, _vp, _vp, _vp]),
    "pcv_metad_get_hills": (_i, [_vp, _vp, _i, ctypes.POINTER(_i), ctypes.POINTER(ctypes.c_int64)]),
    "pcv_metad_set_hills": (_i, [_vp, _vp, _i, ctypes.c_int64]),
    "pcv_metad_last_error": (ctypes.c_char_p, [_vp]),
    "pcv_shard_pack": (_i, [_i, _i, _i, _d, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "pcv_shard_unpack": (_i, [_i, _i, _i, _d, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "pcv_shard_pack_host": (_i, [_i, _i, _i, _d, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "pcv_shard_unpack_host": (_i, [_i, _i, _i, _d, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
}

_lib = None


def library_path() -> Path:
    return build_lib.LIB


def load(path: str | Path | None = None):
    """Load libpcv.so (raises if it is missing: build it first)."""
    global _lib
    if _lib is not None:
        return _lib
    p = Path(path) if path else library_path()
    if not p.exists():
        raise RuntimeError(f"libpcv.so not found at {p}: build it with __graft_entry__.build() "
                           "(the CUDA library is required; there is no fallback)")
    L = ctypes.CDLL(str(p))
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def _check(ctx, st):
    if st != PCV_OK:
        msg = load().pcv_last_error(ctx)
        raise PcvError(st, msg.decode() if msg else "")


# ---- thin wrappers with the C names ------------------------------------------------------
def pcv_create(device: int = 0, stream: int | None = None, precision: int = PCV_FP32):
    h = ctypes.c_void_p()
    st = load().pcv_create(ctypes.byref(h), device, stream, precision)
    _check(None, st)
    return h


def pcv_destroy(ctx):
    load().pcv_destroy(ctx)


def pcv_set_stream(ctx, stream):
    _check(ctx, load().pcv_set_stream(ctx, stream))


def pcv_set_landmarks(ctx, coords: np.ndarray, w: np.ndarray | None = None, q: np.ndarray | None = None):
    coords = np.ascontiguousarray(coords, dtype=np.float64)
    m, n = coords.shape[0], coords.shape[1]
    wp = None if w is None else np.ascontiguousarray(w, dtype=np.float64)
    qp = None if q is None else np.ascontiguousarray(q, dtype=np.float64)
    st = load().pcv_set_landmarks(ctx, m, n, coords.ctypes.data, None if wp is None else wp.ctypes.data,
                                  None if qp is None else qp.ctypes.data)
    _check(ctx, st)


def pcv_set_landmarks_weighted(ctx, coords: np.ndarray, w: np.ndarray | None, w_align: np.ndarray | None,
                               q: np.ndarray | None = None):
    coords = np.ascontiguousarray(coords, dtype=np.float64)
    m, n = coords.shape[0], coords.shape[1]
    arrs = [None if a is None else np.ascontiguousarray(a, dtype=np.float64) for a in (w, w_align, q)]
    st = load().pcv_set_landmarks_weighted(ctx, m, n, coords.ctypes.data,
                                           *[None if a is None else a.ctypes.data for a in arrs])
    _check(ctx, st)


def pcv_set_lambda(ctx, lam: float):
    _check(ctx, load().pcv_set_lambda(ctx, float(lam)))


def pcv_set_close_threshold(ctx, eps: float):
    _check(ctx, load().pcv_set_close_threshold(ctx, float(eps)))


def pcv_set_neighbor_list(ctx, size: int, stride: int):
    _check(ctx, load().pcv_set_neighbor_list(ctx, int(size), int(stride)))


def pcv_set_option(ctx, key: int, value: int):
    _check(ctx, load().pcv_set_option(ctx, key, int(value)))


def pcv_evaluate(ctx, F: int, frames_ptr, s_ptr, z_ptr, dsdx_ptr=None, dzdx_ptr=None, msd_ptr=None,
                 refreshed_ptr=None):
    _check(ctx, load().pcv_evaluate(ctx, F, frames_ptr, s_ptr, z_ptr, dsdx_ptr, dzdx_ptr, msd_ptr, refreshed_ptr))


def pcv_host_chunk_plan(F: int, chunks: int = 0, end_share: int = 25) -> list[int]:
    """Chunk sizes pcv_evaluate_host uses for F frames with these options (host only)."""
    count = ctypes.c_int()
    _check(None, load().pcv_host_chunk_plan(F, chunks, end_share, None, 0, ctypes.byref(count)))
    sizes = (ctypes.c_int * max(count.value, 1))()
    _check(None, load().pcv_host_chunk_plan(F, chunks, end_share, sizes, count.value, ctypes.byref(count)))
    return list(sizes[:count.value])


def pcv_evaluate_host(ctx, F: int, frames_ptr, s_ptr, z_ptr, dsdx_ptr=None, dzdx_ptr=None, msd_ptr=None,
                      refreshed_ptr=None):
    _check(ctx, load().pcv_evaluate_host(ctx, F, frames_ptr, s_ptr, z_ptr, dsdx_ptr, dzdx_ptr, msd_ptr,
                                         refreshed_ptr))


def pcv_combine_grad(ctx, F: int, gs_ptr, gz_ptr, dsdx_ptr, dzdx_ptr, out_ptr):
    _check(ctx, load().pcv_combine_grad(ctx, F, gs_ptr, gz_ptr, dsdx_ptr, dzdx_ptr, out_ptr))


def pcv_reset_close_state(ctx):
    _check(ctx, load().pcv_reset_close_state(ctx))


def pcv_save_state(ctx) -> bytes:
    n = ctypes.c_size_t(0)
    _check(ctx, load().pcv_save_state(ctx, None, ctypes.byref(n)))
    buf = ctypes.create_string_buffer(n.value)
    _check(ctx, load().pcv_save_state(ctx, buf, ctypes.byref(n)))
    return buf.raw[: n.value]


def pcv_load_state(ctx, blob: bytes):
    buf = ctypes.create_string_buffer(blob, len(blob))
    _check(ctx, load().pcv_load_state(ctx, buf, len(blob)))


def pcv_get_stats(ctx) -> dict:
    out = pcv_stats()
    _check(ctx, load().pcv_get_stats(ctx, ctypes.byref(out)))
    return out.as_dict()


def pcv_sync(ctx):
    _check(ctx, load().pcv_sync(ctx))


def pcv_get_profile(ctx) -> dict:
    """{kernel family: (total ms, launches)} collected since the last call."""
    n = PCV_PROFILE_KERNELS
    ms = (ctypes.c_double * n)()
    la = (ctypes.c_int64 * n)()
    _check(ctx, load().pcv_get_profile(ctx, n, ms, la))
    out = {}
    for k in range(n):
        name = load().pcv_profile_name(k).decode()
        if name and la[k]:
            out[name] = (float(ms[k]), int(la[k]))
    return out


def pcv_evaluate_group(ctxs, ios, stream=None):
    """ctxs: context handles; ios: dicts with keys F, frames, s, z and optionally dsdx, dzdx,
    msd, refreshed (device pointers as ints)."""
    n = len(ctxs)
    handles = (_vp * n)(*[c.value if hasattr(c, "value") else c for c in ctxs])
    arr = (pcv_batch_io * n)()
    for k, d in enumerate(ios):
        arr[k].F = int(d["F"])
        for key in ("frames", "s", "z", "dsdx", "dzdx", "msd", "refreshed"):
            setattr(arr[k], key, d.get(key))
    st = load().pcv_evaluate_group(handles, n, arr, stream)
    _check(ctxs[0], st)


def pcv_shard_pack(precision: int, F: int, N: int, lam: float, zmin_ptr, s_ptr, z_ptr, dsdx_ptr, dzdx_ptr,
                   scalars_ptr, elements_ptr, stream=None):
    """Device pointers: shard values -> summable terms (see include/pcv.h)."""
    _check(None, load().pcv_shard_pack(precision, F, N, float(lam), zmin_ptr, s_ptr, z_ptr, dsdx_ptr, dzdx_ptr,
                                       scalars_ptr, elements_ptr, stream))


def pcv_group_tuning(ctx) -> tuple[int, int, int]:
    """(tile frames, tile landmarks, persistent CTAs) the group autotuner chose for the groups
    whose first context is ctx; zeros before any tuned call."""
    tf, tm, b = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(ctx, load().pcv_group_tuning(ctx, ctypes.byref(tf), ctypes.byref(tm), ctypes.byref(b)))
    return tf.value, tm.value, b.value


def pcv_shard_unpack(precision: int, F: int, N: int, lam: float, zmin_ptr, scalars_ptr, elements_ptr, s_ptr,
                     z_ptr, dsdx_ptr, dzdx_ptr, stream=None):
    """Device pointers: summed terms -> whole-path s, z and gradients."""
    _check(None, load().pcv_shard_unpack(precision, F, N, float(lam), zmin_ptr, scalars_ptr, elements_ptr, s_ptr,
                                         z_ptr, dsdx_ptr, dzdx_ptr, stream))


def _np_ptr(a):
    return None if a is None else a.ctypes.data


def pcv_shard_pack_host(lam: float, zmin: np.ndarray, s: np.ndarray, z: np.ndarray, dsdx=None, dzdx=None):
    """Host arrays (FP64 gradients): returns (scalars F x 2, elements F x N x 3 x 3 or None)."""
    F = s.shape[0]
    N = dsdx.shape[1] if dsdx is not None else 1
    zmin, s, z = (np.ascontiguousarray(a, dtype=np.float64) for a in (zmin, s, z))
    g = [None if a is None else np.ascontiguousarray(a, dtype=np.float64) for a in (dsdx, dzdx)]
    scal = np.zeros((F, 2))
    elem = np.zeros((F, N, 3, 3)) if g[0] is not None else None
    _check(None, load().pcv_shard_pack_host(PCV_FP64, F, N, float(lam), _np_ptr(zmin), _np_ptr(s), _np_ptr(z),
                                            _np_ptr(g[0]), _np_ptr(g[1]), _np_ptr(scal), _np_ptr(elem)))
    return scal, elem


def pcv_shard_unpack_host(lam: float, zmin: np.ndarray, scalars: np.ndarray, elements=None):
    """Host arrays: summed terms -> (s, z, dsdx, dzdx) with FP64 gradients (None without elements)."""
    F = scalars.shape[0]
    zmin = np.ascontiguousarray(zmin, dtype=np.float64)
    scalars = np.ascontiguousarray(scalars, dtype=np.float64)
    s, z = np.zeros(F), np.zeros(F)
    gs = gz = None
    N = 1
    if elements is not None:
        elements = np.ascontiguousarray(elements, dtype=np.float64)
        N = elements.shape[1]
        gs, gz = np.zeros((F, N, 3)), np.zeros((F, N, 3))
    _check(None, load().pcv_shard_unpack_host(PCV_FP64, F, N, float(lam), _np_ptr(zmin), _np_ptr(scalars),
                                              _np_ptr(elements), _np_ptr(s), _np_ptr(z), _np_ptr(gs), _np_ptr(gz)))
    return s, z, gs, gz


def _check_metad(m, st):
    if st != PCV_OK:
        msg = load().pcv_metad_last_error(m)
        raise PcvError(st, msg.decode() if msg else "")


def pcv_metad_create(device: int, stream, height: float, sigma_s: float, sigma_z: float, stride: int,
                     max_hills: int):
    h = ctypes.c_void_p()
    _check_metad(None, load().pcv_metad_create(ctypes.byref(h), device, stream, float(height), float(sigma_s),
                                               float(sigma_z), int(stride), int(max_hills)))
    return h


def pcv_metad_destroy(m):
    load().pcv_metad_destroy(m)


def pcv_metad_set_stream(m, stream):
    _check_metad(m, load().pcv_metad_set_stream(m, stream))


def pcv_metad_apply(m, precision: int, F: int, N: int, s_ptr, z_ptr, dsdx_ptr, dzdx_ptr, bias_ptr, force_ptr):
    _check_metad(m, load().pcv_metad_apply(m, precision, F, N, s_ptr, z_ptr, dsdx_ptr, dzdx_ptr, bias_ptr,
                                           force_ptr))


def pcv_metad_get_hills(m):
    """(hills as an (n, 2) array, step count)"""
    n = ctypes.c_int(0)
    steps = ctypes.c_int64(0)
    _check_metad(m, load().pcv_metad_get_hills(m, None, 0, ctypes.byref(n), ctypes.byref(steps)))
    out = np.zeros((max(n.value, 1), 2))
    _check_metad(m, load().pcv_metad_get_hills(m, out.ctypes.data, n.value, ctypes.byref(n), ctypes.byref(steps)))
    return out[:n.value], int(steps.value)


def pcv_metad_set_hills(m, hills: np.ndarray, steps: int):
    h = np.ascontiguousarray(np.asarray(hills, dtype=np.float64).reshape(-1, 2))
    _check_metad(m, load().pcv_metad_set_hills(m, h.ctypes.data if h.size else None, h.shape[0], int(steps)))


def pcv_last_error(ctx) -> str:
    m = load().pcv_last_error(ctx)
    return m.decode() if m else ""


# ---- torch convenience layer ---------------------------------------------------------------
_PREC = {"fp64": PCV_FP64, "fp32": PCV_FP32, "fp16": PCV_FP16_STORAGE}


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


class PathCV:
    """A library context bound to one CUDA device and the current torch stream.

    frames are torch CUDA tensors (F, N, 3): float64 in 'fp64' mode, float32 otherwise.
    """

    def __init__(self, landmarks: np.ndarray, lam: float, eps: float = -1.0, precision: str = "fp32",
                 weights: np.ndarray | None = None, props: np.ndarray | None = None, device: int = 0,
                 band: int | None = None, min_chunk: int | None = None, materialize: int | None = None,
                 tensor_cores: bool | None = None, neighbor_list: tuple[int, int] | None = None,
                 align_weights: np.ndarray | None = None):
        import torch

        self.torch = torch
        self.precision = precision
        self.device = torch.device("cuda", device)
        stream = torch.cuda.current_stream(self.device).cuda_stream
        self.ctx = pcv_create(device, stream, _PREC[precision])
        self.M, self.N = landmarks.shape[0], landmarks.shape[1]
        if align_weights is None:
            pcv_set_landmarks(self.ctx, landmarks, weights, props)
        else:
            pcv_set_landmarks_weighted(self.ctx, landmarks, weights, align_weights, props)
        pcv_set_lambda(self.ctx, lam)
        pcv_set_close_threshold(self.ctx, eps)
        if band is not None:
            pcv_set_option(self.ctx, PCV_OPT_BAND, band)
        if min_chunk is not None:
            pcv_set_option(self.ctx, PCV_OPT_CHUNK, min_chunk)
        if materialize is not None:
            pcv_set_option(self.ctx, PCV_OPT_MATERIALIZE, materialize)
        if tensor_cores is not None:
            pcv_set_option(self.ctx, PCV_OPT_TENSOR_CORES, 1 if tensor_cores else 0)
        if neighbor_list is not None:
            pcv_set_neighbor_list(self.ctx, *neighbor_list)

    @property
    def frame_dtype(self):
        return self.torch.float64 if self.precision == "fp64" else self.torch.float32

    def close(self):
        if getattr(self, "ctx", None):
            pcv_destroy(self.ctx)
            self.ctx = None

    __del__ = close

    def _bind_stream(self):
        pcv_set_stream(self.ctx, self.torch.cuda.current_stream(self.device).cuda_stream)

    def evaluate(self, frames, grad: bool = False, msd: bool = False, refreshed: bool = False) -> dict:
        torch = self.torch
        if frames.dtype != self.frame_dtype or not frames.is_cuda or not frames.is_contiguous():
            raise ValueError(f"frames must be a contiguous CUDA tensor of {self.frame_dtype}")
        F = frames.shape[0]
        dev = frames.device
        out = {"s": torch.empty(F, dtype=torch.float64, device=dev), "z": torch.empty(F, dtype=torch.float64, device=dev)}
        if grad:
            out["dsdx"] = torch.empty_like(frames)
            out["dzdx"] = torch.empty_like(frames)
        if msd:
            out["msd"] = torch.empty((F, self.M), dtype=torch.float64, device=dev)
        if refreshed:
            out["refreshed"] = torch.empty(F, dtype=torch.uint8, device=dev)
        self._bind_stream()
        pcv_evaluate(self.ctx, F, _ptr(frames), _ptr(out["s"]), _ptr(out["z"]), _ptr(out.get("dsdx")),
                     _ptr(out.get("dzdx")), _ptr(out.get("msd")), _ptr(out.get("refreshed")))
        return out

    def combine_grad(self, g_s, g_z, dsdx, dzdx):
        out = self.torch.empty_like(dsdx)
        self._bind_stream()
        pcv_combine_grad(self.ctx, dsdx.shape[0], _ptr(g_s), _ptr(g_z), _ptr(dsdx), _ptr(dzdx), _ptr(out))
        return out

    def stats(self) -> dict:
        return pcv_get_stats(self.ctx)

    def set_profiling(self, on: bool):
        pcv_set_option(self.ctx, PCV_OPT_PROFILE, 1 if on else 0)

    def profile(self) -> dict:
        return pcv_get_profile(self.ctx)

    def sync(self):
        pcv_sync(self.ctx)

    def reset(self):
        pcv_reset_close_state(self.ctx)

    def set_neighbor_list(self, size: int, stride: int):
        """Keep the `size` closest landmarks, updated every `stride` steps (0: all landmarks)."""
        pcv_set_neighbor_list(self.ctx, size, stride)

    def save_state(self) -> bytes:
        return pcv_save_state(self.ctx)

    def load_state(self, blob: bytes):
        pcv_load_state(self.ctx, blob)


class Metad:
    """Gaussian-hill metadynamics bias on (s, z) (pcv_metad_*) bound to a CUDA device and the
    current torch stream."""

    def __init__(self, height: float, sigma_s: float, sigma_z: float, stride: int, max_hills: int = 100_000,
                 device: int = 0):
        import torch

        self.torch = torch
        self.device = torch.device("cuda", device)
        self.m = pcv_metad_create(device, torch.cuda.current_stream(self.device).cuda_stream, height, sigma_s,
                                  sigma_z, stride, max_hills)

    def close(self):
        if getattr(self, "m", None):
            pcv_metad_destroy(self.m)
            self.m = None

    __del__ = close

    def apply(self, s, z, dsdx=None, dzdx=None, precision: str = "fp32") -> dict:
        """bias (F doubles) and, with dsdx / dzdx, the force -dV/dx (same shape and type)."""
        torch = self.torch
        F = s.shape[0]
        out = {"bias": torch.empty(F, dtype=torch.float64, device=s.device)}
        N = 0
        if dsdx is not None:
            out["force"] = torch.empty_like(dsdx)
            N = dsdx.shape[1]
        pcv_metad_set_stream(self.m, torch.cuda.current_stream(self.device).cuda_stream)
        pcv_metad_apply(self.m, _PREC[precision], F, N, _ptr(s), _ptr(z), _ptr(dsdx), _ptr(dzdx), _ptr(out["bias"]),
                        _ptr(out.get("force")))
        return out

    def hills(self):
        return pcv_metad_get_hills(self.m)

    def set_hills(self, hills, steps: int):
        pcv_metad_set_hills(self.m, hills, steps)


def _make_function():
    import torch

    class PathCVFunction(torch.autograd.Function):
        """(s, z) = PathCVFunction.apply(frames, pathcv): the forward evaluates s, z and
        their coordinate derivatives in the library; the backward forms
        g_s * ds/dx + g_z * dz/dx in the library."""

        @staticmethod
        def forward(ctx, frames, pathcv):
            r = pathcv.evaluate(frames.contiguous(), grad=True)
            ctx.pathcv = pathcv
            ctx.save_for_backward(r["dsdx"], r["dzdx"])
            return r["s"], r["z"]

        @staticmethod
        def backward(ctx, g_s, g_z):
            dsdx, dzdx = ctx.saved_tensors
            g_s = None if g_s is None else g_s.contiguous().to(torch.float64)
            g_z = None if g_z is None else g_z.contiguous().to(torch.float64)
            return ctx.pathcv.combine_grad(g_s, g_z, dsdx, dzdx), None

    return PathCVFunction


_function = None


def path_cv(frames, pathcv: PathCV):
    """Differentiable (s, z) of a batch of frames."""
    global _function
    if _function is None:
        _function = _make_function()
    return _function.apply(frames, pathcv)

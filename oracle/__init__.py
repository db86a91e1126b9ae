"""FP64 CPU oracle for the path-CV / MSD hot path (plain C, loaded through ctypes).

TEST INFRASTRUCTURE ONLY: tests/, ``__graft_entry__.smoke()`` and the CPU-baseline /
reference legs of ``bench.py`` are the only users.  The CUDA library never imports or
links this package, and this package never touches the CUDA library.

See ``pcv_oracle.c`` for the paper passages each routine follows.  ``build()`` compiles
the C source with gcc (OpenMP over frames in exact mode, over landmarks and atoms within a
frame; the results do not depend on the thread count).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_SRC = _HERE / "pcv_oracle.c"
_BUILD = _HERE / "_build"
_LIB_PATH = _BUILD / "liborc.so"
_lib = None

ALIGN_FIELDS = 47  # length of the flat record written by orc_align_flat


def build(force: bool = False) -> Path:
    """Compile the oracle with gcc (-O2, IEEE semantics, OpenMP)."""
    _BUILD.mkdir(exist_ok=True)
    if force or not _LIB_PATH.exists() or _LIB_PATH.stat().st_mtime < _SRC.stat().st_mtime:
        tmp = _BUILD / f"liborc.{os.getpid()}.so"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-fno-fast-math",
               "-ffp-contract=off", str(_SRC), "-o", str(tmp), "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(str(_LIB_PATH))
        dp = ctypes.POINTER(ctypes.c_double)
        i64p = ctypes.POINTER(ctypes.c_int64)
        u8p = ctypes.POINTER(ctypes.c_uint8)
        c_int, c_double = ctypes.c_int, ctypes.c_double
        L.orc_align_flat.argtypes = [c_int, dp, dp, dp, dp]
        L.orc_jacobi4.argtypes = [dp, dp, dp]
        L.orc_quat_matrix.argtypes = [dp, dp]
        L.orc_quat_to_rot.argtypes = [dp, dp]
        L.orc_path_cv.argtypes = [c_int, dp, dp, c_double, dp, dp, dp]
        L.orc_exact.argtypes = [c_int, c_int, c_int, dp, dp, dp, dp, dp, c_double, dp, dp, dp, dp, dp]
        i32p = ctypes.POINTER(ctypes.c_int32)
        L.orc_close.argtypes = [c_int, c_int, c_int, dp, dp, dp, dp, dp, c_double, c_double, dp, dp,
                                c_int, c_int, i32p, i64p, dp, dp, dp, u8p, dp, dp, dp, dp]
        L.orc_exact_nl.argtypes = [c_int, c_int, c_int, dp, dp, dp, dp, dp, c_double, c_int, c_int, i32p, i64p,
                                   dp, dp, dp, dp, dp]
        L.orc_nl_select.argtypes = [c_int, dp, c_int, i32p]
        L.orc_hills_value.argtypes = [c_int, dp, c_double, c_double, c_double, c_double, c_double, dp, dp, dp]
        L.orc_metad.argtypes = [c_int, c_int, dp, dp, dp, dp, c_double, c_double, c_double, c_int, c_int, dp, i64p,
                                dp, dp]
        L.orc_close_distance.argtypes = [c_int, dp, dp, dp, dp, dp, dp]
        L.orc_close_distance.restype = c_double
        for name in ("orc_cost_original", "orc_cost_close", "orc_amdahl"):
            getattr(L, name).argtypes = [c_double] * (3 if name == "orc_cost_original" else 2)
            getattr(L, name).restype = c_double
        L.orc_threads.restype = c_int
        L.orc_set_threads.argtypes = [c_int]
        _lib = L
    return _lib


def threads() -> int:
    """Threads the oracle's OpenMP loops use."""
    return int(lib().orc_threads())


def set_threads(n: int) -> None:
    """Set the oracle's OpenMP thread count (the results do not depend on it)."""
    lib().orc_set_threads(int(n))


def _p(a, ctype=ctypes.c_double):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


# --------------------------------------------------------------------------------------
def align(x, a, w=None) -> dict:
    """Optimal superposition of a onto x (uncentred inputs).  Returns D (direct form),
    D_formula, Gx, Ga, R (fits a onto x), q, evals, evecs, H, sweeps."""
    x, a = _f64(x), _f64(a)
    n = x.shape[0]
    w = np.full(n, 1.0 / n) if w is None else _f64(w) / np.sum(w)
    out = np.zeros(ALIGN_FIELDS)
    st = lib().orc_align_flat(n, _p(w), _p(x), _p(a), _p(out))
    return dict(D=out[0], D_formula=out[1], Gx=out[2], Ga=out[3], R=out[4:13].reshape(3, 3),
                q=out[13:17].copy(), evals=out[17:21].copy(), evecs=out[21:37].reshape(4, 4),
                H=out[37:46].reshape(3, 3), sweeps=int(out[46]), status=st)


def quat_matrix(H):
    H = _f64(H).reshape(9)
    K = np.zeros(16)
    lib().orc_quat_matrix(_p(H), _p(K))
    return K.reshape(4, 4)


def quat_to_rot(q):
    q = _f64(q)
    R = np.zeros(9)
    lib().orc_quat_to_rot(_p(q), _p(R))
    return R.reshape(3, 3)


def jacobi4(K):
    K = _f64(K).reshape(16)
    ev = np.zeros(4)
    V = np.zeros(16)
    sweeps = lib().orc_jacobi4(_p(K), _p(ev), _p(V))
    return ev, V.reshape(4, 4), sweeps


def path_cv(D, lam, q=None):
    D = _f64(D)
    m = D.shape[0]
    q = np.arange(1, m + 1, dtype=np.float64) if q is None else _f64(q)
    s = np.zeros(1)
    z = np.zeros(1)
    p = np.zeros(m)
    lib().orc_path_cv(m, _p(D), _p(q), float(lam), _p(s), _p(z), _p(p))
    return s[0], z[0], p


def exact(frames, landmarks, lam, w=None, q=None, want_D=True, want_grad=False, nl=None, state=None, wa=None):
    """Exact path CVs (Algorithm 1) for F frames.

    w: displacement weights, wa: alignment weights (centres; default w), Section 3.1.

    nl = (M_nl, L): neighbour list of the original method (distances to all landmarks
    every L steps, to the M_nl closest of the last such step otherwise; frames in time
    order, state carried in ``state``, a CloseState).  D of unlisted landmarks is +inf."""
    fr, lm = _f64(frames), _f64(landmarks)
    f, n = fr.shape[0], fr.shape[1]
    m = lm.shape[0]
    s = np.zeros(f)
    z = np.zeros(f)
    D = np.zeros((f, m)) if want_D else None
    gs = np.zeros((f, n, 3)) if want_grad else None
    gz = np.zeros((f, n, 3)) if want_grad else None
    if nl is None:
        st = lib().orc_exact(f, m, n, _p(_f64(w)), _p(_f64(wa)), _p(fr), _p(lm), _p(_f64(q)), float(lam), _p(s),
                             _p(z), _p(D), _p(gs), _p(gz))
    else:
        if state is None:
            state = CloseState(n, m)
        st = lib().orc_exact_nl(f, m, n, _p(_f64(w)), _p(_f64(wa)), _p(fr), _p(lm), _p(_f64(q)), float(lam),
                                int(nl[0]),
                                int(nl[1]), _p(state.nl, ctypes.c_int32), _p(state.ctr, ctypes.c_int64), _p(s),
                                _p(z), _p(D), _p(gs), _p(gz))
    if st != 0:
        raise RuntimeError(f"oracle exact: status {st}")
    return dict(s=s, z=z, D=D, dsdx=gs, dzdx=gz, state=state)


def nl_select(D, m_nl):
    """The m_nl landmarks with the smallest D (ties to the lower index), in index order."""
    D = _f64(D)
    out = np.zeros(m_nl, dtype=np.int32)
    lib().orc_nl_select(D.shape[0], _p(D), int(m_nl), _p(out, ctypes.c_int32))
    return out


class CloseState:
    """Close-structure state (Algorithm 2) and neighbour list carried across calls."""

    def __init__(self, n_atoms: int, n_landmarks: int):
        self.y = np.zeros((n_atoms, 3))
        self.B = np.zeros((n_landmarks, 3, 3))
        self.ctr = np.zeros(8, dtype=np.int64)
        self.nl = np.zeros(n_landmarks, dtype=np.int32)

    @property
    def counters(self) -> dict:
        c = self.ctr
        return dict(has_y=int(c[0]), frames=int(c[1]), xy_alignments=int(c[2]),
                    landmark_alignments=int(c[3]), approx_msds=int(c[4]),
                    refreshes_threshold=int(c[5]), refreshes_initial=int(c[6]), has_nl=int(c[7]))

    def copy(self) -> "CloseState":
        o = CloseState(self.y.shape[0], self.B.shape[0])
        o.y[:] = self.y
        o.B[:] = self.B
        o.ctr[:] = self.ctr
        o.nl[:] = self.nl
        return o


def close(frames, landmarks, lam, eps, state: CloseState | None = None, w=None, q=None,
          want_D=True, want_grad=False, nl=None, wa=None, D_in=None):
    """Floating close structure (Algorithm 2) over F time-ordered frames.

    nl = (M_nl, L): neighbour list chosen at reassignments (exact distances) and every L
    steps (approximate distances), used in between.  D of unlisted landmarks is +inf.
    D_in (F x M, NaN = the oracle's own): distances at which s, z and the derivative
    weights are formed instead of the oracle's (the geometry stays the oracle's)."""
    fr, lm = _f64(frames), _f64(landmarks)
    f, n = fr.shape[0], fr.shape[1]
    m = lm.shape[0]
    if state is None:
        state = CloseState(n, m)
    m_nl, stride = (0, 1) if nl is None else (int(nl[0]), int(nl[1]))
    s = np.zeros(f)
    z = np.zeros(f)
    D = np.zeros((f, m)) if want_D else None
    ref = np.zeros(f, dtype=np.uint8)
    dxy = np.zeros(f)
    gs = np.zeros((f, n, 3)) if want_grad else None
    gz = np.zeros((f, n, 3)) if want_grad else None
    st = lib().orc_close(f, m, n, _p(_f64(w)), _p(_f64(wa)), _p(fr), _p(lm), _p(_f64(q)), float(lam), float(eps),
                         _p(state.y), _p(state.B), m_nl, stride, _p(state.nl, ctypes.c_int32),
                         _p(state.ctr, ctypes.c_int64), _p(s), _p(z), _p(D), _p(ref, ctypes.c_uint8), _p(dxy),
                         _p(gs), _p(gz), _p(_f64(D_in)))
    if st != 0:
        raise RuntimeError(f"oracle close: status {st}")
    return dict(s=s, z=z, D=D, refreshed=ref, dxy=dxy, dsdx=gs, dzdx=gz, state=state)


def hills_value(hills, w, sigma_s, sigma_z, s, z):
    """V, dV/ds, dV/dz of the Gaussian-hill bias (Eq. vbias) at (s, z)."""
    h = np.ascontiguousarray(np.asarray(hills, dtype=np.float64).reshape(-1, 2))
    out = np.zeros(3)
    lib().orc_hills_value(h.shape[0], _p(h), float(w), float(sigma_s), float(sigma_z), float(s), float(z),
                          _p(out[0:1]), _p(out[1:2]), _p(out[2:3]))
    return out[0], out[1], out[2]


class MetadState:
    """Hills deposited so far and the step count of a metadynamics run (Eq. vbias)."""

    def __init__(self, cap: int = 4096):
        self.hills = np.zeros((cap, 2))
        self.state = np.zeros(2, dtype=np.int64)

    @property
    def n_hills(self) -> int:
        return int(self.state[0])


def metad(s, z, w, sigma_s, sigma_z, stride, state: MetadState | None = None, dsdx=None, dzdx=None):
    """Bias V of each frame (hills of earlier steps) and force -dV/dx; after frame t is
    evaluated a hill is deposited at (s_t, z_t) when the step index t (counted from 0 across
    calls) is a positive multiple of `stride`: Eq. (vbias) sums over t' = tau_G, 2 tau_G, ..."""
    s, z = _f64(s), _f64(z)
    f = s.shape[0]
    if state is None:
        state = MetadState()
    n = 0 if dsdx is None else dsdx.shape[1]
    V = np.zeros(f)
    force = np.zeros((f, n, 3)) if dsdx is not None else None
    st = lib().orc_metad(f, n, _p(s), _p(z), _p(_f64(dsdx)), _p(_f64(dzdx)), float(w), float(sigma_s),
                         float(sigma_z), int(stride), state.hills.shape[0], _p(state.hills),
                         _p(state.state, ctypes.c_int64), _p(V), _p(force))
    if st != 0:
        raise RuntimeError(f"oracle metad: status {st}")
    return dict(V=V, force=force, state=state)


def close_distance(x, y, B, a, w=None, wa=None):
    x, y, a = _f64(x), _f64(y), _f64(a)
    B = _f64(B).reshape(9)
    n = x.shape[0]
    return lib().orc_close_distance(n, _p(_f64(w)), _p(_f64(wa)), _p(x), _p(y), _p(B), _p(a))


def cost_original(m_nl, n_ref, l_stride):
    return lib().orc_cost_original(float(m_nl), float(n_ref), float(l_stride))


def cost_close(n_ref, k_interval):
    return lib().orc_cost_close(float(n_ref), float(k_interval))


def amdahl(p, s):
    return lib().orc_amdahl(float(p), float(s))


def mean_adjacent_msd(landmarks, w=None) -> float:
    """Mean D(a_k, a_{k+1}) over adjacent landmarks; the workloads set lambda = 2.3 / this."""
    lm = _f64(landmarks)
    vals = [align(lm[k + 1], lm[k], w)["D"] for k in range(lm.shape[0] - 1)]
    return float(np.mean(vals))

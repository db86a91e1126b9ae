"""Seeded synthetic inputs: landmark paths and MD-like frame batches.

This module only draws random numbers and moves coordinates around rigidly.  It holds
none of the method's arithmetic (no centring, no superposition, no distances), so the
CUDA path and the FP64 oracle can both consume its output without sharing any
computation.

Recipe (stand-ins for the paper's cyclooctane / Trp-cage landmark sets and trajectories,
which are not available; Section "Computational Details"):

* chains: self-avoiding 3-D random walks, bond 0.15 nm, uniformly random bond
  directions; a step is rejected if it comes closer than 0.12 nm to any earlier
  non-bonded atom (100 retries, then the chain restarts);
* landmarks: a_k = (1 - t_k) A + t_k B + N(0, sigma_L) per coordinate, with
  t_k = (k - 1)/(M - 1), then a uniform random rotation and a translation drawn
  from U[-5, 5] nm per axis;
* frames: the same interpolation at a path position p_t in [1, M], frame noise
  N(0, sigma_F) per coordinate (optionally Ornstein-Uhlenbeck correlated in time),
  then a fresh random rigid motion per frame.

All arrays are float64; callers round them to the storage type of the precision mode
(``round_to``) before either side sees them.
"""
from __future__ import annotations

import numpy as np

BOND_NM = 0.15
MIN_NONBONDED_NM = 0.12


def saw_chain(rng: np.random.Generator, n_atoms: int, bond: float = BOND_NM,
              min_dist: float = MIN_NONBONDED_NM, retries: int = 100) -> np.ndarray:
    """Self-avoiding random walk of ``n_atoms`` atoms starting at the origin (N x 3)."""
    while True:
        pos = np.zeros((n_atoms, 3))
        ok = True
        for j in range(1, n_atoms):
            placed = False
            for _ in range(retries):
                d = rng.normal(size=3)
                d *= bond / np.linalg.norm(d)
                cand = pos[j - 1] + d
                if j >= 2:
                    diff = pos[: j - 1] - cand
                    if np.min(np.einsum("ij,ij->i", diff, diff)) < min_dist * min_dist:
                        continue
                pos[j] = cand
                placed = True
                break
            if not placed:
                ok = False
                break
        if ok:
            return pos


def random_rotation(rng: np.random.Generator, n: int | None = None) -> np.ndarray:
    """Uniform random rotation matrices from normalised Gaussian quaternions."""
    shape = (1 if n is None else n, 4)
    q = rng.normal(size=shape)
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q.T
    rot = np.empty((shape[0], 3, 3))
    rot[:, 0, 0] = 1 - 2 * (y * y + z * z)
    rot[:, 0, 1] = 2 * (x * y - w * z)
    rot[:, 0, 2] = 2 * (x * z + w * y)
    rot[:, 1, 0] = 2 * (x * y + w * z)
    rot[:, 1, 1] = 1 - 2 * (x * x + z * z)
    rot[:, 1, 2] = 2 * (y * z - w * x)
    rot[:, 2, 0] = 2 * (x * z - w * y)
    rot[:, 2, 1] = 2 * (y * z + w * x)
    rot[:, 2, 2] = 1 - 2 * (x * x + y * y)
    return rot[0] if n is None else rot


def rigid_motion(rng: np.random.Generator, coords: np.ndarray, box: float = 5.0) -> np.ndarray:
    """Apply an independent random rotation + translation U[-box, box] to each structure
    of a (S, N, 3) stack."""
    s = coords.shape[0]
    rot = random_rotation(rng, s)
    shift = rng.uniform(-box, box, size=(s, 1, 3))
    return np.einsum("sab,snb->sna", rot, coords) + shift


class PathModel:
    """Two end chains A and B; structures along the path are linear interpolations."""

    def __init__(self, rng: np.random.Generator, n_atoms: int):
        self.n_atoms = n_atoms
        self.A = saw_chain(rng, n_atoms)
        self.B = saw_chain(rng, n_atoms)

    def at(self, t: np.ndarray) -> np.ndarray:
        t = np.asarray(t, dtype=np.float64).reshape(-1, 1, 1)
        return (1.0 - t) * self.A[None] + t * self.B[None]


def make_landmarks(rng: np.random.Generator, path: PathModel, n_landmarks: int,
                   noise: float = 0.02) -> np.ndarray:
    """M landmark structures (M x N x 3) along the path, noisy and rigidly moved."""
    m = n_landmarks
    t = np.zeros(1) if m == 1 else np.arange(m) / (m - 1)
    lm = path.at(t) + rng.normal(scale=noise, size=(m, path.n_atoms, 3))
    return rigid_motion(rng, lm)


def positions_drift(n_frames: int, n_landmarks: int) -> np.ndarray:
    """Monotone drift p_t = 1 + (M - 1) t / (F - 1) along the path."""
    if n_frames == 1:
        return np.ones(1)
    return 1.0 + (n_landmarks - 1) * np.arange(n_frames) / (n_frames - 1)


def positions_reflecting_walk(rng: np.random.Generator, n_frames: int, n_landmarks: int,
                              step: float = 0.1) -> np.ndarray:
    """Reflecting random walk on [1, M] with N(0, step) increments (in landmark units)."""
    lo, hi = 1.0, float(n_landmarks)
    p = np.empty(n_frames)
    cur = rng.uniform(lo, hi)
    for t in range(n_frames):
        p[t] = cur
        cur += rng.normal(scale=step)
        width = hi - lo
        if width <= 0:
            cur = lo
            continue
        # reflect into [lo, hi]
        u = (cur - lo) % (2 * width)
        cur = lo + (u if u <= width else 2 * width - u)
    return p


def make_frames(rng: np.random.Generator, path: PathModel, positions: np.ndarray,
                n_landmarks: int, noise: float, ou_rho: float = 0.0) -> np.ndarray:
    """Frames (F x N x 3) at path positions ``positions`` (landmark units, 1..M).

    ``ou_rho`` > 0 makes the frame noise an Ornstein-Uhlenbeck sequence in time
    (correlation ``ou_rho`` between consecutive frames, same stationary variance),
    the smooth-MD regime where close-structure refreshes are rare.
    """
    f = positions.shape[0]
    m = n_landmarks
    t = (positions - 1.0) / max(m - 1, 1)
    base = path.at(t)
    if ou_rho <= 0.0:
        eta = rng.normal(scale=noise, size=base.shape)
    else:
        eta = np.empty_like(base)
        cur = rng.normal(scale=noise, size=base.shape[1:])
        kick = np.sqrt(1.0 - ou_rho * ou_rho) * noise
        for k in range(f):
            eta[k] = cur
            cur = ou_rho * cur + rng.normal(scale=kick, size=cur.shape)
    return rigid_motion(rng, base + eta)


def round_to(arr: np.ndarray, dtype) -> np.ndarray:
    """Round to the storage type and hand back float64 holding the rounded values."""
    return np.asarray(arr).astype(dtype).astype(np.float64)


# Named workloads: sizes of the five configurations the library is measured on.
WORKLOADS = {
    "c1_exact_fp64": dict(n_atoms=22, n_landmarks=20, n_frames=1000, frame_noise=0.02,
                          schedule="walk", dtype="float64"),
    "c2_close_fp32": dict(n_atoms=300, n_landmarks=200, n_frames=100_000, frame_noise=0.05,
                          schedule="drift", dtype="float32"),
    "c4_grad_fp32": dict(n_atoms=1000, n_landmarks=500, n_frames=4096, frame_noise=0.05,
                         schedule="drift", dtype="float32"),
    "c5_large_fp16": dict(n_atoms=5000, n_landmarks=2000, n_frames=10_000, frame_noise=0.05,
                          schedule="drift", dtype="float16"),
}


def make_problem(seed: int, n_atoms: int, n_landmarks: int, n_frames: int,
                 frame_noise: float = 0.05, landmark_noise: float = 0.02,
                 schedule: str = "drift", ou_rho: float = 0.0, frame_dtype=np.float32,
                 landmark_dtype=np.float32):
    """Landmarks (M x N x 3) and frames (F x N x 3) as float64 arrays holding values
    already rounded to the given storage types."""
    rng = np.random.default_rng(seed)
    path = PathModel(rng, n_atoms)
    lm = make_landmarks(rng, path, n_landmarks, noise=landmark_noise)
    if schedule == "drift":
        pos = positions_drift(n_frames, n_landmarks)
    elif schedule == "walk":
        pos = positions_reflecting_walk(rng, n_frames, n_landmarks)
    else:
        raise ValueError(schedule)
    fr = make_frames(rng, path, pos, n_landmarks, frame_noise, ou_rho=ou_rho)
    return round_to(lm, landmark_dtype), round_to(fr, frame_dtype)

"""Shared test helpers: seeded problems (from synth) and the error metrics.

Metrics (readings of the required accuracy):
  D: |D_gpu - D_ref| / max(D_ref, 1e-3 (G_x + G_a))   -- FP32 inputs cannot support a
     relative accuracy finer than ~eps32 (G_x + G_a) / D on the cancelling form;
  s: |s_gpu - s_ref| / max(|s_ref|, 1)  (s >= 1 with q_i = i, so this is |ds| / s);
  z: |z_gpu - z_ref| / max(|z_ref|, 1/lambda);
  gradients: max_k |g_gpu - g_ref| / max_k |g_ref| per frame.
Tolerances: FP64 mode 1e-9, FP32 1e-5, FP16 storage 1e-3 (gradients: FP64 1e-8,
FP32 2e-4, FP16 2e-2: the FP32 rounding of the softmax weights p_i with lambda ~ 1e3 nm^-2
and the cancellation in x_k - sum_i p_i R_i a_ik, |x| / |x - U| ~ 20, give ~1e-5 relative
in FP32).
"""
from __future__ import annotations

import numpy as np

import oracle
from paper_1801_02362_gb300 import synth

TOL = {"fp64": 1e-9, "fp32": 1e-5, "fp16": 1e-3}
GRAD_TOL = {"fp64": 1e-8, "fp32": 2e-4, "fp16": 2e-2}
# the adjoint alone, at the GPU's own distances: FP32 rounding of the terms gamma_i dD_i/dx
# and of their sums, amplified by the cancellation of sum_i p_i (q_i - s) dD_i/dx (ten-fold at
# the end of a 2000-landmark path).  A shift of s by its FP32 rounding (6e-5 at s ~ 2000)
# moves every gamma^s_i and alone gives ~1e-4 there.
ADJ_TOL = {"fp64": 1e-9, "fp32": 5e-5, "fp16": 2e-2}


def problem(seed, n, m, f, noise=0.05, schedule="drift", precision="fp32", ou_rho=0.0, lnoise=0.02):
    fdt = np.float64 if precision == "fp64" else np.float32
    lm, fr = synth.make_problem(seed, n_atoms=n, n_landmarks=m, n_frames=f, frame_noise=noise,
                                landmark_noise=lnoise, schedule=schedule, ou_rho=ou_rho, frame_dtype=fdt,
                                landmark_dtype=fdt)
    lam = 2.3 / oracle.mean_adjacent_msd(lm)
    return lm, fr, lam


def gsum(coords, w=None):
    """G = sum_j w_j |c_j - centre|^2 for each structure of a (S, N, 3) stack."""
    n = coords.shape[1]
    w = np.full(n, 1.0 / n) if w is None else w / w.sum()
    c = np.einsum("j,sjk->sk", w, coords)
    d = coords - c[:, None, :]
    return np.einsum("j,sjk,sjk->s", w, d, d)


def d_err(D_gpu, D_ref, frames, landmarks, w=None):
    gx = gsum(frames, w)[:, None]
    ga = gsum(landmarks, w)[None, :]
    return np.max(np.abs(D_gpu - D_ref) / np.maximum(D_ref, 1e-3 * (gx + ga)))


def s_err(s_gpu, s_ref, m=None, kappa=None):
    """Relative error of s per frame, |s_gpu - s_ref| / max(|s_ref|, 1) (m, the landmark
    count, is accepted for the callers' convenience and not used).  kappa (per frame, optional)
    divides the error by 1 + kappa: the first-order condition number of s with respect to
    relative changes of the D_i (s_kappa), for storage whose rounding moves every D by up to
    the D tolerance itself."""
    s_gpu = np.asarray(s_gpu, dtype=np.float64)
    s_ref = np.asarray(s_ref, dtype=np.float64)
    if s_ref.size == 0:
        return 0.0
    den = np.maximum(np.abs(s_ref), 1.0)
    if kappa is not None:
        den = den * (1.0 + np.asarray(kappa))
    return float(np.max(np.abs(s_gpu - s_ref) / den))


def s_kappa(D_ref, lam, frames, landmarks, w=None):
    """First-order condition number of s = sum_i i p_i (p = softmax(-lam D)) with respect to
    relative changes of the distances, each D_i measured against its error floor
    max(D_i, 1e-3 (G_x + G_a)) as d_err does: ds = -lam sum_i p_i (i - s) dD_i, so
    kappa = lam sum_i p_i |i - s| max(D_i, 1e-3 (G_x + G_a)) / max(|s|, 1)."""
    D = np.asarray(D_ref, dtype=np.float64)
    e = np.exp(-lam * (D - D.min(axis=1, keepdims=True)))
    p = e / e.sum(axis=1, keepdims=True)
    q = np.arange(1, D.shape[1] + 1, dtype=np.float64)
    s = p @ q
    floor = np.maximum(D, 1e-3 * (gsum(frames, w)[:, None] + gsum(landmarks, w)[None, :]))
    return lam * np.sum(p * np.abs(q[None, :] - s[:, None]) * floor, axis=1) / np.maximum(np.abs(s), 1.0)


def z_err(z_gpu, z_ref, lam):
    return np.max(np.abs(z_gpu - z_ref) / np.maximum(np.abs(z_ref), 1.0 / lam))


def grad_err(g_gpu, g_ref):
    num = np.max(np.abs(g_gpu - g_ref).reshape(g_gpu.shape[0], -1), axis=1)
    den = np.max(np.abs(g_ref).reshape(g_ref.shape[0], -1), axis=1)
    return float(np.max(num / den))


def check_grads_at_given_distances(g_s, g_z, ref, ref_at_gpu_D, precision):
    """Gradients of one evaluation checked in two parts.  ref: the oracle's own derivatives;
    ref_at_gpu_D: the oracle's derivatives formed at the GPU's distances (oracle.close with
    D_in), so that their difference is the GPU's adjoint error alone.  That part must be
    within the adjoint's tolerance ADJ_TOL; the end-to-end error must be within the gradient
    tolerance, which it may exceed by the oracle's own response to the GPU's distance errors
    (gated by the D tolerance): with lambda ~ 1e3 nm^-2 the softmax weights move by
    lambda |dD|, ~1e-4 for the 1e-7 nm^2 that FP32 rotations can leave in the approximate
    distances of 5000-atom structures."""
    tol = GRAD_TOL[precision]
    for g, k in ((g_s, "dsdx"), (g_z, "dzdx")):
        own = grad_err(g, ref_at_gpu_D[k])
        prop = grad_err(ref_at_gpu_D[k], ref[k])
        assert own < ADJ_TOL[precision], (k, own)
        assert grad_err(g, ref[k]) < tol + prop, (k, grad_err(g, ref[k]), prop)

// pcv_device.cuh -- device-side numerics shared by the path-CV kernels.
//
// Precision plan (GB300 issues FP64 at 1/62 of the FP32 rate):
//  * per-atom sums (correlation matrix, centroids, sums of squares) run in FP32 with an
//    error-free outer accumulator (TwoSum, Knuth) -- never FP64 per atom;
//  * the 4x4 quaternion eigenvalue, on which MSD = G_x + G_a - 2 lambda_max cancels, is
//    found in FP64: characteristic polynomial of K (Section 3, quaternion method of
//    Kearsley / Coutsias), Newton from the upper bound (G_x + G_a)/2, first in FP32 to
//    get close, then FP64 steps; a bounded number of iterations, never a spin;
//  * eigenvectors / rotations, which only need FP32 accuracy (the MSD is stationary in
//    the rotation), come from an adjugate column of K - lambda I in FP32.
#pragma once
#include <cuda_fp16.h>
#include <stdint.h>

namespace pcv {

// ---------------------------------------------------------------------------------------
// the low part of s held as hi + lo, hi = s rounded to ST: q - s is then formed as
// (q - hi) - lo, exact up to one rounding of the difference (q - hi is exact for q within a
// factor two of hi, Sterbenz).  Forming q - (ST)s instead carries the rounding of s itself,
// up to half an ulp of s (6e-5 at s ~ 2000 in FP32), into every gamma^s_i; the shift moves
// the s-gradient by lambda (s - hi) sum_i p_i dD_i/dx, far above the FP32 rounding of the
// terms once s is large.  Zero for ST = double.
template <typename ST>
__device__ __forceinline__ ST s_low(double s, ST hi) {
  return (ST)(s - (double)hi);
}

// ---------------------------------------------------------------------------------------
// compensated FP32 accumulation: (hi, lo) += v without losing the rounding error of the
// addition (TwoSum).  Valid without FMA contraction concerns: no products involved.
__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float v) {
  const float s = __fadd_rn(hi, v);
  const float bp = __fsub_rn(s, hi);
  const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(v, bp));
  hi = s;
  lo = __fadd_rn(lo, err);
}

// (hi, lo) pair sum of two compensated values
__device__ __forceinline__ void two_sum_pair(float& hi, float& lo, float hi2, float lo2) {
  two_sum_acc(hi, lo, hi2);
  lo = __fadd_rn(lo, lo2);
}

__device__ __forceinline__ double pair_to_double(float hi, float lo) {
  return (double)hi + (double)lo;
}

// warp-wide sum of a compensated FP32 value; every lane receives the result
__device__ __forceinline__ void warp_sum_pair(float& hi, float& lo) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const float h2 = __shfl_xor_sync(0xffffffffu, hi, off);
    const float l2 = __shfl_xor_sync(0xffffffffu, lo, off);
    two_sum_pair(hi, lo, h2, l2);
  }
}

__device__ __forceinline__ double warp_sum_double(double v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

__device__ __forceinline__ float warp_sum_float(float v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

// ---------------------------------------------------------------------------------------
// Landmark coordinate (i, j, c) in the working type: the stored value, plus the FP32 block
// offset in FP16 storage (blocks of 16 atoms; off holds M*ceil(N/16)*3 floats).
template <typename ST, typename LT>
__device__ __forceinline__ ST lm_coord(const LT* lm, const float* off, int N, size_t i, int j, int c) {
  (void)off;
  return (ST)lm[(i * N + j) * 3 + c];
}
template <>
__device__ __forceinline__ float lm_coord<float, __half>(const __half* lm, const float* off, int N, size_t i, int j,
                                                        int c) {
  return __half2float(lm[(i * N + j) * 3 + c]) + off[(i * ((N + 15) >> 4) + (j >> 4)) * 3 + c];
}
// the same for a value already read (e.g. from a shared-memory copy of the landmark)
template <typename LT>
__device__ __forceinline__ float lm_plus_off(float v, const float* off, int N, size_t i, int j, int c) {
  (void)off;
  (void)N;
  (void)i;
  (void)j;
  (void)c;
  return v;
}
template <>
__device__ __forceinline__ float lm_plus_off<__half>(float v, const float* off, int N, size_t i, int j, int c) {
  return v + off[(i * ((N + 15) >> 4) + (j >> 4)) * 3 + c];
}

// ---------------------------------------------------------------------------------------
// Packed FP32 pairs (Blackwell f32x2 instructions): one instruction performs two IEEE FP32
// operations with round-to-nearest, bit-identical to two scalar ones, at half the issue
// cost.  A pair lives in a 64-bit register pair: low half = first element.
typedef unsigned long long f2;
__device__ __forceinline__ f2 f2_pack(float lo, float hi) {
  f2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void f2_unpack(f2 v, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ f2 f2_fma(f2 a, f2 b, f2 c) {
  f2 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}

// ---------------------------------------------------------------------------------------
// Quaternion matrix.  For the correlation H[b][c] = sum_j w_j a_jb x_jc of a structure a
// fitted onto x, q^T K q = trace(R(q) H) for unit q, so the largest eigenpair of K gives
// the optimal rotation R(q) of a onto x and lambda_max = max_R trace(R H).
template <typename T>
__device__ __forceinline__ void quat_matrix(const T* H, T* K) {
  const T hxx = H[0], hxy = H[1], hxz = H[2];
  const T hyx = H[3], hyy = H[4], hyz = H[5];
  const T hzx = H[6], hzy = H[7], hzz = H[8];
  K[0] = hxx + hyy + hzz;
  K[1] = hyz - hzy;
  K[2] = hzx - hxz;
  K[3] = hxy - hyx;
  K[5] = hxx - hyy - hzz;
  K[6] = hxy + hyx;
  K[7] = hzx + hxz;
  K[10] = -hxx + hyy - hzz;
  K[11] = hyz + hzy;
  K[15] = -hxx - hyy + hzz;
  K[4] = K[1];
  K[8] = K[2];
  K[9] = K[6];
  K[12] = K[3];
  K[13] = K[7];
  K[14] = K[11];
}

// det of a symmetric 4x4 through complementary 2x2 minors (Laplace expansion on rows 0-1)
template <typename T>
__device__ __forceinline__ T det4(const T* a) {
  const T s0 = a[0] * a[5] - a[4] * a[1];
  const T s1 = a[0] * a[6] - a[4] * a[2];
  const T s2 = a[0] * a[7] - a[4] * a[3];
  const T s3 = a[1] * a[6] - a[5] * a[2];
  const T s4 = a[1] * a[7] - a[5] * a[3];
  const T s5 = a[2] * a[7] - a[6] * a[3];
  const T c5 = a[10] * a[15] - a[14] * a[11];
  const T c4 = a[9] * a[15] - a[13] * a[11];
  const T c3 = a[9] * a[14] - a[13] * a[10];
  const T c2 = a[8] * a[15] - a[12] * a[11];
  const T c1 = a[8] * a[14] - a[12] * a[10];
  const T c0 = a[8] * a[13] - a[12] * a[9];
  return s0 * c5 - s1 * c4 + s2 * c3 + s3 * c2 - s4 * c1 + s5 * c0;
}

template <typename T>
__device__ __forceinline__ T det3(const T* h) {
  return h[0] * (h[4] * h[8] - h[5] * h[7]) - h[1] * (h[3] * h[8] - h[5] * h[6]) +
         h[2] * (h[3] * h[7] - h[4] * h[6]);
}

// Coefficients of det(lambda I - K) = lambda^4 + c2 lambda^2 + c1 lambda + c0
// (trace K = 0): c2 = -2 |H|_F^2, c1 = -8 det H, c0 = det K.
template <typename T>
__device__ __forceinline__ void char_poly(const T* H, const T* K, T& c2, T& c1, T& c0) {
  T f = 0;
#pragma unroll
  for (int e = 0; e < 9; ++e) f += H[e] * H[e];
  c2 = T(-2) * f;
  c1 = T(-8) * det3(H);
  c0 = det4(K);
}

// Largest root of the characteristic polynomial by Newton iteration started from an
// upper bound ub >= lambda_max (e.g. (G_x + G_a)/2, Cauchy-Schwarz); from above, Newton
// on a polynomial with all-real roots decreases monotonically onto the largest root.
// FP32 iterations first (cheap); the FP64 iterations restart slightly above the FP32
// estimate (by 4e-6 ub, well above its rounding error) so that they also approach from
// above, and stop once a step is below 1e-13 ub.
// Returns lambda_max; sets *ok = false if the iteration caps were reached.  dp_out (optional)
// receives P'(l) of the last iteration, which tells a (nearly) double root (near_double_f64).
// cap: iterations of the FP64 phase (the FP32 phase takes at most 40).
__device__ __forceinline__ double lambda_max_newton(const double* H, double ub, bool* ok,
                                                    double* dp_out = nullptr, int cap = 60) {
  double K[16];
  quat_matrix(H, K);
  double c2, c1, c0;
  char_poly(H, K, c2, c1, c0);
  // FP32 phase
  const float f2 = (float)c2, f1 = (float)c1, f0 = (float)c0;
  float lf = (float)ub;
  const float tolf = 2e-6f * fabsf(lf) + 1e-30f;
  for (int it = 0; it < 40; ++it) {
    const float l2 = lf * lf;
    const float p = fmaf(fmaf(l2 + f2, lf, f1), lf, f0);
    const float dp = fmaf(fmaf(4.0f * lf, lf, 2.0f * f2), lf, f1);
    if (!(dp > 0.0f)) break;
    const float step = p / dp;
    lf -= step;
    if (fabsf(step) <= tolf) break;
  }
  // FP64 phase
  double l = (double)lf + 4e-6 * fabs(ub);
  if (!(l <= ub) || !(l == l)) l = ub;
  const double tol = 1e-13 * fabs(ub) + 1e-300;
  *ok = false;
  double prev = 1.0e300, dp_last = 0.0;
  for (int it = 0; it < cap; ++it) {
    const double l2 = l * l;
    const double p = fma(fma(l2 + c2, l, c1), l, c0);
    const double dp = fma(fma(4.0 * l, l, 2.0 * c2), l, c1);
    dp_last = dp;
    if (!(dp > 0.0)) {
      *ok = true;  // at (or numerically on) the root
      break;
    }
    // the step only needs relative accuracy: divide in FP32
    const double step = (double)__fdiv_rn((float)p, (float)dp);
    l -= step;
    const double a = fabs(step);
    // converged, or at the rounding-noise floor of P (steps stop shrinking near the root)
    if (a <= tol || (a < 1e-9 * fabs(ub) && a >= 0.5 * prev)) {
      *ok = true;
      break;
    }
    prev = a;
  }
  if (dp_out) *dp_out = dp_last;
  return l;
}

// P'(l) = prod_k (l - lambda_k) over the other three eigenvalues.  The rounding of P near its
// top root moves l by about 10 u ub^4 / P'(l) (u = 2^-53); D = G_x + G_a - 2 l must stay
// within 1e-9 of 1e-3 (G_x + G_a) = 2e-3 ub, so P'(l) must exceed ~1e-3 ub^3.  Below that the
// top eigenvalue is (nearly) double and the Jacobi iteration takes over.
__device__ __forceinline__ bool near_double_f64(double dp, double ub) { return !(dp > 1e-3 * ub * ub * ub); }


// Rotation of a unit quaternion q = (s, v): R = (s^2 - |v|^2) I + 2 v v^T + 2 s [v]_x,
// divided by |q|^2 so that rounding in q does not spoil orthogonality to first order.
template <typename T>
__device__ __forceinline__ void quat_to_rot(const T* q, T* R) {
  const T s = q[0], x = q[1], y = q[2], z = q[3];
  const T n2 = s * s + x * x + y * y + z * z;
  const T inv = T(1) / n2;
  R[0] = (s * s + x * x - y * y - z * z) * inv;
  R[1] = T(2) * (x * y - s * z) * inv;
  R[2] = T(2) * (x * z + s * y) * inv;
  R[3] = T(2) * (x * y + s * z) * inv;
  R[4] = (s * s - x * x + y * y - z * z) * inv;
  R[5] = T(2) * (y * z - s * x) * inv;
  R[6] = T(2) * (x * z - s * y) * inv;
  R[7] = T(2) * (y * z + s * x) * inv;
  R[8] = (s * s - x * x - y * y + z * z) * inv;
}

// Correlation H = sum_j w_j (y_j - c_y)(x_j - c_x)^T of one frame pair over a warp, with
// compensated FP32 sums (products summed 16 at a time, then folded into a (hi, lo) pair):
// every lane returns H rounded to FP32, no FP64 instruction.
__device__ __forceinline__ void warp_corr_pair_f32(int N, const float* __restrict__ x, float4 cx,
                                                   const float* __restrict__ y, float4 cy,
                                                   const float* __restrict__ wts, float* H) {
  const int lane = threadIdx.x & 31;
  float p[9], hi[9], lo[9];
#pragma unroll
  for (int e = 0; e < 9; ++e) p[e] = hi[e] = lo[e] = 0.0f;
  int cnt = 0;
#pragma unroll 4
  for (int j = lane; j < N; j += 32) {
    float u0 = y[3 * j] - cy.x, u1 = y[3 * j + 1] - cy.y, u2 = y[3 * j + 2] - cy.z;
    const float v0 = x[3 * j] - cx.x, v1 = x[3 * j + 1] - cx.y, v2 = x[3 * j + 2] - cx.z;
    if (wts) {
      const float wj = wts[j];
      u0 *= wj;
      u1 *= wj;
      u2 *= wj;
    }
    const float u[3] = {u0, u1, u2}, v[3] = {v0, v1, v2};
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
      for (int c = 0; c < 3; ++c) p[3 * b + c] = fmaf(u[b], v[c], p[3 * b + c]);
    if (++cnt == 16) {
      cnt = 0;
#pragma unroll
      for (int e = 0; e < 9; ++e) {
        two_sum_acc(hi[e], lo[e], p[e]);
        p[e] = 0.0f;
      }
    }
  }
#pragma unroll
  for (int e = 0; e < 9; ++e) {
    two_sum_acc(hi[e], lo[e], p[e]);
    warp_sum_pair(hi[e], lo[e]);
    H[e] = hi[e] + lo[e];
  }
}

// ---------------------------------------------------------------------------------------
// FP32 top eigenvector of K(H) (the quaternion of the optimal rotation), for the direct
// two-pass MSD: the rotation only needs FP32 accuracy because the directly evaluated
// MSD sum_j w_j |x_j - R a_j|^2 is stationary in R.  H is normalised by an upper bound
// ub >= lambda_max so that the iteration works on O(1) numbers.

// cofactor-based eigenvector of the symmetric 4x4 A = K - lam I; returns the magnitude of
// the adjugate diagonal entry used (small => lam is (nearly) a multiple eigenvalue)
__device__ __forceinline__ float adj_eigvec_f32(const float* A, float* q) {
  float cof[16];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      float m[9];
      int k = 0;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        if (i == r) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          if (j == c) continue;
          m[k++] = A[4 * i + j];
        }
      }
      const float d = det3(m);
      cof[4 * r + c] = ((r + c) & 1) ? -d : d;
    }
  // column of the largest diagonal cofactor, chosen by compares (a run-time index into the
  // array would move it to local memory)
  float bv = fabsf(cof[0]);
#pragma unroll
  for (int i = 0; i < 4; ++i) q[i] = cof[4 * i];
#pragma unroll
  for (int c = 1; c < 4; ++c) {
    const bool take = fabsf(cof[5 * c]) > bv;
    bv = take ? fabsf(cof[5 * c]) : bv;
#pragma unroll
    for (int i = 0; i < 4; ++i) q[i] = take ? cof[4 * i + c] : q[i];
  }
  float n2 = 0.0f;
#pragma unroll
  for (int i = 0; i < 4; ++i) n2 += q[i] * q[i];
  if (n2 > 0.0f) {
    const float inv = rsqrtf(n2) * (q[0] < 0.0f ? -1.0f : 1.0f);
#pragma unroll
    for (int i = 0; i < 4; ++i) q[i] *= inv;
  }
  return bv;
}

// cyclic Jacobi fallback (FP32) for (nearly) degenerate top eigenvalues: top eigenvector.
// The matrix comes by value and every inner loop is unrolled, so A and V stay in registers.
struct Mat4f {
  float v[16];
};
static __device__ __noinline__ float4 jacobi_top_f32(Mat4f Kin) {
  float A[16], V[16];
#pragma unroll
  for (int e = 0; e < 16; ++e) {
    A[e] = Kin.v[e];
    V[e] = (e % 5 == 0) ? 1.0f : 0.0f;
  }
  for (int sweep = 0; sweep < 12; ++sweep) {
    float off = 0.0f;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = i + 1; j < 4; ++j) off += A[4 * i + j] * A[4 * i + j];
    if (off < 1e-30f) break;
#pragma unroll
    for (int p = 0; p < 3; ++p)
#pragma unroll
      for (int r = p + 1; r < 4; ++r) {
        const float apr = A[4 * p + r];
        if (apr != 0.0f) {
          const float th = (A[5 * r] - A[5 * p]) / (2.0f * apr);
          const float t = copysignf(1.0f, th) / (fabsf(th) + sqrtf(th * th + 1.0f));
          const float c = rsqrtf(t * t + 1.0f), sn = t * c;
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const float akp = A[4 * k + p], akr = A[4 * k + r];
            A[4 * k + p] = c * akp - sn * akr;
            A[4 * k + r] = sn * akp + c * akr;
          }
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const float apk = A[4 * p + k], ark = A[4 * r + k];
            A[4 * p + k] = c * apk - sn * ark;
            A[4 * r + k] = sn * apk + c * ark;
          }
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const float vkp = V[4 * k + p], vkr = V[4 * k + r];
            V[4 * k + p] = c * vkp - sn * vkr;
            V[4 * k + r] = sn * vkp + c * vkr;
          }
        }
      }
  }
  float bv = A[0], q[4] = {V[0], V[4], V[8], V[12]};
#pragma unroll
  for (int c = 1; c < 4; ++c) {
    const bool take = A[5 * c] > bv;
    bv = take ? A[5 * c] : bv;
#pragma unroll
    for (int i = 0; i < 4; ++i) q[i] = take ? V[4 * i + c] : q[i];
  }
  const float sg = q[0] < 0.0f ? -1.0f : 1.0f;
  return make_float4(sg * q[0], sg * q[1], sg * q[2], sg * q[3]);
}

// Top eigenvector (unit quaternion, q[0] >= 0) of K(H) in FP32.  Returns false if the
// Newton iteration hit its cap of `cap` iterations (the result is still usable).
__device__ __forceinline__ bool top_quat_f32(const float* Hin, float ub, float* q, int cap = 60) {
  const float sc = 1.0f / ub;
  float H[9];
#pragma unroll
  for (int e = 0; e < 9; ++e) H[e] = Hin[e] * sc;
  float K[16];
  quat_matrix(H, K);
  float c2, c1, c0;
  char_poly(H, K, c2, c1, c0);
  float l = 1.0f;
  bool ok = false;
  float prev = 3.0e38f;
  for (int it = 0; it < cap; ++it) {
    const float p = fmaf(fmaf(fmaf(l, l, c2), l, c1), l, c0);
    const float dp = fmaf(fmaf(4.0f * l, l, 2.0f * c2), l, c1);
    if (!(dp > 0.0f)) {
      ok = true;
      break;
    }
    const float step = p / dp;
    l -= step;
    const float a = fabsf(step);
    // converged: below FP32 resolution, or at the rounding-noise floor of P near the root
    // (steps no longer shrink; happens when the top eigenvalue gap is small)
    if (a <= 2e-7f || (a < 1e-4f && a >= 0.5f * prev)) {
      ok = true;
      break;
    }
    prev = a;
  }
  // P'(l) = prod_k (l - lambda_k) over the other eigenvalues: small when the top eigenvalue
  // is (nearly) double.  Newton then converges only linearly and stops at its noise floor,
  // |l - lambda| ~ sqrt(u) ~ 3e-4 of the bound, which the adjugate column inherits; there
  // P'(l) ~ 2 |l - lambda| prod_{k > 2} (lambda - lambda_k) reaches a few 1e-3 l^3
  // (eigenvalues in [-1, 1] after the scaling).  Below 0.02 l^3 (a double root at the noise floor,
  // or a relative gap below ~5e-3) the eigenvector comes from the Jacobi iteration, which
  // does not degrade there.  (A bar of 0.002 let collinear pairs through to the adjugate,
  // depending on the rounding of H.)
  const float dpl = fmaf(fmaf(4.0f * l, l, 2.0f * c2), l, c1);
  const bool near_double = !(dpl > 0.02f * l * l * l);
  float A[16];
#pragma unroll
  for (int e = 0; e < 16; ++e) A[e] = K[e];
  A[0] -= l;
  A[5] -= l;
  A[10] -= l;
  A[15] -= l;
  const float mag = near_double ? 0.0f : adj_eigvec_f32(A, q);
  if (!(mag > 1e-5f)) {
    Mat4f kk;
#pragma unroll
    for (int e = 0; e < 16; ++e) kk.v[e] = K[e];
    const float4 r = jacobi_top_f32(kk);
    q[0] = r.x;
    q[1] = r.y;
    q[2] = r.z;
    q[3] = r.w;
  }
  return ok;
}

// Unit eigenvector of K for eigenvalue lam in FP64 (adjugate column, as adj_eigvec).
__device__ __forceinline__ void adj_eigvec_f64(const double* K, double lam, double* q) {
  double A[16];
#pragma unroll
  for (int e = 0; e < 16; ++e) A[e] = K[e];
  A[0] -= lam;
  A[5] -= lam;
  A[10] -= lam;
  A[15] -= lam;
  double cof[16];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      double m[9];
      int k = 0;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        if (i == r) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          if (j == c) continue;
          m[k++] = A[4 * i + j];
        }
      }
      const double d = det3(m);
      cof[4 * r + c] = ((r + c) & 1) ? -d : d;
    }
  // column of the largest diagonal cofactor, chosen by compares (no run-time index)
  double bv = fabs(cof[0]);
#pragma unroll
  for (int i = 0; i < 4; ++i) q[i] = cof[4 * i];
#pragma unroll
  for (int c = 1; c < 4; ++c) {
    const bool take = fabs(cof[5 * c]) > bv;
    bv = take ? fabs(cof[5 * c]) : bv;
#pragma unroll
    for (int i = 0; i < 4; ++i) q[i] = take ? cof[4 * i + c] : q[i];
  }
  double n2 = 0.0;
#pragma unroll
  for (int i = 0; i < 4; ++i) n2 += q[i] * q[i];
  if (!(n2 > 0.0)) {
    q[0] = 1.0;
    q[1] = q[2] = q[3] = 0.0;
    return;
  }
  const double inv = (q[0] < 0.0 ? -1.0 : 1.0) / sqrt(n2);
#pragma unroll
  for (int i = 0; i < 4; ++i) q[i] *= inv;
}

// FP64 cyclic Jacobi for the symmetric 4x4 K: the top eigenvalue and its unit eigenvector
// (q[0] >= 0), for (nearly) double top eigenvalues, where Newton on the characteristic
// quartic converges only linearly and the adjugate column is ill-conditioned.  Jacobi
// rotations keep the eigenvalues accurate to ~u |K|_F whatever the gap.  Stops when the
// off-diagonal mass is below 1e-32 of |K|_F^2; ok = 0 if 30 sweeps do not get there.
// The matrix comes by value and the function is not inlined, so the callers' registers do
// not grow with it.
struct Mat4d {
  double v[16];
};
struct TopEig4d {
  double lam;
  double q[4];
  int ok;
};
static __device__ __noinline__ TopEig4d jacobi_top_f64(Mat4d Kin) {
  double A[16], V[16], fro = 0.0;
#pragma unroll
  for (int e = 0; e < 16; ++e) {
    A[e] = Kin.v[e];
    V[e] = (e % 5 == 0) ? 1.0 : 0.0;
    fro += A[e] * A[e];
  }
  TopEig4d out;
  out.ok = 0;
  for (int sweep = 0; sweep < 30; ++sweep) {
    double off = 0.0;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = i + 1; j < 4; ++j) off += A[4 * i + j] * A[4 * i + j];
    if (!(off > 1e-32 * fro)) {
      out.ok = 1;
      break;
    }
#pragma unroll
    for (int p = 0; p < 3; ++p)
#pragma unroll
      for (int r = p + 1; r < 4; ++r) {
        const double apr = A[4 * p + r];
        if (apr != 0.0) {
          const double th = (A[5 * r] - A[5 * p]) / (2.0 * apr);
          const double t = copysign(1.0, th) / (fabs(th) + sqrt(th * th + 1.0));
          const double c = 1.0 / sqrt(t * t + 1.0), sn = t * c;
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const double akp = A[4 * k + p], akr = A[4 * k + r];
            A[4 * k + p] = c * akp - sn * akr;
            A[4 * k + r] = sn * akp + c * akr;
          }
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const double apk = A[4 * p + k], ark = A[4 * r + k];
            A[4 * p + k] = c * apk - sn * ark;
            A[4 * r + k] = sn * apk + c * ark;
          }
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const double vkp = V[4 * k + p], vkr = V[4 * k + r];
            V[4 * k + p] = c * vkp - sn * vkr;
            V[4 * k + r] = sn * vkp + c * vkr;
          }
        }
      }
  }
  double bv = A[0], q[4] = {V[0], V[4], V[8], V[12]};
#pragma unroll
  for (int c = 1; c < 4; ++c) {
    const bool take = A[5 * c] > bv;
    bv = take ? A[5 * c] : bv;
#pragma unroll
    for (int i = 0; i < 4; ++i) q[i] = take ? V[4 * i + c] : q[i];
  }
  const double sg = q[0] < 0.0 ? -1.0 : 1.0;
  out.lam = bv;
#pragma unroll
  for (int i = 0; i < 4; ++i) out.q[i] = sg * q[i];
  return out;
}

// Top eigenpair of K(H) in FP64 for one pair: Newton on the characteristic quartic from the
// upper bound ub and (when q is requested) the adjugate column; at a (nearly) double top
// eigenvalue (near_double_f64) the Jacobi iteration gives both instead.  Returns lambda_max;
// *ok = false if an iteration cap was reached.
__device__ __forceinline__ double top_eig_f64(const double* H, double ub, bool* ok, double* q) {
  double dp = 0.0;
  const double lam = lambda_max_newton(H, ub, ok, &dp);
  if (near_double_f64(dp, ub)) {
    Mat4d k;
    quat_matrix(H, k.v);
    const TopEig4d e = jacobi_top_f64(k);
    *ok = e.ok != 0;
    if (q) {
#pragma unroll
      for (int a = 0; a < 4; ++a) q[a] = e.q[a];
    }
    return e.lam;
  }
  if (q) {
    double K[16];
    quat_matrix(H, K);
    adj_eigvec_f64(K, lam, q);
  }
  return lam;
}

// Solve the 4x4 symmetric positive definite system A p = g by Cholesky.
// Returns false if A is not numerically positive definite.
template <typename T>
__device__ __forceinline__ bool spd_solve4(const T* A, const T* g, T* p) {
  T L[16];
#pragma unroll
  for (int e = 0; e < 16; ++e) L[e] = 0;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
#pragma unroll
    for (int j = 0; j <= i; ++j) {
      T sum = A[4 * i + j];
#pragma unroll
      for (int k = 0; k < j; ++k) sum -= L[4 * i + k] * L[4 * j + k];
      if (i == j) {
        if (!(sum > T(0))) return false;
        L[4 * i + i] = sqrt(sum);
      } else {
        L[4 * i + j] = sum / L[4 * j + j];
      }
    }
  }
  T y[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    T sum = g[i];
#pragma unroll
    for (int k = 0; k < i; ++k) sum -= L[4 * i + k] * y[k];
    y[i] = sum / L[4 * i + i];
  }
#pragma unroll
  for (int i = 3; i >= 0; --i) {
    T sum = y[i];
#pragma unroll
    for (int k = i + 1; k < 4; ++k) sum -= L[4 * k + i] * p[k];
    p[i] = sum / L[4 * i + i];
  }
  return true;
}

// top eigenpair (lambda0, unit q0) of K(H) in the working precision
__device__ __forceinline__ void top_eig(const float* H, const float* K, float* l0, float* q0) {
  float ub = 0.0f;  // Gershgorin bound >= lambda_max
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    float rs = 0.0f;
#pragma unroll
    for (int b = 0; b < 4; ++b) rs += fabsf(K[4 * a + b]);
    ub = fmaxf(ub, rs);
  }
  top_quat_f32(H, ub + 1e-30f, q0);
  float t = 0.0f;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) t += q0[a] * K[4 * a + b] * q0[b];
  *l0 = t;
}
__device__ __forceinline__ void top_eig(const double* H, const double* K, double* l0, double* q0) {
  double ub = 0.0;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    double rs = 0.0;
#pragma unroll
    for (int b = 0; b < 4; ++b) rs += fabs(K[4 * a + b]);
    ub = fmax(ub, rs);
  }
  bool ok = true;
  *l0 = lambda_max_newton(H, ub + 1e-300, &ok);
  adj_eigvec_f64(K, *l0, q0);
}

// Rotation term of Eq. (close_der_dist) summed over the landmarks with weights gamma_i:
// sum_ab Ghat_ab dR_xy,ab / dx_kc = w_k (T^T y_k)_c, where
//   Ghat = -2 (X - R_xy Phi),  X = sum_j w_j x_j beta_j^T,  Phi = sum_i gamma_i B_i A_i B_i^T,
//   q0, l0: top eigenpair of K(H_xy), H_xy = sum_j w_j y_j x_j^T,
//   g = 2 K(Ghat^T) q0 (gradient of sum_ab Ghat_ab R(q)_ab at q0),
//   p solves (l0 I - K + q0 q0^T) p = g - (q0.g) q0 (first-order eigenvector perturbation
//   dq0 = (l0 I - K)^+ dK q0, with dK = K(w_k y_k e_c^T)),
//   T_bc = p^T K(E_bc) q0.
template <typename T>
__device__ __forceinline__ void adjoint_rotation_term(const T* H, const T* R, const T* X, const T* Phi, T* Tout) {
  T K[16];
  quat_matrix(H, K);
  T l0, q0[4];
  top_eig(H, K, &l0, q0);
  T Gh[9];
#pragma unroll
  for (int b = 0; b < 3; ++b)
#pragma unroll
    for (int c = 0; c < 3; ++c)
      Gh[3 * b + c] = T(-2) * (X[3 * b + c] - (R[3 * b] * Phi[c] + R[3 * b + 1] * Phi[3 + c] + R[3 * b + 2] * Phi[6 + c]));
  T GhT[9];
#pragma unroll
  for (int b = 0; b < 3; ++b)
#pragma unroll
    for (int c = 0; c < 3; ++c) GhT[3 * b + c] = Gh[3 * c + b];
  T KG[16];
  quat_matrix(GhT, KG);
  T g[4];
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    g[a] = 0;
#pragma unroll
    for (int b = 0; b < 4; ++b) g[a] += T(2) * KG[4 * a + b] * q0[b];
  }
  const T gq = g[0] * q0[0] + g[1] * q0[1] + g[2] * q0[2] + g[3] * q0[3];
#pragma unroll
  for (int a = 0; a < 4; ++a) g[a] -= gq * q0[a];
  T Am[16];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) Am[4 * a + b] = (a == b ? l0 : T(0)) - K[4 * a + b] + q0[a] * q0[b];
  T pv[4] = {0, 0, 0, 0};
  spd_solve4(Am, g, pv);
#pragma unroll
  for (int b = 0; b < 3; ++b)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      T E[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
      E[3 * b + c] = 1;
      T KE[16];
      quat_matrix(E, KE);
      T t = 0;
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int d = 0; d < 4; ++d) t += pv[a] * KE[4 * a + d] * q0[d];
      Tout[3 * b + c] = t;
    }
}


// The rotation terms of gamma^s and gamma^z together (as adjoint_rotation_term), given the
// top eigenvector q0 of K(H) -- the alignment quaternion of x onto y, known from the
// refresh search -- so the eigen-solve and the factorisation of (l0 I - K + q0 q0^T) are
// done once for both.  q0 may have either sign: T is quadratic in q0.
template <typename T>
__device__ __forceinline__ void adjoint_rotation_terms2(const T* H, const T* R, const T* q0in, const T* Xs,
                                                        const T* Xz, const T* Ps, const T* Pz, T* Ts, T* Tz) {
  T K[16];
  quat_matrix(H, K);
  T q0[4];
  {
    const T rn = T(1) / sqrt(q0in[0] * q0in[0] + q0in[1] * q0in[1] + q0in[2] * q0in[2] + q0in[3] * q0in[3]);
#pragma unroll
    for (int a = 0; a < 4; ++a) q0[a] = q0in[a] * rn;
  }
  T l0 = 0;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) l0 += q0[a] * K[4 * a + b] * q0[b];
  T g2[2][4];
#pragma unroll
  for (int which = 0; which < 2; ++which) {
    const T* X = which ? Xz : Xs;
    const T* Phi = which ? Pz : Ps;
    T GhT[9];  // Ghat^T, Ghat = -2 (X - R Phi)
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
      for (int c = 0; c < 3; ++c)
        GhT[3 * c + b] = T(-2) * (X[3 * b + c] - (R[3 * b] * Phi[c] + R[3 * b + 1] * Phi[3 + c] + R[3 * b + 2] * Phi[6 + c]));
    T KG[16];
    quat_matrix(GhT, KG);
    T* g = g2[which];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      g[a] = 0;
#pragma unroll
      for (int b = 0; b < 4; ++b) g[a] += T(2) * KG[4 * a + b] * q0[b];
    }
    const T gq = g[0] * q0[0] + g[1] * q0[1] + g[2] * q0[2] + g[3] * q0[3];
#pragma unroll
    for (int a = 0; a < 4; ++a) g[a] -= gq * q0[a];
  }
  // Cholesky factor of l0 I - K + q0 q0^T, then two solves (one reciprocal per diagonal
  // entry, products instead of divisions on the serial chain)
  T L[16], iL[4];
#pragma unroll
  for (int e = 0; e < 16; ++e) L[e] = 0;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
#pragma unroll
    for (int j = 0; j <= i; ++j) {
      T sum = (i == j ? l0 : T(0)) - K[4 * i + j] + q0[i] * q0[j];
#pragma unroll
      for (int k = 0; k < j; ++k) sum -= L[4 * i + k] * L[4 * j + k];
      if (i == j) {
        L[4 * i + i] = sqrt(sum > T(0) ? sum : T(1e-30));
        iL[i] = T(1) / L[4 * i + i];
      } else {
        L[4 * i + j] = sum * iL[j];
      }
    }
  }
  T pv[2][4];
#pragma unroll
  for (int which = 0; which < 2; ++which) {
    T y[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      T sum = g2[which][i];
#pragma unroll
      for (int k = 0; k < i; ++k) sum -= L[4 * i + k] * y[k];
      y[i] = sum * iL[i];
    }
#pragma unroll
    for (int i = 3; i >= 0; --i) {
      T sum = y[i];
#pragma unroll
      for (int k = i + 1; k < 4; ++k) sum -= L[4 * k + i] * pv[which][k];
      pv[which][i] = sum * iL[i];
    }
  }
#pragma unroll
  for (int b = 0; b < 3; ++b)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      T E[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
      E[3 * b + c] = 1;
      T KE[16];
      quat_matrix(E, KE);
      T ts = 0, tz = 0;
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int d = 0; d < 4; ++d) {
          ts += pv[0][a] * KE[4 * a + d] * q0[d];
          tz += pv[1][a] * KE[4 * a + d] * q0[d];
        }
      Ts[3 * b + c] = ts;
      Tz[3 * b + c] = tz;
    }
}

}  // namespace pcv

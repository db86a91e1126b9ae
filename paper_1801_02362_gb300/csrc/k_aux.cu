// k_aux.cu -- per-frame kernels around the pair kernels:
//   frame preparation (centres, sums of squares), frame-vs-structure alignments for the
//   close-structure decision of Algorithm 2 (band of previous frames, speculative chunks,
//   FP64 re-check of undecidable cases), the parallel refresh-search scan, compaction,
//   path-CV finalisation (Eq. property_map_cv and z) and the chain-rule combination of
//   the gradients.
#include <cuda_fp16.h>

#include <algorithm>

#include "pcv_device.cuh"
#include "pcv_internal.h"

namespace pcv {
namespace {

constexpr int WARPS_PER_BLOCK = 4;

__device__ __forceinline__ int warp_global() {
  return (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
}

// ---------------------------------------------------------------------------------------
// frame preparation: one warp per frame.
//   FP32 frames: centre c = sum_j w_j x_j with compensated FP32 sums, c32 = fl(c);
//   G = sum_j wk_j |fl(x_j - c32)|^2 over exactly the values the pair kernels stage
//   (error-free squares, compensated sums).  FP64 frames: plain FP64.
// centre and G of frame f, one warp.  The centre is weighted by the alignment weights wc
// when given (they set the translation, Section 3.1), else by wts; G by wts.
__device__ __forceinline__ void frame_prep_warp_f32(int f, int N, const float* __restrict__ frames,
                                                    const float* __restrict__ wts, float4* __restrict__ c32,
                                                    double* __restrict__ G, const float* __restrict__ wc = nullptr) {
  const int lane = threadIdx.x & 31;
  const float* x = frames + (size_t)f * N * 3;
  const float* cw = wc ? wc : wts;
  float hi[3] = {0, 0, 0}, lo[3] = {0, 0, 0};
#pragma unroll 4
  for (int j = lane; j < N; j += 32) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float v = x[3 * j + c];
      if (cw) {
        const float p = cw[j] * v;
        const float e = fmaf(cw[j], v, -p);
        two_sum_acc(hi[c], lo[c], p);
        lo[c] += e;
      } else {
        two_sum_acc(hi[c], lo[c], v);
      }
    }
  }
  // FP32 centre: any centre works as long as G is taken over the same staged values;
  // FP64 per frame would cost ~16 SM cycles per warp instruction on this chip
  float cf[3];
  const float invn = 1.0f / (float)N;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    warp_sum_pair(hi[k], lo[k]);
    cf[k] = cw ? hi[k] + lo[k] : (hi[k] + lo[k]) * invn;
  }
  float gh = 0.0f, gl = 0.0f;
#pragma unroll 4
  for (int j = lane; j < N; j += 32) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float v = x[3 * j + k] - cf[k];
      const float vw = wts ? v * wts[j] : v;  // the staged frame value in the exact kernel
      const float p = vw * v;
      const float e = fmaf(vw, v, -p);
      two_sum_acc(gh, gl, p);
      gl += e;
    }
  }
  warp_sum_pair(gh, gl);
  if (lane == 0) {
    c32[f] = make_float4(cf[0], cf[1], cf[2], 0.0f);
    G[f] = pair_to_double(gh, gl);
  }
}

__global__ void frame_prep_f32(int F, int N, const float* __restrict__ frames, const float* __restrict__ wts,
                               float4* __restrict__ c32, double4* __restrict__ c64, double* __restrict__ G,
                               const float* __restrict__ wc) {
  const int f = warp_global();
  if (f >= F) return;
  frame_prep_warp_f32(f, N, frames, wts, c32, G, wc);
}

// The same per frame with one 256-thread block per frame, for a few large frames (the
// per-step case): warp sums, then the 8 warps' compensated pairs combined in shared memory.
__device__ __forceinline__ void block_sum_pair(float& hi, float& lo, float (*sh)[2]) {
  warp_sum_pair(hi, lo);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0) {
    sh[w][0] = hi;
    sh[w][1] = lo;
  }
  __syncthreads();
  hi = 0.0f;
  lo = 0.0f;
  for (int k = 0; k < nw; ++k) two_sum_pair(hi, lo, sh[k][0], sh[k][1]);
}

__global__ void frame_prep_f32_block(int F, int N, const float* __restrict__ frames, const float* __restrict__ wts,
                                     float4* __restrict__ c32, double* __restrict__ G, const float* __restrict__ wc) {
  __shared__ float sh[32][2];
  const int f = blockIdx.x;
  const float* x = frames + (size_t)f * N * 3;
  const float* cw = wc ? wc : wts;
  float cf[3];
  const float invn = 1.0f / (float)N;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    float hi = 0.0f, lo = 0.0f;
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
      const float v = x[3 * j + k];
      if (cw) {
        const float p = cw[j] * v;
        const float e = fmaf(cw[j], v, -p);
        two_sum_acc(hi, lo, p);
        lo += e;
      } else {
        two_sum_acc(hi, lo, v);
      }
    }
    block_sum_pair(hi, lo, sh);
    cf[k] = cw ? hi + lo : (hi + lo) * invn;
  }
  float gh = 0.0f, gl = 0.0f;
  for (int j = threadIdx.x; j < N; j += blockDim.x) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float v = x[3 * j + k] - cf[k];
      const float vw = wts ? v * wts[j] : v;
      const float p = vw * v;
      const float e = fmaf(vw, v, -p);
      two_sum_acc(gh, gl, p);
      gl += e;
    }
  }
  block_sum_pair(gh, gl, sh);
  if (threadIdx.x == 0) {
    c32[f] = make_float4(cf[0], cf[1], cf[2], 0.0f);
    G[f] = pair_to_double(gh, gl);
  }
}

__global__ void frame_prep_f64(int F, int N, const double* __restrict__ frames,
                               const double* __restrict__ w64, float4* __restrict__ c32,
                               double4* __restrict__ c64, double* __restrict__ G, const double* __restrict__ wc64) {
  const int f = warp_global();
  if (f >= F) return;
  const int lane = threadIdx.x & 31;
  const double* x = frames + (size_t)f * N * 3;
  const double* cw = wc64 ? wc64 : w64;  // the centre: alignment weights when given
  double c[3] = {0, 0, 0};
  for (int j = lane; j < N; j += 32) {
    const double wj = cw ? cw[j] : 1.0;
#pragma unroll
    for (int k = 0; k < 3; ++k) c[k] += wj * x[3 * j + k];
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    c[k] = warp_sum_double(c[k]);
    if (!cw) c[k] /= (double)N;
  }
  double g = 0.0;
  for (int j = lane; j < N; j += 32) {
    const double wj = w64 ? w64[j] : 1.0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const double v = x[3 * j + k] - c[k];
      g += wj * v * v;
    }
  }
  g = warp_sum_double(g);
  if (lane == 0) {
    c32[f] = make_float4((float)c[0], (float)c[1], (float)c[2], 0.0f);
    c64[f] = make_double4(c[0], c[1], c[2], 0.0);
    G[f] = g;
  }
}

// ---------------------------------------------------------------------------------------
// Alignment of frame t onto a reference structure y (fit y onto x_t): H = sum_j wk_j
// y_j x_j^T over centred values, FP64 eigenvalue, D = (G_x + G_y - 2 lambda) dscale.
struct RefView {
  const void* coords;
  float4 c32;
  double4 c64;
  double G;
};

__device__ __forceinline__ void warp_corr_f64(int N, const double* __restrict__ x, double4 cx,
                                              const double* __restrict__ y, double4 cy,
                                              const double* __restrict__ w64, double* H) {
  const int lane = threadIdx.x & 31;
  double h[9];
#pragma unroll
  for (int e = 0; e < 9; ++e) h[e] = 0.0;
  for (int j = lane; j < N; j += 32) {
    const double wj = w64 ? w64[j] : 1.0;
    const double u[3] = {wj * (y[3 * j] - cy.x), wj * (y[3 * j + 1] - cy.y), wj * (y[3 * j + 2] - cy.z)};
    const double v[3] = {x[3 * j] - cx.x, x[3 * j + 1] - cx.y, x[3 * j + 2] - cx.z};
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
      for (int c = 0; c < 3; ++c) h[3 * b + c] = fma(u[b], v[c], h[3 * b + c]);
  }
#pragma unroll
  for (int e = 0; e < 9; ++e) H[e] = warp_sum_double(h[e]);
}

// D from H (lane 0 only), quaternion and decision flag
__device__ __forceinline__ void finish_alignment(const double* H, double Gx, double Gy, double dscale,
                                                 double eps, bool amb_check, double* outD, double4* outQ,
                                                 uint8_t* outFlag, bool* amb_out) {
  bool ok = true;
  double q[4];
  const double lam = top_eig_f64(H, 0.5 * (Gx + Gy), &ok, q);
  double D = (Gx + Gy - 2.0 * lam) * dscale;
  if (D < 0.0) D = 0.0;
  *outD = D;
  *outQ = make_double4(q[0], q[1], q[2], q[3]);
  // Worst-case error of the compensated FP32 correlation: chunks of 16 products are
  // summed in FP32 (|err| <= 16 u sum|terms| per entry), so |dD| <= ~100 u (Gx + Gy).
  // Decisions inside 1e-5 (Gx + Gy) of eps are re-done in FP64.
  const bool amb = amb_check && fabs(D - eps) <= 1e-5 * (Gx + Gy) * dscale;
  *amb_out = amb;
  *outFlag = (uint8_t)((D > eps ? 1 : 0) | (amb ? 2 : 0));
}

// FP32 decision alignment (one warp): pass 1 the correlation in FP32 and an FP32 eigen-
// solve for R (fits y onto x); pass 2 D = sum_j w_j |x_j - R y_j|^2 directly.  Returns D in
// true units on every lane together with a bound on |D - D_exact|:
//   lane sums of ~N/32 positive terms and a 5-level tree: (N/32 + 8) u D;
//   FP32 centring, rotation and residual rounding: <= 20 u sqrt(D (G_x + G_y));
// times a safety factor of 4 (u = 2^-24).
__device__ __forceinline__ double warp_direct_f32(int N, const float* __restrict__ x, float4 cx,
                                                  const float* __restrict__ y, float4 cy, const float* __restrict__ wts,
                                                  double Gx, double Gy, double dscale, double* bound) {
  const int lane = threadIdx.x & 31;
  float h[9];
#pragma unroll
  for (int e = 0; e < 9; ++e) h[e] = 0.0f;
#pragma unroll 4
  for (int j = lane; j < N; j += 32) {
    float u[3] = {y[3 * j] - cy.x, y[3 * j + 1] - cy.y, y[3 * j + 2] - cy.z};
    const float v[3] = {x[3 * j] - cx.x, x[3 * j + 1] - cx.y, x[3 * j + 2] - cx.z};
    if (wts) {
      const float wj = wts[j];
      u[0] *= wj;
      u[1] *= wj;
      u[2] *= wj;
    }
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
      for (int c = 0; c < 3; ++c) h[3 * b + c] = fmaf(u[b], v[c], h[3 * b + c]);
  }
#pragma unroll
  for (int e = 0; e < 9; ++e) h[e] = warp_sum_float(h[e]);
  float q[4], R[9];
  top_quat_f32(h, (float)(0.5 * (Gx + Gy)) * 1.00001f + 1e-30f, q);
  quat_to_rot(q, R);
  float dsum = 0.0f;
#pragma unroll 4
  for (int j = lane; j < N; j += 32) {
    const float u0 = y[3 * j] - cy.x, u1 = y[3 * j + 1] - cy.y, u2 = y[3 * j + 2] - cy.z;
    const float v0 = x[3 * j] - cx.x, v1 = x[3 * j + 1] - cx.y, v2 = x[3 * j + 2] - cx.z;
    const float d0 = v0 - fmaf(R[0], u0, fmaf(R[1], u1, R[2] * u2));
    const float d1 = v1 - fmaf(R[3], u0, fmaf(R[4], u1, R[5] * u2));
    const float d2 = v2 - fmaf(R[6], u0, fmaf(R[7], u1, R[8] * u2));
    const float t = fmaf(d0, d0, fmaf(d1, d1, d2 * d2));
    dsum = wts ? fmaf(wts[j], t, dsum) : dsum + t;
  }
  const double D = (double)warp_sum_float(dsum) * dscale;
  const double u32 = 5.9604644775390625e-8;
  const double G = (Gx + Gy) * dscale;
  *bound = 4.0 * (((double)N / 32.0 + 8.0) * u32 * D + 20.0 * u32 * sqrt(fmax(D, 0.0) * G)) + 1e-30;
  return D;
}

// One alignment of frame t onto the structure `ref` (-1: the stored prior y), written to
// slot `slot` of the outputs.  Returns, on every lane, whether the frame definitely exceeds
// eps (bit 0 of the flag set, outside the FP64 recheck band).
template <bool F64>
__device__ __forceinline__ bool align_frame(int mode, int t, int ref, int slot, int N, const void* __restrict__ frames_v,
                                            const RefView& prior, const float4* __restrict__ c32,
                                            const double4* __restrict__ c64, const double* __restrict__ fG,
                                            const float* __restrict__ wts, const double* __restrict__ w64,
                                            double dscale, double eps, double* __restrict__ outD,
                                            double4* __restrict__ outQ, uint8_t* __restrict__ outFlag,
                                            int* __restrict__ recheck_list, int* __restrict__ recheck_count) {
  const int lane = threadIdx.x & 31;
  const double Gx = fG[t];
  const double Gy = ref >= 0 ? fG[ref] : prior.G;
  if (F64) {
    double H[9];
    const double* frames = (const double*)frames_v;
    const double* y = ref >= 0 ? frames + (size_t)ref * N * 3 : (const double*)prior.coords;
    const double4 cy = ref >= 0 ? c64[ref] : prior.c64;
    warp_corr_f64(N, frames + (size_t)t * N * 3, c64[t], y, cy, w64, H);
    int ex = 0;
    if (lane == 0) {
      bool amb = false;
      finish_alignment(H, Gx, Gy, dscale, eps, false, outD + slot, outQ + slot, outFlag + slot, &amb);
      ex = outFlag[slot] & 1;
    }
    return __shfl_sync(0xffffffffu, ex, 0) != 0;
  }
  const float* frames = (const float*)frames_v;
  const float* y = ref >= 0 ? frames + (size_t)ref * N * 3 : (const float*)prior.coords;
  const float4 cy = ref >= 0 ? c32[ref] : prior.c32;
  double bound = 0.0;
  const double D = warp_direct_f32(N, frames + (size_t)t * N * 3, c32[t], y, cy, wts, Gx, Gy, dscale, &bound);
  const bool amb = fabs(D - eps) <= bound;  // the same on every lane (D and bound are)
  if (lane == 0) {
    outD[slot] = D;
    outFlag[slot] = (uint8_t)((D > eps ? 1 : 0) | (amb ? 2 : 0));
    if (amb) {
      const int pos = atomicAdd(recheck_count, 1);
      recheck_list[pos] = (slot << 1) | (mode == 0 ? 0 : 1);
    }
  }
  return D > eps && !amb;
}

// mode 0: band rows, one warp per (frame t in [t0, t1), offset k in 1..W).
// mode 1: chunk [t0, t1) against `ref_index`.  The warps take the frames in order with a
// grid stride; a frame that definitely exceeds eps lowers *stop (set to t1 beforehand), and
// frames past *stop are skipped: only the first exceeding frame matters to the search, and
// every frame t <= the final *stop is aligned (a warp skips t only when t > *stop at its
// check, and *stop never rises).  The frames aligned beyond the first exceed are bounded by
// the warps in flight instead of the chunk length.
template <bool F64>
__global__ void align_kernel(int mode, int F, int W, int t0, int t1, int ref_index, int N,
                             const void* __restrict__ frames_v, RefView prior,
                             const float4* __restrict__ c32, const double4* __restrict__ c64,
                             const double* __restrict__ fG, const float* __restrict__ wts,
                             const double* __restrict__ w64, double dscale, double eps,
                             double* __restrict__ outD, double4* __restrict__ outQ,
                             uint8_t* __restrict__ outFlag, int* __restrict__ recheck_list,
                             int* __restrict__ recheck_count, int* __restrict__ stop) {
  const int wid = warp_global();
  const int lane = threadIdx.x & 31;
  if (mode == 0) {  // band rows t in [t0, t1)
    const int t = t0 + wid / W;
    const int k = 1 + wid % W;
    if (t >= t1) return;
    const int ref = t - k;
    const int slot = t * W + k - 1;
    if (ref < 0) {
      if (lane == 0) {
        outD[slot] = -1.0;
        outFlag[slot] = 0;
      }
      return;
    }
    align_frame<F64>(0, t, ref, slot, N, frames_v, prior, c32, c64, fG, wts, w64, dscale, eps, outD, outQ, outFlag,
                     recheck_list, recheck_count);
    return;
  }
  const int nw = gridDim.x * (blockDim.x >> 5);
  for (int t = t0 + wid; t < t1; t += nw) {
    int lim = 0;
    if (lane == 0) lim = *(volatile int*)stop;
    lim = __shfl_sync(0xffffffffu, lim, 0);  // one value for the whole warp
    if (t > lim) return;
    const bool ex = align_frame<F64>(1, t, ref_index, t, N, frames_v, prior, c32, c64, fG, wts, w64, dscale, eps,
                                     outD, outQ, outFlag, recheck_list, recheck_count);
    if (ex && lane == 0) atomicMin(stop, t);
  }
}

// Chunk mode for large structures in FP32: one block of AT_THREADS per frame.  A round of
// the search lasts as long as one frame's alignment (the frames run side by side), and with
// one warp per frame that is two passes over N atoms by 32 lanes; here 256 threads share
// them.  The decision, its bound and the outputs are those of align_frame<false>, with the
// summation term of the bound counting ceil(N / 256) terms per thread, the 5-level warp
// tree and the sum over the 8 warps: (N / 256 + 16) u D.
constexpr int AT_WARPS = 8, AT_THREADS = 32 * AT_WARPS;
constexpr int AT_MIN_ATOMS = 1024;  // below this a warp per frame keeps more frames in flight

__global__ void __launch_bounds__(AT_THREADS)
align_chunk_block(int t0, int t1, int ref_index, int N, const float* __restrict__ frames, RefView prior,
                  const float4* __restrict__ c32, const double* __restrict__ fG, const float* __restrict__ wts,
                  double dscale, double eps, double* __restrict__ outD, uint8_t* __restrict__ outFlag,
                  int* __restrict__ recheck_list, int* __restrict__ recheck_count, int* __restrict__ stop) {
  __shared__ float red[AT_WARPS][9];
  __shared__ float sR[9];
  __shared__ int s_lim;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const float* y = ref_index >= 0 ? frames + (size_t)ref_index * N * 3 : (const float*)prior.coords;
  const float4 cy = ref_index >= 0 ? c32[ref_index] : prior.c32;
  const double Gy = ref_index >= 0 ? fG[ref_index] : prior.G;
  for (int t = t0 + blockIdx.x; t < t1; t += gridDim.x) {
    if (tid == 0) s_lim = *(volatile int*)stop;
    __syncthreads();
    if (t > s_lim) return;  // the same value for the whole block
    const float* x = frames + (size_t)t * N * 3;
    const float4 cx = c32[t];
    // pass 1: correlation of y onto x
    float h[9];
#pragma unroll
    for (int e = 0; e < 9; ++e) h[e] = 0.0f;
#pragma unroll 4
    for (int j = tid; j < N; j += AT_THREADS) {
      float u[3] = {y[3 * j] - cy.x, y[3 * j + 1] - cy.y, y[3 * j + 2] - cy.z};
      const float v[3] = {x[3 * j] - cx.x, x[3 * j + 1] - cx.y, x[3 * j + 2] - cx.z};
      if (wts) {
        const float wj = wts[j];
        u[0] *= wj;
        u[1] *= wj;
        u[2] *= wj;
      }
#pragma unroll
      for (int b = 0; b < 3; ++b)
#pragma unroll
        for (int c = 0; c < 3; ++c) h[3 * b + c] = fmaf(u[b], v[c], h[3 * b + c]);
    }
#pragma unroll
    for (int e = 0; e < 9; ++e) h[e] = warp_sum_float(h[e]);
    if (lane == 0)
#pragma unroll
      for (int e = 0; e < 9; ++e) red[warp][e] = h[e];
    __syncthreads();
    const double Gx = fG[t];
    if (tid == 0) {
      float H[9], q[4], R[9];
#pragma unroll
      for (int e = 0; e < 9; ++e) {
        float v = 0.0f;
        for (int w = 0; w < AT_WARPS; ++w) v += red[w][e];
        H[e] = v;
      }
      top_quat_f32(H, (float)(0.5 * (Gx + Gy)) * 1.00001f + 1e-30f, q);
      quat_to_rot(q, R);
#pragma unroll
      for (int e = 0; e < 9; ++e) sR[e] = R[e];
    }
    __syncthreads();
    float R[9];
#pragma unroll
    for (int e = 0; e < 9; ++e) R[e] = sR[e];
    // pass 2: D = sum_j w_j |x_j - R y_j|^2
    float dsum = 0.0f;
#pragma unroll 4
    for (int j = tid; j < N; j += AT_THREADS) {
      const float u0 = y[3 * j] - cy.x, u1 = y[3 * j + 1] - cy.y, u2 = y[3 * j + 2] - cy.z;
      const float v0 = x[3 * j] - cx.x, v1 = x[3 * j + 1] - cx.y, v2 = x[3 * j + 2] - cx.z;
      const float d0 = v0 - fmaf(R[0], u0, fmaf(R[1], u1, R[2] * u2));
      const float d1 = v1 - fmaf(R[3], u0, fmaf(R[4], u1, R[5] * u2));
      const float d2 = v2 - fmaf(R[6], u0, fmaf(R[7], u1, R[8] * u2));
      const float tt = fmaf(d0, d0, fmaf(d1, d1, d2 * d2));
      dsum = wts ? fmaf(wts[j], tt, dsum) : dsum + tt;
    }
    dsum = warp_sum_float(dsum);
    if (lane == 0) red[warp][0] = dsum;  // red's pass-1 values were consumed before the last barrier
    __syncthreads();
    if (tid == 0) {
      float ds = 0.0f;
      for (int w = 0; w < AT_WARPS; ++w) ds += red[w][0];
      const double D = (double)ds * dscale;
      const double u32 = 5.9604644775390625e-8;
      const double G = (Gx + Gy) * dscale;
      const double bound =
          4.0 * (((double)N / AT_THREADS + 16.0) * u32 * D + 20.0 * u32 * sqrt(fmax(D, 0.0) * G)) + 1e-30;
      const bool amb = fabs(D - eps) <= bound;
      outD[t] = D;
      outFlag[t] = (uint8_t)((D > eps ? 1 : 0) | (amb ? 2 : 0));
      if (amb) {
        const int pos = atomicAdd(recheck_count, 1);
        recheck_list[pos] = (t << 1) | 1;
      }
      if (D > eps && !amb) atomicMin(stop, t);
    }
    __syncthreads();  // red and sR are reused by the next frame
  }
}

// Accurate R_xy for the approximate frames (FP32 modes): compensated correlation, FP64
// eigenvalue and FP64 eigenvector.  The approximate MSD of Eq. (close_dist) is not
// stationary in R_xy, so R_xy must be accurate to FP32 rounding.  One warp per frame.
__global__ void xy_refine_kernel(int F, int N, const float* __restrict__ frames, RefView prior,
                                 const float4* __restrict__ c32, const double* __restrict__ fG,
                                 const float* __restrict__ wts, double dscale, FrameRec rec) {
  const int t = warp_global();
  if (t >= F) return;
  if (rec.flag[t] != 0) return;
  const int lane = threadIdx.x & 31;
  const int ref = rec.ref[t];
  const float* y = ref >= 0 ? frames + (size_t)ref * N * 3 : (const float*)prior.coords;
  const float4 cy = ref >= 0 ? c32[ref] : prior.c32;
  float H[9];
  warp_corr_pair_f32(N, frames + (size_t)t * N * 3, c32[t], y, cy, wts, H);
  if (lane == 0) {
    // H is accurate to ~1e-8 relative (compensated sums); the FP32 eigen-solve then gives
    // q to ~u / (relative gap) ~ 1e-7 with no FP64 instruction
    const float Gx = (float)fG[t], Gy = (float)(ref >= 0 ? fG[ref] : prior.G);
    float q[4];
    top_quat_f32(H, 0.5f * (Gx + Gy) * 1.00001f + 1e-30f, q);
    rec.qxy[t] = make_double4(q[0], q[1], q[2], q[3]);
  }
}

// R_xy of few large frames (FP32 modes): xy_refine_kernel's arithmetic with one block of
// XR_THREADS per frame instead of one warp (a single 5000-atom frame per call took 45 us on
// one warp).  Each thread keeps compensated (hi, lo) totals of its atoms' products (chunks of
// 16 folded by TwoSum), the warps add the pairs, and thread 0 adds the warps' pairs in order.
constexpr int XR_THREADS = 256, XR_WARPS = XR_THREADS / 32;
__global__ void __launch_bounds__(XR_THREADS, 2)
xy_refine_block(int F, int N, const float* __restrict__ frames, RefView prior, const float4* __restrict__ c32,
                const double* __restrict__ fG, const float* __restrict__ wts, FrameRec rec) {
  __shared__ float red[XR_WARPS][18];
  const int t = blockIdx.x;
  if (t >= F || rec.flag[t] != 0) return;  // uniform over the block
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int ref = rec.ref[t];
  const float* y = ref >= 0 ? frames + (size_t)ref * N * 3 : (const float*)prior.coords;
  const float4 cy = ref >= 0 ? c32[ref] : prior.c32;
  const float* x = frames + (size_t)t * N * 3;
  const float4 cx = c32[t];
  float p[9], hi[9], lo[9];
#pragma unroll
  for (int e = 0; e < 9; ++e) p[e] = hi[e] = lo[e] = 0.0f;
  int cnt = 0;
#pragma unroll 4
  for (int j = tid; j < N; j += XR_THREADS) {
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
    if (lane == 0) {
      red[warp][2 * e] = hi[e];
      red[warp][2 * e + 1] = lo[e];
    }
  }
  __syncthreads();
  if (tid == 0) {
    float H[9];
#pragma unroll
    for (int e = 0; e < 9; ++e) {
      float h = red[0][2 * e], l = red[0][2 * e + 1];
      for (int w = 1; w < XR_WARPS; ++w) two_sum_pair(h, l, red[w][2 * e], red[w][2 * e + 1]);
      H[e] = h + l;
    }
    const float Gx = (float)fG[t], Gy = (float)(ref >= 0 ? fG[ref] : prior.G);
    float q[4];
    top_quat_f32(H, 0.5f * (Gx + Gy) * 1.00001f + 1e-30f, q);
    rec.qxy[t] = make_double4(q[0], q[1], q[2], q[3]);
  }
}

// Full FP64 re-evaluation of D(x_t, y) from the raw FP32 coordinates: FP64 correlation
// and sums of squares, FP64 eigenvalue.  Centres: when they are weighted like the distance
// (no separate alignment weights) the frames' stored centres c32 serve: at the exact
// centres sum_j w_j (x_j - c_x) = 0 = sum_j w_j (y_j - c_y), so a centre error d enters
// G_x, G_y, H and hence D only at second order (|d|^2 sum w, ~1e-13 nm^2 for FP32 centres
// from compensated sums).  With alignment weights w' != w that first-order term does not
// vanish and the centres are summed in FP64 first.
//
// FP64 issues at a small fraction of the FP32 rate on this part, so one warp per entry
// would leave a 5000-atom structure's ~1.5e5 FP64 operations to one SM (~0.2 ms, and an
// entry ends a search round).  The first RC_CAP entries are therefore shared by all the
// blocks of the launch: block b sums its slice of the atoms and stores its 11 partials
// (H, G_x, G_y), and the entry's last block -- found by an atomic count after a fence;
// nothing waits -- adds the partials in block order, solves for the eigenvalue and writes
// the decision.  Entries past RC_CAP, and all entries with FP64 centres, take one warp each.
constexpr int RC_CAP = 32;         // entries shared by the blocks
constexpr int RC_BLOCKS_MAX = 76;  // grid cap (the partial buffer holds RC_CAP x this)
constexpr int RC_THREADS = 128;
constexpr int RC_PARTS = 11;  // H (9), G_x, G_y

__device__ __forceinline__ void recheck_decode(int code, int W, int chunk_ref, int& t, int& ref, int& slot,
                                               bool& is_chunk) {
  slot = code >> 1;
  is_chunk = code & 1;
  if (is_chunk) {
    t = slot;
    ref = chunk_ref;
  } else {
    t = slot / W;
    ref = t - (slot % W + 1);
  }
}

// the decision from the FP64 sums (one thread)
__device__ __forceinline__ void recheck_finish(const double* h, double gx, double gy, double dscale, double eps,
                                               int slot, bool is_chunk, double* bandD, uint8_t* bandFlag,
                                               double* chunkD, uint8_t* chunkFlag,
                                               unsigned long long* n_rechecks) {
  bool ok = true;
  const double lam = top_eig_f64(h, 0.5 * (gx + gy), &ok, nullptr);
  double D = (gx + gy - 2.0 * lam) * dscale;
  if (D < 0.0) D = 0.0;
  const uint8_t fl = (uint8_t)(D > eps ? 1 : 0);
  if (is_chunk) {
    chunkD[slot] = D;
    chunkFlag[slot] = fl;
  } else {
    bandD[slot] = D;
    bandFlag[slot] = fl;
  }
  atomicAdd(n_rechecks, 1ull);
}

// FP64 sums over atoms j = j0 + k * stride < j1 of one entry (this thread's share)
__device__ __forceinline__ void recheck_sums(int j0, int j1, int stride, const float* __restrict__ x,
                                             const float* __restrict__ y, const double* cx, const double* cy,
                                             const double* __restrict__ w64, double* h, double& gx, double& gy) {
  for (int j = j0; j < j1; j += stride) {
    const double wj = w64 ? w64[j] : 1.0;
    double u[3], v[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      u[c] = (double)y[3 * j + c] - cy[c];
      v[c] = (double)x[3 * j + c] - cx[c];
      gx += wj * v[c] * v[c];
      gy += wj * u[c] * u[c];
    }
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
      for (int c = 0; c < 3; ++c) h[3 * b + c] += wj * u[b] * v[c];
  }
}

__device__ __forceinline__ void recheck_centres_c32(int t, int ref, const float4* __restrict__ c32,
                                                    const RefView& prior, double* cx, double* cy) {
  const float4 a = c32[t];
  const float4 b = ref >= 0 ? c32[ref] : prior.c32;
  cx[0] = a.x;
  cx[1] = a.y;
  cx[2] = a.z;
  cy[0] = b.x;
  cy[1] = b.y;
  cy[2] = b.z;
}

__global__ void __launch_bounds__(RC_THREADS)
recheck_kernel(const int* __restrict__ list, const int* __restrict__ count, int W, int N,
               const float* __restrict__ frames, RefView prior, int chunk_ref, const double* __restrict__ w64,
               double dscale, double eps, double* bandD, uint8_t* bandFlag, double* chunkD, uint8_t* chunkFlag,
               unsigned long long* n_rechecks, const double* __restrict__ wc64, const float4* __restrict__ c32,
               double* __restrict__ part, int* __restrict__ done) {
  __shared__ double red[RC_THREADS / 32][RC_PARTS];
  __shared__ int s_last;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int n = *count, nb = gridDim.x, blk = blockIdx.x;
  const int nshared = wc64 ? 0 : min(n, RC_CAP);
  const int per = (N + nb - 1) / nb, j0 = blk * per, j1 = min(N, j0 + per);
  for (int e = 0; e < nshared; ++e) {
    int t, ref, slot;
    bool is_chunk;
    recheck_decode(list[e], W, chunk_ref, t, ref, slot, is_chunk);
    const float* x = frames + (size_t)t * N * 3;
    const float* y = ref >= 0 ? frames + (size_t)ref * N * 3 : (const float*)prior.coords;
    double cx[3], cy[3];
    recheck_centres_c32(t, ref, c32, prior, cx, cy);
    double h[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0}, gx = 0.0, gy = 0.0;
    recheck_sums(j0 + tid, j1, RC_THREADS, x, y, cx, cy, w64, h, gx, gy);
#pragma unroll
    for (int k = 0; k < 9; ++k) h[k] = warp_sum_double(h[k]);
    gx = warp_sum_double(gx);
    gy = warp_sum_double(gy);
    if (lane == 0) {
#pragma unroll
      for (int k = 0; k < 9; ++k) red[warp][k] = h[k];
      red[warp][9] = gx;
      red[warp][10] = gy;
    }
    __syncthreads();
    if (tid == 0) {
      double* my = part + ((size_t)e * RC_BLOCKS_MAX + blk) * RC_PARTS;
      for (int k = 0; k < RC_PARTS; ++k) {
        double v = 0.0;
        for (int w = 0; w < RC_THREADS / 32; ++w) v += red[w][k];
        my[k] = v;
      }
      __threadfence();  // the partials are visible before the count says so
      s_last = atomicAdd(&done[e], 1) == nb - 1;
    }
    __syncthreads();
    if (s_last && tid == 0) {
      __threadfence();
      double acc[RC_PARTS];
      for (int k = 0; k < RC_PARTS; ++k) acc[k] = 0.0;
      for (int bb = 0; bb < nb; ++bb) {  // block order: the same sums whichever block is last
        const double* pp = part + ((size_t)e * RC_BLOCKS_MAX + bb) * RC_PARTS;
        for (int k = 0; k < RC_PARTS; ++k) acc[k] += __ldcg(pp + k);
      }
      recheck_finish(acc, acc[9], acc[10], dscale, eps, slot, is_chunk, bandD, bandFlag, chunkD, chunkFlag,
                     n_rechecks);
      done[e] = 0;  // ready for the next launch
    }
    __syncthreads();  // red and s_last are reused by the next entry
  }
  // the rest: one warp per entry
  const int nw = nb * (RC_THREADS / 32);
  for (int wid = nshared + blk * (RC_THREADS / 32) + warp; wid < n; wid += nw) {
    int t, ref, slot;
    bool is_chunk;
    recheck_decode(list[wid], W, chunk_ref, t, ref, slot, is_chunk);
    const float* x = frames + (size_t)t * N * 3;
    const float* y = ref >= 0 ? frames + (size_t)ref * N * 3 : (const float*)prior.coords;
    double cx[3], cy[3];
    if (!wc64) {
      recheck_centres_c32(t, ref, c32, prior, cx, cy);
    } else {
#pragma unroll
      for (int c = 0; c < 3; ++c) cx[c] = cy[c] = 0.0;
      for (int j = lane; j < N; j += 32) {
        const double wj = wc64[j];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          cx[c] += wj * (double)x[3 * j + c];
          cy[c] += wj * (double)y[3 * j + c];
        }
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        cx[c] = warp_sum_double(cx[c]);
        cy[c] = warp_sum_double(cy[c]);
      }
    }
    double h[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0}, gx = 0.0, gy = 0.0;
    recheck_sums(lane, N, 32, x, y, cx, cy, w64, h, gx, gy);
#pragma unroll
    for (int k = 0; k < 9; ++k) h[k] = warp_sum_double(h[k]);
    gx = warp_sum_double(gx);
    gy = warp_sum_double(gy);
    if (lane == 0)
      recheck_finish(h, gx, gy, dscale, eps, slot, is_chunk, bandD, bandFlag, chunkD, chunkFlag, n_rechecks);
  }
}

__global__ void set_int_kernel(int* p, int v) { *p = v; }
__global__ void set_chunk_round_kernel(int* recheck_count, int* stop, int* first, int t1) {
  *recheck_count = 0;
  *stop = t1;
  *first = t1;
}

// frames past *stop may not have been aligned by the chunk kernel: the scan ends at *stop
__global__ void first_exceed_kernel(int t0, int t1, const uint8_t* __restrict__ flag, const int* __restrict__ stop,
                                    int* first) {
  const int t = t0 + blockIdx.x * blockDim.x + threadIdx.x;
  const int hi = stop ? min(t1, *stop + 1) : t1;
  if (t < hi && (flag[t] & 1)) atomicMin(first, t);
}

// ---------------------------------------------------------------------------------------
// Refresh search over the band.  After frame t the state is the offset o = t - r of t from
// its close structure r (0 = frame t refreshed).  Frame t+1 compares with x_r at offset
// o+1: it refreshes if D(x_{t+1}, x_{t+1-(o+1)}) > eps, otherwise its state is o+1.  With
// only W offsets computed, state W cannot be continued (OVF).  Each frame's transition is
// a map of the 8 states {0..6, OVF=7}, packed 4 bits per state; maps compose
// associatively, so a block-wide scan decides 1024 frames at a time.
constexpr unsigned OVF = 7u;
__device__ __forceinline__ unsigned map_apply(unsigned m, unsigned s) { return (m >> (4 * s)) & 15u; }
__device__ __forceinline__ unsigned map_compose(unsigned later, unsigned earlier) {
  unsigned out = 0;
#pragma unroll
  for (int s = 0; s < 8; ++s) out |= map_apply(later, map_apply(earlier, s)) << (4 * s);
  return out;
}
__device__ __forceinline__ unsigned frame_map(const uint8_t* bflag, int t, int W) {
  unsigned m = 0;
#pragma unroll
  for (int s = 0; s < 8; ++s) {
    unsigned nxt = OVF;
    if (s < W) nxt = (bflag[(size_t)t * W + s] & 1) ? 0u : (unsigned)(s + 1);
    m |= nxt << (4 * s);
  }
  return m;
}

constexpr int SCAN_THREADS = 1024;
__global__ void __launch_bounds__(SCAN_THREADS) band_scan_kernel(int F, int W, int t0, int o_init,
                                                                 const double* __restrict__ bandD,
                                                                 const double4* __restrict__ bandQ,
                                                                 const uint8_t* __restrict__ bandFlag,
                                                                 FrameRec rec, ScanResult* res) {
  __shared__ unsigned s_warp[32];
  __shared__ unsigned s_state[SCAN_THREADS];
  __shared__ int s_stop;
  const int tid = threadIdx.x, lane = tid & 31, wrp = tid >> 5;
  unsigned s_in = (unsigned)o_init;
  int nref = 0;
  for (int base = t0; base < F; base += SCAN_THREADS) {
    const int t = base + tid;
    unsigned m = (t < F) ? frame_map(bandFlag, t, W) : 0x76543210u;  // identity beyond F
    // warp inclusive scan (later o earlier)
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const unsigned other = __shfl_up_sync(0xffffffffu, m, d);
      if (lane >= d) m = map_compose(m, other);
    }
    if (lane == 31) s_warp[wrp] = m;
    if (tid == 0) s_stop = F;
    __syncthreads();
    if (wrp == 0) {
      unsigned wm = s_warp[lane];
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const unsigned other = __shfl_up_sync(0xffffffffu, wm, d);
        if (lane >= d) wm = map_compose(wm, other);
      }
      s_warp[lane] = wm;  // inclusive prefix over warps
    }
    __syncthreads();
    if (wrp > 0) m = map_compose(m, s_warp[wrp - 1]);
    const unsigned after = map_apply(m, s_in);
    s_state[tid] = after;
    __syncthreads();
    const unsigned before = tid == 0 ? s_in : s_state[tid - 1];
    if (t < F && after == OVF) atomicMin(&s_stop, t);
    __syncthreads();
    const int stop = s_stop;
    if (t < F && t < stop) {
      if (after == 0) {
        rec.flag[t] = 1;
        rec.ref[t] = t;
        rec.dxy[t] = bandD[(size_t)t * W + before];  // offset before+1 triggered
        rec.qxy[t] = make_double4(1.0, 0.0, 0.0, 0.0);
      } else {
        const size_t sl = (size_t)t * W + (after - 1);
        rec.flag[t] = 0;
        rec.ref[t] = t - (int)after;
        rec.dxy[t] = bandD[sl];
        rec.qxy[t] = bandQ[sl];
      }
    }
    nref += __syncthreads_count(t < F && t < stop && after == 0);
    if (stop < F) {
      if (tid == 0) {
        // frame stop-1 had offset W from its close structure
        res->t_stop = stop;
        res->ref = stop - 1 - W;
        res->nref = nref;
      }
      return;
    }
    s_in = s_state[SCAN_THREADS - 1];
    __syncthreads();
  }
  if (tid == 0) {
    res->t_stop = F;
    res->ref = -2;
    res->nref = nref;
  }
}

__global__ void chunk_records_kernel(int t0, int t_end, int t1, int ref, const double* __restrict__ cD,
                                     const double4* __restrict__ cQ, FrameRec rec, const int* __restrict__ t_end_dev) {
  if (t_end_dev) t_end = *t_end_dev;  // the first exceed as found on the device
  const int t = t0 + blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= t1 || t > t_end) return;
  if (t < t_end) {
    rec.flag[t] = 0;
    rec.ref[t] = ref;
    rec.dxy[t] = cD[t];
    rec.qxy[t] = cQ[t];
  } else {  // t == t_end < t1: reassignment
    rec.flag[t] = 1;
    rec.ref[t] = t;
    rec.dxy[t] = cD[t];
    rec.qxy[t] = make_double4(1.0, 0.0, 0.0, 0.0);
  }
}

__global__ void initial_record_kernel(FrameRec rec) {
  rec.flag[0] = 2;
  rec.ref[0] = 0;
  rec.dxy[0] = -1.0;
  rec.qxy[0] = make_double4(1.0, 0.0, 0.0, 0.0);
}

// Stream compaction of refresh / approximate frames in time order (single block).
// seg_of_frame[t] = prior_seg + number of reassignments in [0, t].
__global__ void __launch_bounds__(SCAN_THREADS) compact_kernel(int F, const uint8_t* __restrict__ flag,
                                                               int* refresh_list, int* refresh_count,
                                                               int* seg_of_frame, int* approx_list,
                                                               int* approx_count, int* approx_seg, int prior_seg) {
  // 4 consecutive frames per thread, 4096 per block scan.  The approximate frames of a
  // round are compacted into shared memory first and copied out by the whole block, so the
  // global stores stay contiguous across the warp; seg_of_frame goes out as one 16-byte
  // store per thread.
  constexpr int CI = 4;
  __shared__ int s_r[32], s_a[32];
  __shared__ int s_list[SCAN_THREADS * CI], s_seg[SCAN_THREADS * CI];
  const int tid = threadIdx.x, lane = tid & 31, wrp = tid >> 5;
  int nref = 0, napp = 0;
  for (int base = 0; base < F; base += SCAN_THREADS * CI) {
    const int t0 = base + tid * CI;
    uint8_t fl[CI];
    int cr = 0, ca = 0;
#pragma unroll
    for (int k = 0; k < CI; ++k) {
      const bool in = t0 + k < F;
      fl[k] = in ? flag[t0 + k] : (uint8_t)0;
      cr += (in && fl[k] != 0) ? 1 : 0;
      ca += (in && fl[k] == 0) ? 1 : 0;
    }
    int r = cr, a = ca;  // inclusive scans over the block
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int ro = __shfl_up_sync(0xffffffffu, r, d);
      const int ao = __shfl_up_sync(0xffffffffu, a, d);
      if (lane >= d) {
        r += ro;
        a += ao;
      }
    }
    if (lane == 31) {
      s_r[wrp] = r;
      s_a[wrp] = a;
    }
    __syncthreads();
    if (wrp == 0) {
      int rr = s_r[lane], aa = s_a[lane];
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const int ro = __shfl_up_sync(0xffffffffu, rr, d);
        const int ao = __shfl_up_sync(0xffffffffu, aa, d);
        if (lane >= d) {
          rr += ro;
          aa += ao;
        }
      }
      s_r[lane] = rr;
      s_a[lane] = aa;
    }
    __syncthreads();
    if (wrp > 0) {
      r += s_r[wrp - 1];
      a += s_a[wrp - 1];
    }
    const int tot_r = s_r[31], tot_a = s_a[31];
    int pr = nref + r - cr, pa = a - ca;  // refreshes before t0 (global), approximate (block-local)
    int seg[CI];
#pragma unroll
    for (int k = 0; k < CI; ++k) {
      const int t = t0 + k;
      if (t < F && fl[k] != 0) refresh_list[pr++] = t;
      seg[k] = prior_seg + pr;  // inclusive count of reassignments
      if (t < F && fl[k] == 0) {
        s_list[pa] = t;
        s_seg[pa] = seg[k];
        ++pa;
      }
    }
    if (t0 + CI <= F)
      *reinterpret_cast<int4*>(seg_of_frame + t0) = make_int4(seg[0], seg[1], seg[2], seg[3]);
    else
#pragma unroll
      for (int k = 0; k < CI; ++k)
        if (t0 + k < F) seg_of_frame[t0 + k] = seg[k];
    __syncthreads();
    for (int i = tid; i < tot_a; i += SCAN_THREADS) {
      approx_list[napp + i] = s_list[i];
      approx_seg[napp + i] = s_seg[i];
    }
    nref += tot_r;
    napp += tot_a;
    __syncthreads();
  }
  if (tid == 0) {
    *refresh_count = nref;
    *approx_count = napp;
  }
}

// ---------------------------------------------------------------------------------------
// Path CVs: m = min D, l = sum exp(-lambda (D - m)), s = sum q e / l, z = m - ln(l)/lambda.
// FP32 modes: exponentials and sums in FP32 (relative error ~1e-7, far inside the
// tolerance).  s is accumulated about q_m, the index of a landmark at the minimum:
// s = q_m + sum (q_i - q_m) e_i / l, so that its FP32 error is relative to the spread of the
// weights (a few landmarks) instead of to s itself (up to M): the adjoint's gamma^s_i =
// -lambda p_i (q_i - s) carries any error of s as a shift of every term.  One warp per
// frame.
// With want_p the distances are overwritten by the softmax weights p_i = exp(-lambda (D_i -
// m)) / l that the adjoint consumes (gamma^z_i = p_i, gamma^s_i = -lambda p_i (q_i - s)).
// s, z of frame f from its MSD row (Eqs. 5-6, shifted log-sum-exp), one warp
__device__ __forceinline__ void finalize_warp_f32(int f, int M, float* __restrict__ D, const float* __restrict__ q,
                                                  float lambda, double* __restrict__ s, double* __restrict__ z,
                                                  float* __restrict__ mstat, double* __restrict__ msd, int want_p) {
  const int lane = threadIdx.x & 31;
  float* d = D + (size_t)f * M;
  float m = 3.4e38f, qm = 0.0f;  // the minimum and the q of a landmark attaining it
  for (int i = lane; i < M; i += 32) {
    const float v = d[i];
    if (v < m) {
      m = v;
      qm = q[i];
    }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {  // (m, qm) in lexicographic order: one result on all lanes
    const float m2 = __shfl_xor_sync(0xffffffffu, m, off), q2 = __shfl_xor_sync(0xffffffffu, qm, off);
    if (m2 < m || (m2 == m && q2 < qm)) {
      m = m2;
      qm = q2;
    }
  }
  // l >= 1 and every term is in (0, 1]: FP32 sums are accurate to ~1e-7 relative
  float l = 0.0f, sq = 0.0f;
  for (int i = lane; i < M; i += 32) {
    const float e = expf(-lambda * (d[i] - m));
    l += e;
    sq = fmaf(q[i] - qm, e, sq);
    if (msd) msd[(size_t)f * M + i] = (double)d[i];
  }
  l = warp_sum_float(l);
  sq = warp_sum_float(sq);
  if (want_p) {
    const float il = 1.0f / l;
    for (int i = lane; i < M; i += 32) d[i] = expf(-lambda * (d[i] - m)) * il;
  }
  if (lane == 0) {
    s[f] = (double)qm + (double)(sq / l);
    z[f] = (double)(m - __logf(l) / lambda);
    mstat[2 * f] = m;
    mstat[2 * f + 1] = l;
  }
}

// The path CVs of few frames against many landmarks (FP32 modes): finalize_warp_f32's
// arithmetic with one block of FN_THREADS per frame (one 2000-landmark frame per call took
// 29 us on one warp).  The minimum and q_m reduce in (value, q) order, the sums over the
// block's warps in warp order.
constexpr int FN_THREADS = 256, FN_WARPS = FN_THREADS / 32;
__global__ void __launch_bounds__(FN_THREADS)
finalize_block_f32(int F, int M, float* __restrict__ D, const float* __restrict__ q, float lambda,
                   double* __restrict__ s, double* __restrict__ z, float* __restrict__ mstat,
                   double* __restrict__ msd, int want_p) {
  __shared__ float sm_m[FN_WARPS], sm_q[FN_WARPS], sm_l[FN_WARPS], sm_s[FN_WARPS];
  const int f = blockIdx.x;
  if (f >= F) return;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  float* d = D + (size_t)f * M;
  float m = 3.4e38f, qm = 0.0f;
  for (int i = tid; i < M; i += FN_THREADS) {
    const float v = d[i];
    if (v < m) {
      m = v;
      qm = q[i];
    }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const float m2 = __shfl_xor_sync(0xffffffffu, m, off), q2 = __shfl_xor_sync(0xffffffffu, qm, off);
    if (m2 < m || (m2 == m && q2 < qm)) {
      m = m2;
      qm = q2;
    }
  }
  if (lane == 0) {
    sm_m[warp] = m;
    sm_q[warp] = qm;
  }
  __syncthreads();
  m = sm_m[0];
  qm = sm_q[0];
  for (int w = 1; w < FN_WARPS; ++w)
    if (sm_m[w] < m || (sm_m[w] == m && sm_q[w] < qm)) {
      m = sm_m[w];
      qm = sm_q[w];
    }
  float l = 0.0f, sq = 0.0f;
  for (int i = tid; i < M; i += FN_THREADS) {
    const float e = expf(-lambda * (d[i] - m));
    l += e;
    sq = fmaf(q[i] - qm, e, sq);
    if (msd) msd[(size_t)f * M + i] = (double)d[i];
  }
  l = warp_sum_float(l);
  sq = warp_sum_float(sq);
  if (lane == 0) {
    sm_l[warp] = l;
    sm_s[warp] = sq;
  }
  __syncthreads();
  l = 0.0f;
  sq = 0.0f;
  for (int w = 0; w < FN_WARPS; ++w) {
    l += sm_l[w];
    sq += sm_s[w];
  }
  if (want_p) {
    const float il = 1.0f / l;
    for (int i = tid; i < M; i += FN_THREADS) d[i] = expf(-lambda * (d[i] - m)) * il;
  }
  if (tid == 0) {
    s[f] = (double)qm + (double)(sq / l);
    z[f] = (double)(m - __logf(l) / lambda);
    mstat[2 * f] = m;
    mstat[2 * f + 1] = l;
  }
}

__global__ void finalize_f32(int F, int M, float* __restrict__ D, const float* __restrict__ q, float lambda,
                             double* __restrict__ s, double* __restrict__ z, float* __restrict__ mstat,
                             double* __restrict__ msd, int want_p) {
  const int f = warp_global();
  if (f >= F) return;
  finalize_warp_f32(f, M, D, q, lambda, s, z, mstat, msd, want_p);
}

// ---- group forms: frames of many instances, one warp per frame, instance found by
// binary search over the instances' first global frame index
__device__ __forceinline__ int group_instance(const GroupInst* __restrict__ I, int n, int g) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (I[mid].fbase <= g) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__global__ void frame_prep_group_f32(const GroupInst* __restrict__ I, int n, int Ftot) {
  const int g = warp_global();
  if (g >= Ftot) return;
  const GroupInst& t = I[group_instance(I, n, g)];
  frame_prep_warp_f32(g - t.fbase, t.N, t.frames, t.w, t.c32, t.fG);
}

__global__ void finalize_group_f32(const GroupInst* __restrict__ I, int n, int Ftot) {
  const int g = warp_global();
  if (g >= Ftot) return;
  const GroupInst& t = I[group_instance(I, n, g)];
  finalize_warp_f32(g - t.fbase, t.M, t.D, t.q32, t.lambda, t.s, t.z, t.mstat, t.msd, 0);
}

__global__ void finalize_f64(int F, int M, double* __restrict__ D, const double* __restrict__ q,
                             double lambda, double* __restrict__ s, double* __restrict__ z,
                             double* __restrict__ mstat64, double* __restrict__ msd, int want_p) {
  const int f = warp_global();
  if (f >= F) return;
  const int lane = threadIdx.x & 31;
  double* d = D + (size_t)f * M;
  double m = 1.0e300;
  for (int i = lane; i < M; i += 32) m = fmin(m, d[i]);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) m = fmin(m, __shfl_xor_sync(0xffffffffu, m, off));
  double l = 0.0, sq = 0.0;
  for (int i = lane; i < M; i += 32) {
    const double e = exp(-lambda * (d[i] - m));
    l += e;
    sq += q[i] * e;
    if (msd) msd[(size_t)f * M + i] = d[i];
  }
  l = warp_sum_double(l);
  sq = warp_sum_double(sq);
  if (want_p)
    for (int i = lane; i < M; i += 32) d[i] = exp(-lambda * (d[i] - m)) / l;
  if (lane == 0) {
    s[f] = sq / l;
    z[f] = m - log(l) / lambda;
    mstat64[2 * f] = m;
    mstat64[2 * f + 1] = l;
  }
}

template <typename T>
__global__ void combine_grad_kernel(size_t n, int N3, const double* __restrict__ g_s,
                                    const double* __restrict__ g_z, const T* __restrict__ gs,
                                    const T* __restrict__ gz, T* __restrict__ out) {
  const size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (k >= n) return;
  const size_t f = k / (size_t)N3;
  const double a = g_s ? g_s[f] : 0.0, b = g_z ? g_z[f] : 0.0;
  out[k] = (T)(a * (double)gs[k] + b * (double)gz[k]);
}

// FP32 rows: one block per frame row (grid-stride over rows), 16-byte vectors when the row
// length 3N is a multiple of 4 and the buffers are 16-byte aligned; FP32 arithmetic (the
// output is FP32)
template <bool VEC>
__global__ void combine_rows_f32(int F, int N3, const double* __restrict__ g_s, const double* __restrict__ g_z,
                                 const float* __restrict__ gs, const float* __restrict__ gz, float* __restrict__ out) {
  for (int f = blockIdx.x; f < F; f += gridDim.x) {
    const float a = g_s ? (float)g_s[f] : 0.0f, b = g_z ? (float)g_z[f] : 0.0f;
    const size_t base = (size_t)f * N3;
    if (VEC) {
      const float4* x = reinterpret_cast<const float4*>(gs + base);
      const float4* y = reinterpret_cast<const float4*>(gz + base);
      float4* o = reinterpret_cast<float4*>(out + base);
      for (int e = threadIdx.x; e < N3 / 4; e += blockDim.x) {
        const float4 u = x[e], v = y[e];
        o[e] = make_float4(fmaf(a, u.x, b * v.x), fmaf(a, u.y, b * v.y), fmaf(a, u.z, b * v.z), fmaf(a, u.w, b * v.w));
      }
    } else {
      for (int e = threadIdx.x; e < N3; e += blockDim.x) out[base + e] = fmaf(a, gs[base + e], b * gz[base + e]);
    }
  }
}

__global__ void fill_u8_kernel(uint8_t* p, uint8_t v, size_t n) {
  const size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (k < n) p[k] = v;
}

inline unsigned blocks_for(size_t n, unsigned per) { return (unsigned)((n + per - 1) / per); }

RefView view_of(const RefDesc& r) { return RefView{r.coords, r.c32, r.c64, r.G}; }

}  // namespace

// ---------------------------------------------------------------------------------------
void launch_frame_prep(Prec p, int F, const void* frames, const LandmarkDev& L, FrameInfo fi,
                       cudaStream_t st) {
  if (F <= 0) return;
  const unsigned blocks = blocks_for((size_t)F, WARPS_PER_BLOCK);
  if (p == P_F64)
    frame_prep_f64<<<blocks, 32 * WARPS_PER_BLOCK, 0, st>>>(F, L.N, (const double*)frames, L.w64, fi.c32,
                                                            fi.c64, fi.G, L.wa64);
  else if (F <= 1216 && L.N >= 256)  // few large frames: one block per frame
    frame_prep_f32_block<<<F, 256, 0, st>>>(F, L.N, (const float*)frames, L.w, fi.c32, fi.G, L.wa);
  else
    frame_prep_f32<<<blocks, 32 * WARPS_PER_BLOCK, 0, st>>>(F, L.N, (const float*)frames, L.w, fi.c32, fi.c64,
                                                            fi.G, L.wa);
  note_launch();
}

void launch_align_band(Prec p, int F, int W, int t_lo, int t_hi, const void* frames, const LandmarkDev& L,
                       FrameInfo fi, double eps, AlignOut out, int* recheck_list, int* recheck_count,
                       cudaStream_t st) {
  t_lo = t_lo < 1 ? 1 : t_lo;
  if (t_hi > F) t_hi = F;
  if (t_hi <= t_lo) return;
  const size_t warps = (size_t)(t_hi - t_lo) * W;
  const unsigned blocks = blocks_for(warps, WARPS_PER_BLOCK);
  RefView none{nullptr, make_float4(0, 0, 0, 0), make_double4(0, 0, 0, 0), 0.0};
  if (p == P_F64)
    align_kernel<true><<<blocks, 32 * WARPS_PER_BLOCK, 0, st>>>(0, F, W, t_lo, t_hi, 0, L.N, frames, none, fi.c32,
                                                                fi.c64, fi.G, L.w, L.w64, L.dscale, eps, out.D, out.q,
                                                                out.flag, recheck_list, recheck_count, nullptr);
  else
    align_kernel<false><<<blocks, 32 * WARPS_PER_BLOCK, 0, st>>>(0, F, W, t_lo, t_hi, 0, L.N, frames, none, fi.c32,
                                                                 fi.c64, fi.G, L.w, L.w64, L.dscale, eps, out.D, out.q,
                                                                 out.flag, recheck_list, recheck_count, nullptr);
  note_launch();
}

// resident blocks of the chunk kernel on the whole device (the grid of its frame loop)
template <bool F64>
unsigned align_chunk_grid() {
  thread_local int dev = -1;
  thread_local unsigned grid = 0;
  int d = 0;
  cudaGetDevice(&d);
  if (d != dev || grid == 0) {
    int sms = 0, per = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, d);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, align_kernel<F64>, 32 * WARPS_PER_BLOCK, 0);
    grid = (unsigned)std::max(1, sms * std::max(per, 1));
    dev = d;
  }
  return grid;
}

void launch_align_chunk(Prec p, int t0, int t1, const void* frames, const LandmarkDev& L, FrameInfo fi,
                        int ref_index, const RefDesc& prior, double eps, AlignOut out, int* recheck_list,
                        int* recheck_count, int* stop, cudaStream_t st) {
  if (t1 <= t0) return;
  if (p != P_F64 && L.N >= AT_MIN_ATOMS) {
    thread_local int dev = -1;
    thread_local unsigned grid = 0;
    int d = 0;
    cudaGetDevice(&d);
    if (d != dev || grid == 0) {
      int sms = 0, per = 0;
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, d);
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, align_chunk_block, AT_THREADS, 0);
      grid = (unsigned)std::max(1, sms * std::max(per, 1));
      dev = d;
    }
    align_chunk_block<<<std::min((unsigned)(t1 - t0), grid), AT_THREADS, 0, st>>>(
        t0, t1, ref_index, L.N, (const float*)frames, view_of(prior), fi.c32, fi.G, L.w, L.dscale, eps, out.D,
        out.flag, recheck_list, recheck_count, stop);
    note_launch();
    return;
  }
  const unsigned need = blocks_for((size_t)(t1 - t0), WARPS_PER_BLOCK);
  if (p == P_F64)
    align_kernel<true><<<std::min(need, align_chunk_grid<true>()), 32 * WARPS_PER_BLOCK, 0, st>>>(
        1, 0, 1, t0, t1, ref_index, L.N, frames, view_of(prior), fi.c32, fi.c64, fi.G, L.w, L.w64, L.dscale, eps,
        out.D, out.q, out.flag, recheck_list, recheck_count, stop);
  else
    align_kernel<false><<<std::min(need, align_chunk_grid<false>()), 32 * WARPS_PER_BLOCK, 0, st>>>(
        1, 0, 1, t0, t1, ref_index, L.N, frames, view_of(prior), fi.c32, fi.c64, fi.G, L.w, L.w64, L.dscale, eps,
        out.D, out.q, out.flag, recheck_list, recheck_count, stop);
  note_launch();
}

void launch_recheck(Prec p, int max_entries, const int* list, const int* count, int W, const void* frames,
                    const LandmarkDev& L, const float4* c32, const RefDesc& prior, int chunk_ref, double eps,
                    AlignOut band, AlignOut chunk, unsigned long long* n_rechecks, RecheckScratch scr,
                    cudaStream_t st) {
  if (p == P_F64 || max_entries <= 0) return;
  // the list holds the decisions within the FP32 error bound of eps, a few per round: the
  // blocks share each of the first RC_CAP entries (a slice of ~256 atoms or more each) and
  // loop over the rest one warp per entry; at most RC_BLOCKS_MAX blocks (a grid sized for
  // max_entries would spend its time starting and retiring empty blocks)
  const unsigned by_atoms = blocks_for((size_t)L.N, 256);
  const unsigned by_list = blocks_for((size_t)max_entries, RC_THREADS / 32);
  const unsigned blocks = std::max(1u, std::min((unsigned)RC_BLOCKS_MAX, std::max(by_atoms, by_list)));
  recheck_kernel<<<blocks, RC_THREADS, 0, st>>>(list, count, W, L.N, (const float*)frames, view_of(prior), chunk_ref,
                                                L.w64, L.dscale, eps, band.D, band.flag, chunk.D, chunk.flag,
                                                n_rechecks, L.wa64, c32, scr.part, scr.done);
  note_launch();
}

size_t recheck_scratch_bytes() {
  return sizeof(double) * (size_t)RC_CAP * RC_BLOCKS_MAX * RC_PARTS + sizeof(int) * (size_t)RC_CAP;
}

RecheckScratch recheck_scratch_at(void* base) {
  double* part = (double*)base;
  return RecheckScratch{part, (int*)(part + (size_t)RC_CAP * RC_BLOCKS_MAX * RC_PARTS)};
}

void launch_xy_refine(Prec p, int F, const void* frames, const LandmarkDev& L, FrameInfo fi, const RefDesc& prior,
                      FrameRec rec, cudaStream_t st) {
  if (p == P_F64 || F <= 0) return;
  if (F <= 152 && L.N >= 1024) {  // few large frames: a block per frame
    xy_refine_block<<<F, XR_THREADS, 0, st>>>(F, L.N, (const float*)frames, view_of(prior), fi.c32, fi.G, L.w, rec);
    note_launch();
    return;
  }
  xy_refine_kernel<<<blocks_for((size_t)F, WARPS_PER_BLOCK), 32 * WARPS_PER_BLOCK, 0, st>>>(
      F, L.N, (const float*)frames, view_of(prior), fi.c32, fi.G, L.w, L.dscale, rec);
  note_launch();
}

void launch_set_int(int* p, int v, cudaStream_t st) { set_int_kernel<<<1, 1, 0, st>>>(p, v); note_launch(); }

void launch_chunk_round_init(int* recheck_count, int* stop, int* first, int t1, cudaStream_t st) {
  set_chunk_round_kernel<<<1, 1, 0, st>>>(recheck_count, stop, first, t1);
  note_launch();
}

void launch_first_exceed(int t0, int t1, const uint8_t* flag, const int* stop, int* first, cudaStream_t st) {
  if (t1 <= t0) return;
  first_exceed_kernel<<<blocks_for((size_t)(t1 - t0), 256), 256, 0, st>>>(t0, t1, flag, stop, first); note_launch();
}

void launch_band_scan(int F, int W, int t0, int o_init, const AlignOut band, FrameRec rec, ScanResult* res,
                      cudaStream_t st) {
  band_scan_kernel<<<1, SCAN_THREADS, 0, st>>>(F, W, t0, o_init, band.D, band.q, band.flag, rec, res); note_launch();
}

void launch_chunk_records(int t0, int t_end, int t1, int ref, const AlignOut chunk, FrameRec rec,
                          cudaStream_t st) {
  const int n = (t_end < t1 ? t_end + 1 : t1) - t0;
  if (n <= 0) return;
  chunk_records_kernel<<<blocks_for((size_t)n, 256), 256, 0, st>>>(t0, t_end, t1, ref, chunk.D, chunk.q, rec,
                                                                    nullptr); note_launch();
}

void launch_chunk_records_dev(int t0, const int* t_end_dev, int t1, int ref, const AlignOut chunk, FrameRec rec,
                              cudaStream_t st) {
  const int n = t1 - t0;
  if (n <= 0) return;
  chunk_records_kernel<<<blocks_for((size_t)n, 256), 256, 0, st>>>(t0, 0, t1, ref, chunk.D, chunk.q, rec, t_end_dev);
  note_launch();
}

void launch_initial_record(FrameRec rec, cudaStream_t st) { initial_record_kernel<<<1, 1, 0, st>>>(rec); note_launch(); }

void launch_compact(int F, const FrameRec rec, int* refresh_list, int* refresh_count, int* seg_of_frame,
                    int* approx_list, int* approx_count, int* approx_seg, int prior_seg, cudaStream_t st) {
  compact_kernel<<<1, SCAN_THREADS, 0, st>>>(F, rec.flag, refresh_list, refresh_count, seg_of_frame, approx_list,
                                             approx_count, approx_seg, prior_seg); note_launch();
}

void launch_finalize(Prec p, int F, int M, void* D, const double* q, const float* q32, double lambda, double* s,
                     double* z, float* mstat, double* mstat64, double* msd_out, bool want_p, cudaStream_t st) {
  if (F <= 0) return;
  const unsigned blocks = blocks_for((size_t)F, WARPS_PER_BLOCK);
  if (p == P_F64)
    finalize_f64<<<blocks, 32 * WARPS_PER_BLOCK, 0, st>>>(F, M, (double*)D, q, lambda, s, z, mstat64, msd_out,
                                                          want_p ? 1 : 0);
  else if (F <= 152 && M >= 1024)  // few frames against many landmarks: a block per frame
    finalize_block_f32<<<F, FN_THREADS, 0, st>>>(F, M, (float*)D, q32, (float)lambda, s, z, mstat, msd_out,
                                                 want_p ? 1 : 0);
  else
    finalize_f32<<<blocks, 32 * WARPS_PER_BLOCK, 0, st>>>(F, M, (float*)D, q32, (float)lambda, s, z, mstat, msd_out,
                                                          want_p ? 1 : 0);
  note_launch();
}

void launch_frame_prep_group(const GroupInst* I, int n, int Ftot, cudaStream_t st) {
  if (Ftot <= 0) return;
  frame_prep_group_f32<<<blocks_for((size_t)Ftot, WARPS_PER_BLOCK), 32 * WARPS_PER_BLOCK, 0, st>>>(I, n, Ftot);
  note_launch();
}

void launch_finalize_group(const GroupInst* I, int n, int Ftot, cudaStream_t st) {
  if (Ftot <= 0) return;
  finalize_group_f32<<<blocks_for((size_t)Ftot, WARPS_PER_BLOCK), 32 * WARPS_PER_BLOCK, 0, st>>>(I, n, Ftot);
  note_launch();
}

void launch_combine_grad(Prec p, int F, int N3, const double* g_s, const double* g_z, const void* gs,
                         const void* gz, void* out, cudaStream_t st) {
  const size_t n = (size_t)F * N3;
  if (n == 0) return;
  if (p == P_F64)
    combine_grad_kernel<double><<<blocks_for(n, 256), 256, 0, st>>>(n, N3, g_s, g_z, (const double*)gs,
                                                                     (const double*)gz, (double*)out);
  else {
    const bool vec = N3 % 4 == 0 && ((uintptr_t)gs % 16) == 0 && ((uintptr_t)gz % 16) == 0 && ((uintptr_t)out % 16) == 0;
    const unsigned blocks = (unsigned)(F < 152 * 16 ? F : 152 * 16);
    const unsigned threads = N3 >= 1024 ? 256 : 128;
    if (vec)
      combine_rows_f32<true><<<blocks, threads, 0, st>>>(F, N3, g_s, g_z, (const float*)gs, (const float*)gz,
                                                          (float*)out);
    else
      combine_rows_f32<false><<<blocks, threads, 0, st>>>(F, N3, g_s, g_z, (const float*)gs, (const float*)gz,
                                                           (float*)out);
  }
  note_launch();
}

// device-to-device copy by the SMs (16-byte pieces when both ends are aligned): keeps the
// copy engines free for host transfers running next to the evaluation
__global__ void dev_copy_kernel(uint8_t* __restrict__ dst, const uint8_t* __restrict__ src, size_t n, int vec) {
  const size_t i0 = blockIdx.x * (size_t)blockDim.x + threadIdx.x, step = (size_t)gridDim.x * blockDim.x;
  if (vec) {
    const size_t n16 = n / 16;
    for (size_t i = i0; i < n16; i += step)
      reinterpret_cast<uint4*>(dst)[i] = reinterpret_cast<const uint4*>(src)[i];
    for (size_t i = n16 * 16 + i0; i < n; i += step) dst[i] = src[i];
  } else {
    for (size_t i = i0; i < n; i += step) dst[i] = src[i];
  }
}

void launch_dev_copy(void* dst, const void* src, size_t bytes, cudaStream_t st) {
  if (bytes == 0) return;
  const int vec = ((uintptr_t)dst % 16) == 0 && ((uintptr_t)src % 16) == 0;
  const size_t units = vec ? bytes / 16 + 1 : bytes;
  const unsigned blocks = (unsigned)std::min<size_t>((units + 255) / 256, 152 * 8);
  dev_copy_kernel<<<blocks, 256, 0, st>>>((uint8_t*)dst, (const uint8_t*)src, bytes, vec);
  note_launch();
}

void launch_fill_u8(uint8_t* p, uint8_t v, size_t n, cudaStream_t st) {
  if (n == 0) return;
  fill_u8_kernel<<<blocks_for(n, 256), 256, 0, st>>>(p, v, n); note_launch();
}

}  // namespace pcv

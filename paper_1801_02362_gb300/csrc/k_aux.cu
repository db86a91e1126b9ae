// k_aux.cu -- per-frame kernels around the pair kernels:
//   frame preparation (centres, sums of squares), frame-vs-structure alignments for the
//   close-structure decision of Algorithm 2 (band of previous frames, speculative chunks,
//   FP64 re-check of undecidable cases), the parallel refresh-search scan, compaction,
//   path-CV finalisation (Eq. property_map_cv and z) and the adjoint of
//   Eq. (der_dist) / Eq. (close_der_dist).
#include <cuda_fp16.h>

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
__global__ void frame_prep_f32(int F, int N, const float* __restrict__ frames,
                               const float* __restrict__ wts, float4* __restrict__ c32,
                               double4* __restrict__ c64, double* __restrict__ G) {
  const int f = warp_global();
  if (f >= F) return;
  const int lane = threadIdx.x & 31;
  const float* x = frames + (size_t)f * N * 3;
  float hi[3] = {0, 0, 0}, lo[3] = {0, 0, 0};
  for (int j = lane; j < N; j += 32) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float v = x[3 * j + c];
      if (wts) {
        const float p = wts[j] * v;
        const float e = fmaf(wts[j], v, -p);
        two_sum_acc(hi[c], lo[c], p);
        lo[c] += e;
      } else {
        two_sum_acc(hi[c], lo[c], v);
      }
    }
  }
  double c[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    warp_sum_pair(hi[k], lo[k]);
    c[k] = pair_to_double(hi[k], lo[k]);
    if (!wts) c[k] /= (double)N;
  }
  const float cf[3] = {(float)c[0], (float)c[1], (float)c[2]};
  float gh = 0.0f, gl = 0.0f;
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
    c64[f] = make_double4(c[0], c[1], c[2], 0.0);
    G[f] = pair_to_double(gh, gl);
  }
}

__global__ void frame_prep_f64(int F, int N, const double* __restrict__ frames,
                               const double* __restrict__ w64, float4* __restrict__ c32,
                               double4* __restrict__ c64, double* __restrict__ G) {
  const int f = warp_global();
  if (f >= F) return;
  const int lane = threadIdx.x & 31;
  const double* x = frames + (size_t)f * N * 3;
  double c[3] = {0, 0, 0};
  for (int j = lane; j < N; j += 32) {
    const double wj = w64 ? w64[j] : 1.0;
#pragma unroll
    for (int k = 0; k < 3; ++k) c[k] += wj * x[3 * j + k];
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    c[k] = warp_sum_double(c[k]);
    if (!w64) c[k] /= (double)N;
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

// FP32 frames: compensated correlation, returns H in FP64 on every lane
__device__ __forceinline__ void warp_corr_f32(int N, const float* __restrict__ x, float4 cx,
                                              const float* __restrict__ y, float4 cy,
                                              const float* __restrict__ wts, double* H) {
  const int lane = threadIdx.x & 31;
  float p[9], hi[9], lo[9];
#pragma unroll
  for (int e = 0; e < 9; ++e) p[e] = hi[e] = lo[e] = 0.0f;
  int cnt = 0;
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
    H[e] = pair_to_double(hi[e], lo[e]);
  }
}

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
  const double lam = lambda_max_newton(H, 0.5 * (Gx + Gy), &ok);
  double D = (Gx + Gy - 2.0 * lam) * dscale;
  if (D < 0.0) D = 0.0;
  double K[16];
  quat_matrix(H, K);
  double q[4];
  adj_eigvec_f64(K, lam, q);
  *outD = D;
  *outQ = make_double4(q[0], q[1], q[2], q[3]);
  // Worst-case error of the compensated FP32 correlation: chunks of 16 products are
  // summed in FP32 (|err| <= 16 u sum|terms| per entry), so |dD| <= ~100 u (Gx + Gy).
  // Decisions inside 1e-5 (Gx + Gy) of eps are re-done in FP64.
  const bool amb = amb_check && fabs(D - eps) <= 1e-5 * (Gx + Gy) * dscale;
  *amb_out = amb;
  *outFlag = (uint8_t)((D > eps ? 1 : 0) | (amb ? 2 : 0));
}

template <bool F64>
__global__ void align_kernel(int mode, int F, int W, int t0, int t1, int ref_index, int N,
                             const void* __restrict__ frames_v, RefView prior,
                             const float4* __restrict__ c32, const double4* __restrict__ c64,
                             const double* __restrict__ fG, const float* __restrict__ wts,
                             const double* __restrict__ w64, double dscale, double eps,
                             double* __restrict__ outD, double4* __restrict__ outQ,
                             uint8_t* __restrict__ outFlag, int* __restrict__ recheck_list,
                             int* __restrict__ recheck_count) {
  const int wid = warp_global();
  const int lane = threadIdx.x & 31;
  int t, ref, slot;
  if (mode == 0) {  // band
    t = 1 + wid / W;
    const int k = 1 + wid % W;
    if (t >= F) return;
    ref = t - k;
    slot = t * W + k - 1;
    if (ref < 0) {
      if (lane == 0) {
        outD[slot] = -1.0;
        outFlag[slot] = 0;
      }
      return;
    }
  } else {  // chunk
    t = t0 + wid;
    if (t >= t1) return;
    ref = ref_index;
    slot = t;
  }
  double H[9];
  const double Gx = fG[t];
  const double Gy = ref >= 0 ? fG[ref] : prior.G;
  if (F64) {
    const double* frames = (const double*)frames_v;
    const double* y = ref >= 0 ? frames + (size_t)ref * N * 3 : (const double*)prior.coords;
    const double4 cy = ref >= 0 ? c64[ref] : prior.c64;
    warp_corr_f64(N, frames + (size_t)t * N * 3, c64[t], y, cy, w64, H);
  } else {
    const float* frames = (const float*)frames_v;
    const float* y = ref >= 0 ? frames + (size_t)ref * N * 3 : (const float*)prior.coords;
    const float4 cy = ref >= 0 ? c32[ref] : prior.c32;
    warp_corr_f32(N, frames + (size_t)t * N * 3, c32[t], y, cy, wts, H);
  }
  if (lane == 0) {
    bool amb = false;
    finish_alignment(H, Gx, Gy, dscale, eps, !F64, outD + slot, outQ + slot, outFlag + slot, &amb);
    if (amb) {
      const int pos = atomicAdd(recheck_count, 1);
      recheck_list[pos] = (slot << 1) | (mode == 0 ? 0 : 1);
    }
  }
}

// Full FP64 re-evaluation of D(x_t, y) from the raw FP32 coordinates: FP64 centres,
// FP64 correlation and sums of squares, FP64 eigenvalue.  One warp per listed entry.
__global__ void recheck_kernel(const int* __restrict__ list, const int* __restrict__ count, int W,
                               int N, const float* __restrict__ frames, RefView prior, int chunk_ref,
                               const double* __restrict__ w64, double dscale, double eps,
                               double* bandD, uint8_t* bandFlag, double* chunkD, uint8_t* chunkFlag,
                               unsigned long long* n_rechecks) {
  const int wid = warp_global();
  if (wid >= *count) return;
  const int lane = threadIdx.x & 31;
  const int code = list[wid];
  const int slot = code >> 1;
  const bool is_chunk = code & 1;
  int t, ref;
  if (is_chunk) {
    t = slot;
    ref = chunk_ref;
  } else {
    t = slot / W;
    ref = t - (slot % W + 1);
  }
  const float* x = frames + (size_t)t * N * 3;
  const float* y = ref >= 0 ? frames + (size_t)ref * N * 3 : (const float*)prior.coords;
  double cx[3] = {0, 0, 0}, cy[3] = {0, 0, 0};
  for (int j = lane; j < N; j += 32) {
    const double wj = w64 ? w64[j] : 1.0;
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
    if (!w64) {
      cx[c] /= (double)N;
      cy[c] /= (double)N;
    }
  }
  double h[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0}, gx = 0.0, gy = 0.0;
  for (int j = lane; j < N; j += 32) {
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
#pragma unroll
  for (int e = 0; e < 9; ++e) h[e] = warp_sum_double(h[e]);
  gx = warp_sum_double(gx);
  gy = warp_sum_double(gy);
  if (lane == 0) {
    bool ok = true;
    const double lam = lambda_max_newton(h, 0.5 * (gx + gy), &ok);
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
}

__global__ void set_int_kernel(int* p, int v) { *p = v; }

__global__ void first_exceed_kernel(int t0, int t1, const uint8_t* __restrict__ flag, int* first) {
  const int t = t0 + blockIdx.x * blockDim.x + threadIdx.x;
  if (t < t1 && (flag[t] & 1)) atomicMin(first, t);
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
    if (stop < F) {
      if (tid == 0) {
        // frame stop-1 had offset W from its close structure
        res->t_stop = stop;
        res->ref = stop - 1 - W;
      }
      return;
    }
    s_in = s_state[SCAN_THREADS - 1];
    __syncthreads();
  }
  if (tid == 0) {
    res->t_stop = F;
    res->ref = -2;
  }
}

__global__ void chunk_records_kernel(int t0, int t_end, int t1, int ref, const double* __restrict__ cD,
                                     const double4* __restrict__ cQ, FrameRec rec) {
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
  __shared__ int s_r[32], s_a[32];
  const int tid = threadIdx.x, lane = tid & 31, wrp = tid >> 5;
  int nref = 0, napp = 0;
  for (int base = 0; base < F; base += SCAN_THREADS) {
    const int t = base + tid;
    const int isr = (t < F && flag[t] != 0) ? 1 : 0;
    const int isa = (t < F && flag[t] == 0) ? 1 : 0;
    int r = isr, a = isa;
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
    if (t < F) {
      const int seg = prior_seg + nref + r;  // inclusive count of reassignments
      seg_of_frame[t] = seg;
      if (isr) refresh_list[nref + r - 1] = t;
      if (isa) {
        approx_list[napp + a - 1] = t;
        approx_seg[napp + a - 1] = seg;
      }
    }
    nref += s_r[31];
    napp += s_a[31];
    __syncthreads();
  }
  if (tid == 0) {
    *refresh_count = nref;
    *approx_count = napp;
  }
}

// ---------------------------------------------------------------------------------------
// Path CVs: m = min D, l = sum exp(-lambda (D - m)), s = sum q e / l, z = m - ln(l)/lambda.
// FP32 modes: exponentials in FP32 (relative error ~1e-7, far inside the tolerance),
// lane partials combined in FP64.  One warp per frame.
__global__ void finalize_f32(int F, int M, const float* __restrict__ D, const double* __restrict__ q,
                             double lambda, double* __restrict__ s, double* __restrict__ z,
                             float* __restrict__ mstat, double* __restrict__ msd) {
  const int f = warp_global();
  if (f >= F) return;
  const int lane = threadIdx.x & 31;
  const float* d = D + (size_t)f * M;
  float m = 3.4e38f;
  for (int i = lane; i < M; i += 32) m = fminf(m, d[i]);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) m = fminf(m, __shfl_xor_sync(0xffffffffu, m, off));
  const float lf = (float)lambda;
  float l = 0.0f, sq = 0.0f;
  for (int i = lane; i < M; i += 32) {
    const float e = expf(-lf * (d[i] - m));
    l += e;
    sq = fmaf((float)q[i], e, sq);
    if (msd) msd[(size_t)f * M + i] = (double)d[i];
  }
  const double L = warp_sum_double((double)l);
  const double SQ = warp_sum_double((double)sq);
  if (lane == 0) {
    s[f] = SQ / L;
    z[f] = (double)m - log(L) / lambda;
    mstat[2 * f] = m;
    mstat[2 * f + 1] = (float)L;
  }
}

__global__ void finalize_f64(int F, int M, const double* __restrict__ D, const double* __restrict__ q,
                             double lambda, double* __restrict__ s, double* __restrict__ z,
                             double* __restrict__ mstat64, double* __restrict__ msd) {
  const int f = warp_global();
  if (f >= F) return;
  const int lane = threadIdx.x & 31;
  const double* d = D + (size_t)f * M;
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
  if (lane == 0) {
    s[f] = sq / l;
    z[f] = m - log(l) / lambda;
    mstat64[2 * f] = m;
    mstat64[2 * f + 1] = l;
  }
}

// ---------------------------------------------------------------------------------------
// Adjoint.  For L = s and L = z, dL/dD_i = gamma_i with p_i = exp(-lambda (D_i - m))/l:
// gamma^z_i = p_i, gamma^s_i = -lambda p_i (q_i - s).  The direct part of Eq. (der_dist)
// summed over landmarks is 2 w_k ((sum_i gamma_i) x_k - beta_k) with
// beta_k = sum_i gamma_i Rot_i a_ik: a (3F x 3M)(3M x N) contraction computed here, with
// Rot_i = R_{a_i x} (exact) or R_{a_i y} (close structure, R_{xy} applied afterwards).
constexpr int AB_TF = 32, AB_TJ = 64, AB_KL = 8, AB_THREADS = 128;

template <typename ST, typename LT>
__device__ __forceinline__ ST lm_load(const LT* p) {
  return (ST)(*p);
}
template <>
__device__ __forceinline__ float lm_load<float, __half>(const __half* p) {
  return __half2float(*p);
}

template <typename ST, typename LT, typename MT>
__global__ void __launch_bounds__(AB_THREADS)
adjoint_beta_kernel(int F, int M, int N, const LT* __restrict__ lm, const double* __restrict__ q,
                    const ST* __restrict__ D, const MT* __restrict__ mstat, const double* __restrict__ s,
                    double lambda, const ST* __restrict__ Rpair, const ST* __restrict__ Bseg,
                    const int* __restrict__ seg_of_frame, ST* __restrict__ gs, ST* __restrict__ gz) {
  // thread: 2 frames (ty) x 8 atoms (tx); CTA: 32 frames x 64 atoms
  __shared__ __align__(16) ST Ws[AB_KL * 3][AB_TF * 3];  // W^s[(i,c)][(f,b)] = gamma^s_fi Rot_fi[b][c]
  __shared__ __align__(16) ST Wz[AB_KL * 3][AB_TF * 3];
  __shared__ __align__(16) ST As[AB_KL * 3][AB_TJ];      // a_ij[c]
  const int f0 = blockIdx.y * AB_TF, j0 = blockIdx.x * AB_TJ;
  const int tid = threadIdx.x, tx = tid & 7, ty = tid >> 3;
  ST bs[2][3][8], bz[2][3][8];
#pragma unroll
  for (int u = 0; u < 2; ++u)
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
      for (int k = 0; k < 8; ++k) bs[u][b][k] = bz[u][b][k] = 0;

  for (int i0 = 0; i0 < M; i0 += AB_KL) {
    // weights W for (frame, landmark) pairs of this chunk
    for (int e = tid; e < AB_TF * AB_KL; e += AB_THREADS) {
      const int ff = e / AB_KL, ii = e - ff * AB_KL;
      const int f = f0 + ff, i = i0 + ii;
      ST rot[9];
      ST gsv = 0, gzv = 0;
#pragma unroll
      for (int c = 0; c < 9; ++c) rot[c] = 0;
      if (f < F && i < M) {
        const double m = (double)mstat[2 * f], l = (double)mstat[2 * f + 1];
        const double p = exp(-lambda * ((double)D[(size_t)f * M + i] - m)) / l;
        gzv = (ST)p;
        gsv = (ST)(-lambda * p * (q[i] - s[f]));
        const ST* R = Rpair ? Rpair + ((size_t)f * M + i) * 9 : Bseg + ((size_t)seg_of_frame[f] * M + i) * 9;
#pragma unroll
        for (int c = 0; c < 9; ++c) rot[c] = R[c];
      }
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
          Ws[ii * 3 + c][ff * 3 + b] = gsv * rot[3 * b + c];
          Wz[ii * 3 + c][ff * 3 + b] = gzv * rot[3 * b + c];
        }
    }
    for (int e = tid; e < AB_KL * AB_TJ; e += AB_THREADS) {
      const int ii = e / AB_TJ, jj = e - ii * AB_TJ;
      const int i = i0 + ii, j = j0 + jj;
#pragma unroll
      for (int c = 0; c < 3; ++c) As[ii * 3 + c][jj] = (i < M && j < N) ? lm_load<ST>(lm + ((size_t)i * N + j) * 3 + c) : (ST)0;
    }
    __syncthreads();
#pragma unroll 2
    for (int kk = 0; kk < AB_KL * 3; ++kk) {
      ST a[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) a[k] = As[kk][tx * 8 + k];
#pragma unroll
      for (int u = 0; u < 2; ++u)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
          const ST ws = Ws[kk][(ty * 2 + u) * 3 + b];
          const ST wz = Wz[kk][(ty * 2 + u) * 3 + b];
#pragma unroll
          for (int k = 0; k < 8; ++k) {
            bs[u][b][k] = fma(ws, a[k], bs[u][b][k]);
            bz[u][b][k] = fma(wz, a[k], bz[u][b][k]);
          }
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    const int f = f0 + ty * 2 + u;
    if (f >= F) continue;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int j = j0 + tx * 8 + k;
      if (j >= N) continue;
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        gs[((size_t)f * N + j) * 3 + b] = bs[u][b][k];
        gz[((size_t)f * N + j) * 3 + b] = bz[u][b][k];
      }
    }
  }
}

// block-wide FP64 sum of per-thread values (blockDim.x == 128)
__device__ __forceinline__ double block_sum128(double v, double* scratch) {
  v = warp_sum_double(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) scratch[w] = v;
  __syncthreads();
  return scratch[0] + scratch[1] + scratch[2] + scratch[3];
}

// Per-frame finish: from beta (in gs/gz) to ds/dx and dz/dx.
//  exact / reassignment frames: ds/dx_k = -2 w_k beta^s_k, dz/dx_k = 2 w_k (x_k - beta^z_k);
//  approximate frames (beta in the close-structure frame): the direct term uses R_xy beta,
//  plus the rotation term sum_ab Ghat_ab dR_xy,ab/dx_k of Eq. (close_der_dist).  With
//  Ghat = -2 (sum_j w_j x_j beta_j^T - R_xy Phi), Phi = sum_i gamma_i R_{a_i y} A_i
//  R_{a_i y}^T (A_i = sum_j w_j a_ij a_ij^T), the rotation term is w_k T^T y_k with
//  T_bc = p^T K(E_bc) q0, where q0 is the top eigenvector of K(H_xy) (eigenvalue l0) and
//  p solves (l0 I - K + q0 q0^T) p = g - (q0.g) q0, g = 2 K(Ghat^T) q0 (first-order
//  eigenvector perturbation).
template <typename ST, typename FT>
__global__ void __launch_bounds__(128)
adjoint_finish_kernel(int F, int M, int N, const FT* __restrict__ frames, const float4* __restrict__ c32,
                      const double4* __restrict__ c64, const float* __restrict__ wts,
                      const double* __restrict__ w64, const double* __restrict__ LA,
                      const double* __restrict__ q, double dscale, const ST* __restrict__ D,
                      const float* __restrict__ mstat, const double* __restrict__ mstat64,
                      const double* __restrict__ s, double lambda, const ST* __restrict__ Bseg,
                      const int* __restrict__ seg_of_frame, FrameRec rec, RefView prior,
                      ST* __restrict__ gs, ST* __restrict__ gz, unsigned* __restrict__ status) {
  const int f = blockIdx.x;
  if (f >= F) return;
  const int tid = threadIdx.x;
  __shared__ double scratch[4];
  __shared__ double s_T[2][9];  // rotation-term matrices T^s, T^z
  __shared__ double s_R[9];     // R_xy
  __shared__ double s_yc[3];
  const bool approx = rec.flag && rec.flag[f] == 0;
  const bool f64 = sizeof(ST) == 8;
  double cx[3];
  if (f64) {
    const double4 c = c64[f];
    cx[0] = c.x; cx[1] = c.y; cx[2] = c.z;
  } else {
    const float4 c = c32[f];
    cx[0] = c.x; cx[1] = c.y; cx[2] = c.z;
  }
  const FT* x = frames + (size_t)f * N * 3;
  auto wt = [&](int j) -> double { return f64 ? (w64 ? w64[j] : dscale) : (wts ? (double)wts[j] : dscale); };

  if (!approx) {
    for (int j = tid; j < N; j += 128) {
      const double w = wt(j);
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        const size_t idx = ((size_t)f * N + j) * 3 + b;
        const ST v = (ST)x[3 * j + b] - (ST)cx[b];
        gs[idx] = (ST)(-2.0 * w * (double)gs[idx]);
        gz[idx] = (ST)(2.0 * w * (double)(v - gz[idx]));
      }
    }
    return;
  }

  // ---- approximate frame ----
  const int r = rec.ref[f];
  const FT* y = r >= 0 ? frames + (size_t)r * N * 3 : (const FT*)prior.coords;
  double cy[3];
  if (r >= 0) {
    if (f64) { const double4 c = c64[r]; cy[0] = c.x; cy[1] = c.y; cy[2] = c.z; }
    else { const float4 c = c32[r]; cy[0] = c.x; cy[1] = c.y; cy[2] = c.z; }
  } else {
    if (f64) { cy[0] = prior.c64.x; cy[1] = prior.c64.y; cy[2] = prior.c64.z; }
    else { cy[0] = prior.c32.x; cy[1] = prior.c32.y; cy[2] = prior.c32.z; }
  }
  if (tid == 0) {
    const double4 qq = rec.qxy[f];
    const double qd[4] = {qq.x, qq.y, qq.z, qq.w};
    quat_to_rot(qd, s_R);
  }
  __syncthreads();
  // X = sum_j w_j x_j beta_j^T (s and z) and H_xy = sum_j w_j y_j x_j^T, true weights
  double Xs[9], Xz[9], Hy[9];
#pragma unroll
  for (int e = 0; e < 9; ++e) Xs[e] = Xz[e] = Hy[e] = 0.0;
  for (int j = tid; j < N; j += 128) {
    const double w = wt(j);
    double v[3], u[3], bsj[3], bzj[3];
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      v[b] = (double)((ST)x[3 * j + b] - (ST)cx[b]);
      u[b] = (double)((ST)y[3 * j + b] - (ST)cy[b]);
      const size_t idx = ((size_t)f * N + j) * 3 + b;
      bsj[b] = (double)gs[idx];
      bzj[b] = (double)gz[idx];
    }
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        Xs[3 * b + c] += w * v[b] * bsj[c];
        Xz[3 * b + c] += w * v[b] * bzj[c];
        Hy[3 * b + c] += w * u[b] * v[c];
      }
  }
#pragma unroll
  for (int e = 0; e < 9; ++e) {
    Xs[e] = block_sum128(Xs[e], scratch);
    Xz[e] = block_sum128(Xz[e], scratch);
    Hy[e] = block_sum128(Hy[e], scratch);
  }
  // Phi = sum_i gamma_i B_i A_i B_i^T
  double Ps[9], Pz[9];
#pragma unroll
  for (int e = 0; e < 9; ++e) Ps[e] = Pz[e] = 0.0;
  const int seg = seg_of_frame[f];
  const double mm = f64 ? mstat64[2 * f] : (double)mstat[2 * f];
  const double ll = f64 ? mstat64[2 * f + 1] : (double)mstat[2 * f + 1];
  for (int i = tid; i < M; i += 128) {
    const double p = exp(-lambda * ((double)D[(size_t)f * M + i] - mm)) / ll;
    const double gzv = p, gsv = -lambda * p * (q[i] - s[f]);
    const ST* B = Bseg + ((size_t)seg * M + i) * 9;
    const double* A6 = LA + (size_t)i * 6;
    const double A[9] = {A6[0], A6[1], A6[2], A6[1], A6[3], A6[4], A6[2], A6[4], A6[5]};
    double BA[9];
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
      for (int c = 0; c < 3; ++c)
        BA[3 * b + c] = (double)B[3 * b] * A[c] + (double)B[3 * b + 1] * A[3 + c] + (double)B[3 * b + 2] * A[6 + c];
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const double S = BA[3 * b] * (double)B[3 * c] + BA[3 * b + 1] * (double)B[3 * c + 1] + BA[3 * b + 2] * (double)B[3 * c + 2];
        Ps[3 * b + c] += gsv * S;
        Pz[3 * b + c] += gzv * S;
      }
  }
#pragma unroll
  for (int e = 0; e < 9; ++e) {
    Ps[e] = block_sum128(Ps[e], scratch);
    Pz[e] = block_sum128(Pz[e], scratch);
  }
  if (tid == 0) {
    // eigen-decomposition data of K(H_xy) in true units
    double K[16];
    quat_matrix(Hy, K);
    double Gx = 0.0, Gy = 0.0;  // upper bound from the trace-free structure: use |K| bound
    // lambda_max via Newton from an upper bound: the largest absolute row sum of K
    double ub = 0.0;
    for (int a = 0; a < 4; ++a) {
      double rs = 0.0;
      for (int b = 0; b < 4; ++b) rs += fabs(K[4 * a + b]);
      ub = fmax(ub, rs);
    }
    (void)Gx;
    (void)Gy;
    bool ok = true;
    const double l0 = lambda_max_newton(Hy, ub, &ok);
    if (!ok) atomicOr(status, STATUS_NOCONV);
    double q0[4];
    adj_eigvec_f64(K, l0, q0);
    double Amat[16];
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b) Amat[4 * a + b] = (a == b ? l0 : 0.0) - K[4 * a + b] + q0[a] * q0[b];
    for (int which = 0; which < 2; ++which) {
      const double* X = which == 0 ? Xs : Xz;
      const double* P = which == 0 ? Ps : Pz;
      // Ghat = -2 (X - R_xy Phi)
      double Gh[9];
      for (int b = 0; b < 3; ++b)
        for (int c = 0; c < 3; ++c)
          Gh[3 * b + c] = -2.0 * (X[3 * b + c] - (s_R[3 * b] * P[c] + s_R[3 * b + 1] * P[3 + c] + s_R[3 * b + 2] * P[6 + c]));
      double GhT[9];
      for (int b = 0; b < 3; ++b)
        for (int c = 0; c < 3; ++c) GhT[3 * b + c] = Gh[3 * c + b];
      double KG[16];
      quat_matrix(GhT, KG);
      double g[4];
      for (int a = 0; a < 4; ++a) {
        g[a] = 0.0;
        for (int b = 0; b < 4; ++b) g[a] += 2.0 * KG[4 * a + b] * q0[b];
      }
      const double gq = g[0] * q0[0] + g[1] * q0[1] + g[2] * q0[2] + g[3] * q0[3];
      for (int a = 0; a < 4; ++a) g[a] -= gq * q0[a];
      double pv[4] = {0, 0, 0, 0};
      if (!spd_solve4(Amat, g, pv)) atomicOr(status, STATUS_NOCONV);
      // T_bc = p^T K(E_bc) q0
      for (int b = 0; b < 3; ++b)
        for (int c = 0; c < 3; ++c) {
          double E[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
          E[3 * b + c] = 1.0;
          double KE[16];
          quat_matrix(E, KE);
          double t = 0.0;
          for (int a = 0; a < 4; ++a)
            for (int d = 0; d < 4; ++d) t += pv[a] * KE[4 * a + d] * q0[d];
          s_T[which][3 * b + c] = t;
        }
    }
  }
  __syncthreads();
  for (int j = tid; j < N; j += 128) {
    const double w = wt(j);
    double v[3], u[3], bsj[3], bzj[3];
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      v[b] = (double)((ST)x[3 * j + b] - (ST)cx[b]);
      u[b] = (double)((ST)y[3 * j + b] - (ST)cy[b]);
      const size_t idx = ((size_t)f * N + j) * 3 + b;
      bsj[b] = (double)gs[idx];
      bzj[b] = (double)gz[idx];
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double Rbs = s_R[3 * c] * bsj[0] + s_R[3 * c + 1] * bsj[1] + s_R[3 * c + 2] * bsj[2];
      const double Rbz = s_R[3 * c] * bzj[0] + s_R[3 * c + 1] * bzj[1] + s_R[3 * c + 2] * bzj[2];
      const double Ts = s_T[0][c] * u[0] + s_T[0][3 + c] * u[1] + s_T[0][6 + c] * u[2];
      const double Tz = s_T[1][c] * u[0] + s_T[1][3 + c] * u[1] + s_T[1][6 + c] * u[2];
      const size_t idx = ((size_t)f * N + j) * 3 + c;
      gs[idx] = (ST)(-2.0 * w * Rbs + w * Ts);
      gz[idx] = (ST)(2.0 * w * (v[c] - Rbz) + w * Tz);
    }
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
                                                            fi.c64, fi.G);
  else
    frame_prep_f32<<<blocks, 32 * WARPS_PER_BLOCK, 0, st>>>(F, L.N, (const float*)frames, L.w, fi.c32, fi.c64,
                                                            fi.G); note_launch();
}

void launch_align_band(Prec p, int F, int W, const void* frames, const LandmarkDev& L, FrameInfo fi,
                       double eps, AlignOut out, int* recheck_list, int* recheck_count, cudaStream_t st) {
  if (F <= 1) return;
  const size_t warps = (size_t)(F - 1) * W;
  const unsigned blocks = blocks_for(warps, WARPS_PER_BLOCK);
  RefView none{nullptr, make_float4(0, 0, 0, 0), make_double4(0, 0, 0, 0), 0.0};
  if (p == P_F64)
    align_kernel<true><<<blocks, 32 * WARPS_PER_BLOCK, 0, st>>>(0, F, W, 0, 0, 0, L.N, frames, none, fi.c32, fi.c64,
                                                                fi.G, L.w, L.w64, L.dscale, eps, out.D, out.q,
                                                                out.flag, recheck_list, recheck_count);
  else
    align_kernel<false><<<blocks, 32 * WARPS_PER_BLOCK, 0, st>>>(0, F, W, 0, 0, 0, L.N, frames, none, fi.c32,
                                                                 fi.c64, fi.G, L.w, L.w64, L.dscale, eps, out.D,
                                                                 out.q, out.flag, recheck_list, recheck_count); note_launch();
}

void launch_align_chunk(Prec p, int t0, int t1, const void* frames, const LandmarkDev& L, FrameInfo fi,
                        int ref_index, const RefDesc& prior, double eps, AlignOut out, int* recheck_list,
                        int* recheck_count, cudaStream_t st) {
  if (t1 <= t0) return;
  const unsigned blocks = blocks_for((size_t)(t1 - t0), WARPS_PER_BLOCK);
  if (p == P_F64)
    align_kernel<true><<<blocks, 32 * WARPS_PER_BLOCK, 0, st>>>(1, 0, 1, t0, t1, ref_index, L.N, frames,
                                                                view_of(prior), fi.c32, fi.c64, fi.G, L.w, L.w64,
                                                                L.dscale, eps, out.D, out.q, out.flag,
                                                                recheck_list, recheck_count);
  else
    align_kernel<false><<<blocks, 32 * WARPS_PER_BLOCK, 0, st>>>(1, 0, 1, t0, t1, ref_index, L.N, frames,
                                                                 view_of(prior), fi.c32, fi.c64, fi.G, L.w,
                                                                 L.w64, L.dscale, eps, out.D, out.q, out.flag,
                                                                 recheck_list, recheck_count); note_launch();
}

void launch_recheck(Prec p, int max_entries, const int* list, const int* count, int W, const void* frames,
                    const LandmarkDev& L, const RefDesc& prior, int chunk_ref, double eps, AlignOut band,
                    AlignOut chunk, unsigned long long* n_rechecks, cudaStream_t st) {
  if (p == P_F64 || max_entries <= 0) return;
  const unsigned blocks = blocks_for((size_t)max_entries, WARPS_PER_BLOCK);
  recheck_kernel<<<blocks, 32 * WARPS_PER_BLOCK, 0, st>>>(list, count, W, L.N, (const float*)frames,
                                                          view_of(prior), chunk_ref, L.w64, L.dscale, eps, band.D,
                                                          band.flag, chunk.D, chunk.flag, n_rechecks); note_launch();
}

void launch_set_int(int* p, int v, cudaStream_t st) { set_int_kernel<<<1, 1, 0, st>>>(p, v); note_launch(); }

void launch_first_exceed(int t0, int t1, const uint8_t* flag, int* first, cudaStream_t st) {
  set_int_kernel<<<1, 1, 0, st>>>(first, t1); note_launch();
  if (t1 <= t0) return;
  first_exceed_kernel<<<blocks_for((size_t)(t1 - t0), 256), 256, 0, st>>>(t0, t1, flag, first); note_launch();
}

void launch_band_scan(int F, int W, int t0, int o_init, const AlignOut band, FrameRec rec, ScanResult* res,
                      cudaStream_t st) {
  band_scan_kernel<<<1, SCAN_THREADS, 0, st>>>(F, W, t0, o_init, band.D, band.q, band.flag, rec, res); note_launch();
}

void launch_chunk_records(int t0, int t_end, int t1, int ref, const AlignOut chunk, FrameRec rec,
                          cudaStream_t st) {
  const int n = (t_end < t1 ? t_end + 1 : t1) - t0;
  if (n <= 0) return;
  chunk_records_kernel<<<blocks_for((size_t)n, 256), 256, 0, st>>>(t0, t_end, t1, ref, chunk.D, chunk.q, rec); note_launch();
}

void launch_initial_record(FrameRec rec, cudaStream_t st) { initial_record_kernel<<<1, 1, 0, st>>>(rec); note_launch(); }

void launch_compact(int F, const FrameRec rec, int* refresh_list, int* refresh_count, int* seg_of_frame,
                    int* approx_list, int* approx_count, int* approx_seg, int prior_seg, cudaStream_t st) {
  compact_kernel<<<1, SCAN_THREADS, 0, st>>>(F, rec.flag, refresh_list, refresh_count, seg_of_frame, approx_list,
                                             approx_count, approx_seg, prior_seg); note_launch();
}

void launch_finalize(Prec p, int F, int M, const void* D, const double* q, double lambda, double* s, double* z,
                     float* mstat, double* mstat64, double* msd_out, cudaStream_t st) {
  if (F <= 0) return;
  const unsigned blocks = blocks_for((size_t)F, WARPS_PER_BLOCK);
  if (p == P_F64)
    finalize_f64<<<blocks, 32 * WARPS_PER_BLOCK, 0, st>>>(F, M, (const double*)D, q, lambda, s, z, mstat64,
                                                          msd_out);
  else
    finalize_f32<<<blocks, 32 * WARPS_PER_BLOCK, 0, st>>>(F, M, (const float*)D, q, lambda, s, z, mstat, msd_out); note_launch();
}

void launch_adjoint_beta(Prec p, int F, const LandmarkDev& L, const void* D, const float* mstat, const double* s,
                         double lambda, const void* Rpair, const void* Bseg, const int* seg_of_frame, void* gs,
                         void* gz, cudaStream_t st) {
  if (F <= 0) return;
  dim3 grid((L.N + AB_TJ - 1) / AB_TJ, (F + AB_TF - 1) / AB_TF);
  switch (p) {
    case P_F64:
      adjoint_beta_kernel<double, double, double><<<grid, AB_THREADS, 0, st>>>(
          F, L.M, L.N, (const double*)L.coords, L.q, (const double*)D, (const double*)(const void*)mstat, s, lambda,
          (const double*)Rpair, (const double*)Bseg, seg_of_frame, (double*)gs, (double*)gz); note_launch();
      break;
    case P_F32:
      adjoint_beta_kernel<float, float, float><<<grid, AB_THREADS, 0, st>>>(
          F, L.M, L.N, (const float*)L.coords, L.q, (const float*)D, mstat, s, lambda, (const float*)Rpair,
          (const float*)Bseg, seg_of_frame, (float*)gs, (float*)gz); note_launch();
      break;
    case P_F16:
      adjoint_beta_kernel<float, __half, float><<<grid, AB_THREADS, 0, st>>>(
          F, L.M, L.N, (const __half*)L.coords, L.q, (const float*)D, mstat, s, lambda, (const float*)Rpair,
          (const float*)Bseg, seg_of_frame, (float*)gs, (float*)gz); note_launch();
      break;
  }
}

void launch_adjoint_finish(Prec p, int F, const void* frames, const LandmarkDev& L, FrameInfo fi, const void* D,
                           const float* mstat, const double* s, double lambda, const void* Bseg,
                           const int* seg_of_frame, const FrameRec rec, const RefDesc& prior, void* gs, void* gz,
                           unsigned* status, cudaStream_t st) {
  if (F <= 0) return;
  if (p == P_F64)
    adjoint_finish_kernel<double, double><<<F, 128, 0, st>>>(
        F, L.M, L.N, (const double*)frames, fi.c32, fi.c64, L.w, L.w64, L.A, L.q, L.dscale, (const double*)D,
        nullptr, (const double*)(const void*)mstat, s, lambda, (const double*)Bseg, seg_of_frame, rec,
        view_of(prior), (double*)gs, (double*)gz, status);
  else
    adjoint_finish_kernel<float, float><<<F, 128, 0, st>>>(
        F, L.M, L.N, (const float*)frames, fi.c32, fi.c64, L.w, L.w64, L.A, L.q, L.dscale, (const float*)D, mstat,
        nullptr, s, lambda, (const float*)Bseg, seg_of_frame, rec, view_of(prior), (float*)gs, (float*)gz, status); note_launch();
}

void launch_combine_grad(Prec p, int F, int N3, const double* g_s, const double* g_z, const void* gs,
                         const void* gz, void* out, cudaStream_t st) {
  const size_t n = (size_t)F * N3;
  if (n == 0) return;
  if (p == P_F64)
    combine_grad_kernel<double><<<blocks_for(n, 256), 256, 0, st>>>(n, N3, g_s, g_z, (const double*)gs,
                                                                     (const double*)gz, (double*)out);
  else
    combine_grad_kernel<float><<<blocks_for(n, 256), 256, 0, st>>>(n, N3, g_s, g_z, (const float*)gs,
                                                                    (const float*)gz, (float*)out); note_launch();
}

void launch_fill_u8(uint8_t* p, uint8_t v, size_t n, cudaStream_t st) {
  if (n == 0) return;
  fill_u8_kernel<<<blocks_for(n, 256), 256, 0, st>>>(p, v, n); note_launch();
}

}  // namespace pcv

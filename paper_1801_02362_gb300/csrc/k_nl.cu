// k_nl.cu -- the neighbour list of the original method and of the close-structure method.
//
// The paper evaluates the distances to all M landmarks only at neighbour-list update steps
// (every L steps, Section 6.2: M_nl + (M - M_nl)/L expensive distances per step) and to
// the M_nl closest ones of the last update in between (Section 2).  With the close
// structure (end of Section 3.2) a reassignment computes every distance exactly and the
// other update steps choose the list from the approximate distances of Eq. (close_dist).
// Eq. (property_map_cv) then sums over the listed landmarks only.
//
// A batch of F frames is handled as:
//   nl_schedule_kernel  update flag and list slot of every frame (one block-wide scan):
//                       slot 0 is the list carried over from the previous call, slot k+1
//                       the list chosen at the k-th update frame of this call;
//   (all-landmark distances of the update frames: the existing exact / approximate pair
//    kernels over a compacted frame list)
//   nl_select_kernel    the M_nl smallest distances of each update frame (radix select
//                       on 64-bit order-preserving keys; ties to the lower index), written
//                       in increasing landmark index;
//   nl_exact_* / nl_approx_kernel  one CTA per frame between updates, one warp per listed
//                       landmark: exact MSD (eigen-solved rotation, then the direct sum) or
//                       the approximate MSD of Eq. (close_dist); unlisted landmarks get +inf,
//                       which the softmax turns into a weight of exactly 0;
//   nl_beta_kernel      the contraction beta = sum_i gamma_i Rot_i a_i of the adjoint over
//                       each frame's own landmarks (all at update frames, the list otherwise).
#include <cuda_fp16.h>

#include <cmath>

#include "pcv_device.cuh"
#include "pcv_internal.h"

namespace pcv {
namespace {

constexpr int NL_SCAN_THREADS = 1024;

// exclusive block-wide prefix counts of up to three 0/1 flags per thread; returns the
// block totals in tot[]; every thread of the block must call it
__device__ __forceinline__ void block_scan3(const bool v[3], int ex[3], int tot[3], int* wsum /* 3 * 32 */) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  int wpre[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const unsigned b = __ballot_sync(0xffffffffu, v[k]);
    wpre[k] = __popc(b & lt);
    if (lane == 0) wsum[k * 32 + w] = __popc(b);
  }
  __syncthreads();
  if (w == 0) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const int x = lane < nw ? wsum[k * 32 + lane] : 0;
      int incl = x;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
      }
      wsum[k * 32 + lane] = incl - x;  // exclusive warp offsets
      const int total = __shfl_sync(0xffffffffu, incl, 31);
      if (lane == 0) wsum[96 + k] = total;
    }
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    ex[k] = wsum[k * 32 + w] + wpre[k];
    tot[k] = wsum[96 + k];
  }
  __syncthreads();  // wsum is reused by the next call
}

// frame t is an update step when (step0 + t) % L == 0, when no list is held yet (t = 0
// only), and in close mode at reassignments (flag != 0)
__global__ void __launch_bounds__(NL_SCAN_THREADS)
nl_schedule_kernel(int F, long long step0, int L, int have_list, const uint8_t* __restrict__ flag,
                   const int* __restrict__ segof, int* __restrict__ slot, uint8_t* __restrict__ upd,
                   int* __restrict__ ulist, int* __restrict__ uapp_list, int* __restrict__ uapp_seg,
                   int* __restrict__ nlist, int* __restrict__ counts) {
  __shared__ int wsum[3 * 32 + 3];
  int base[3] = {0, 0, 0};
  for (int t0 = 0; t0 < F; t0 += NL_SCAN_THREADS) {
    const int t = t0 + threadIdx.x;
    bool v[3] = {false, false, false};
    if (t < F) {
      const bool refresh = flag && flag[t] != 0;
      const bool u = refresh || ((step0 + t) % L == 0) || (t == 0 && !have_list);
      v[0] = u;                      // update frame
      v[1] = u && flag && !refresh;  // update frame evaluated approximately (close mode)
      v[2] = !u;                     // frame between updates
    }
    int ex[3], tot[3];
    block_scan3(v, ex, tot, wsum);
    if (t < F) {
      const int ucount = base[0] + ex[0] + (v[0] ? 1 : 0);  // updates in [0, t]
      slot[t] = ucount;
      upd[t] = v[0] ? 1 : 0;
      if (v[0]) ulist[base[0] + ex[0]] = t;
      if (v[1]) {
        uapp_list[base[1] + ex[1]] = t;
        uapp_seg[base[1] + ex[1]] = segof[t];
      }
      if (v[2]) nlist[base[2] + ex[2]] = t;
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) base[k] += tot[k];
  }
  if (threadIdx.x == 0) {
    counts[0] = base[0];
    counts[1] = base[1];
    counts[2] = base[2];
  }
}

// ---------------------------------------------------------------------------------------
// order-preserving 64-bit key of a distance (IEEE total order for non-NaN values)
__device__ __forceinline__ unsigned long long dist_key(double d) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(d);
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
template <typename DT>
__device__ __forceinline__ double as_double(DT v) {
  return (double)v;
}

constexpr int NL_SEL_THREADS = 256;

// the Mnl smallest of row D[f * M + 0..M) for update frame k = blockIdx.x (f = ulist[k]),
// ties to the lower index, into NLtab[(k + 1) * Mnl ...] in increasing landmark index
template <typename DT>
__global__ void __launch_bounds__(NL_SEL_THREADS)
nl_select_kernel(const int* __restrict__ ulist, const int* __restrict__ counts, int M, int Mnl,
                 const DT* __restrict__ D, int* __restrict__ NLtab) {
  __shared__ unsigned hist[256];
  __shared__ int s_digit, s_rank;
  __shared__ int wsum[3 * 32 + 3];
  const int k = blockIdx.x;
  if (k >= counts[0]) return;  // uniform over the block
  const DT* row = D + (size_t)ulist[k] * M;
  int* out = NLtab + (size_t)(k + 1) * Mnl;
  unsigned long long prefix = 0, mask = 0;
  int rank = Mnl;  // 1-based rank of the wanted key among the keys matching prefix
  for (int pass = 0; pass < 8; ++pass) {
    const int shift = 56 - 8 * pass;
    for (int b = threadIdx.x; b < 256; b += blockDim.x) hist[b] = 0u;
    __syncthreads();
    for (int i = threadIdx.x; i < M; i += blockDim.x) {
      const unsigned long long key = dist_key(as_double(row[i]));
      if ((key & mask) == prefix) atomicAdd(&hist[(key >> shift) & 255u], 1u);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      int cum = 0, b = 0;
      for (; b < 255; ++b) {
        if (cum + (int)hist[b] >= rank) break;
        cum += (int)hist[b];
      }
      s_digit = b;
      s_rank = rank - cum;
    }
    __syncthreads();
    prefix |= (unsigned long long)s_digit << shift;
    mask |= 255ull << shift;
    rank = s_rank;
    __syncthreads();  // s_digit / s_rank are rewritten by the next pass
  }
  // members: keys below the threshold key, and the first `rank` keys equal to it
  int base_eq = 0, base_sel = 0;
  for (int i0 = 0; i0 < M; i0 += blockDim.x) {
    const int i = i0 + threadIdx.x;
    bool lt = false, eq = false;
    if (i < M) {
      const unsigned long long key = dist_key(as_double(row[i]));
      lt = key < prefix;
      eq = key == prefix;
    }
    bool v[3] = {eq, false, false};
    int ex[3], tot[3];
    block_scan3(v, ex, tot, wsum);
    const bool sel = lt || (eq && base_eq + ex[0] < rank);
    const int eq_total = tot[0];
    v[0] = sel;
    block_scan3(v, ex, tot, wsum);
    if (sel) out[base_sel + ex[0]] = i;
    base_eq += eq_total;
    base_sel += tot[0];
  }
}

// ---------------------------------------------------------------------------------------
// Distances to the listed landmarks of the frames between updates.  One CTA per frame
// (k-th entry of nlist), one warp per listed landmark.  The CTA first writes +inf over
// the whole row of D.
constexpr int NL_PAIR_THREADS = 256;

template <typename DT>
__device__ __forceinline__ void fill_row_inf(DT* row, int M) {
  for (int i = threadIdx.x; i < M; i += blockDim.x) row[i] = (DT)INFINITY;
  __syncthreads();
}

// FP32 / FP16 storage: FP32 correlation in compensated chunks of 16 atoms, FP32 eigen-solve
// for the rotation, then Eq. (dist) summed directly (stationary in R), compensated
template <typename LT>
__global__ void __launch_bounds__(NL_PAIR_THREADS)
nl_exact_f32(const int* __restrict__ nlist, const int* __restrict__ counts, const int* __restrict__ slot,
             const int* __restrict__ NLtab, int Mnl, int M, int N, const float* __restrict__ frames,
             const float4* __restrict__ c32, const double* __restrict__ fG, const LT* __restrict__ lm,
             const float* __restrict__ lmoff, const double* __restrict__ lG, const float* __restrict__ wts,
             double dscale, float* __restrict__ D, float* __restrict__ Rnl, unsigned* __restrict__ status) {
  const int k = blockIdx.x;
  if (k >= counts[2]) return;  // uniform over the block
  const int f = nlist[k];
  float* row = D + (size_t)f * M;
  fill_row_inf(row, M);
  const int* members = NLtab + (size_t)slot[f] * Mnl;
  const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const float4 c = c32[f];
  const float* x = frames + (size_t)f * N * 3;
  const double Gx = fG[f];
  for (int r = threadIdx.x >> 5; r < Mnl; r += nw) {
    const int i = members[r];
    float p[9], hi[9], lo[9];
#pragma unroll
    for (int e = 0; e < 9; ++e) p[e] = hi[e] = lo[e] = 0.0f;
    int cnt = 0;
    for (int j = lane; j < N; j += 32) {
      float u[3] = {lm_coord<float, LT>(lm, lmoff, N, i, j, 0), lm_coord<float, LT>(lm, lmoff, N, i, j, 1),
                    lm_coord<float, LT>(lm, lmoff, N, i, j, 2)};
      const float v[3] = {x[3 * j] - c.x, x[3 * j + 1] - c.y, x[3 * j + 2] - c.z};
      if (wts) {
        const float wj = wts[j];
        u[0] *= wj;
        u[1] *= wj;
        u[2] *= wj;
      }
#pragma unroll
      for (int b = 0; b < 3; ++b)
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) p[3 * b + cc] = fmaf(u[b], v[cc], p[3 * b + cc]);
      if (++cnt == 16) {
        cnt = 0;
#pragma unroll
        for (int e = 0; e < 9; ++e) {
          two_sum_acc(hi[e], lo[e], p[e]);
          p[e] = 0.0f;
        }
      }
    }
    float H[9];
#pragma unroll
    for (int e = 0; e < 9; ++e) {
      two_sum_acc(hi[e], lo[e], p[e]);
      warp_sum_pair(hi[e], lo[e]);
      H[e] = hi[e] + lo[e];
    }
    const double Ga = lG[i];
    float q[4], R[9];
    const bool ok = top_quat_f32(H, (float)(0.5 * (Gx + Ga)) * 1.00001f + 1e-30f, q);
    quat_to_rot(q, R);
    float s = 0.0f, shi = 0.0f, slo = 0.0f;
    cnt = 0;
    for (int j = lane; j < N; j += 32) {
      const float a0 = lm_coord<float, LT>(lm, lmoff, N, i, j, 0), a1 = lm_coord<float, LT>(lm, lmoff, N, i, j, 1),
                  a2 = lm_coord<float, LT>(lm, lmoff, N, i, j, 2);
      const float d0 = (x[3 * j] - c.x) - fmaf(R[0], a0, fmaf(R[1], a1, R[2] * a2));
      const float d1 = (x[3 * j + 1] - c.y) - fmaf(R[3], a0, fmaf(R[4], a1, R[5] * a2));
      const float d2 = (x[3 * j + 2] - c.z) - fmaf(R[6], a0, fmaf(R[7], a1, R[8] * a2));
      const float t = fmaf(d0, d0, fmaf(d1, d1, d2 * d2));
      s = wts ? fmaf(wts[j], t, s) : s + t;
      if (++cnt == 16) {
        cnt = 0;
        two_sum_acc(shi, slo, s);
        s = 0.0f;
      }
    }
    two_sum_acc(shi, slo, s);
    warp_sum_pair(shi, slo);
    if (lane == 0) {
      row[i] = (float)(pair_to_double(shi, slo) * dscale);
      if (Rnl) {
        float* dst = Rnl + ((size_t)f * Mnl + r) * 9;
#pragma unroll
        for (int e = 0; e < 9; ++e) dst[e] = R[e];
      }
      if (!ok) atomicOr(status, STATUS_NOCONV);
    }
  }
}

// FP64 mode: FP64 correlation, eigenvalue by Newton on the characteristic polynomial,
// D = (G_x + G_a - 2 lambda_max) dscale as in the FP64 pair kernel
__global__ void __launch_bounds__(NL_PAIR_THREADS)
nl_exact_f64(const int* __restrict__ nlist, const int* __restrict__ counts, const int* __restrict__ slot,
             const int* __restrict__ NLtab, int Mnl, int M, int N, const double* __restrict__ frames,
             const double4* __restrict__ c64, const double* __restrict__ fG, const double* __restrict__ lm,
             const double* __restrict__ lG, const double* __restrict__ w64, double dscale, double* __restrict__ D,
             double* __restrict__ Rnl, unsigned* __restrict__ status) {
  const int k = blockIdx.x;
  if (k >= counts[2]) return;
  const int f = nlist[k];
  double* row = D + (size_t)f * M;
  fill_row_inf(row, M);
  const int* members = NLtab + (size_t)slot[f] * Mnl;
  const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const double4 c = c64[f];
  const double* x = frames + (size_t)f * N * 3;
  const double Gx = fG[f];
  for (int r = threadIdx.x >> 5; r < Mnl; r += nw) {
    const int i = members[r];
    const double* a = lm + (size_t)i * N * 3;
    double h[9];
#pragma unroll
    for (int e = 0; e < 9; ++e) h[e] = 0.0;
    for (int j = lane; j < N; j += 32) {
      const double wj = w64 ? w64[j] : 1.0;
      const double u[3] = {wj * a[3 * j], wj * a[3 * j + 1], wj * a[3 * j + 2]};
      const double v[3] = {x[3 * j] - c.x, x[3 * j + 1] - c.y, x[3 * j + 2] - c.z};
#pragma unroll
      for (int b = 0; b < 3; ++b)
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) h[3 * b + cc] = fma(u[b], v[cc], h[3 * b + cc]);
    }
#pragma unroll
    for (int e = 0; e < 9; ++e) h[e] = warp_sum_double(h[e]);
    if (lane == 0) {
      const double Ga = lG[i];
      bool ok = true;
      double q[4];
      const double lam = top_eig_f64(h, 0.5 * (Gx + Ga), &ok, Rnl ? q : nullptr);
      double d = (Gx + Ga - 2.0 * lam) * dscale;
      row[i] = d < 0.0 ? 0.0 : d;
      if (Rnl) {
        double Rm[9];
        quat_to_rot(q, Rm);
        double* dst = Rnl + ((size_t)f * Mnl + r) * 9;
#pragma unroll
        for (int e = 0; e < 9; ++e) dst[e] = Rm[e];
      }
      if (!ok) atomicOr(status, STATUS_NOCONV);
    }
  }
}

// Approximate MSD of Eq. (close_dist), D~ = sum_j w_j |R_xy^T (x_j - c) - R_{a_i y} a_ij|^2,
// summed directly (positive terms); ST is the arithmetic type (float, or double in FP64 mode)
template <typename ST>
__device__ __forceinline__ void frame_c(const float4* c32, const double4* c64, int f, ST* c);
template <>
__device__ __forceinline__ void frame_c<float>(const float4* c32, const double4*, int f, float* c) {
  const float4 v = c32[f];
  c[0] = v.x;
  c[1] = v.y;
  c[2] = v.z;
}
template <>
__device__ __forceinline__ void frame_c<double>(const float4*, const double4* c64, int f, double* c) {
  const double4 v = c64[f];
  c[0] = v.x;
  c[1] = v.y;
  c[2] = v.z;
}

template <typename ST, typename LT>
__global__ void __launch_bounds__(NL_PAIR_THREADS)
nl_approx_kernel(const int* __restrict__ nlist, const int* __restrict__ counts, const int* __restrict__ slot,
                 const int* __restrict__ NLtab, int Mnl, int M, int N, const ST* __restrict__ frames,
                 const float4* __restrict__ c32, const double4* __restrict__ c64, const LT* __restrict__ lm,
                 const float* __restrict__ lmoff, const float* __restrict__ wts, const double* __restrict__ w64,
                 double dscale, const double4* __restrict__ qxy, const ST* __restrict__ Bseg,
                 const int* __restrict__ segof, ST* __restrict__ D) {
  const int k = blockIdx.x;
  if (k >= counts[2]) return;
  const int f = nlist[k];
  ST* row = D + (size_t)f * M;
  fill_row_inf(row, M);
  const int* members = NLtab + (size_t)slot[f] * Mnl;
  const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  ST c[3];
  frame_c<ST>(c32, c64, f, c);
  ST Rxy[9];
  {
    const double4 qq = qxy[f];
    const ST q[4] = {(ST)qq.x, (ST)qq.y, (ST)qq.z, (ST)qq.w};
    quat_to_rot(q, Rxy);
  }
  const ST* x = frames + (size_t)f * N * 3;
  const int seg = segof[f];
  for (int r = threadIdx.x >> 5; r < Mnl; r += nw) {
    const int i = members[r];
    const ST* B = Bseg + ((size_t)seg * M + i) * 9;
    ST Bm[9];
#pragma unroll
    for (int e = 0; e < 9; ++e) Bm[e] = B[e];
    ST s = 0, shi = 0, slo = 0;  // FP32: chunks of 16 terms into a compensated (hi, lo) total
    int cnt = 0;
    for (int j = lane; j < N; j += 32) {
      const ST v0 = x[3 * j] - c[0], v1 = x[3 * j + 1] - c[1], v2 = x[3 * j + 2] - c[2];
      const ST a0 = lm_coord<ST, LT>(lm, lmoff, N, i, j, 0), a1 = lm_coord<ST, LT>(lm, lmoff, N, i, j, 1),
               a2 = lm_coord<ST, LT>(lm, lmoff, N, i, j, 2);
      const ST d0 = (Rxy[0] * v0 + Rxy[3] * v1 + Rxy[6] * v2) - (Bm[0] * a0 + Bm[1] * a1 + Bm[2] * a2);
      const ST d1 = (Rxy[1] * v0 + Rxy[4] * v1 + Rxy[7] * v2) - (Bm[3] * a0 + Bm[4] * a1 + Bm[5] * a2);
      const ST d2 = (Rxy[2] * v0 + Rxy[5] * v1 + Rxy[8] * v2) - (Bm[6] * a0 + Bm[7] * a1 + Bm[8] * a2);
      const ST t = d0 * d0 + d1 * d1 + d2 * d2;
      if constexpr (sizeof(ST) == 8) {
        s += (w64 ? w64[j] : 1.0) * t;
      } else {
        s += wts ? wts[j] * t : t;
        if (++cnt == 16) {
          cnt = 0;
          two_sum_acc(shi, slo, s);
          s = 0;
        }
      }
    }
    double tot;
    if constexpr (sizeof(ST) == 8) {
      tot = warp_sum_double(s);
    } else {
      two_sum_acc(shi, slo, s);
      warp_sum_pair(shi, slo);
      tot = pair_to_double(shi, slo);
    }
    if (lane == 0) row[i] = (ST)(tot * dscale);
  }
}

// ---------------------------------------------------------------------------------------
// beta_f = sum_i gamma_fi Rot_fi a_i over the frame's landmarks: all M at update frames,
// the list otherwise.  Rot: close mode Bseg[segof[f]] (R_{a_i y}; R_{a_i x} at
// reassignments, whose segment is their own); exact mode Rupd rows of the update frames
// (row = slot - 1) or Rnl (frame, list position).  One CTA per frame, one thread per atom,
// landmarks staged in chunks of NL_BK (gamma^s, gamma^z, Rot, index).
constexpr int NL_BETA_THREADS = 128, NL_BK = 32;

template <typename ST, typename LT>
__global__ void __launch_bounds__(NL_BETA_THREADS)
nl_beta_kernel(int F, int M, int N, int Mnl, const uint8_t* __restrict__ upd, const int* __restrict__ slot,
               const int* __restrict__ NLtab, const LT* __restrict__ lm, const float* __restrict__ lmoff,
               const double* __restrict__ q, const ST* __restrict__ P, const double* __restrict__ s, double lambda,
               const ST* __restrict__ Rupd, const ST* __restrict__ Rnl, const ST* __restrict__ Bseg,
               const int* __restrict__ segof, ST* __restrict__ gs, ST* __restrict__ gz) {
  __shared__ ST sg[NL_BK], zg[NL_BK], sR[NL_BK][9];
  __shared__ int sidx[NL_BK];
  const int f = blockIdx.x;
  if (f >= F) return;
  const bool u = upd[f] != 0;
  const int cnt = u ? M : Mnl;
  const int* members = u ? nullptr : NLtab + (size_t)slot[f] * Mnl;
  const ST sf = (ST)s[f], sl = s_low<ST>(s[f], sf), lam = (ST)lambda;
  for (int j0 = 0; j0 < N; j0 += blockDim.x) {
    const int j = j0 + threadIdx.x;
    ST bs[3] = {0, 0, 0}, bz[3] = {0, 0, 0};
    for (int k0 = 0; k0 < cnt; k0 += NL_BK) {
      __syncthreads();  // the previous chunk's readers are done
      if (threadIdx.x < NL_BK) {
        const int kk = k0 + threadIdx.x;
        ST gsv = 0, gzv = 0;
        ST R[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
        int i = -1;
        if (kk < cnt) {
          i = members ? members[kk] : kk;
          const ST p = P[(size_t)f * M + i];
          gzv = p;
          gsv = -lam * p * (((ST)q[i] - sf) - sl);
          const ST* src = Bseg ? Bseg + ((size_t)segof[f] * M + i) * 9
                               : (u ? Rupd + ((size_t)(slot[f] - 1) * M + i) * 9 : Rnl + ((size_t)f * Mnl + kk) * 9);
#pragma unroll
          for (int e = 0; e < 9; ++e) R[e] = src[e];
        }
        sg[threadIdx.x] = gsv;
        zg[threadIdx.x] = gzv;
#pragma unroll
        for (int e = 0; e < 9; ++e) sR[threadIdx.x][e] = R[e];
        sidx[threadIdx.x] = i;
      }
      __syncthreads();
      if (j < N) {
        const int kn = cnt - k0 < NL_BK ? cnt - k0 : NL_BK;
        for (int kk = 0; kk < kn; ++kk) {
          const ST gsv = sg[kk], gzv = zg[kk];
          if (gsv == (ST)0 && gzv == (ST)0) continue;  // weight underflowed: no contribution
          const int i = sidx[kk];
          const ST a0 = lm_coord<ST, LT>(lm, lmoff, N, i, j, 0), a1 = lm_coord<ST, LT>(lm, lmoff, N, i, j, 1),
                   a2 = lm_coord<ST, LT>(lm, lmoff, N, i, j, 2);
#pragma unroll
          for (int b = 0; b < 3; ++b) {
            const ST ra = sR[kk][3 * b] * a0 + sR[kk][3 * b + 1] * a1 + sR[kk][3 * b + 2] * a2;
            bs[b] += gsv * ra;
            bz[b] += gzv * ra;
          }
        }
      }
    }
    if (j < N) {
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        gs[((size_t)f * N + j) * 3 + b] = bs[b];
        gz[((size_t)f * N + j) * 3 + b] = bz[b];
      }
    }
  }
}

// Tiles of the frames between updates: the frames of list slot s are the consecutive
// frames strictly between update frames ulist[s-1] and ulist[s] (-1 and F at the ends), so
// a tile starts at every NL_TILE_F-th frame of its run
__global__ void __launch_bounds__(NL_SCAN_THREADS)
nl_tiles_kernel(int F, int* __restrict__ counts, const int* __restrict__ nlist, const int* __restrict__ slot,
                const int* __restrict__ ulist, NlTile* __restrict__ tiles) {
  __shared__ int wsum[3 * 32 + 3];
  const int nb = counts[2], nu = counts[0];
  int base = 0;
  for (int p0 = 0; p0 < nb; p0 += NL_SCAN_THREADS) {
    const int p = p0 + threadIdx.x;
    bool v[3] = {false, false, false};
    int rows = 0, sl = 0;
    if (p < nb) {
      const int t = nlist[p];
      sl = slot[t];
      const int u = sl > 0 ? ulist[sl - 1] : -1;
      const int nxt = sl < nu ? ulist[sl] : F;
      const int off = t - u - 1;
      v[0] = off % NL_TILE_F == 0;
      rows = min(NL_TILE_F, nxt - u - 1 - off);
    }
    int ex[3], tot[3];
    block_scan3(v, ex, tot, wsum);
    if (v[0]) tiles[base + ex[0]] = NlTile{p, rows, sl, 0};
    base += tot[0];
  }
  if (threadIdx.x == 0) counts[3] = base;
}

template <typename DT>
__global__ void nl_fill_inf_kernel(const int* __restrict__ counts, const int* __restrict__ nlist, int M,
                                   DT* __restrict__ D) {
  const int p = blockIdx.x;
  if (p >= counts[2]) return;
  DT* row = D + (size_t)nlist[p] * M;
  for (int i = threadIdx.x; i < M; i += blockDim.x) row[i] = (DT)INFINITY;
}

// the list of the last update frame of this call becomes the carried-over list
__global__ void nl_carry_kernel(const int* __restrict__ counts, const int* __restrict__ NLtab, int Mnl,
                                int* __restrict__ keep) {
  const int n = counts[0];
  if (n == 0) return;
  for (int r = threadIdx.x; r < Mnl; r += blockDim.x) keep[r] = NLtab[(size_t)n * Mnl + r];
}

}  // namespace

// ---------------------------------------------------------------------------------------
void launch_nl_schedule(int F, long long step0, int L, bool have_list, const uint8_t* flag, const int* segof,
                        const NlLists& nl, cudaStream_t st) {
  if (F <= 0) return;
  nl_schedule_kernel<<<1, NL_SCAN_THREADS, 0, st>>>(F, step0, L, have_list ? 1 : 0, flag, segof, nl.slot, nl.upd,
                                                    nl.ulist, nl.uapp_list, nl.uapp_seg, nl.nlist, nl.counts);
  note_launch();
}

void launch_nl_select(Prec p, int max_upd, const NlLists& nl, int M, int Mnl, const void* D, int* NLtab,
                      cudaStream_t st) {
  if (max_upd <= 0) return;
  if (p == P_F64)
    nl_select_kernel<double><<<max_upd, NL_SEL_THREADS, 0, st>>>(nl.ulist, nl.counts, M, Mnl, (const double*)D, NLtab);
  else
    nl_select_kernel<float><<<max_upd, NL_SEL_THREADS, 0, st>>>(nl.ulist, nl.counts, M, Mnl, (const float*)D, NLtab);
  note_launch();
}

void launch_nl_exact(Prec p, int max_rows, const NlLists& nl, const int* NLtab, int Mnl, const void* frames,
                     const LandmarkDev& L, FrameInfo fi, void* D, void* Rnl, unsigned* status, cudaStream_t st) {
  if (max_rows <= 0) return;
  switch (p) {
    case P_F64:
      nl_exact_f64<<<max_rows, NL_PAIR_THREADS, 0, st>>>(nl.nlist, nl.counts, nl.slot, NLtab, Mnl, L.M, L.N,
                                                         (const double*)frames, fi.c64, fi.G, (const double*)L.coords,
                                                         L.G, L.w64, L.dscale, (double*)D, (double*)Rnl, status);
      break;
    case P_F32:
      nl_exact_f32<float><<<max_rows, NL_PAIR_THREADS, 0, st>>>(nl.nlist, nl.counts, nl.slot, NLtab, Mnl, L.M, L.N,
                                                                (const float*)frames, fi.c32, fi.G,
                                                                (const float*)L.coords, L.off, L.G, L.w, L.dscale,
                                                                (float*)D, (float*)Rnl, status);
      break;
    case P_F16:
      nl_exact_f32<__half><<<max_rows, NL_PAIR_THREADS, 0, st>>>(nl.nlist, nl.counts, nl.slot, NLtab, Mnl, L.M, L.N,
                                                                 (const float*)frames, fi.c32, fi.G,
                                                                 (const __half*)L.coords, L.off, L.G, L.w, L.dscale,
                                                                 (float*)D, (float*)Rnl, status);
      break;
  }
  note_launch();
}

void launch_nl_approx(Prec p, int max_rows, const NlLists& nl, const int* NLtab, int Mnl, const void* frames,
                      const LandmarkDev& L, FrameInfo fi, const double4* qxy, const void* Bseg, const int* segof,
                      void* D, cudaStream_t st) {
  if (max_rows <= 0) return;
  switch (p) {
    case P_F64:
      nl_approx_kernel<double, double><<<max_rows, NL_PAIR_THREADS, 0, st>>>(
          nl.nlist, nl.counts, nl.slot, NLtab, Mnl, L.M, L.N, (const double*)frames, fi.c32, fi.c64,
          (const double*)L.coords, L.off, L.w, L.w64, L.dscale, qxy, (const double*)Bseg, segof, (double*)D);
      break;
    case P_F32:
      nl_approx_kernel<float, float><<<max_rows, NL_PAIR_THREADS, 0, st>>>(
          nl.nlist, nl.counts, nl.slot, NLtab, Mnl, L.M, L.N, (const float*)frames, fi.c32, fi.c64,
          (const float*)L.coords, L.off, L.w, L.w64, L.dscale, qxy, (const float*)Bseg, segof, (float*)D);
      break;
    case P_F16:
      nl_approx_kernel<float, __half><<<max_rows, NL_PAIR_THREADS, 0, st>>>(
          nl.nlist, nl.counts, nl.slot, NLtab, Mnl, L.M, L.N, (const float*)frames, fi.c32, fi.c64,
          (const __half*)L.coords, L.off, L.w, L.w64, L.dscale, qxy, (const float*)Bseg, segof, (float*)D);
      break;
  }
  note_launch();
}

void launch_nl_beta(Prec p, int F, const NlLists& nl, const int* NLtab, int Mnl, const LandmarkDev& L, const void* P,
                    const double* s, double lambda, const void* Rupd, const void* Rnl, const void* Bseg,
                    const int* segof, void* gs, void* gz, cudaStream_t st) {
  if (F <= 0) return;
  switch (p) {
    case P_F64:
      nl_beta_kernel<double, double><<<F, NL_BETA_THREADS, 0, st>>>(
          F, L.M, L.N, Mnl, nl.upd, nl.slot, NLtab, (const double*)L.coords, L.off, L.q, (const double*)P, s, lambda,
          (const double*)Rupd, (const double*)Rnl, (const double*)Bseg, segof, (double*)gs, (double*)gz);
      break;
    case P_F32:
      nl_beta_kernel<float, float><<<F, NL_BETA_THREADS, 0, st>>>(
          F, L.M, L.N, Mnl, nl.upd, nl.slot, NLtab, (const float*)L.coords, L.off, L.q, (const float*)P, s, lambda,
          (const float*)Rupd, (const float*)Rnl, (const float*)Bseg, segof, (float*)gs, (float*)gz);
      break;
    case P_F16:
      nl_beta_kernel<float, __half><<<F, NL_BETA_THREADS, 0, st>>>(
          F, L.M, L.N, Mnl, nl.upd, nl.slot, NLtab, (const __half*)L.coords, L.off, L.q, (const float*)P, s, lambda,
          (const float*)Rupd, (const float*)Rnl, (const float*)Bseg, segof, (float*)gs, (float*)gz);
      break;
  }
  note_launch();
}

void launch_nl_tiles(int F, const NlLists& nl, NlTile* tiles, cudaStream_t st) {
  if (F <= 0) return;
  nl_tiles_kernel<<<1, NL_SCAN_THREADS, 0, st>>>(F, nl.counts, nl.nlist, nl.slot, nl.ulist, tiles);
  note_launch();
}

void launch_nl_fill_inf(Prec p, int max_between, const NlLists& nl, int M, void* D, cudaStream_t st) {
  if (max_between <= 0) return;
  if (p == P_F64)
    nl_fill_inf_kernel<double><<<max_between, 128, 0, st>>>(nl.counts, nl.nlist, M, (double*)D);
  else
    nl_fill_inf_kernel<float><<<max_between, 128, 0, st>>>(nl.counts, nl.nlist, M, (float*)D);
  note_launch();
}

void launch_nl_carry(const NlLists& nl, const int* NLtab, int Mnl, int* keep, cudaStream_t st) {
  nl_carry_kernel<<<1, 256, 0, st>>>(nl.counts, NLtab, Mnl, keep);
  note_launch();
}

}  // namespace pcv

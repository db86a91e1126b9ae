// k_pair.cu -- frame x landmark pair kernels (the O(F M N) part of the path).
//
// exact pair kernels: Algorithm 1 (and the reassignment branch of Algorithm 2) for a tile
//   of TF frames x TM landmarks.  The 3x3 correlation H_fi[b][c] = sum_j wk_j a_ijb x_fjc
//   is a dense (3 TM x N)(N x 3 TF) contraction; each thread owns 2 frames x 2 landmarks
//   (36 sums), atoms are streamed through shared memory in chunks of KC.  The quaternion
//   eigen-solve (Section 3, Kearsley / Coutsias) gives R per pair.  FP32 modes then
//   evaluate Eq. (dist) directly in a second pass; FP64 mode assembles
//   D = G_x + G_a - 2 lambda_max.
// approx_pair_kernel: Eq. (close_dist) for frames of Algorithm 2's "else" branch.  With
//   x' = R_{xy}^T x and b_i = R_{a_i y} a_i the approximate distance is
//   D~ = sum_j w_j |x'_j - b_ij|^2, evaluated directly (positive terms, no cancellation);
//   landmarks are rotated by their stored R_{a_i y} while being staged, frames by the
//   transpose of their R_{xy}.
#include <cuda_fp16.h>

#include "pcv_device.cuh"
#include "pcv_internal.h"

namespace pcv {
namespace {

template <typename ST>
__device__ __forceinline__ void load2(const ST* p, ST& a, ST& b);
template <>
__device__ __forceinline__ void load2<float>(const float* p, float& a, float& b) {
  const float2 v = *reinterpret_cast<const float2*>(p);
  a = v.x;
  b = v.y;
}
template <>
__device__ __forceinline__ void load2<double>(const double* p, double& a, double& b) {
  const double2 v = *reinterpret_cast<const double2*>(p);
  a = v.x;
  b = v.y;
}
template <typename ST>
__device__ __forceinline__ void load4(const ST* p, ST* o);
template <>
__device__ __forceinline__ void load4<float>(const float* p, float* o) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  o[0] = v.x;
  o[1] = v.y;
  o[2] = v.z;
  o[3] = v.w;
}
template <>
__device__ __forceinline__ void load4<double>(const double* p, double* o) {
  const double2 v0 = *reinterpret_cast<const double2*>(p);
  const double2 v1 = *reinterpret_cast<const double2*>(p + 2);
  o[0] = v0.x;
  o[1] = v0.y;
  o[2] = v1.x;
  o[3] = v1.y;
}

template <typename ST>
__device__ __forceinline__ void frame_centre(const float4* c32, const double4* c64, int f, ST* c);
template <>
__device__ __forceinline__ void frame_centre<float>(const float4* c32, const double4*, int f, float* c) {
  const float4 v = c32[f];
  c[0] = v.x;
  c[1] = v.y;
  c[2] = v.z;
}
template <>
__device__ __forceinline__ void frame_centre<double>(const float4*, const double4* c64, int f, double* c) {
  const double4 v = c64[f];
  c[0] = v.x;
  c[1] = v.y;
  c[2] = v.z;
}

// ---------------------------------------------------------------------------------------
constexpr int EX_TF = 16, EX_TM = 32, EX_THREADS = 128;

// Stage one chunk of KC atoms of the tile: frames centred (weight mode 1: x w_j,
// 2: x sqrt(w_j)), landmarks (mode 2: a sqrt(w_j)).  Layout [jj*3 + c][row].  Landmark
// column c of the tile is landmark i0 + c, or with a column list cols (a neighbour list of
// ncol entries) landmark cols[i0 + c].
template <typename FT, typename LT, typename ST, int TF, int TM, int KC, int PF, int PM>
__device__ __forceinline__ void stage_exact(int j0, int N, int M, int i0, const FT* __restrict__ frames,
                                            const LT* __restrict__ lm, const float* __restrict__ lmoff,
                                            const ST* __restrict__ wts, int wmode, const int* s_frame,
                                            const ST (*s_c)[3],
                                            ST (*Xs)[PF], ST (*As)[PM], const int* __restrict__ cols = nullptr,
                                            int ncol = 0) {
  const int tid = threadIdx.x;
  for (int e = tid; e < TF * KC; e += EX_THREADS) {
    const int ff = e / KC, jj = e - ff * KC;
    const int j = j0 + jj;
    const int f = s_frame[ff];
    ST v0 = 0, v1 = 0, v2 = 0;
    if (f >= 0 && j < N) {
      const FT* src = frames + ((size_t)f * N + j) * 3;
      v0 = (ST)src[0] - s_c[ff][0];
      v1 = (ST)src[1] - s_c[ff][1];
      v2 = (ST)src[2] - s_c[ff][2];
      if (wts && wmode) {
        const ST wj = wmode == 1 ? (ST)wts[j] : (ST)sqrt((double)wts[j]);
        v0 *= wj;
        v1 *= wj;
        v2 *= wj;
      }
    }
    Xs[jj * 3 + 0][ff] = v0;
    Xs[jj * 3 + 1][ff] = v1;
    Xs[jj * 3 + 2][ff] = v2;
  }
  for (int e = tid; e < TM * KC; e += EX_THREADS) {
    const int ll = e / KC, jj = e - ll * KC;
    const int j = j0 + jj, ci = i0 + ll;
    ST v0 = 0, v1 = 0, v2 = 0;
    if ((cols ? ci < ncol : ci < M) && j < N) {
      const int i = cols ? cols[ci] : ci;
      v0 = lm_coord<ST, LT>(lm, lmoff, N, i, j, 0);
      v1 = lm_coord<ST, LT>(lm, lmoff, N, i, j, 1);
      v2 = lm_coord<ST, LT>(lm, lmoff, N, i, j, 2);
      if (wts && wmode == 2) {
        const ST sw = (ST)sqrt((double)wts[j]);
        v0 *= sw;
        v1 *= sw;
        v2 *= sw;
      }
    }
    As[jj * 3 + 0][ll] = v0;
    As[jj * 3 + 1][ll] = v1;
    As[jj * 3 + 2][ll] = v2;
  }
}

template <typename FT, typename ST, int TF = EX_TF>
__device__ __forceinline__ void load_tile_frames(int rows, const int* __restrict__ row_frame, int row0,
                                                 const float4* __restrict__ c32, const double4* __restrict__ c64,
                                                 int* s_frame, ST (*s_c)[3]) {
  const int tid = threadIdx.x;
  if (tid < TF) {
    const int r = row0 + tid;
    int f = -1;
    if (r < rows) f = row_frame ? row_frame[r] : r;
    s_frame[tid] = f;
    ST c[3] = {0, 0, 0};
    if (f >= 0) frame_centre<ST>(c32, c64, f, c);
    s_c[tid][0] = c[0];
    s_c[tid][1] = c[1];
    s_c[tid][2] = c[2];
  }
}

// FP32 modes: two passes over the atoms of a TF x TM tile (frames x landmarks; 16 x 32 by
// default, 32 x 16 and 8 x 64 for the group launch's autotuner), 128 threads, each on 2
// frames x 2 landmarks.
//  pass 1: H = sum_j w_j a_j x_j^T in FP32 (2 frames x 2 landmarks x 9 sums per thread);
//          per pair, the top eigenvector of the quaternion matrix in FP32 -> R_{a x};
//  pass 2: D = sum_j w_j |x_j - R a_j|^2 directly in FP32 (Eq. dist): positive terms, no
//          cancellation, stationary in R -- so D is accurate to ~1e-7 relative although
//          every operation is FP32.
// one TF-frame x TM-landmark tile with origin (row0, i0); the per-call kernel, the
// persistent group kernel and the neighbour-list kernels (column list cols of ncol
// landmarks; rotations then go to Rout[(f * ncol + column) * 9]) run it.
// APPROX: the approximate MSD of Eq. (close_dist) instead: no pass 1, the rotation of each
// pair is R_xy R_{a_i y} from the frame's alignment quaternion qxy[f] and the stored
// rotations Bseg[segof[f] * M + i], then the direct pass 2.
template <typename LT, bool APPROX = false, int TF = EX_TF, int TM = EX_TM>
__device__ __forceinline__ void exact_tile_f32(int rows, const int* __restrict__ row_frame,
                                               const float* __restrict__ frames, const float4* __restrict__ c32,
                                               const double* __restrict__ fG, const LT* __restrict__ lm,
                                               const float* __restrict__ lmoff, const double* __restrict__ lG,
                                               const float* __restrict__ wts, int M, int N, double dscale,
                                               float* __restrict__ Dout, float* __restrict__ Rout,
                                               unsigned* __restrict__ status, int row0, int i0,
                                               const int* __restrict__ cols = nullptr, int ncol = 0,
                                               const double4* __restrict__ qxy = nullptr,
                                               const float* __restrict__ Bseg = nullptr,
                                               const int* __restrict__ segof = nullptr, int cap = 60) {
  constexpr int KC = 32;
  constexpr int PF = TF + 2, PM = TM + 2;
  static_assert(TF * TM == 4 * EX_THREADS && 64 % TM == 0 && TF % 2 == 0, "tile shape: 128 threads of 2 x 2 pairs");
  __shared__ __align__(16) float Xs[KC * 3][PF];
  __shared__ __align__(16) float As[KC * 3][PM];
  __shared__ int s_frame[TF];
  __shared__ float s_c[TF][3];
  // per-thread totals of the correlation sums: each KC-atom chunk is summed in registers
  // and then added here, so the longest rounding chain is KC + N / KC terms instead of N
  // (at 4400 atoms the single chain put ~1e-4 into H, hence into R and the exact frames'
  // gradients; the MSD itself is stationary in R)
  __shared__ float Hs[36][EX_THREADS];

  if (row0 >= rows) return;
  const int tid = threadIdx.x;
  const int tx = tid % (TM / 2);  // landmark pair: i0 + 2 tx + {0,1}
  const int ty = tid / (TM / 2);  // frame pair: rows 2 ty + {0,1}
  load_tile_frames<float, float, TF>(rows, row_frame, row0, c32, nullptr, s_frame, s_c);
  __syncthreads();
  // a warp holds the rows row0 + (128 / TM) w onwards (128 / TM of them): warps wholly past
  // the rows skip the products (a tile of few frames, e.g. one MD step)
  const int kc_live = row0 + (tid >> 5) * (128 / TM) < rows ? KC : 0;

  float h[2][2][9];
#pragma unroll
  for (int u = 0; u < 2; ++u)
#pragma unroll
    for (int v = 0; v < 2; ++v)
#pragma unroll
      for (int e = 0; e < 9; ++e) h[u][v][e] = 0.0f;
  if (!APPROX)
#pragma unroll
    for (int e = 0; e < 36; ++e) Hs[e][tid] = 0.0f;

  for (int j0 = 0; j0 < (APPROX ? 0 : N); j0 += KC) {
    stage_exact<float, LT, float, TF, TM, KC, PF, PM>(j0, N, M, i0, frames, lm, lmoff, wts, 1, s_frame, s_c, Xs, As,
                                                      cols, ncol);
    __syncthreads();
#pragma unroll 4
    for (int jj = 0; jj < kc_live; ++jj) {
      float x[2][3], a[2][3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        load2<float>(&Xs[jj * 3 + c][ty * 2], x[0][c], x[1][c]);
        load2<float>(&As[jj * 3 + c][tx * 2], a[0][c], a[1][c]);
      }
#pragma unroll
      for (int u = 0; u < 2; ++u)
#pragma unroll
        for (int v = 0; v < 2; ++v)
#pragma unroll
          for (int b = 0; b < 3; ++b)
#pragma unroll
            for (int c = 0; c < 3; ++c) h[u][v][3 * b + c] = fmaf(a[v][b], x[u][c], h[u][v][3 * b + c]);
    }
#pragma unroll
    for (int u = 0; u < 2; ++u)
#pragma unroll
      for (int v = 0; v < 2; ++v)
#pragma unroll
        for (int e = 0; e < 9; ++e) {
          Hs[(2 * u + v) * 9 + e][tid] += h[u][v][e];
          h[u][v][e] = 0.0f;
        }
    __syncthreads();
  }
  if (!APPROX)
#pragma unroll
    for (int u = 0; u < 2; ++u)
#pragma unroll
      for (int v = 0; v < 2; ++v)
#pragma unroll
        for (int e = 0; e < 9; ++e) h[u][v][e] = Hs[(2 * u + v) * 9 + e][tid];

  // rotations of the four pairs
  float R[2][2][9];
  bool all_ok = true;
#pragma unroll
  for (int u = 0; u < 2; ++u)
#pragma unroll
    for (int v = 0; v < 2; ++v) {
      const int f = s_frame[ty * 2 + u];
      const int ci = i0 + tx * 2 + v;
      float q[4] = {1.0f, 0.0f, 0.0f, 0.0f};
      if (APPROX) {
        float Rxy[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1}, B[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
        if (f >= 0 && (cols ? ci < ncol : ci < M)) {
          const int i = cols ? cols[ci] : ci;
          const double4 qq = qxy[f];
          const float qf[4] = {(float)qq.x, (float)qq.y, (float)qq.z, (float)qq.w};
          quat_to_rot(qf, Rxy);
          const float* Bi = Bseg + ((size_t)segof[f] * M + i) * 9;
#pragma unroll
          for (int e = 0; e < 9; ++e) B[e] = Bi[e];
        }
#pragma unroll
        for (int b = 0; b < 3; ++b)
#pragma unroll
          for (int cc = 0; cc < 3; ++cc)
            R[u][v][3 * b + cc] = fmaf(Rxy[3 * b], B[cc], fmaf(Rxy[3 * b + 1], B[3 + cc], Rxy[3 * b + 2] * B[6 + cc]));
        continue;
      }
      if (f >= 0 && (cols ? ci < ncol : ci < M)) {
        const int i = cols ? cols[ci] : ci;
        const float ub = (float)(0.5 * (fG[f] + lG[i])) * 1.00001f + 1e-30f;
        all_ok &= top_quat_f32(h[u][v], ub, q, cap);
      }
      quat_to_rot(q, R[u][v]);
    }

  // per-chunk FP32 partials, added into an error-free (hi, lo) total after each chunk
  const float dsf = (float)dscale;
  float acc[2][2] = {{0.0f, 0.0f}, {0.0f, 0.0f}};
  float thi[2][2] = {{0.0f, 0.0f}, {0.0f, 0.0f}}, tlo[2][2] = {{0.0f, 0.0f}, {0.0f, 0.0f}};
  for (int j0 = 0; j0 < N; j0 += KC) {
    stage_exact<float, LT, float, TF, TM, KC, PF, PM>(j0, N, M, i0, frames, lm, lmoff, wts, 2, s_frame, s_c, Xs, As,
                                                      cols, ncol);
    __syncthreads();
#pragma unroll 4
    for (int jj = 0; jj < kc_live; ++jj) {
      float x[2][3], a[2][3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        load2<float>(&Xs[jj * 3 + c][ty * 2], x[0][c], x[1][c]);
        load2<float>(&As[jj * 3 + c][tx * 2], a[0][c], a[1][c]);
      }
#pragma unroll
      for (int u = 0; u < 2; ++u)
#pragma unroll
        for (int v = 0; v < 2; ++v) {
          const float* Rr = R[u][v];
          const float d0 = x[u][0] - fmaf(Rr[0], a[v][0], fmaf(Rr[1], a[v][1], Rr[2] * a[v][2]));
          const float d1 = x[u][1] - fmaf(Rr[3], a[v][0], fmaf(Rr[4], a[v][1], Rr[5] * a[v][2]));
          const float d2 = x[u][2] - fmaf(Rr[6], a[v][0], fmaf(Rr[7], a[v][1], Rr[8] * a[v][2]));
          acc[u][v] = fmaf(d0, d0, fmaf(d1, d1, fmaf(d2, d2, acc[u][v])));
        }
    }
#pragma unroll
    for (int u = 0; u < 2; ++u)
#pragma unroll
      for (int v = 0; v < 2; ++v) {
        two_sum_acc(thi[u][v], tlo[u][v], acc[u][v]);
        acc[u][v] = 0.0f;
      }
    __syncthreads();
  }

#pragma unroll
  for (int u = 0; u < 2; ++u)
#pragma unroll
    for (int v = 0; v < 2; ++v) {
      const int r = row0 + ty * 2 + u;
      const int f = s_frame[ty * 2 + u];
      const int ci = i0 + tx * 2 + v;
      if (f < 0 || !(cols ? ci < ncol : ci < M)) continue;
      const int i = cols ? cols[ci] : ci;
      Dout[(size_t)f * M + i] = (thi[u][v] + tlo[u][v]) * dsf;
      if (Rout && !APPROX) {
        float* dst = cols ? Rout + ((size_t)f * ncol + ci) * 9 : Rout + ((size_t)r * M + i) * 9;
#pragma unroll
        for (int e = 0; e < 9; ++e) dst[e] = R[u][v][e];
      }
    }
  if (!all_ok) atomicOr(status, STATUS_NOCONV);
}

// ---------------------------------------------------------------------------------------
// The exact tiles with the atoms split over SPLITS slices (FP32 modes): for batches of few
// frames against many landmarks (the reassignment frames of a batch: 34 frames x 2000
// landmarks gave 189 tiles, one CTA each, a long serial chain per CTA on a mostly idle GPU).
// exact_split_pass1: the 16 x 32 tile's correlation sums over its slice of the atoms, to
//   Hp[((s * rows + r) * M + i) * 9 + e];
// exact_split_pass2: every slice's CTA adds the partials in slice order (the same H, hence
//   the same R, in every slice), solves for R (slice 0 writes it to Rout), and sums
//   w |x - R a|^2 over its slice (compensated) to Dp[((s * rows + r) * M + i) * 2 + {0,1}];
// exact_split_finish: D = the slices' (hi, lo) pairs added in slice order.
// Arithmetic per atom as exact_tile_f32; the sums are split, not reordered within a chunk.
// atoms [j_beg, j_end) of slice s: whole chunks of 32, the last slice ending at N
__device__ __forceinline__ void split_range(int N, int nsplit, int s, int& j_beg, int& j_end) {
  const int chunks = (N + 31) / 32, per = (chunks + nsplit - 1) / nsplit;
  j_beg = min(N, s * per * 32);
  j_end = min(N, (s + 1) * per * 32);
}

template <typename LT>
__global__ void __launch_bounds__(EX_THREADS, 4)
exact_split_pass1(int rows, const int* __restrict__ row_frame, const float* __restrict__ frames,
                  const float4* __restrict__ c32, const LT* __restrict__ lm, const float* __restrict__ lmoff,
                  const float* __restrict__ wts, int M, int N, int nsplit, float* __restrict__ Hp) {
  constexpr int TF = EX_TF, TM = EX_TM, KC = 32, PF = TF + 2, PM = TM + 2;
  __shared__ __align__(16) float Xs[KC * 3][PF];
  __shared__ __align__(16) float As[KC * 3][PM];
  __shared__ int s_frame[TF];
  __shared__ float s_c[TF][3];
  const int row0 = blockIdx.y * TF, i0 = blockIdx.x * TM, sp = blockIdx.z;
  const int tid = threadIdx.x, tx = tid % (TM / 2), ty = tid / (TM / 2);
  int j_beg, j_end;
  split_range(N, nsplit, sp, j_beg, j_end);
  load_tile_frames<float, float, TF>(rows, row_frame, row0, c32, nullptr, s_frame, s_c);
  __syncthreads();
  const int kc_live = row0 + (tid >> 5) * (128 / TM) < rows ? KC : 0;
  float h[2][2][9], t[2][2][9];
#pragma unroll
  for (int u = 0; u < 2; ++u)
#pragma unroll
    for (int v = 0; v < 2; ++v)
#pragma unroll
      for (int e = 0; e < 9; ++e) h[u][v][e] = t[u][v][e] = 0.0f;
  for (int j0 = j_beg; j0 < j_end; j0 += KC) {
    stage_exact<float, LT, float, TF, TM, KC, PF, PM>(j0, N, M, i0, frames, lm, lmoff, wts, 1, s_frame, s_c, Xs,
                                                      As);  // chunks never cross j_end (whole chunks per slice)
    __syncthreads();
#pragma unroll 4
    for (int jj = 0; jj < kc_live; ++jj) {
      float x[2][3], a[2][3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        load2<float>(&Xs[jj * 3 + c][ty * 2], x[0][c], x[1][c]);
        load2<float>(&As[jj * 3 + c][tx * 2], a[0][c], a[1][c]);
      }
#pragma unroll
      for (int u = 0; u < 2; ++u)
#pragma unroll
        for (int v = 0; v < 2; ++v)
#pragma unroll
          for (int b = 0; b < 3; ++b)
#pragma unroll
            for (int c = 0; c < 3; ++c) h[u][v][3 * b + c] = fmaf(a[v][b], x[u][c], h[u][v][3 * b + c]);
    }
#pragma unroll
    for (int u = 0; u < 2; ++u)
#pragma unroll
      for (int v = 0; v < 2; ++v)
#pragma unroll
        for (int e = 0; e < 9; ++e) {
          t[u][v][e] += h[u][v][e];  // chunk totals: chains of KC + chunks-per-slice terms
          h[u][v][e] = 0.0f;
        }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 2; ++u)
#pragma unroll
    for (int v = 0; v < 2; ++v) {
      const int r = row0 + ty * 2 + u, i = i0 + tx * 2 + v;
      if (r >= rows || i >= M) continue;
      float* dst = Hp + (((size_t)sp * rows + r) * M + i) * 9;
#pragma unroll
      for (int e = 0; e < 9; ++e) dst[e] = t[u][v][e];
    }
}

template <typename LT>
__global__ void __launch_bounds__(EX_THREADS, 4)
exact_split_pass2(int rows, const int* __restrict__ row_frame, const float* __restrict__ frames,
                  const float4* __restrict__ c32, const double* __restrict__ fG, const LT* __restrict__ lm,
                  const float* __restrict__ lmoff, const double* __restrict__ lG, const float* __restrict__ wts, int M,
                  int N, int nsplit, const float* __restrict__ Hp, float* __restrict__ Dp, float* __restrict__ Rout,
                  unsigned* __restrict__ status, int cap) {
  constexpr int TF = EX_TF, TM = EX_TM, KC = 32, PF = TF + 2, PM = TM + 2;
  __shared__ __align__(16) float Xs[KC * 3][PF];
  __shared__ __align__(16) float As[KC * 3][PM];
  __shared__ int s_frame[TF];
  __shared__ float s_c[TF][3];
  const int row0 = blockIdx.y * TF, i0 = blockIdx.x * TM, sp = blockIdx.z;
  const int tid = threadIdx.x, tx = tid % (TM / 2), ty = tid / (TM / 2);
  int j_beg, j_end;
  split_range(N, nsplit, sp, j_beg, j_end);
  load_tile_frames<float, float, TF>(rows, row_frame, row0, c32, nullptr, s_frame, s_c);
  __syncthreads();
  const int kc_live = row0 + (tid >> 5) * (128 / TM) < rows ? KC : 0;
  float R[2][2][9];
  bool all_ok = true;
#pragma unroll
  for (int u = 0; u < 2; ++u)
#pragma unroll
    for (int v = 0; v < 2; ++v) {
      const int r = row0 + ty * 2 + u, i = i0 + tx * 2 + v;
      const int f = s_frame[ty * 2 + u];
      float q[4] = {1.0f, 0.0f, 0.0f, 0.0f};
      if (f >= 0 && i < M) {
        float H[9];
#pragma unroll
        for (int e = 0; e < 9; ++e) H[e] = 0.0f;
        for (int k = 0; k < nsplit; ++k) {  // slice order: the same H in every slice's CTA
          const float* src = Hp + (((size_t)k * rows + r) * M + i) * 9;
#pragma unroll
          for (int e = 0; e < 9; ++e) H[e] += src[e];
        }
        const float ub = (float)(0.5 * (fG[f] + lG[i])) * 1.00001f + 1e-30f;
        all_ok &= top_quat_f32(H, ub, q, cap);
      }
      quat_to_rot(q, R[u][v]);
    }
  float acc[2][2] = {{0.0f, 0.0f}, {0.0f, 0.0f}};
  float thi[2][2] = {{0.0f, 0.0f}, {0.0f, 0.0f}}, tlo[2][2] = {{0.0f, 0.0f}, {0.0f, 0.0f}};
  for (int j0 = j_beg; j0 < j_end; j0 += KC) {
    stage_exact<float, LT, float, TF, TM, KC, PF, PM>(j0, N, M, i0, frames, lm, lmoff, wts, 2, s_frame, s_c, Xs,
                                                      As);  // chunks never cross j_end (whole chunks per slice)
    __syncthreads();
#pragma unroll 4
    for (int jj = 0; jj < kc_live; ++jj) {
      float x[2][3], a[2][3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        load2<float>(&Xs[jj * 3 + c][ty * 2], x[0][c], x[1][c]);
        load2<float>(&As[jj * 3 + c][tx * 2], a[0][c], a[1][c]);
      }
#pragma unroll
      for (int u = 0; u < 2; ++u)
#pragma unroll
        for (int v = 0; v < 2; ++v) {
          const float* Rr = R[u][v];
          const float d0 = x[u][0] - fmaf(Rr[0], a[v][0], fmaf(Rr[1], a[v][1], Rr[2] * a[v][2]));
          const float d1 = x[u][1] - fmaf(Rr[3], a[v][0], fmaf(Rr[4], a[v][1], Rr[5] * a[v][2]));
          const float d2 = x[u][2] - fmaf(Rr[6], a[v][0], fmaf(Rr[7], a[v][1], Rr[8] * a[v][2]));
          acc[u][v] = fmaf(d0, d0, fmaf(d1, d1, fmaf(d2, d2, acc[u][v])));
        }
    }
#pragma unroll
    for (int u = 0; u < 2; ++u)
#pragma unroll
      for (int v = 0; v < 2; ++v) {
        two_sum_acc(thi[u][v], tlo[u][v], acc[u][v]);
        acc[u][v] = 0.0f;
      }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 2; ++u)
#pragma unroll
    for (int v = 0; v < 2; ++v) {
      const int r = row0 + ty * 2 + u, i = i0 + tx * 2 + v;
      if (s_frame[ty * 2 + u] < 0 || i >= M) continue;
      float* dp = Dp + (((size_t)sp * rows + r) * M + i) * 2;
      dp[0] = thi[u][v];
      dp[1] = tlo[u][v];
      if (Rout && sp == 0) {
        float* dst = Rout + ((size_t)r * M + i) * 9;
#pragma unroll
        for (int e = 0; e < 9; ++e) dst[e] = R[u][v][e];
      }
    }
  if (!all_ok && sp == 0) atomicOr(status, STATUS_NOCONV);
}

__global__ void exact_split_finish(int rows, const int* __restrict__ row_frame, int M, int nsplit, float dscale,
                                   const float* __restrict__ Dp, float* __restrict__ Dout) {
  const size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (k >= (size_t)rows * M) return;
  const int r = (int)(k / M), i = (int)(k - (size_t)r * M);
  const int f = row_frame ? row_frame[r] : r;
  float hi = 0.0f, lo = 0.0f;
  for (int sp = 0; sp < nsplit; ++sp) {
    const float* d = Dp + (((size_t)sp * rows + r) * M + i) * 2;
    two_sum_acc(hi, lo, d[0]);
    lo += d[1];
  }
  Dout[(size_t)f * M + i] = (hi + lo) * dscale;
}

template <typename LT, int TF = EX_TF, int TM = EX_TM>
__global__ void __launch_bounds__(EX_THREADS, 4)
exact_pair_f32(int rows, const int* __restrict__ row_frame, const float* __restrict__ frames,
               const float4* __restrict__ c32, const double* __restrict__ fG, const LT* __restrict__ lm,
               const float* __restrict__ lmoff, const double* __restrict__ lG, const float* __restrict__ wts, int M,
               int N, double dscale, float* __restrict__ Dout, float* __restrict__ Rout,
               unsigned* __restrict__ status, int cap) {
  exact_tile_f32<LT, false, TF, TM>(rows, row_frame, frames, c32, fG, lm, lmoff, lG, wts, M, N, dscale, Dout, Rout,
                                    status, blockIdx.y * TF, blockIdx.x * TM, nullptr, 0, nullptr, nullptr, nullptr,
                                    cap);
}

// Many instances in one persistent launch: CTA b takes tiles b, b + grid, ... (tiles of
// TF x TM: the host lists them for the shape it launches)
template <typename LT, int TF = EX_TF, int TM = EX_TM>
__global__ void __launch_bounds__(EX_THREADS, 4)
exact_group_f32(const GroupInst* __restrict__ I, const GroupTile* __restrict__ tiles, int ntiles) {
  for (int k = blockIdx.x; k < ntiles; k += gridDim.x) {
    const GroupTile w = tiles[k];
    const GroupInst& t = I[w.inst];
    exact_tile_f32<LT, false, TF, TM>(t.F, nullptr, t.frames, t.c32, t.fG, (const LT*)t.lm, t.lmoff, t.lG, t.w, t.M,
                                      t.N, t.dscale, t.D, nullptr, t.status, w.row0, w.i0);
    __syncthreads();  // the tile's shared staging is reused by the next tile
  }
}

// Neighbour list: tile k = blockIdx.y covers `rows` consecutive entries of the list of
// frames between list updates (all sharing the list `slot`), blockIdx.x the listed
// landmarks in columns of 32.  APPROX: Eq. (close_dist) with the frames' close structures.
template <typename LT, bool APPROX>
__global__ void __launch_bounds__(EX_THREADS, 4)
nl_list_f32(const NlTile* __restrict__ tiles, const int* __restrict__ ntiles, const int* __restrict__ nlist,
            const int* __restrict__ NLtab, int Mnl, const float* __restrict__ frames, const float4* __restrict__ c32,
            const double* __restrict__ fG, const LT* __restrict__ lm, const float* __restrict__ lmoff,
            const double* __restrict__ lG, const float* __restrict__ wts, int M, int N, double dscale,
            float* __restrict__ Dout, float* __restrict__ Rnl, unsigned* __restrict__ status,
            const double4* __restrict__ qxy, const float* __restrict__ Bseg, const int* __restrict__ segof) {
  if ((int)blockIdx.y >= *ntiles) return;  // uniform over the block
  const NlTile w = tiles[blockIdx.y];
  exact_tile_f32<LT, APPROX>(w.rows, nlist + w.p0, frames, c32, fG, lm, lmoff, lG, wts, M, N, dscale, Dout, Rnl,
                             status, 0, blockIdx.x * EX_TM, NLtab + (size_t)w.slot * Mnl, Mnl, qxy, Bseg, segof);
}

// Eq. (close_dist) for every landmark of the frames row_frame[0 .. *count) (frames of
// different close structures may share a tile: the rotation is per pair)
template <typename LT>
__global__ void __launch_bounds__(EX_THREADS, 4)
approx_rows_f32(const int* __restrict__ row_frame, const int* __restrict__ count, const float* __restrict__ frames,
                const float4* __restrict__ c32, const LT* __restrict__ lm, const float* __restrict__ lmoff,
                const float* __restrict__ wts, int M, int N, double dscale, float* __restrict__ Dout,
                const double4* __restrict__ qxy, const float* __restrict__ Bseg, const int* __restrict__ segof) {
  const int rows = *count;
  exact_tile_f32<LT, true>(rows, row_frame, frames, c32, nullptr, lm, lmoff, nullptr, wts, M, N, dscale, Dout, nullptr,
                           nullptr, blockIdx.y * EX_TF, blockIdx.x * EX_TM, nullptr, 0, qxy, Bseg, segof);
}

// FP64 mode: one pass, FP64 correlation, FP64 eigenvalue and D = G_x + G_a - 2 lambda_max
// (FP64 sums carry ~1e-16 relative error, far below the cancellation's needs).  A pair whose
// top eigenvalue is (nearly) double (near_double_f64) gets D = -1 as a mark and is redone by
// exact_redo_f64 with the Jacobi iteration, which keeps the Jacobi code out of this tile's
// registers.
__global__ void __launch_bounds__(EX_THREADS, 3)
exact_pair_f64(int rows, const int* __restrict__ row_frame, const double* __restrict__ frames,
               const double4* __restrict__ c64, const double* __restrict__ fG, const double* __restrict__ lm,
               const double* __restrict__ lG, const double* __restrict__ wts, int M, int N, double dscale,
               double* __restrict__ Dout, double* __restrict__ Rout, unsigned* __restrict__ status, int cap) {
  const float* lmoff = nullptr;  // FP64 storage has no block offsets
  constexpr int TF = EX_TF, TM = EX_TM, KC = 16;
  constexpr int PF = TF + 2, PM = TM + 2;
  __shared__ __align__(16) double Xs[KC * 3][PF];
  __shared__ __align__(16) double As[KC * 3][PM];
  __shared__ int s_frame[TF];
  __shared__ double s_c[TF][3];

  const int row0 = blockIdx.y * TF;
  if (row0 >= rows) return;
  const int i0 = blockIdx.x * TM;
  const int tid = threadIdx.x;
  const int tx = tid & 15;
  const int ty = tid >> 4;
  load_tile_frames<double, double>(rows, row_frame, row0, nullptr, c64, s_frame, s_c);
  __syncthreads();
  double h[2][2][9];
#pragma unroll
  for (int u = 0; u < 2; ++u)
#pragma unroll
    for (int v = 0; v < 2; ++v)
#pragma unroll
      for (int e = 0; e < 9; ++e) h[u][v][e] = 0.0;
  // a warp holds the rows row0 + 4 w .. row0 + 4 w + 3: warps wholly past the rows skip the
  // products (FP64 issue slots are shared by the SM's warps)
  const bool live = row0 + (tid >> 5) * 4 < rows;
  for (int j0 = 0; j0 < N; j0 += KC) {
    stage_exact<double, double, double, TF, TM, KC, PF, PM>(j0, N, M, i0, frames, lm, lmoff, wts, 1, s_frame, s_c, Xs, As);
    __syncthreads();
#pragma unroll 4
    for (int jj = 0; jj < (live ? KC : 0); ++jj) {
      double x[2][3], a[2][3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        load2<double>(&Xs[jj * 3 + c][ty * 2], x[0][c], x[1][c]);
        load2<double>(&As[jj * 3 + c][tx * 2], a[0][c], a[1][c]);
      }
#pragma unroll
      for (int u = 0; u < 2; ++u)
#pragma unroll
        for (int v = 0; v < 2; ++v)
#pragma unroll
          for (int b = 0; b < 3; ++b)
#pragma unroll
            for (int c = 0; c < 3; ++c) h[u][v][3 * b + c] = fma(a[v][b], x[u][c], h[u][v][3 * b + c]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 2; ++u)
#pragma unroll
    for (int v = 0; v < 2; ++v) {
      const int r = row0 + ty * 2 + u;
      const int f = s_frame[ty * 2 + u];
      const int i = i0 + tx * 2 + v;
      if (f < 0 || i >= M) continue;
      const double Gx = fG[f], Ga = lG[i];
      bool ok = true;
      double dp = 0.0;
      const double ub = 0.5 * (Gx + Ga);
      const double lam = lambda_max_newton(h[u][v], ub, &ok, &dp, cap);
      if (near_double_f64(dp, ub)) {
        Dout[(size_t)f * M + i] = -1.0;  // redone by exact_redo_f64
        continue;
      }
      double D = (Gx + Ga - 2.0 * lam) * dscale;
      if (D < 0.0) D = 0.0;
      Dout[(size_t)f * M + i] = D;
      if (Rout) {
        double K[16], q[4], Rm[9];
        quat_matrix(h[u][v], K);
        adj_eigvec_f64(K, lam, q);
        quat_to_rot(q, Rm);
        double* dst = Rout + ((size_t)r * M + i) * 9;
#pragma unroll
        for (int e = 0; e < 9; ++e) dst[e] = Rm[e];
      }
      if (!ok) atomicOr(status, STATUS_NOCONV);
    }
}

// The pairs exact_pair_f64 marked with D = -1 (a (nearly) double top eigenvalue): the
// correlation is summed again, one warp per pair in FP64, and the top eigenpair comes from
// the Jacobi iteration.  Each warp scans 32 consecutive (row, landmark) entries at a time;
// marked pairs are rare, so the scan of rows x M values is the usual cost.
constexpr int REDO_THREADS = 256;
__global__ void __launch_bounds__(REDO_THREADS)
exact_redo_f64(int rows, const int* __restrict__ row_frame, const double* __restrict__ frames,
               const double4* __restrict__ c64, const double* __restrict__ fG, const double* __restrict__ lm,
               const double* __restrict__ lG, const double* __restrict__ wts, int M, int N, double dscale,
               double* __restrict__ Dout, double* __restrict__ Rout, unsigned* __restrict__ status) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const long long total = (long long)rows * M;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long base = warp * 32; base < total; base += nwarps * 32) {
    const long long e = base + lane;
    int r = 0, i = 0, f = -1;
    bool mark = false;
    if (e < total) {
      r = (int)(e / M);
      i = (int)(e - (long long)r * M);
      f = row_frame ? row_frame[r] : r;
      mark = f >= 0 && Dout[(size_t)f * M + i] < 0.0;
    }
    unsigned bal = __ballot_sync(full, mark);
    while (bal) {
      const int src = __ffs(bal) - 1;
      bal &= bal - 1;
      const int rr = __shfl_sync(full, r, src), ii = __shfl_sync(full, i, src), ff = __shfl_sync(full, f, src);
      const double* x = frames + (size_t)ff * N * 3;
      const double* a = lm + (size_t)ii * N * 3;
      const double4 c = c64[ff];
      double h[9];
#pragma unroll
      for (int k = 0; k < 9; ++k) h[k] = 0.0;
      for (int j = lane; j < N; j += 32) {
        const double wj = wts ? wts[j] : 1.0;
        const double xv[3] = {wj * (x[3 * j] - c.x), wj * (x[3 * j + 1] - c.y), wj * (x[3 * j + 2] - c.z)};
#pragma unroll
        for (int b = 0; b < 3; ++b)
#pragma unroll
          for (int cc = 0; cc < 3; ++cc) h[3 * b + cc] = fma(a[3 * j + b], xv[cc], h[3 * b + cc]);
      }
#pragma unroll
      for (int k = 0; k < 9; ++k) h[k] = warp_sum_double(h[k]);
      if (lane == 0) {
        Mat4d km;
        quat_matrix(h, km.v);
        const TopEig4d ev = jacobi_top_f64(km);
        double D = (fG[ff] + lG[ii] - 2.0 * ev.lam) * dscale;
        if (D < 0.0) D = 0.0;
        Dout[(size_t)ff * M + ii] = D;
        if (Rout) {
          double Rm[9];
          quat_to_rot(ev.q, Rm);
          double* dst = Rout + ((size_t)rr * M + ii) * 9;
#pragma unroll
          for (int k = 0; k < 9; ++k) dst[k] = Rm[k];
        }
        if (!ev.ok) atomicOr(status, STATUS_NOCONV);
      }
    }
  }
}

// ---------------------------------------------------------------------------------------
// Approximate pairs.  Tile: 64 frames x (8 RM) landmarks, 128 threads, each 4 frames x RM
// landmarks.  Atoms in chunks of 16, software-pipelined: raw coordinates of chunk c+1 are
// loaded into registers while chunk c is computed from one of two shared buffers, then
// rotated (frames by R_xy^T after centring, landmarks by R_{a_i y}) into the other buffer.
constexpr int AP_TF = 64, AP_THREADS = 128, AP_KC = 16;

template <typename FT, typename LT, typename ST, int RM>
__global__ void __launch_bounds__(AP_THREADS, 3)
approx_pair_kernel(const int* __restrict__ alist, const int* __restrict__ aseg,
                   const int* __restrict__ acount, const FT* __restrict__ frames,
                   const float4* __restrict__ c32, const double4* __restrict__ c64,
                   const double4* __restrict__ qxy, const LT* __restrict__ lm, const float* __restrict__ lmoff,
                   const ST* __restrict__ Bseg, const ST* __restrict__ wts, int M, int N,
                   double dscale, ST* __restrict__ Dout) {
  constexpr int TF = AP_TF, TM = 8 * RM, KC = sizeof(ST) == 8 ? AP_KC / 2 : AP_KC;
  constexpr int PF = TF + 4, PM = TM + 4;
  constexpr int NF = TF * KC / AP_THREADS;  // frame-atom items per thread per chunk
  constexpr int NL = (TM * KC + AP_THREADS - 1) / AP_THREADS;
  __shared__ __align__(16) ST Xs[2][KC * 3][PF];
  __shared__ __align__(16) ST Bs[2][KC * 3][PM];
  __shared__ ST s_R[TF][9];
  __shared__ ST s_B[TM][9];
  __shared__ ST s_c[TF][3];
  __shared__ ST s_sw[2][KC];
  __shared__ int s_frame[TF], s_seg[TF];

  const int count = *acount;
  const int row0 = blockIdx.y * TF;
  if (row0 >= count) return;
  const ST dsc = (ST)dscale;
  const int i0 = blockIdx.x * TM;
  const int tid = threadIdx.x;
  const int tx = tid & 7;   // landmarks i0 + RM tx + {0..RM-1}
  const int ty = tid >> 3;  // rows 4 ty + {0..3}

  if (tid < TF) {
    const int r = row0 + tid;
    int f = -1, sg = -1;
    if (r < count) {
      f = alist[r];
      sg = aseg[r];
    }
    s_frame[tid] = f;
    s_seg[tid] = sg;
    ST c[3] = {0, 0, 0};
    ST R[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
    if (f >= 0) {
      frame_centre<ST>(c32, c64, f, c);
      const double4 qq = qxy[f];
      if (sizeof(ST) == 8) {
        const double qd[4] = {qq.x, qq.y, qq.z, qq.w};
        double Rd[9];
        quat_to_rot(qd, Rd);
#pragma unroll
        for (int e = 0; e < 9; ++e) R[e] = (ST)Rd[e];
      } else {
        const float qf[4] = {(float)qq.x, (float)qq.y, (float)qq.z, (float)qq.w};
        float Rf[9];
        quat_to_rot(qf, Rf);
#pragma unroll
        for (int e = 0; e < 9; ++e) R[e] = (ST)Rf[e];
      }
    }
#pragma unroll
    for (int e = 0; e < 9; ++e) s_R[tid][e] = R[e];
    s_c[tid][0] = c[0];
    s_c[tid][1] = c[1];
    s_c[tid][2] = c[2];
  }
  __syncthreads();

  const int nchunk = (N + KC - 1) / KC;
  int k = 0;
  while (k < TF && s_frame[k] >= 0) {
    const int seg = s_seg[k];
    int kend = k;
    while (kend < TF && s_frame[kend] >= 0 && s_seg[kend] == seg) ++kend;
    for (int e = tid; e < TM * 9; e += AP_THREADS) {
      const int ll = e / 9, c = e - ll * 9;
      const int i = i0 + ll;
      s_B[ll][c] = (i < M) ? Bseg[((size_t)seg * M + i) * 9 + c] : (ST)0;
    }
    ST acc[4][RM], thi[4][RM], tlo[4][RM];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < RM; ++v) acc[u][v] = thi[u][v] = tlo[u][v] = 0;

    ST rf[NF][3], rl[NL][3], rsw = 1;
    auto load_chunk = [&](int c) {
      const int j0 = c * KC;
#pragma unroll
      for (int r = 0; r < NF; ++r) {
        const int e = tid + r * AP_THREADS;
        const int ff = e / KC, jj = e - ff * KC;
        const int j = j0 + jj;
        if (ff >= k && ff < kend && j < N) {
          const FT* src = frames + ((size_t)s_frame[ff] * N + j) * 3;
          rf[r][0] = (ST)src[0];
          rf[r][1] = (ST)src[1];
          rf[r][2] = (ST)src[2];
        } else {
          rf[r][0] = rf[r][1] = rf[r][2] = 0;
        }
      }
#pragma unroll
      for (int r = 0; r < NL; ++r) {
        const int e = tid + r * AP_THREADS;
        const int ll = e / KC, jj = e - ll * KC;
        const int j = j0 + jj, i = i0 + ll;
        if (e < TM * KC && i < M && j < N) {
          rl[r][0] = lm_coord<ST, LT>(lm, lmoff, N, i, j, 0);
          rl[r][1] = lm_coord<ST, LT>(lm, lmoff, N, i, j, 1);
          rl[r][2] = lm_coord<ST, LT>(lm, lmoff, N, i, j, 2);
        } else {
          rl[r][0] = rl[r][1] = rl[r][2] = 0;
        }
      }
      if (tid < KC) {
        const int j = j0 + tid;
        rsw = 1;
        if (wts) rsw = (j < N) ? (ST)sqrt(wts[j]) : (ST)0;
      }
    };
    auto store_chunk = [&](int c, int buf) {
      const int j0 = c * KC;
      if (tid < KC) s_sw[buf][tid] = rsw;
#pragma unroll
      for (int r = 0; r < NF; ++r) {
        const int e = tid + r * AP_THREADS;
        const int ff = e / KC, jj = e - ff * KC;
        ST o0 = 0, o1 = 0, o2 = 0;
        if (ff >= k && ff < kend && j0 + jj < N) {
          const ST v0 = rf[r][0] - s_c[ff][0];
          const ST v1 = rf[r][1] - s_c[ff][1];
          const ST v2 = rf[r][2] - s_c[ff][2];
          const ST* R = s_R[ff];
          ST sw = 1;
          if (wts) sw = (ST)sqrt(wts[j0 + jj]);
          o0 = (R[0] * v0 + R[3] * v1 + R[6] * v2) * sw;
          o1 = (R[1] * v0 + R[4] * v1 + R[7] * v2) * sw;
          o2 = (R[2] * v0 + R[5] * v1 + R[8] * v2) * sw;
        }
        Xs[buf][jj * 3 + 0][ff] = o0;
        Xs[buf][jj * 3 + 1][ff] = o1;
        Xs[buf][jj * 3 + 2][ff] = o2;
      }
#pragma unroll
      for (int r = 0; r < NL; ++r) {
        const int e = tid + r * AP_THREADS;
        if (e >= TM * KC) continue;
        const int ll = e / KC, jj = e - ll * KC;
        const ST* B = s_B[ll];
        ST sw = 1;
        if (wts && j0 + jj < N) sw = (ST)sqrt(wts[j0 + jj]);
        Bs[buf][jj * 3 + 0][ll] = (B[0] * rl[r][0] + B[1] * rl[r][1] + B[2] * rl[r][2]) * sw;
        Bs[buf][jj * 3 + 1][ll] = (B[3] * rl[r][0] + B[4] * rl[r][1] + B[5] * rl[r][2]) * sw;
        Bs[buf][jj * 3 + 2][ll] = (B[6] * rl[r][0] + B[7] * rl[r][1] + B[8] * rl[r][2]) * sw;
      }
    };
    __syncthreads();  // s_B ready
    load_chunk(0);
    store_chunk(0, 0);
    __syncthreads();
    for (int c = 0; c < nchunk; ++c) {
      const int buf = c & 1;
      const bool more = c + 1 < nchunk;
      if (more) load_chunk(c + 1);
#pragma unroll 4
      for (int jj = 0; jj < KC; ++jj) {
        ST x[3][4], b[3][RM];
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) {
          load4<ST>(&Xs[buf][jj * 3 + cc][ty * 4], x[cc]);
#pragma unroll
          for (int v = 0; v < RM; ++v) b[cc][v] = Bs[buf][jj * 3 + cc][tx * RM + v];
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < RM; ++v) {
            const ST d0 = x[0][u] - b[0][v];
            const ST d1 = x[1][u] - b[1][v];
            const ST d2 = x[2][u] - b[2][v];
            ST t = acc[u][v];
            t = fma(d0, d0, t);
            t = fma(d1, d1, t);
            t = fma(d2, d2, t);
            acc[u][v] = t;
          }
      }
      // every 2 chunks: chunk partials into the error-free (hi, lo) totals
      if ((c & 1) || !more) {
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < RM; ++v) {
            if (sizeof(ST) == 4) {
              float h = (float)thi[u][v], l = (float)tlo[u][v];
              two_sum_acc(h, l, (float)acc[u][v]);
              thi[u][v] = (ST)h;
              tlo[u][v] = (ST)l;
            } else {
              thi[u][v] += acc[u][v];
            }
            acc[u][v] = 0;
          }
      }
      if (more) store_chunk(c + 1, buf ^ 1);
      __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int ff = ty * 4 + u;
      if (ff < k || ff >= kend) continue;
      const int f = s_frame[ff];
#pragma unroll
      for (int v = 0; v < RM; ++v) {
        const int i = i0 + tx * RM + v;
        if (i < M) Dout[(size_t)f * M + i] = (thi[u][v] + tlo[u][v]) * dsc;
      }
    }
    k = kend;
    __syncthreads();
  }
}

// FP32 modes.  Tile: 128 frames x (8 RM) landmarks, 128 threads, each 8 frames x RM
// landmarks (40 pairs for RM = 5): per atom 8 x 3 frame values (6 LDS.128) and RM x 3
// landmark values feed 6 RM x 8 FP32 operations.  Atoms come in chunks of 8; the chunk
// sums of each pair go into an FP32 total every 32 atoms (relative rounding ~u sqrt(N/32),
// 7.5e-7 at N = 5000).  Frames are centred and rotated by R_xy^T while staged, landmarks
// rotated by R_{a_i y}.
constexpr int AQ_TF = 128, AQ_THREADS = 128, AQ_KC = 8;

template <typename LT, int RM>
__global__ void __launch_bounds__(AQ_THREADS, 3)
approx_pair_f32t(const int* __restrict__ alist, const int* __restrict__ aseg, const int* __restrict__ acount,
                 const float* __restrict__ frames, const float4* __restrict__ c32, const double4* __restrict__ qxy,
                 const LT* __restrict__ lm, const float* __restrict__ lmoff, const float* __restrict__ Bseg,
                 const float* __restrict__ wts, int M, int N, float dscale, float* __restrict__ Dout) {
  constexpr int TF = AQ_TF, TM = 8 * RM, KC = AQ_KC;
  __shared__ __align__(16) float Xs[KC * 3][TF + 4];
  __shared__ __align__(16) float Bs[KC * 3][TM + 4];
  __shared__ float s_R[TF][9];
  __shared__ float s_B[TM][9];
  __shared__ float s_c[TF][3];
  __shared__ int s_frame[TF], s_seg[TF];

  const int count = *acount;
  const int row0 = blockIdx.y * TF;
  if (row0 >= count) return;
  const int i0 = blockIdx.x * TM;
  const int tid = threadIdx.x;
  const int tx = tid & 7;   // landmarks i0 + RM tx + {0..RM-1}
  const int ty = tid >> 3;  // rows 8 ty + {0..7}

  if (tid < TF) {
    const int r = row0 + tid;
    int f = -1, sg = -1;
    if (r < count) {
      f = alist[r];
      sg = aseg[r];
    }
    s_frame[tid] = f;
    s_seg[tid] = sg;
    float R[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
    float4 c = make_float4(0.f, 0.f, 0.f, 0.f);
    if (f >= 0) {
      c = c32[f];
      const double4 qq = qxy[f];
      const float qf[4] = {(float)qq.x, (float)qq.y, (float)qq.z, (float)qq.w};
      quat_to_rot(qf, R);
    }
#pragma unroll
    for (int e = 0; e < 9; ++e) s_R[tid][e] = R[e];
    s_c[tid][0] = c.x;
    s_c[tid][1] = c.y;
    s_c[tid][2] = c.z;
  }
  __syncthreads();

  int k = 0;
  while (k < TF && s_frame[k] >= 0) {
    const int seg = s_seg[k];
    int kend = k;
    while (kend < TF && s_frame[kend] >= 0 && s_seg[kend] == seg) ++kend;
    for (int e = tid; e < TM * 9; e += AQ_THREADS) {
      const int ll = e / 9, c = e - ll * 9;
      const int i = i0 + ll;
      s_B[ll][c] = (i < M) ? Bseg[((size_t)seg * M + i) * 9 + c] : 0.0f;
    }
    float acc[8][RM], tot[8][RM];
#pragma unroll
    for (int u = 0; u < 8; ++u)
#pragma unroll
      for (int v = 0; v < RM; ++v) acc[u][v] = tot[u][v] = 0.0f;
    __syncthreads();
    for (int j0 = 0, c = 0; j0 < N; j0 += KC, ++c) {
      for (int e = tid; e < TF * KC; e += AQ_THREADS) {
        const int ff = e / KC, jj = e - ff * KC;
        const int j = j0 + jj;
        float o0 = 0.0f, o1 = 0.0f, o2 = 0.0f;
        if (ff >= k && ff < kend && j < N) {
          const float* src = frames + ((size_t)s_frame[ff] * N + j) * 3;
          const float v0 = src[0] - s_c[ff][0], v1 = src[1] - s_c[ff][1], v2 = src[2] - s_c[ff][2];
          const float* R = s_R[ff];
          const float sw = wts ? sqrtf(wts[j]) : 1.0f;
          o0 = (R[0] * v0 + R[3] * v1 + R[6] * v2) * sw;
          o1 = (R[1] * v0 + R[4] * v1 + R[7] * v2) * sw;
          o2 = (R[2] * v0 + R[5] * v1 + R[8] * v2) * sw;
        }
        Xs[jj * 3 + 0][ff] = o0;
        Xs[jj * 3 + 1][ff] = o1;
        Xs[jj * 3 + 2][ff] = o2;
      }
      for (int e = tid; e < TM * KC; e += AQ_THREADS) {
        const int ll = e / KC, jj = e - ll * KC;
        const int j = j0 + jj, i = i0 + ll;
        float b0 = 0.0f, b1 = 0.0f, b2 = 0.0f;
        if (i < M && j < N) {
          const float a0 = lm_coord<float, LT>(lm, lmoff, N, i, j, 0);
          const float a1 = lm_coord<float, LT>(lm, lmoff, N, i, j, 1);
          const float a2 = lm_coord<float, LT>(lm, lmoff, N, i, j, 2);
          const float* B = s_B[ll];
          const float sw = wts ? sqrtf(wts[j]) : 1.0f;
          b0 = (B[0] * a0 + B[1] * a1 + B[2] * a2) * sw;
          b1 = (B[3] * a0 + B[4] * a1 + B[5] * a2) * sw;
          b2 = (B[6] * a0 + B[7] * a1 + B[8] * a2) * sw;
        }
        Bs[jj * 3 + 0][ll] = b0;
        Bs[jj * 3 + 1][ll] = b1;
        Bs[jj * 3 + 2][ll] = b2;
      }
      __syncthreads();
#pragma unroll 2
      for (int jj = 0; jj < KC; ++jj) {
        float x[3][8], b[3][RM];
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) {
          const float4 xa = *reinterpret_cast<const float4*>(&Xs[jj * 3 + cc][ty * 8]);
          const float4 xb = *reinterpret_cast<const float4*>(&Xs[jj * 3 + cc][ty * 8 + 4]);
          x[cc][0] = xa.x; x[cc][1] = xa.y; x[cc][2] = xa.z; x[cc][3] = xa.w;
          x[cc][4] = xb.x; x[cc][5] = xb.y; x[cc][6] = xb.z; x[cc][7] = xb.w;
#pragma unroll
          for (int v = 0; v < RM; ++v) b[cc][v] = Bs[jj * 3 + cc][tx * RM + v];
        }
#pragma unroll
        for (int u = 0; u < 8; ++u)
#pragma unroll
          for (int v = 0; v < RM; ++v) {
            const float d0 = x[0][u] - b[0][v];
            const float d1 = x[1][u] - b[1][v];
            const float d2 = x[2][u] - b[2][v];
            acc[u][v] = fmaf(d0, d0, fmaf(d1, d1, fmaf(d2, d2, acc[u][v])));
          }
      }
      if ((c & 3) == 3 || j0 + KC >= N) {
#pragma unroll
        for (int u = 0; u < 8; ++u)
#pragma unroll
          for (int v = 0; v < RM; ++v) {
            tot[u][v] += acc[u][v];
            acc[u][v] = 0.0f;
          }
      }
      __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int ff = ty * 8 + u;
      if (ff < k || ff >= kend) continue;
      const int f = s_frame[ff];
#pragma unroll
      for (int v = 0; v < RM; ++v) {
        const int i = i0 + tx * RM + v;
        if (i < M) Dout[(size_t)f * M + i] = tot[u][v] * dscale;
      }
    }
    k = kend;
    __syncthreads();
  }
}

}  // namespace

// ---------------------------------------------------------------------------------------
int exact_split_count(int rows, int M, int N) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const long long tiles = (long long)((M + EX_TM - 1) / EX_TM) * ((rows + EX_TF - 1) / EX_TF);
  if (tiles >= 2LL * sms) return 1;  // the tiles alone fill two waves
  const int chunks = (N + 31) / 32;
  int k = 1;
  while (k < 16 && tiles * k < 4LL * sms && chunks / (2 * k) >= 4) k *= 2;  // at least 4 chunks per slice
  return k;
}

size_t exact_split_bytes(int rows, int M, int nsplit) {
  return sizeof(float) * (size_t)nsplit * rows * M * (9 + 2);
}

void launch_exact_pairs(Prec p, int rows, const int* row_frame, const int* rows_dev, const void* frames,
                        const LandmarkDev& L, FrameInfo fi, void* D, void* Rout, unsigned* status,
                        cudaStream_t st, const ScratchView* scr) {
  (void)rows_dev;
  if (rows <= 0) return;
  if (p != P_F64 && rows <= STREAM_FRAMES && stream_fits(p, L.N)) {  // a few frames: one CTA per landmark
    launch_exact_stream(p, rows, row_frame, frames, L, fi, D, Rout, status, st);
    return;
  }
  if (p != P_F64 && scr && L.exact_tile == 0) {
    // few tiles: the atoms split over slices so that the grid fills the GPU
    const int nsplit = exact_split_count(rows, L.M, L.N);
    if (nsplit > 1 && scr->bytes >= exact_split_bytes(rows, L.M, nsplit)) {
      float* Hp = (float*)scr->ptr;
      float* Dp = Hp + (size_t)nsplit * rows * L.M * 9;
      const dim3 g((L.M + EX_TM - 1) / EX_TM, (rows + EX_TF - 1) / EX_TF, nsplit);
      const bool h = p == P_F16;
      if (h)
        exact_split_pass1<__half><<<g, EX_THREADS, 0, st>>>(rows, row_frame, (const float*)frames, fi.c32,
                                                            (const __half*)L.coords, L.off, L.w, L.M, L.N, nsplit, Hp);
      else
        exact_split_pass1<float><<<g, EX_THREADS, 0, st>>>(rows, row_frame, (const float*)frames, fi.c32,
                                                           (const float*)L.coords, L.off, L.w, L.M, L.N, nsplit, Hp);
      if (h)
        exact_split_pass2<__half><<<g, EX_THREADS, 0, st>>>(rows, row_frame, (const float*)frames, fi.c32, fi.G,
                                                            (const __half*)L.coords, L.off, L.G, L.w, L.M, L.N, nsplit,
                                                            Hp, Dp, (float*)Rout, status, L.newton_cap);
      else
        exact_split_pass2<float><<<g, EX_THREADS, 0, st>>>(rows, row_frame, (const float*)frames, fi.c32, fi.G,
                                                           (const float*)L.coords, L.off, L.G, L.w, L.M, L.N, nsplit,
                                                           Hp, Dp, (float*)Rout, status, L.newton_cap);
      const size_t n = (size_t)rows * L.M;
      exact_split_finish<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(rows, row_frame, L.M, nsplit, (float)L.dscale,
                                                                     Dp, (float*)D);
      note_launch(3);
      return;
    }
  }
  const int shape = L.exact_tile > 0 && L.exact_tile <= EXACT_SHAPES ? L.exact_tile - 1 : 0;
  if (p != P_F64 && shape > 0) {  // a chosen shape (FP32 / FP16 storage)
    const ExactShape sh = kExactShape[shape];
    const dim3 g((L.M + sh.tm - 1) / sh.tm, (rows + sh.tf - 1) / sh.tf);
    const bool h = p == P_F16;
#define PCV_EXACT_SHAPED(TF, TM)                                                                                   \
  if (h)                                                                                                           \
    exact_pair_f32<__half, TF, TM><<<g, EX_THREADS, 0, st>>>(rows, row_frame, (const float*)frames, fi.c32, fi.G,  \
                                                             (const __half*)L.coords, L.off, L.G, L.w, L.M, L.N,   \
                                                             L.dscale, (float*)D, (float*)Rout, status,            \
                                                             L.newton_cap);                                         \
  else                                                                                                             \
    exact_pair_f32<float, TF, TM><<<g, EX_THREADS, 0, st>>>(rows, row_frame, (const float*)frames, fi.c32, fi.G,   \
                                                            (const float*)L.coords, L.off, L.G, L.w, L.M, L.N,     \
                                                            L.dscale, (float*)D, (float*)Rout, status, L.newton_cap);
    if (shape == 1) {
      PCV_EXACT_SHAPED(32, 16)
    } else {
      PCV_EXACT_SHAPED(8, 64)
    }
#undef PCV_EXACT_SHAPED
    note_launch();
    return;
  }
  dim3 grid((L.M + EX_TM - 1) / EX_TM, (rows + EX_TF - 1) / EX_TF);
  switch (p) {
    case P_F64:
      exact_pair_f64<<<grid, EX_THREADS, 0, st>>>(rows, row_frame, (const double*)frames, fi.c64, fi.G,
                                                  (const double*)L.coords, L.G, L.w64, L.M, L.N, L.dscale,
                                                  (double*)D, (double*)Rout, status, L.newton_cap); note_launch();
      {
        const long long warps = ((long long)rows * L.M + 31) / 32;
        const int blocks = (int)std::min<long long>((warps + REDO_THREADS / 32 - 1) / (REDO_THREADS / 32), 152 * 8);
        exact_redo_f64<<<blocks, REDO_THREADS, 0, st>>>(rows, row_frame, (const double*)frames, fi.c64, fi.G,
                                                         (const double*)L.coords, L.G, L.w64, L.M, L.N, L.dscale,
                                                         (double*)D, (double*)Rout, status); note_launch();
      }
      break;
    case P_F32:
      exact_pair_f32<float><<<grid, EX_THREADS, 0, st>>>(rows, row_frame, (const float*)frames, fi.c32, fi.G,
                                                         (const float*)L.coords, L.off, L.G, L.w, L.M, L.N,
                                                         L.dscale,
                                                         (float*)D, (float*)Rout, status, L.newton_cap);
      note_launch();
      break;
    case P_F16:
      exact_pair_f32<__half><<<grid, EX_THREADS, 0, st>>>(rows, row_frame, (const float*)frames, fi.c32, fi.G,
                                                          (const __half*)L.coords, L.off, L.G, L.w, L.M, L.N,
                                                          L.dscale,
                                                          (float*)D, (float*)Rout, status, L.newton_cap);
      note_launch();
      break;
  }
}

template <int TF, int TM>
static void exact_group_launch(bool fp16, const GroupInst* I, const GroupTile* tiles, int ntiles, int blocks,
                               cudaStream_t st) {
  if (fp16)
    exact_group_f32<__half, TF, TM><<<blocks, EX_THREADS, 0, st>>>(I, tiles, ntiles);
  else
    exact_group_f32<float, TF, TM><<<blocks, EX_THREADS, 0, st>>>(I, tiles, ntiles);
}

void launch_exact_group(bool fp16, int shape, const GroupInst* I, const GroupTile* tiles, int ntiles, int blocks,
                        cudaStream_t st) {
  if (ntiles <= 0) return;
  static_assert(kExactShape[0].tf == EX_TF && kExactShape[0].tm == EX_TM, "shape 0 is the default tile");
  static_assert(kExactShape[1].tf == 32 && kExactShape[1].tm == 16 && kExactShape[2].tf == 8 &&
                    kExactShape[2].tm == 64,
                "the shapes instantiated below");
  switch (shape) {
    case 1: exact_group_launch<32, 16>(fp16, I, tiles, ntiles, blocks, st); break;
    case 2: exact_group_launch<8, 64>(fp16, I, tiles, ntiles, blocks, st); break;
    default: exact_group_launch<16, 32>(fp16, I, tiles, ntiles, blocks, st); break;
  }
  note_launch();
}

// landmark tile of 32 or 40 (whichever wastes fewer rows of the last tile)
static int approx_rm(int M) {
  const int w4 = (M + 31) / 32 * 32 - M, w5 = (M + 39) / 40 * 40 - M;
  return w5 < w4 ? 5 : 4;
}

template <int RM>
static void approx_launch(Prec p, int max_rows, const int* approx_list, const int* approx_seg, const int* count,
                          const void* frames, const LandmarkDev& L, FrameInfo fi, const double4* qxy,
                          const void* Bseg, void* D, cudaStream_t st) {
  dim3 grid((L.M + 8 * RM - 1) / (8 * RM), (max_rows + AP_TF - 1) / AP_TF);
  if (p == P_F32 || p == P_F16) {
    dim3 gq((L.M + 8 * RM - 1) / (8 * RM), (max_rows + AQ_TF - 1) / AQ_TF);
    if (p == P_F32)
      approx_pair_f32t<float, RM><<<gq, AQ_THREADS, 0, st>>>(approx_list, approx_seg, count, (const float*)frames,
                                                             fi.c32, qxy, (const float*)L.coords, L.off,
                                                             (const float*)Bseg,
                                                             L.w, L.M, L.N, (float)L.dscale, (float*)D);
    else
      approx_pair_f32t<__half, RM><<<gq, AQ_THREADS, 0, st>>>(approx_list, approx_seg, count, (const float*)frames,
                                                              fi.c32, qxy, (const __half*)L.coords, L.off,
                                                              (const float*)Bseg,
                                                              L.w, L.M, L.N, (float)L.dscale, (float*)D);
    note_launch();
    return;
  }
  switch (p) {
    case P_F64:
      approx_pair_kernel<double, double, double, RM><<<grid, AP_THREADS, 0, st>>>(
          approx_list, approx_seg, count, (const double*)frames, fi.c32, fi.c64, qxy, (const double*)L.coords,
          nullptr, (const double*)Bseg, L.w64, L.M, L.N, L.dscale, (double*)D);
      break;
    case P_F32:
      approx_pair_kernel<float, float, float, RM><<<grid, AP_THREADS, 0, st>>>(
          approx_list, approx_seg, count, (const float*)frames, fi.c32, fi.c64, qxy, (const float*)L.coords,
          L.off, (const float*)Bseg, L.w, L.M, L.N, L.dscale, (float*)D);
      break;
    case P_F16:
      approx_pair_kernel<float, __half, float, RM><<<grid, AP_THREADS, 0, st>>>(
          approx_list, approx_seg, count, (const float*)frames, fi.c32, fi.c64, qxy, (const __half*)L.coords,
          L.off, (const float*)Bseg, L.w, L.M, L.N, L.dscale, (float*)D);
      break;
  }
  note_launch();
}

void launch_nl_exact_tiles(Prec p, int max_tiles, const NlLists& nl, const NlTile* tiles, const int* NLtab, int Mnl,
                           const void* frames, const LandmarkDev& L, FrameInfo fi, void* D, void* Rnl,
                           unsigned* status, cudaStream_t st) {
  if (max_tiles <= 0 || p == P_F64) return;
  dim3 grid((Mnl + EX_TM - 1) / EX_TM, max_tiles);
  if (p == P_F32)
    nl_list_f32<float, false><<<grid, EX_THREADS, 0, st>>>(
        tiles, nl.counts + 3, nl.nlist, NLtab, Mnl, (const float*)frames, fi.c32, fi.G, (const float*)L.coords, L.off,
        L.G, L.w, L.M, L.N, L.dscale, (float*)D, (float*)Rnl, status, nullptr, nullptr, nullptr);
  else
    nl_list_f32<__half, false><<<grid, EX_THREADS, 0, st>>>(
        tiles, nl.counts + 3, nl.nlist, NLtab, Mnl, (const float*)frames, fi.c32, fi.G, (const __half*)L.coords,
        L.off, L.G, L.w, L.M, L.N, L.dscale, (float*)D, (float*)Rnl, status, nullptr, nullptr, nullptr);
  note_launch();
}

void launch_nl_approx_tiles(Prec p, int max_uapp, int max_tiles, const NlLists& nl, const NlTile* tiles,
                            const int* NLtab, int Mnl, const void* frames, const LandmarkDev& L, FrameInfo fi,
                            const double4* qxy, const void* Bseg, const int* segof, void* D, cudaStream_t st) {
  if (p == P_F64) return;
  if (max_uapp > 0) {  // update frames that are not reassignments: every landmark
    dim3 grid((L.M + EX_TM - 1) / EX_TM, (max_uapp + EX_TF - 1) / EX_TF);
    if (p == P_F32)
      approx_rows_f32<float><<<grid, EX_THREADS, 0, st>>>(nl.uapp_list, nl.counts + 1, (const float*)frames, fi.c32,
                                                          (const float*)L.coords, L.off, L.w, L.M, L.N, L.dscale,
                                                          (float*)D, qxy, (const float*)Bseg, segof);
    else
      approx_rows_f32<__half><<<grid, EX_THREADS, 0, st>>>(nl.uapp_list, nl.counts + 1, (const float*)frames, fi.c32,
                                                           (const __half*)L.coords, L.off, L.w, L.M, L.N, L.dscale,
                                                           (float*)D, qxy, (const float*)Bseg, segof);
    note_launch();
  }
  if (max_tiles > 0) {  // frames between updates: their lists
    dim3 grid((Mnl + EX_TM - 1) / EX_TM, max_tiles);
    if (p == P_F32)
      nl_list_f32<float, true><<<grid, EX_THREADS, 0, st>>>(
          tiles, nl.counts + 3, nl.nlist, NLtab, Mnl, (const float*)frames, fi.c32, nullptr, (const float*)L.coords,
          L.off, nullptr, L.w, L.M, L.N, L.dscale, (float*)D, nullptr, nullptr, qxy, (const float*)Bseg, segof);
    else
      nl_list_f32<__half, true><<<grid, EX_THREADS, 0, st>>>(
          tiles, nl.counts + 3, nl.nlist, NLtab, Mnl, (const float*)frames, fi.c32, nullptr, (const __half*)L.coords,
          L.off, nullptr, L.w, L.M, L.N, L.dscale, (float*)D, nullptr, nullptr, qxy, (const float*)Bseg, segof);
    note_launch();
  }
}

void launch_approx_pairs(Prec p, int max_rows, const int* approx_list, const int* approx_seg, const int* count,
                         const void* frames, const LandmarkDev& L, FrameInfo fi, const double4* qxy, const void* Bseg,
                         void* D, cudaStream_t st) {
  if (max_rows <= 0) return;
  if (p != P_F64 && max_rows <= STREAM_FRAMES && stream_fits(p, L.N)) {  // a few frames: one CTA per landmark
    launch_approx_stream(p, max_rows, approx_list, approx_seg, count, frames, L, fi, qxy, Bseg, D, st);
    return;
  }
  if (approx_rm(L.M) == 5)
    approx_launch<5>(p, max_rows, approx_list, approx_seg, count, frames, L, fi, qxy, Bseg, D, st);
  else
    approx_launch<4>(p, max_rows, approx_list, approx_seg, count, frames, L, fi, qxy, Bseg, D, st);
}

}  // namespace pcv

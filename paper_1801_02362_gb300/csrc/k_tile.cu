// k_tile.cu -- close-structure kernels on materialised, rotated operands (FP32 modes,
// uniform weights).
//
// With the close structure every approximate frame x enters only as x' = R_xy^T (x - c),
// and every landmark of segment s (frames sharing the close structure y(s)) only as
// b = R_{a_i y} a (Eq. close_dist).  Both are written once, as deviations from the centred
// close structure y' of their segment: dx = x' - y' and d_i = b_i - y', with their squared
// norms.  Then
//   approx_pair_tile:   D~_fi = (|dx_f|^2 + |d_i|^2 - 2 dx_f . d_i) / N,
//   adjoint_beta_tile:  beta_f = Gamma_f y' + sum_i gamma_fi d_i  (gamma^s and gamma^z).
// The identity |x' - b|^2 = |dx - d|^2 is exact; the cancelling form costs one FMA per
// coordinate instead of a subtraction and an FMA, and stays accurate in FP32 because the
// deviations are small: frames are within the close threshold of y, and the landmarks that
// matter (large softmax weight) are near the frame, hence near y.
// Rows are padded to N16 (a multiple of 16 atoms, zeros), so each chunk is a run of
// 16-byte pieces moved global -> shared with cp.async in a 3-stage pipeline: copies of chunk
// c+2 are in flight while chunk c is used, and no register holds staged data.
//
// The approximate-MSD loop uses packed FP32 pairs (f32x2) over adjacent coordinates of dx
// and d: each instruction performs two IEEE FP32 operations, which frees issue slots for the
// shared-memory loads (the packed operations run on one of the two FP32 sub-pipes, so the
// FP32 rate itself is unchanged).
#include <cuda_fp16.h>

#include <algorithm>

#include "pcv_device.cuh"
#include "pcv_internal.h"

namespace pcv {
namespace {

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, bool pred) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  const int n = pred ? 16 : 0;  // 0 source bytes: the 16 shared bytes are zero-filled
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(s), "l"(gmem), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int K>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(K) : "memory");
}

// ---------------------------------------------------------------------------------------
// block sum of one value per thread (blockDim.x a multiple of 32, at most 1024)
__device__ __forceinline__ float block_sum(float v, float* red) {
  v = warp_sum_float(v);
  const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[w] = v;
  __syncthreads();
  float t = 0.0f;
  for (int k = 0; k < nw; ++k) t += red[k];
  return t;
}

// y' (centred close structure) of segment slot s: the prior structure for segment 0, else
// the frame refresh_list[seg - 1]
__device__ __forceinline__ const float* seg_structure(int seg, const float* frames, int N3, const float4* c32,
                                                      const int* refresh_list, const float* prior, float4 prior_c,
                                                      float4& c) {
  if (seg == 0) {
    c = prior_c;
    return prior;
  }
  const int f = refresh_list[seg - 1];
  c = c32[f];
  return frames + (size_t)f * N3;
}

// d_{s,i} = R_{a_i y(s)} a_i - y'(s) for segments s in [s0, s0 + gridDim.y): rows of N16
// atoms in Bm, |d_{s,i}|^2 in Nb[s * M + i]; block i == 0 also writes y'(s) to Yc[s].
template <typename LT>
__global__ void materialize_landmarks_kernel(int s0, int M, int N, int N16, const LT* __restrict__ lm,
                                             const float* __restrict__ lmoff, const float* __restrict__ Bseg, const float* __restrict__ frames,
                                             const float4* __restrict__ c32, const int* __restrict__ refresh_list,
                                             const float* __restrict__ prior, float4 prior_c, float* __restrict__ Bm,
                                             float* __restrict__ Nb, float* __restrict__ Yc) {
  __shared__ float red[32];
  const int i = blockIdx.x, slot = blockIdx.y, seg = s0 + slot;
  float4 c;
  const float* y = seg_structure(seg, frames, 3 * N, c32, refresh_list, prior, prior_c, c);
  const float* B = Bseg + ((size_t)seg * M + i) * 9;
  float R[9];
#pragma unroll
  for (int e = 0; e < 9; ++e) R[e] = B[e];
  const LT* a = lm + (size_t)i * N * 3;
  const size_t row = (size_t)slot * M + i;
  float* out = Bm + row * N16 * 3;
  float nrm = 0.0f;
  for (int j = threadIdx.x; j < N16; j += blockDim.x) {
    float o0 = 0.0f, o1 = 0.0f, o2 = 0.0f;
    if (j < N) {
      const float a0 = lm_coord<float, LT>(lm, lmoff, N, i, j, 0);
      const float a1 = lm_coord<float, LT>(lm, lmoff, N, i, j, 1);
      const float a2 = lm_coord<float, LT>(lm, lmoff, N, i, j, 2);
      const float y0 = y[3 * j] - c.x, y1 = y[3 * j + 1] - c.y, y2 = y[3 * j + 2] - c.z;
      o0 = (R[0] * a0 + R[1] * a1 + R[2] * a2) - y0;
      o1 = (R[3] * a0 + R[4] * a1 + R[5] * a2) - y1;
      o2 = (R[6] * a0 + R[7] * a1 + R[8] * a2) - y2;
      if (i == 0) {
        Yc[(size_t)slot * 3 * N + 3 * j] = y0;
        Yc[(size_t)slot * 3 * N + 3 * j + 1] = y1;
        Yc[(size_t)slot * 3 * N + 3 * j + 2] = y2;
      }
    }
    out[3 * j] = o0;
    out[3 * j + 1] = o1;
    out[3 * j + 2] = o2;
    nrm = fmaf(o0, o0, fmaf(o1, o1, fmaf(o2, o2, nrm)));
  }
  nrm = block_sum(nrm, red);
  if (threadIdx.x == 0) Nb[row] = nrm;
}

// dx_k = R_xy^T (x_f - c_f) - y'(seg), f = alist[k], one row of N16 atoms per approximate
// frame, and |dx_k|^2 in Nx[k].  Runs after materialize_landmarks (y' from Yc).  One warp
// per frame; with VEC (N % 4 == 0 and 16-byte aligned frame rows) a lane moves 4 atoms as
// three 16-byte loads of x and of y' and three 16-byte stores.
// REFINE: the accurate R_xy is formed here first (compensated FP32 correlation of x with its
// close structure, FP32 eigen-solve; the arithmetic of the separate refinement kernel) and
// its quaternion stored in qxy, so the frame is read once for both.
struct RefineArgs {
  const int* ref;           // close-structure frame of each frame (-1: the stored prior)
  const float* prior;       // prior structure coordinates
  float4 prior_c;           // and its centre
  double prior_G;           // and its G
  const double* fG;         // G of every frame
  const float* wts;         // distance weights (null: uniform)
};
template <bool VEC, bool REFINE>
__global__ void materialize_frames_kernel(int napp_max, const int* __restrict__ acount, const int* __restrict__ alist,
                                          const int* __restrict__ aseg, int seg_base, int N, int N16,
                                          const float* __restrict__ frames, const float4* __restrict__ c32,
                                          double4* __restrict__ qxy, const float* __restrict__ Yc,
                                          float* __restrict__ Xr, float* __restrict__ Nx, RefineArgs ra) {
  const int k = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (k >= napp_max || k >= *acount) return;  // uniform over the warp
  const int f = alist[k];
  const float4 c = c32[f];
  const float* x = frames + (size_t)f * N * 3;
  float qf[4];
  if (REFINE) {
    const int ref = ra.ref[f];
    const float* y = ref >= 0 ? frames + (size_t)ref * N * 3 : ra.prior;
    const float4 cy = ref >= 0 ? c32[ref] : ra.prior_c;
    float H[9];
    warp_corr_pair_f32(N, x, c, y, cy, ra.wts, H);  // every lane holds H
    const float Gx = (float)ra.fG[f], Gy = (float)(ref >= 0 ? ra.fG[ref] : ra.prior_G);
    top_quat_f32(H, 0.5f * (Gx + Gy) * 1.00001f + 1e-30f, qf);
    if (lane == 0) qxy[f] = make_double4(qf[0], qf[1], qf[2], qf[3]);
  } else {
    const double4 qq = qxy[f];
    qf[0] = (float)qq.x;
    qf[1] = (float)qq.y;
    qf[2] = (float)qq.z;
    qf[3] = (float)qq.w;
  }
  float R[9];
  quat_to_rot(qf, R);
  const float* yc = Yc + (size_t)(aseg[k] - seg_base) * 3 * N;
  float* out = Xr + (size_t)k * N16 * 3;
  float nrm = 0.0f;
  auto atom = [&](float x0, float x1, float x2, float y0, float y1, float y2, float* o) {
    const float v0 = x0 - c.x, v1 = x1 - c.y, v2 = x2 - c.z;
    o[0] = (R[0] * v0 + R[3] * v1 + R[6] * v2) - y0;
    o[1] = (R[1] * v0 + R[4] * v1 + R[7] * v2) - y1;
    o[2] = (R[2] * v0 + R[5] * v1 + R[8] * v2) - y2;
    nrm = fmaf(o[0], o[0], fmaf(o[1], o[1], fmaf(o[2], o[2], nrm)));
  };
  if (VEC) {
    const float4* x4 = reinterpret_cast<const float4*>(x);
    const float4* y4 = reinterpret_cast<const float4*>(yc);
    float4* o4 = reinterpret_cast<float4*>(out);
    for (int qd = lane; qd < N16 / 4; qd += 32) {  // atoms 4 qd .. 4 qd + 3 (all < N or all >= N)
      float o[12];
      if (4 * qd < N) {
        float xv[12], yv[12];
#pragma unroll
        for (int h = 0; h < 3; ++h) {
          const float4 a = x4[3 * qd + h], b = y4[3 * qd + h];
          xv[4 * h] = a.x;
          xv[4 * h + 1] = a.y;
          xv[4 * h + 2] = a.z;
          xv[4 * h + 3] = a.w;
          yv[4 * h] = b.x;
          yv[4 * h + 1] = b.y;
          yv[4 * h + 2] = b.z;
          yv[4 * h + 3] = b.w;
        }
#pragma unroll
        for (int m = 0; m < 4; ++m)
          atom(xv[3 * m], xv[3 * m + 1], xv[3 * m + 2], yv[3 * m], yv[3 * m + 1], yv[3 * m + 2], o + 3 * m);
      } else {
#pragma unroll
        for (int e = 0; e < 12; ++e) o[e] = 0.0f;
      }
#pragma unroll
      for (int h = 0; h < 3; ++h) o4[3 * qd + h] = make_float4(o[4 * h], o[4 * h + 1], o[4 * h + 2], o[4 * h + 3]);
    }
  } else {
    for (int j = lane; j < N16; j += 32) {
      float o[3] = {0.0f, 0.0f, 0.0f};
      if (j < N) atom(x[3 * j], x[3 * j + 1], x[3 * j + 2], yc[3 * j], yc[3 * j + 1], yc[3 * j + 2], o);
      out[3 * j] = o[0];
      out[3 * j + 1] = o[1];
      out[3 * j + 2] = o[2];
    }
  }
  nrm = warp_sum_float(nrm);
  if (lane == 0) Nx[k] = nrm;
}

// gamma^s_fi = -lambda p_fi (q_i - s_f), gamma^z_fi = p_fi (Eqs. 5-6 differentiated), rows of
// Mp >= M entries (zero beyond M), and Gamma^s_f, Gamma^z_f in Gsum.  One warp per frame.
__global__ void gamma_kernel(int F, int M, int Mp, const float* __restrict__ P, const float* __restrict__ q32,
                             const double* __restrict__ s, float lambda, float* __restrict__ GS, float* __restrict__ GZ,
                             float* __restrict__ Gsum) {
  const int lane = threadIdx.x & 31;
  const int f = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (f >= F) return;
  const float sf = (float)s[f], sl = s_low<float>(s[f], sf);
  float ss = 0.0f, sz = 0.0f;
  for (int i = lane; i < Mp; i += 32) {
    float gs = 0.0f, gz = 0.0f;
    if (i < M) {
      const float p = P[(size_t)f * M + i];
      gz = p;
      gs = -lambda * p * ((q32[i] - sf) - sl);
    }
    GS[(size_t)f * Mp + i] = gs;
    GZ[(size_t)f * Mp + i] = gz;
    ss += gs;
    sz += gz;
  }
  ss = warp_sum_float(ss);
  sz = warp_sum_float(sz);
  if (lane == 0) {
    Gsum[2 * f] = ss;
    Gsum[2 * f + 1] = sz;
  }
}

// ---------------------------------------------------------------------------------------
// approximate MSDs.  Tile: 64 approximate frames x 8 RM landmarks, 128 threads; thread
// (tx, ty) holds frames u*16 + ty (u < 4) and landmarks v*8 + tx (v < RM).  Chunks of 16
// atoms (192 bytes per row); shared rows of 52 floats, so the 4 frame rows and the 8 landmark
// rows a warp reads at one step fall in distinct banks.  Two atoms per step: 3 LDS.64 per
// row, each an adjacent coordinate pair; per (frame, landmark) 3 FMA2 of dx . d.
constexpr int AT_TF = 64, AT_THREADS = 128, AT_KC = 16, AT_STAGES = 3;
constexpr int AT_ROWF = AT_KC * 3 + 4;

template <int RM>
__global__ void __launch_bounds__(AT_THREADS, 3)
approx_pair_tile(const int* __restrict__ alist, const int* __restrict__ aseg, const int* __restrict__ acount,
                 int seg_base, int M, int N16, const float* __restrict__ Xr, const float* __restrict__ Bm,
                 const float* __restrict__ Nx, const float* __restrict__ Nb, float dscale, float* __restrict__ Dout) {
  constexpr int TF = AT_TF, TM = 8 * RM;
  extern __shared__ __align__(16) float smem[];
  float* Xs = smem;                            // [stage][TF][ROWF]
  float* Ls = smem + AT_STAGES * TF * AT_ROWF;  // [stage][TM][ROWF]
  __shared__ int s_seg[TF];
  __shared__ int s_frame[TF];
  const int count = *acount;
  const int i0 = blockIdx.x * TM;
  const int tid = threadIdx.x, tx = tid & 7, ty = tid >> 3;
  const int nchunk = N16 / AT_KC;
  const size_t rowlen = (size_t)N16 * 3;
  for (int row0 = blockIdx.y * TF; row0 < count; row0 += gridDim.y * TF) {
    __syncthreads();  // the previous tile's reads of s_seg / s_frame are done
    if (tid < TF) {
      const int r = row0 + tid;
      s_seg[tid] = r < count ? aseg[r] : -1;
      s_frame[tid] = r < count ? alist[r] : -1;
    }
    __syncthreads();
    int k = 0;
    while (k < TF && s_seg[k] >= 0) {
      const int seg = s_seg[k];
      int kend = k;
      while (kend < TF && s_seg[kend] == seg) ++kend;
      const float* Bsrc = Bm + (size_t)(seg - seg_base) * M * rowlen;
      auto issue = [&](int c) {
        const int st = c % AT_STAGES;
        float* xs = Xs + st * TF * AT_ROWF;
        float* ls = Ls + st * TM * AT_ROWF;
        const size_t col = (size_t)c * AT_KC * 3;
        for (int e = tid; e < (TF + TM) * 12; e += AT_THREADS) {  // 12 pieces of 16 bytes per row
          const int row = e / 12, piece = e - row * 12;
          if (row < TF) {
            const bool ok = row >= k && row < kend;
            const float* src = ok ? Xr + (size_t)(row0 + row) * rowlen + col + piece * 4 : Xr;
            cp_async16(xs + row * AT_ROWF + piece * 4, src, ok);
          } else {
            const int ll = row - TF, i = i0 + ll;
            const bool ok = i < M;
            const float* src = ok ? Bsrc + (size_t)i * rowlen + col + piece * 4 : Bm;
            cp_async16(ls + ll * AT_ROWF + piece * 4, src, ok);
          }
        }
      };
      f2 acc[4][RM];
      float thi[4][RM], tlo[4][RM];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < RM; ++v) {
          acc[u][v] = 0ull;  // the bit pattern of (+0, +0)
          thi[u][v] = tlo[u][v] = 0.0f;
        }
#pragma unroll
      for (int st = 0; st < AT_STAGES - 1; ++st) {
        if (st < nchunk) issue(st);
        cp_async_commit();
      }
      for (int c = 0; c < nchunk; ++c) {
        cp_async_wait<AT_STAGES - 2>();
        __syncthreads();
        if (c + AT_STAGES - 1 < nchunk) issue(c + AT_STAGES - 1);
        cp_async_commit();
        const int st = c % AT_STAGES;
        const float* xs = Xs + st * TF * AT_ROWF;
        const float* ls = Ls + st * TM * AT_ROWF;
#pragma unroll 2
        for (int a = 0; a < AT_KC; a += 2) {
          f2 x[4][3], b[RM][3];
#pragma unroll
          for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int h = 0; h < 3; ++h)
              x[u][h] = *reinterpret_cast<const f2*>(xs + (u * 16 + ty) * AT_ROWF + a * 3 + 2 * h);
#pragma unroll
          for (int v = 0; v < RM; ++v)
#pragma unroll
            for (int h = 0; h < 3; ++h)
              b[v][h] = *reinterpret_cast<const f2*>(ls + (v * 8 + tx) * AT_ROWF + a * 3 + 2 * h);
#pragma unroll
          for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < RM; ++v) {
              f2 t = acc[u][v];
#pragma unroll
              for (int h = 0; h < 3; ++h) {
                t = f2_fma(x[u][h], b[v][h], t);
              }
              acc[u][v] = t;
            }
        }
        if ((c & 3) == 3 || c + 1 == nchunk) {  // every 64 atoms into the compensated totals
#pragma unroll
          for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < RM; ++v) {
              float lo, hi;
              f2_unpack(acc[u][v], lo, hi);
              two_sum_acc(thi[u][v], tlo[u][v], lo + hi);
              acc[u][v] = 0ull;
            }
        }
      }
      cp_async_wait<0>();
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int ff = u * 16 + ty;
        if (ff < k || ff >= kend) continue;
        const int f = s_frame[ff];
        const float nx = Nx[row0 + ff];
        const float* nb = Nb + (size_t)(seg - seg_base) * M;
#pragma unroll
        for (int v = 0; v < RM; ++v) {
          const int i = i0 + v * 8 + tx;
          if (i < M) {
            // |dx|^2 + |d|^2 - 2 dx.d with the compensated cross term
            const float two_c = 2.0f * thi[u][v];
            const float base = nx + nb[i];
            Dout[(size_t)f * M + i] = ((base - two_c) - 2.0f * tlo[u][v]) * dscale;
          }
        }
      }
      k = kend;
      __syncthreads();  // the next run's first copies overwrite stages still being read
    }
  }
}

// ---------------------------------------------------------------------------------------
// beta for frames grouped by segment.  Tile: 64 consecutive frames x 32 atoms, 256 threads,
// each 4 frames x 2 atoms x 3 components x {s, z}.  Landmark chunks of 16: per frame a row
// of 16 gamma^s and 16 gamma^z, per landmark 32 atoms of b (384 bytes, 24 pieces).  Per
// four landmarks: one LDS.128 of each gamma per frame, 3 LDS.64 of b per landmark.
constexpr int BT_TF = 64, BT_TJ = 32, BT_KL = 16, BT_THREADS = 256, BT_STAGES = 3;
constexpr int BT_GROW = BT_KL + 4;
constexpr int BT_BROW = BT_TJ * 3 + 4;

__global__ void __launch_bounds__(BT_THREADS, 2)
adjoint_beta_tile(int F, int M, int Mp, int N, int N16, int seg_base, const float* __restrict__ GS,
                  const float* __restrict__ GZ, const float* __restrict__ Bm, const float* __restrict__ Gsum,
                  const float* __restrict__ Yc, const int* __restrict__ seg_of_frame, float* __restrict__ gs,
                  float* __restrict__ gz) {
  extern __shared__ __align__(16) float smem[];
  float* Gss = smem;                               // [stage][TF][GROW]
  float* Gzs = Gss + BT_STAGES * BT_TF * BT_GROW;  // [stage][TF][GROW]
  float* Bbs = Gzs + BT_STAGES * BT_TF * BT_GROW;  // [stage][KL][BROW]
  __shared__ int s_seg[BT_TF];
  const int j0 = blockIdx.x * BT_TJ;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int nchunk = Mp / BT_KL;
  const size_t rowlen = (size_t)N16 * 3;
  const int colend = N16 * 3 - j0 * 3;  // floats of the row left from this tile's first atom
  for (int f0 = blockIdx.y * BT_TF; f0 < F; f0 += gridDim.y * BT_TF) {
    __syncthreads();  // the previous tile's reads of s_seg are done
    if (tid < BT_TF) s_seg[tid] = f0 + tid < F ? seg_of_frame[f0 + tid] : -1;
    float acs[4][6], acz[4][6];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int e = 0; e < 6; ++e) acs[u][e] = acz[u][e] = 0.0f;
    __syncthreads();
    int k = 0;
    while (k < BT_TF && s_seg[k] >= 0) {
      const int seg = s_seg[k];
      int kend = k;
      while (kend < BT_TF && s_seg[kend] == seg) ++kend;
      const float* Bsrc = Bm + (size_t)(seg - seg_base) * M * rowlen + (size_t)j0 * 3;
      auto issue = [&](int c) {
        const int st = c % BT_STAGES;
        float* gss = Gss + st * BT_TF * BT_GROW;
        float* gzs = Gzs + st * BT_TF * BT_GROW;
        float* bbs = Bbs + st * BT_KL * BT_BROW;
        const int i0 = c * BT_KL;
        for (int e = tid; e < BT_TF * 8 + BT_KL * 24; e += BT_THREADS) {
          if (e < BT_TF * 8) {  // per frame 4 pieces of gamma^s, then 4 of gamma^z
            const int row = e >> 3, pc = e & 7, piece = pc & 3;
            const bool ok = row >= k && row < kend;
            const float* base = pc < 4 ? GS : GZ;
            const float* src = ok ? base + (size_t)(f0 + row) * Mp + i0 + piece * 4 : GS;
            cp_async16((pc < 4 ? gss : gzs) + row * BT_GROW + piece * 4, src, ok);
          } else {
            const int e2 = e - BT_TF * 8;
            const int ll = e2 / 24, piece = e2 - ll * 24;
            const int i = i0 + ll;
            const bool ok = i < M && piece * 4 < colend;
            const float* src = ok ? Bsrc + (size_t)i * rowlen + piece * 4 : Bm;
            cp_async16(bbs + ll * BT_BROW + piece * 4, src, ok);
          }
        }
      };
#pragma unroll
      for (int st = 0; st < BT_STAGES - 1; ++st) {
        if (st < nchunk) issue(st);
        cp_async_commit();
      }
      for (int c = 0; c < nchunk; ++c) {
        cp_async_wait<BT_STAGES - 2>();
        __syncthreads();
        if (c + BT_STAGES - 1 < nchunk) issue(c + BT_STAGES - 1);
        cp_async_commit();
        const int st = c % BT_STAGES;
        const float* gss = Gss + st * BT_TF * BT_GROW;
        const float* gzs = Gzs + st * BT_TF * BT_GROW;
        const float* bbs = Bbs + st * BT_KL * BT_BROW;
#pragma unroll
        for (int i4 = 0; i4 < BT_KL; i4 += 4) {
          float g1[4][4], g2[4][4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const float4 a = *reinterpret_cast<const float4*>(gss + (ty * 4 + u) * BT_GROW + i4);
            const float4 b = *reinterpret_cast<const float4*>(gzs + (ty * 4 + u) * BT_GROW + i4);
            g1[u][0] = a.x;
            g1[u][1] = a.y;
            g1[u][2] = a.z;
            g1[u][3] = a.w;
            g2[u][0] = b.x;
            g2[u][1] = b.y;
            g2[u][2] = b.z;
            g2[u][3] = b.w;
          }
#pragma unroll
          for (int l = 0; l < 4; ++l) {
            float bv[6];
#pragma unroll
            for (int h = 0; h < 3; ++h) {
              const float2 t = *reinterpret_cast<const float2*>(bbs + (i4 + l) * BT_BROW + tx * 6 + 2 * h);
              bv[2 * h] = t.x;
              bv[2 * h + 1] = t.y;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
              for (int e = 0; e < 6; ++e) {
                acs[u][e] = fmaf(g1[u][l], bv[e], acs[u][e]);
                acz[u][e] = fmaf(g2[u][l], bv[e], acz[u][e]);
              }
          }
        }
      }
      cp_async_wait<0>();
      __syncthreads();  // the next run's first copies overwrite stages still being read
      k = kend;
    }
    // beta = Gamma_f y' + sum_i gamma_fi d_i
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int f = f0 + ty * 4 + u;
      if (f >= F) continue;
      const float Gs = Gsum[2 * f], Gz = Gsum[2 * f + 1];
      const float* yc = Yc + (size_t)(s_seg[ty * 4 + u] - seg_base) * 3 * N;
#pragma unroll
      for (int a = 0; a < 2; ++a) {
        const int j = j0 + tx * 2 + a;
        if (j >= N) continue;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const float yv = yc[3 * j + c];
          gs[((size_t)f * N + j) * 3 + c] = fmaf(Gs, yv, acs[u][3 * a + c]);
          gz[((size_t)f * N + j) * 3 + c] = fmaf(Gz, yv, acz[u][3 * a + c]);
        }
      }
    }
  }
}

template <typename K>
void set_smem(K kernel, size_t bytes) {
  cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

int tile_rm(int M) {
  const int w4 = (M + 31) / 32 * 32 - M, w5 = (M + 39) / 40 * 40 - M;
  return w5 < w4 ? 5 : 4;
}

}  // namespace

// ---------------------------------------------------------------------------------------
size_t tile_bytes_frames(int napp, int N) { return (size_t)napp * round_up16(N) * 3 * sizeof(float); }
size_t tile_bytes_landmarks(int nseg, int M, int N) {
  return (size_t)nseg * M * round_up16(N) * 3 * sizeof(float);
}
size_t tile_bytes_gamma(int F, int M) { return (size_t)F * round_up16(M) * sizeof(float); }

void launch_materialize_landmarks(Prec p, int s0, int ns, const LandmarkDev& L, const float* Bseg, const void* frames,
                                  FrameInfo fi, const int* refresh_list, const RefDesc& prior, float* Bm, float* Nb,
                                  float* Yc, cudaStream_t st) {
  if (ns <= 0 || L.M <= 0) return;
  const dim3 grid(L.M, ns);
  const int N16 = round_up16(L.N);
  if (p == P_F16)
    materialize_landmarks_kernel<__half><<<grid, 128, 0, st>>>(s0, L.M, L.N, N16, (const __half*)L.coords, L.off, Bseg,
                                                               (const float*)frames, fi.c32, refresh_list,
                                                               (const float*)prior.coords, prior.c32, Bm, Nb, Yc);
  else
    materialize_landmarks_kernel<float><<<grid, 128, 0, st>>>(s0, L.M, L.N, N16, (const float*)L.coords, L.off, Bseg,
                                                              (const float*)frames, fi.c32, refresh_list,
                                                              (const float*)prior.coords, prior.c32, Bm, Nb, Yc);
  note_launch();
}

void launch_materialize_frames(int napp, const int* acount, const int* alist, const int* aseg, int seg_base,
                               const LandmarkDev& L, const void* frames, FrameInfo fi, double4* qxy,
                               const float* Yc, float* Xr, float* Nx, const int* refine_ref, const RefDesc& prior,
                               cudaStream_t st) {
  if (napp <= 0) return;
  const bool vec = L.N % 4 == 0 && ((uintptr_t)frames % 16) == 0 && ((uintptr_t)Yc % 16) == 0 &&
                   ((uintptr_t)Xr % 16) == 0;
  const unsigned blocks = (unsigned)((napp + 7) / 8);  // 8 warps (frames) per block
  RefineArgs ra{refine_ref, (const float*)prior.coords, prior.c32, prior.G, fi.G, L.w};
  const float* fr = (const float*)frames;
  const int N16 = round_up16(L.N);
  if (refine_ref) {
    if (vec)
      materialize_frames_kernel<true, true><<<blocks, 256, 0, st>>>(napp, acount, alist, aseg, seg_base, L.N, N16,
                                                                    fr, fi.c32, qxy, Yc, Xr, Nx, ra);
    else
      materialize_frames_kernel<false, true><<<blocks, 256, 0, st>>>(napp, acount, alist, aseg, seg_base, L.N, N16,
                                                                     fr, fi.c32, qxy, Yc, Xr, Nx, ra);
  } else {
    if (vec)
      materialize_frames_kernel<true, false><<<blocks, 256, 0, st>>>(napp, acount, alist, aseg, seg_base, L.N, N16,
                                                                     fr, fi.c32, qxy, Yc, Xr, Nx, ra);
    else
      materialize_frames_kernel<false, false><<<blocks, 256, 0, st>>>(napp, acount, alist, aseg, seg_base, L.N,
                                                                      N16, fr, fi.c32, qxy, Yc, Xr, Nx, ra);
  }
  note_launch();
}

void launch_gamma(int F, const LandmarkDev& L, const float* P, const double* s, double lambda, float* GS, float* GZ,
                  float* Gsum, cudaStream_t st) {
  if (F <= 0) return;
  gamma_kernel<<<(F + 7) / 8, 256, 0, st>>>(F, L.M, round_up16(L.M), P, L.q32, s, (float)lambda, GS, GZ, Gsum);
  note_launch();
}

void launch_approx_pairs_tile(int napp, const int* alist, const int* aseg, const int* acount, int seg_base,
                              const LandmarkDev& L, const float* Xr, const float* Bm, const float* Nx, const float* Nb,
                              float* D, cudaStream_t st) {
  if (napp <= 0 || L.M <= 0) return;
  const int rm = tile_rm(L.M), tm = 8 * rm, N16 = round_up16(L.N);
  const size_t smem = (size_t)AT_STAGES * (AT_TF + tm) * AT_ROWF * sizeof(float);
  const dim3 grid((L.M + tm - 1) / tm, std::min((napp + AT_TF - 1) / AT_TF, 65535));
  if (rm == 5) {
    set_smem(approx_pair_tile<5>, smem);
    approx_pair_tile<5><<<grid, AT_THREADS, smem, st>>>(alist, aseg, acount, seg_base, L.M, N16, Xr, Bm, Nx, Nb,
                                                         (float)L.dscale, D);
  } else {
    set_smem(approx_pair_tile<4>, smem);
    approx_pair_tile<4><<<grid, AT_THREADS, smem, st>>>(alist, aseg, acount, seg_base, L.M, N16, Xr, Bm, Nx, Nb,
                                                         (float)L.dscale, D);
  }
  note_launch();
}

void launch_adjoint_beta_tile(int F, const LandmarkDev& L, int seg_base, const float* GS, const float* GZ,
                              const float* Bm, const float* Gsum, const float* Yc, const int* seg_of_frame, float* gs,
                              float* gz, cudaStream_t st) {
  if (F <= 0) return;
  const size_t smem = (size_t)BT_STAGES * (2 * BT_TF * BT_GROW + BT_KL * BT_BROW) * sizeof(float);
  const dim3 grid((L.N + BT_TJ - 1) / BT_TJ, std::min((F + BT_TF - 1) / BT_TF, 65535));
  set_smem(adjoint_beta_tile, smem);
  adjoint_beta_tile<<<grid, BT_THREADS, smem, st>>>(F, L.M, round_up16(L.M), L.N, round_up16(L.N), seg_base, GS, GZ,
                                                    Bm, Gsum, Yc, seg_of_frame, gs, gz);
  note_launch();
}

}  // namespace pcv

// k_adjoint.cu -- the adjoint of the path CVs: ds/dx and dz/dx of every frame.
//
// With gamma_i = dL/dD_i (gamma^z_i = p_i, gamma^s_i = -lambda p_i (q_i - s),
// p_i = exp(-lambda (D_i - m)) / l), the direct part of Eq. (der_dist) summed over the
// landmarks is 2 w_k ((sum_i gamma_i) x_k - beta_k) with beta_k = sum_i gamma_i Rot_i a_ik,
// Rot_i = R_{a_i x} at exact / reassignment frames and R_{a_i y} at approximate frames
// (R_xy is applied afterwards).  Two contraction kernels compute beta:
//   adjoint_beta_pair: any per-(frame, landmark) rotation (exact mode, frequent
//     reassignments): 18 FMA per (frame, landmark, atom) for s and z together;
//   adjoint_beta_seg: frames that share a close structure share Rot_i, so b_i = Rot_i a_i
//     is formed once per tile and beta = sum_i gamma_i b_i is a plain GEMM: 6 FMA.
// The finish kernels turn beta into gradients and add, at approximate frames, the rotation
// term of Eq. (close_der_dist) (derivation in pcv_device.cuh: adjoint_rotation_term):
// adjoint_finish_staged (FP32 modes, a warp per frame staged in shared memory),
// adjoint_finish_block (FP32 modes, structures too large to stage: a block per frame) and
// adjoint_finish_warp (FP64: a warp per frame).
#include <algorithm>

#include <cuda_fp16.h>

#include "pcv_device.cuh"
#include "pcv_internal.h"

namespace pcv {
namespace {

// gamma^s, gamma^z of one (frame, landmark) pair from the softmax weight p; s = sh + sl
// (s_low)
template <typename ST>
__device__ __forceinline__ void gammas(ST p, ST lambda, ST qi, ST sh, ST sl, ST& gs, ST& gz) {
  gz = p;
  gs = -lambda * p * ((qi - sh) - sl);
}

// ---------------------------------------------------------------------------------------
constexpr int BP_TF = 32, BP_TJ = 64, BP_THREADS = 128;

template <typename ST, typename LT>
__global__ void __launch_bounds__(BP_THREADS)
adjoint_beta_pair(int F, int M, int N, const LT* __restrict__ lm, const float* __restrict__ lmoff,
                  const double* __restrict__ q,
                  const float* __restrict__ q32, const ST* __restrict__ P, const double* __restrict__ s, double lambda,
                  const ST* __restrict__ Rpair, const ST* __restrict__ Bseg, const int* __restrict__ seg_of_frame,
                  ST* __restrict__ gs, ST* __restrict__ gz, ST* __restrict__ part) {
  constexpr int KL = sizeof(ST) == 8 ? 4 : 8;
  __shared__ __align__(16) ST Ws[KL * 3][BP_TF * 3];  // gamma^s_fi Rot_fi[b][c] at [(i,c)][(f,b)]
  __shared__ __align__(16) ST Wz[KL * 3][BP_TF * 3];
  __shared__ __align__(16) ST As[KL * 3][BP_TJ];
  const int f0 = blockIdx.y * BP_TF, j0 = blockIdx.x * BP_TJ;
  const int tid = threadIdx.x, tx = tid & 7, ty = tid >> 3;
  ST bs[2][3][8], bz[2][3][8];
#pragma unroll
  for (int u = 0; u < 2; ++u)
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
      for (int k = 0; k < 8; ++k) bs[u][b][k] = bz[u][b][k] = 0;
  const ST lam = (ST)lambda;
  // landmark range of this CTA: a split over gridDim.z when the frames give less than a wave
  const int per = ((M + gridDim.z - 1) / gridDim.z + KL - 1) / KL * KL;
  const int ibeg = blockIdx.z * per, iend = min(M, ibeg + per);
  // a warp holds the frames f0 + 8 w .. f0 + 8 w + 7: warps wholly past F skip the products
  const bool live = f0 + (tid >> 5) * 8 < F;
  for (int i0 = ibeg; i0 < iend; i0 += KL) {
    for (int e = tid; e < BP_TF * KL; e += BP_THREADS) {
      const int ff = e / KL, ii = e - ff * KL;
      const int f = f0 + ff, i = i0 + ii;
      ST rot[9];
      ST gsv = 0, gzv = 0;
#pragma unroll
      for (int c = 0; c < 9; ++c) rot[c] = 0;
      if (f < F && i < iend) {
        const ST qi = sizeof(ST) == 8 ? (ST)q[i] : (ST)q32[i];
        const ST sh = (ST)s[f];
        gammas<ST>(P[(size_t)f * M + i], lam, qi, sh, s_low<ST>(s[f], sh), gsv, gzv);
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
    for (int e = tid; e < KL * BP_TJ; e += BP_THREADS) {
      const int ii = e / BP_TJ, jj = e - ii * BP_TJ;
      const int i = i0 + ii, j = j0 + jj;
#pragma unroll
      for (int c = 0; c < 3; ++c) As[ii * 3 + c][jj] = (i < iend && j < N) ? lm_coord<ST, LT>(lm, lmoff, N, i, j, c) : (ST)0;
    }
    __syncthreads();
#pragma unroll 2
    for (int kk = 0; kk < (live ? KL * 3 : 0); ++kk) {
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
      if (part) {
        ST* dst = part + (((size_t)blockIdx.z * F + f) * N + j) * 6;
#pragma unroll
        for (int b = 0; b < 3; ++b) {
          dst[b] = bs[u][b][k];
          dst[3 + b] = bz[u][b][k];
        }
      } else {
#pragma unroll
        for (int b = 0; b < 3; ++b) {
          gs[((size_t)f * N + j) * 3 + b] = bs[u][b][k];
          gz[((size_t)f * N + j) * 3 + b] = bz[u][b][k];
        }
      }
    }
  }
}

// beta of every frame from the landmark ranges' partial sums part[z][f][atom][6], in range
// order
template <typename ST>
__global__ void beta_pair_part_sum(int F, int N, int nsplit, const ST* __restrict__ part, ST* __restrict__ gs,
                                   ST* __restrict__ gz) {
  const size_t total = (size_t)F * N * 6;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    ST v = 0;
    for (int k = 0; k < nsplit; ++k) v += part[(size_t)k * total + e];
    const size_t fj = e / 6;
    const int comp = (int)(e - fj * 6);
    if (comp < 3)
      gs[fj * 3 + comp] = v;
    else
      gz[fj * 3 + comp - 3] = v;
  }
}

// ---------------------------------------------------------------------------------------
// Exact-mode beta with a neighbour list (FP32 / FP16 storage): tile of up to 16 frames of a
// frame list x 64 atoms, 128 threads, each 1 frame x 8 atoms x 3 components x {s, z}.
// mode 0: entries [16 y, 16 y + 16) of the update-frame list, every landmark, rotations
//         Rupd[(row * M + i) * 9] (row = position in the list); the landmarks are split
//         into gridDim.z ranges (the update frames are few and the landmarks many), each
//         CTA writing its partial sums to part[z][row][atom][6], summed by beta_part_sum;
// mode 1: tile y of the between-update tiles, the landmarks of the tile's list, rotations
//         Rnl[(f * Mnl + column) * 9].
// With Bseg (close structure) the rotations are the stored R_{a_i y} of each frame's segment,
// Bseg[(segof[f] * M + i) * 9], in both modes.
// Per chunk of 8 landmarks the weights gamma R (3 x 3 per frame and landmark) and the
// landmark coordinates are staged in shared memory, as in adjoint_beta_pair.
constexpr int BL_TF = NL_TILE_F, BL_TJ = 64, BL_THREADS = 128, BL_KL = 8;

template <typename LT>
__global__ void __launch_bounds__(BL_THREADS)
adjoint_beta_list(int mode, const NlTile* __restrict__ tiles, const int* __restrict__ counts,
                  const int* __restrict__ ulist, const int* __restrict__ nlist, const int* __restrict__ NLtab,
                  int Mnl, int M, int N, const LT* __restrict__ lm, const float* __restrict__ lmoff,
                  const float* __restrict__ q32, const float* __restrict__ P, const double* __restrict__ s,
                  float lambda, const float* __restrict__ Rupd, const float* __restrict__ Rnl,
                  const float* __restrict__ Bseg, const int* __restrict__ segof, float* __restrict__ gs,
                  float* __restrict__ gz, float* __restrict__ part) {
  __shared__ __align__(16) float Ws[BL_KL * 3][BL_TF * 3];
  __shared__ __align__(16) float Wz[BL_KL * 3][BL_TF * 3];
  __shared__ __align__(16) float As[BL_KL * 3][BL_TJ];
  __shared__ int s_frame[BL_TF];
  __shared__ float s_s[BL_TF];
  __shared__ float s_l[BL_TF];
  int p0, rows, ncol;
  const int* fl;
  const int* cols;
  if (mode == 0) {
    p0 = blockIdx.y * BL_TF;
    const int n = counts[0];
    if (p0 >= n) return;  // uniform over the block
    rows = min(BL_TF, n - p0);
    fl = ulist;
    cols = nullptr;
    ncol = M;
  } else {
    if ((int)blockIdx.y >= counts[3]) return;
    const NlTile w = tiles[blockIdx.y];
    p0 = w.p0;
    rows = w.rows;
    fl = nlist;
    cols = NLtab + (size_t)w.slot * Mnl;
    ncol = Mnl;
  }
  // landmark range of this CTA (split of the update frames' landmarks over gridDim.z)
  const int per = ((ncol + gridDim.z - 1) / gridDim.z + BL_KL - 1) / BL_KL * BL_KL;
  const int cbeg = blockIdx.z * per, cend = min(ncol, cbeg + per);
  const int j0 = blockIdx.x * BL_TJ;
  const int tid = threadIdx.x, tx = tid & 7, ty = tid >> 3;
  if (tid < BL_TF) {
    const int f = tid < rows ? fl[p0 + tid] : -1;
    s_frame[tid] = f;
    s_s[tid] = f >= 0 ? (float)s[f] : 0.0f;
    s_l[tid] = f >= 0 ? s_low<float>(s[f], s_s[tid]) : 0.0f;
  }
  __syncthreads();
  float bs[3][8], bz[3][8];
#pragma unroll
  for (int b = 0; b < 3; ++b)
#pragma unroll
    for (int k = 0; k < 8; ++k) bs[b][k] = bz[b][k] = 0.0f;
  for (int c0 = cbeg; c0 < cend; c0 += BL_KL) {
    for (int e = tid; e < BL_TF * BL_KL; e += BL_THREADS) {
      const int ff = e / BL_KL, cc = e - ff * BL_KL;
      const int f = s_frame[ff], c = c0 + cc;
      float rot[9];
      float gsv = 0.0f, gzv = 0.0f;
#pragma unroll
      for (int k = 0; k < 9; ++k) rot[k] = 0.0f;
      if (f >= 0 && c < cend) {
        const int i = cols ? cols[c] : c;
        gammas<float>(P[(size_t)f * M + i], lambda, q32[i], s_s[ff], s_l[ff], gsv, gzv);
        const float* R = Bseg ? Bseg + ((size_t)segof[f] * M + i) * 9
                              : (mode == 0 ? Rupd + ((size_t)(p0 + ff) * M + i) * 9 : Rnl + ((size_t)f * Mnl + c) * 9);
#pragma unroll
        for (int k = 0; k < 9; ++k) rot[k] = R[k];
      }
#pragma unroll
      for (int cx = 0; cx < 3; ++cx)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
          Ws[cc * 3 + cx][ff * 3 + b] = gsv * rot[3 * b + cx];
          Wz[cc * 3 + cx][ff * 3 + b] = gzv * rot[3 * b + cx];
        }
    }
    for (int e = tid; e < BL_KL * BL_TJ; e += BL_THREADS) {
      const int cc = e / BL_TJ, jj = e - cc * BL_TJ;
      const int c = c0 + cc, j = j0 + jj;
      const bool ok = c < cend && j < N;
      const int i = ok ? (cols ? cols[c] : c) : 0;
#pragma unroll
      for (int cx = 0; cx < 3; ++cx) As[cc * 3 + cx][jj] = ok ? lm_coord<float, LT>(lm, lmoff, N, i, j, cx) : 0.0f;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < BL_KL * 3; ++kk) {
      float a[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) a[k] = As[kk][tx * 8 + k];
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        const float ws = Ws[kk][ty * 3 + b], wz = Wz[kk][ty * 3 + b];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          bs[b][k] = fmaf(ws, a[k], bs[b][k]);
          bz[b][k] = fmaf(wz, a[k], bz[b][k]);
        }
      }
    }
    __syncthreads();
  }
  const int f = s_frame[ty];
  if (f < 0) return;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int j = j0 + tx * 8 + k;
    if (j >= N) continue;
    if (part) {
      float* dst = part + (((size_t)blockIdx.z * counts[0] + p0 + ty) * N + j) * 6;
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        dst[b] = bs[b][k];
        dst[3 + b] = bz[b][k];
      }
    } else {
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        gs[((size_t)f * N + j) * 3 + b] = bs[b][k];
        gz[((size_t)f * N + j) * 3 + b] = bz[b][k];
      }
    }
  }
}

// beta of the update frames: the sum of the landmark ranges' partial sums, in range order
__global__ void beta_part_sum(const int* __restrict__ counts, const int* __restrict__ ulist, int N, int nsplit,
                              const float* __restrict__ part, float* __restrict__ gs, float* __restrict__ gz) {
  const int n = counts[0];
  const size_t total = (size_t)n * N * 6;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    float v = 0.0f;
    for (int k = 0; k < nsplit; ++k) v += part[(size_t)k * total + e];
    const size_t rj = e / 6;
    const int comp = (int)(e - rj * 6), row = (int)(rj / N), j = (int)(rj - (size_t)row * N);
    const size_t o = ((size_t)ulist[row] * N + j) * 3 + (comp % 3);
    if (comp < 3)
      gs[o] = v;
    else
      gz[o] = v;
  }
}

// ---------------------------------------------------------------------------------------
// beta for frames sharing close structures: tile of 64 consecutive frames x 32 atoms, 256
// threads, each 4 frames x 2 atoms x 3 components x {s, z} (48 FP32 sums): per landmark
// two LDS.128 of gamma and 6 landmark values feed 48 FMAs.  Frames of the tile are grouped
// into runs of equal segment; per run, landmark chunks are rotated by R_{a_i y} into shared
// memory and gamma is formed from p (coalesced rows of P).
constexpr int BS_TF = 64, BS_TJ = 32, BS_KL = 16, BS_THREADS = 256;

template <typename LT>
__global__ void __launch_bounds__(BS_THREADS, 3)
adjoint_beta_seg(int F, int M, int N, const LT* __restrict__ lm, const float* __restrict__ lmoff,
                 const float* __restrict__ q32,
                 const float* __restrict__ P, const double* __restrict__ s, float lambda,
                 const float* __restrict__ Bseg, const int* __restrict__ seg_of_frame, float* __restrict__ gs,
                 float* __restrict__ gz) {
  __shared__ __align__(16) float Gs[BS_KL][BS_TF + 4];  // gamma^s of (landmark, frame), 0 outside the run
  __shared__ __align__(16) float Gz[BS_KL][BS_TF + 4];
  __shared__ __align__(16) float Bb[BS_KL][BS_TJ * 3 + 4];  // b_ij = R_{a_i y} a_ij, (atom, xyz) packed
  __shared__ float s_B[BS_KL][9];
  __shared__ int s_seg[BS_TF];
  __shared__ float s_s[BS_TF];
  __shared__ float s_l[BS_TF];
  const int f0 = blockIdx.y * BS_TF, j0 = blockIdx.x * BS_TJ;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;  // atoms j0 + 2 tx + {0,1}; frames 4 ty + {0..3}
  if (tid < BS_TF) {
    const int f = f0 + tid;
    s_seg[tid] = f < F ? seg_of_frame[f] : -1;
    s_s[tid] = f < F ? (float)s[f] : 0.0f;
    s_l[tid] = f < F ? s_low<float>(s[f], s_s[tid]) : 0.0f;
  }
  float acs[4][6], acz[4][6];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int k = 0; k < 6; ++k) acs[u][k] = acz[u][k] = 0.0f;
  __syncthreads();
  int k = 0;
  while (k < BS_TF && s_seg[k] >= 0) {
    const int seg = s_seg[k];
    int kend = k;
    while (kend < BS_TF && s_seg[kend] == seg) ++kend;
    for (int i0 = 0; i0 < M; i0 += BS_KL) {
      if (tid < BS_KL * 9) {
        const int ii = tid / 9, c = tid - ii * 9;
        const int i = i0 + ii;
        s_B[ii][c] = i < M ? Bseg[((size_t)seg * M + i) * 9 + c] : 0.0f;
      }
      for (int e = tid; e < BS_KL * BS_TF; e += BS_THREADS) {
        const int ff = e / BS_KL, ii = e - ff * BS_KL;
        const int f = f0 + ff, i = i0 + ii;
        float gsv = 0.0f, gzv = 0.0f;
        if (ff >= k && ff < kend && i < M)
          gammas<float>(P[(size_t)f * M + i], lambda, q32[i], s_s[ff], s_l[ff], gsv, gzv);
        Gs[ii][ff] = gsv;
        Gz[ii][ff] = gzv;
      }
      __syncthreads();
      for (int e = tid; e < BS_KL * BS_TJ; e += BS_THREADS) {
        const int ii = e / BS_TJ, jj = e - ii * BS_TJ;
        const int i = i0 + ii, j = j0 + jj;
        float b0 = 0.0f, b1 = 0.0f, b2 = 0.0f;
        if (i < M && j < N) {
          const float a0 = lm_coord<float, LT>(lm, lmoff, N, i, j, 0);
          const float a1 = lm_coord<float, LT>(lm, lmoff, N, i, j, 1);
          const float a2 = lm_coord<float, LT>(lm, lmoff, N, i, j, 2);
          const float* B = s_B[ii];
          b0 = B[0] * a0 + B[1] * a1 + B[2] * a2;
          b1 = B[3] * a0 + B[4] * a1 + B[5] * a2;
          b2 = B[6] * a0 + B[7] * a1 + B[8] * a2;
        }
        Bb[ii][jj * 3 + 0] = b0;
        Bb[ii][jj * 3 + 1] = b1;
        Bb[ii][jj * 3 + 2] = b2;
      }
      __syncthreads();
#pragma unroll 4
      for (int ii = 0; ii < BS_KL; ++ii) {
        const float4 g1 = *reinterpret_cast<const float4*>(&Gs[ii][ty * 4]);
        const float4 g2 = *reinterpret_cast<const float4*>(&Gz[ii][ty * 4]);
        const float gsv[4] = {g1.x, g1.y, g1.z, g1.w}, gzv[4] = {g2.x, g2.y, g2.z, g2.w};
        // 6 floats at byte offset 24 tx: three 8-byte aligned float2 loads
        const float2 ba = *reinterpret_cast<const float2*>(&Bb[ii][tx * 6]);
        const float2 bb = *reinterpret_cast<const float2*>(&Bb[ii][tx * 6 + 2]);
        const float2 bc = *reinterpret_cast<const float2*>(&Bb[ii][tx * 6 + 4]);
        const float b[6] = {ba.x, ba.y, bb.x, bb.y, bc.x, bc.y};
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int c = 0; c < 6; ++c) {
            acs[u][c] = fmaf(gsv[u], b[c], acs[u][c]);
            acz[u][c] = fmaf(gzv[u], b[c], acz[u][c]);
          }
      }
      __syncthreads();
    }
    k = kend;
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int f = f0 + ty * 4 + u;
    if (f >= F) continue;
#pragma unroll
    for (int a = 0; a < 2; ++a) {
      const int j = j0 + tx * 2 + a;
      if (j >= N) continue;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        gs[((size_t)f * N + j) * 3 + c] = acs[u][3 * a + c];
        gz[((size_t)f * N + j) * 3 + c] = acz[u][3 * a + c];
      }
    }
  }
}

// ---------------------------------------------------------------------------------------
// warp-wide FP32 / FP64 sums
__device__ __forceinline__ float wsum(float v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}
__device__ __forceinline__ double wsum(double v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

// Per-frame finish, one warp per frame.  beta (in gs / gz) -> gradients; approximate
// frames add w_k T^T y_k (see adjoint_rotation_term).
// Alignment weights w' (wa / wa64, null when w' = w; Section 3.1): the centre of Eq.
// (der_dist) adds -2 w'_k S with S = sum_i gamma_i sum_j w_j d_ij = Gamma X_w - (R) sum_j w_j
// beta_j, X_w = sum_j w_j (x_j - c'), and the rotation term's dH/dx_k = (w_k y_k - w'_k Y_w) e_c^T
// adds -w'_k T^T Y_w, Y_w = sum_j w_j (y_j - c'_y).
template <typename ST, typename FT>
__global__ void __launch_bounds__(128)
adjoint_finish_warp(int F, int M, int N, const FT* __restrict__ frames, const float4* __restrict__ c32,
                    const double4* __restrict__ c64, const float* __restrict__ wts, const double* __restrict__ w64,
                    const float* __restrict__ wa, const double* __restrict__ wa64,
                    const float* __restrict__ A32, const double* __restrict__ A64, const double* __restrict__ q,
                    const float* __restrict__ q32, double dscale, const ST* __restrict__ P,
                    const double* __restrict__ s, double lambda, const ST* __restrict__ Bseg,
                    const int* __restrict__ seg_of_frame, FrameRec rec, const FT* __restrict__ prior_coords,
                    double4 prior_c, ST* __restrict__ gs, ST* __restrict__ gz) {
  const int f = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
  if (f >= F) return;
  const int lane = threadIdx.x & 31;
  const bool f64 = sizeof(ST) == 8;
  ST cx[3];
  if (f64) {
    const double4 c = c64[f];
    cx[0] = (ST)c.x; cx[1] = (ST)c.y; cx[2] = (ST)c.z;
  } else {
    const float4 c = c32[f];
    cx[0] = (ST)c.x; cx[1] = (ST)c.y; cx[2] = (ST)c.z;
  }
  const FT* x = frames + (size_t)f * N * 3;
  ST* bsp = gs + (size_t)f * N * 3;
  ST* bzp = gz + (size_t)f * N * 3;
  const ST wuni = (ST)dscale;  // uniform weight; converted once, not per atom
  auto wt = [&](int j) -> ST {
    if (f64) return w64 ? (ST)w64[j] : wuni;
    return wts ? (ST)wts[j] : wuni;
  };
  const bool split = f64 ? wa64 != nullptr : wa != nullptr;
  auto wat = [&](int j) -> ST { return f64 ? (ST)wa64[j] : (ST)wa[j]; };
  const bool approx = rec.flag && rec.flag[f] == 0;
  // Gamma = sum_i gamma_i from the same p the contraction used.  In exact arithmetic
  // Gamma^s = 0 and Gamma^z = 1, but the FP32 value of s and the p-weighted sum of q differ
  // by ~u s, which lambda ~ 1e3 amplifies: keeping the term makes the gradient exactly that
  // of sum_i gamma_i D_i for the gammas used.
  const ST sf = (ST)s[f], sl = s_low<ST>(s[f], sf), lamw = (ST)lambda;
  ST Gs = 0, Gz = 0;
  for (int i = lane; i < M; i += 32) {
    ST gsv, gzv;
    const ST qi = f64 ? (ST)q[i] : (ST)q32[i];
    gammas<ST>(P[(size_t)f * M + i], lamw, qi, sf, sl, gsv, gzv);
    Gs += gsv;
    Gz += gzv;
  }
  Gs = wsum(Gs);
  Gz = wsum(Gz);
  if (!approx) {
    ST Ss[3] = {0, 0, 0}, Sz[3] = {0, 0, 0};  // centre term (alignment weights)
    if (split) {
      ST xw[3] = {0, 0, 0}, bws[3] = {0, 0, 0}, bwz[3] = {0, 0, 0};
      for (int j = lane; j < N; j += 32) {
        const ST w = wt(j);
#pragma unroll
        for (int b = 0; b < 3; ++b) {
          xw[b] += w * ((ST)x[3 * j + b] - cx[b]);
          bws[b] += w * bsp[3 * j + b];
          bwz[b] += w * bzp[3 * j + b];
        }
      }
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        xw[b] = wsum(xw[b]);
        Ss[b] = Gs * xw[b] - wsum(bws[b]);
        Sz[b] = Gz * xw[b] - wsum(bwz[b]);
      }
    }
    for (int j = lane; j < N; j += 32) {
      const ST w = wt(j), w2 = split ? wat(j) : ST(0);
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        const ST v = (ST)x[3 * j + b] - cx[b];
        bsp[3 * j + b] = (ST)2 * w * (Gs * v - bsp[3 * j + b]) - (ST)2 * w2 * Ss[b];
        bzp[3 * j + b] = (ST)2 * w * (Gz * v - bzp[3 * j + b]) - (ST)2 * w2 * Sz[b];
      }
    }
    return;
  }
  const int r = rec.ref[f];
  const FT* y = r >= 0 ? frames + (size_t)r * N * 3 : prior_coords;
  ST cy[3];
  if (r >= 0) {
    if (f64) { const double4 c = c64[r]; cy[0] = (ST)c.x; cy[1] = (ST)c.y; cy[2] = (ST)c.z; }
    else { const float4 c = c32[r]; cy[0] = (ST)c.x; cy[1] = (ST)c.y; cy[2] = (ST)c.z; }
  } else {
    cy[0] = (ST)prior_c.x;
    cy[1] = (ST)prior_c.y;
    cy[2] = (ST)prior_c.z;
  }
  ST R[9];
  {
    const double4 qq = rec.qxy[f];
    const ST qd[4] = {(ST)qq.x, (ST)qq.y, (ST)qq.z, (ST)qq.w};
    quat_to_rot(qd, R);
  }
  // X = sum_j w x_j beta_j^T (s, z) and H_xy = sum_j w y_j x_j^T, centred, true weights
  ST acc[27];
#pragma unroll
  for (int e = 0; e < 27; ++e) acc[e] = 0;
  ST xw[3] = {0, 0, 0}, yw[3] = {0, 0, 0}, bws[3] = {0, 0, 0}, bwz[3] = {0, 0, 0};  // alignment weights
  for (int j = lane; j < N; j += 32) {
    const ST w = wt(j);
    ST v[3], u[3];
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      v[b] = (ST)x[3 * j + b] - cx[b];
      u[b] = (ST)y[3 * j + b] - cy[b];
    }
    if (split) {
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        xw[b] += w * v[b];
        yw[b] += w * u[b];
        bws[b] += w * bsp[3 * j + b];
        bwz[b] += w * bzp[3 * j + b];
      }
    }
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const ST wv = w * v[b], wu = w * u[b];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        acc[3 * b + c] = fma(wv, bsp[3 * j + c], acc[3 * b + c]);
        acc[9 + 3 * b + c] = fma(wv, bzp[3 * j + c], acc[9 + 3 * b + c]);
        acc[18 + 3 * b + c] = fma(wu, v[c], acc[18 + 3 * b + c]);
      }
    }
  }
  // Phi = sum_i gamma_i R_{a_i y} A_i R_{a_i y}^T (s, z)
  ST ph[12];
#pragma unroll
  for (int e = 0; e < 12; ++e) ph[e] = 0;
  const int seg = seg_of_frame[f];
  for (int i = lane; i < M; i += 32) {
    ST gsv, gzv;
    const ST qi = f64 ? (ST)q[i] : (ST)q32[i];
    gammas<ST>(P[(size_t)f * M + i], lamw, qi, sf, sl, gsv, gzv);
    const ST* B = Bseg + ((size_t)seg * M + i) * 9;
    ST A6[6];
#pragma unroll
    for (int e = 0; e < 6; ++e) A6[e] = f64 ? (ST)A64[(size_t)i * 6 + e] : (ST)A32[(size_t)i * 6 + e];
    const ST A[9] = {A6[0], A6[1], A6[2], A6[1], A6[3], A6[4], A6[2], A6[4], A6[5]};
    ST BA[9];
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
      for (int c = 0; c < 3; ++c) BA[3 * b + c] = B[3 * b] * A[c] + B[3 * b + 1] * A[3 + c] + B[3 * b + 2] * A[6 + c];
    // symmetric S = BA B^T: xx xy xz yy yz zz
    const int ib[6] = {0, 0, 0, 1, 1, 2}, ic[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
    for (int e = 0; e < 6; ++e) {
      const int b = ib[e], c = ic[e];
      const ST S = BA[3 * b] * B[3 * c] + BA[3 * b + 1] * B[3 * c + 1] + BA[3 * b + 2] * B[3 * c + 2];
      ph[e] = fma(gsv, S, ph[e]);
      ph[6 + e] = fma(gzv, S, ph[6 + e]);
    }
  }
#pragma unroll
  for (int e = 0; e < 27; ++e) acc[e] = wsum(acc[e]);
#pragma unroll
  for (int e = 0; e < 12; ++e) ph[e] = wsum(ph[e]);
  // every lane holds the totals; all lanes do the (tiny) 4x4 algebra
  ST Ts[9], Tz[9];
  {
    const ST Ps[9] = {ph[0], ph[1], ph[2], ph[1], ph[3], ph[4], ph[2], ph[4], ph[5]};
    const ST Pz[9] = {ph[6], ph[7], ph[8], ph[7], ph[9], ph[10], ph[8], ph[10], ph[11]};
    adjoint_rotation_term<ST>(acc + 18, R, acc, Ps, Ts);
    adjoint_rotation_term<ST>(acc + 18, R, acc + 9, Pz, Tz);
  }
  // alignment weights: -w'_k (2 S + T^T Y_w), S = Gamma X_w - R sum_j w_j beta^y_j
  ST Cs[3] = {0, 0, 0}, Cz[3] = {0, 0, 0};
  if (split) {
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      xw[b] = wsum(xw[b]);
      yw[b] = wsum(yw[b]);
      bws[b] = wsum(bws[b]);
      bwz[b] = wsum(bwz[b]);
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const ST Rbs = R[3 * c] * bws[0] + R[3 * c + 1] * bws[1] + R[3 * c + 2] * bws[2];
      const ST Rbz = R[3 * c] * bwz[0] + R[3 * c + 1] * bwz[1] + R[3 * c + 2] * bwz[2];
      Cs[c] = (ST)2 * (Gs * xw[c] - Rbs) + Ts[c] * yw[0] + Ts[3 + c] * yw[1] + Ts[6 + c] * yw[2];
      Cz[c] = (ST)2 * (Gz * xw[c] - Rbz) + Tz[c] * yw[0] + Tz[3 + c] * yw[1] + Tz[6 + c] * yw[2];
    }
  }
  for (int j = lane; j < N; j += 32) {
    const ST w = wt(j), w2 = split ? wat(j) : ST(0);
    ST v[3], u[3], bsj[3], bzj[3];
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      v[b] = (ST)x[3 * j + b] - cx[b];
      u[b] = (ST)y[3 * j + b] - cy[b];
      bsj[b] = bsp[3 * j + b];
      bzj[b] = bzp[3 * j + b];
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const ST Rbs = R[3 * c] * bsj[0] + R[3 * c + 1] * bsj[1] + R[3 * c + 2] * bsj[2];
      const ST Rbz = R[3 * c] * bzj[0] + R[3 * c + 1] * bzj[1] + R[3 * c + 2] * bzj[2];
      const ST ts = Ts[c] * u[0] + Ts[3 + c] * u[1] + Ts[6 + c] * u[2];
      const ST tz = Tz[c] * u[0] + Tz[3 + c] * u[1] + Tz[6 + c] * u[2];
      bsp[3 * j + c] = (ST)2 * w * (Gs * v[c] - Rbs) + w * ts - w2 * Cs[c];
      bzp[3 * j + c] = (ST)2 * w * (Gz * v[c] - Rbz) + w * tz - w2 * Cz[c];
    }
  }
}

// ---------------------------------------------------------------------------------------
// Per-frame finish for the FP32 modes on structures too large to stage (12 N floats over
// 200 KB: N > 4266 atoms): one block of FB_THREADS per frame, in a persistent grid of
// FB_BLOCKS_PER_SM blocks per SM.  A warp per frame left each 5000-atom frame's passes to
// 32 lanes (17% of the warps active, 25% of the DRAM peak); here 128 threads share them,
// and four blocks per SM let one frame's reductions and 4x4 algebra overlap the other
// frames' passes (5000 atoms, 2000 landmarks, 10k frames: 1.65 -> 1.41 ms).  256-thread
// blocks, 2 per SM, took 1.71 ms; staging the rows through shared memory in coalesced
// chunks, 1.49 ms; unrolling the atom loops, no change.  Gamma comes from Gsum and Phi
// from the segment moments S6 when given (else from P, Bseg and A32); the arithmetic is
// that of adjoint_finish_staged, with block sums in place of warp sums.
constexpr int FB_THREADS = 128, FB_WARPS = FB_THREADS / 32, FB_BLOCKS_PER_SM = 4;
constexpr int FB_SUMS = 51;  // 27 (X^s, X^z, H_xy) + 12 (Phi) + 12 (alignment-weight sums)

// totals of the K per-thread values v over the block, in tot[0..K) (every thread calls it;
// two barriers; red holds FB_WARPS x FB_SUMS floats)
template <int K>
__device__ __forceinline__ void fb_block_sums(const float* v, float (*red)[FB_SUMS], float* tot) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const float t = wsum(v[k]);
    if (lane == 0) red[w][k] = t;
  }
  __syncthreads();
  if ((int)threadIdx.x < K) {
    float t = 0.0f;
    for (int ww = 0; ww < FB_WARPS; ++ww) t += red[ww][threadIdx.x];
    tot[threadIdx.x] = t;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(FB_THREADS)
adjoint_finish_block(int F, int M, int N, const float* __restrict__ frames, const float4* __restrict__ c32,
                     const float* __restrict__ wts, const float* __restrict__ wa, float wuni,
                     const float* __restrict__ A32, const float* __restrict__ q32, const float* __restrict__ P,
                     const double* __restrict__ s, float lambda, const float* __restrict__ Gsum,
                     const float* __restrict__ S6, int seg_base, const float* __restrict__ Bseg,
                     const int* __restrict__ seg_of_frame, FrameRec rec, const float* __restrict__ prior_coords,
                     float4 prior_c, float* __restrict__ gs, float* __restrict__ gz) {
  __shared__ float red[FB_WARPS][FB_SUMS];
  __shared__ float tot[FB_SUMS + 2];  // the sums, then Gamma^s, Gamma^z when not given
  __shared__ float s_T[24];           // Ts, Tz, Cs, Cz
  const int tid = threadIdx.x, N3 = 3 * N;
  for (int f = blockIdx.x; f < F; f += gridDim.x) {
    const float4 c = c32[f];
    const float cx[3] = {c.x, c.y, c.z};
    const float* x = frames + (size_t)f * N3;
    float* gsp = gs + (size_t)f * N3;
    float* gzp = gz + (size_t)f * N3;
    const bool approx = rec.flag && rec.flag[f] == 0;
    const int r = rec.flag ? rec.ref[f] : 0;
    const int seg = rec.flag ? seg_of_frame[f] : 0;
    const float sf = (float)s[f], sl = s_low<float>(s[f], sf);
    // landmarks: Gamma when not given; Phi = sum_i gamma_i S_i at approximate frames
    float lv[14];
#pragma unroll
    for (int e = 0; e < 14; ++e) lv[e] = 0.0f;
    if (approx || !Gsum) {
      for (int i = tid; i < M; i += FB_THREADS) {
        float gsv, gzv;
        gammas<float>(P[(size_t)f * M + i], lambda, q32[i], sf, sl, gsv, gzv);
        lv[12] += gsv;
        lv[13] += gzv;
        if (approx) {
          float S[6];
          if (S6) {
            const float* sp = S6 + ((size_t)(seg - seg_base) * M + i) * 6;
#pragma unroll
            for (int e = 0; e < 6; ++e) S[e] = sp[e];
          } else {
            const float* B = Bseg + ((size_t)seg * M + i) * 9;
            const float* a = A32 + (size_t)i * 6;
            const float A[9] = {a[0], a[1], a[2], a[1], a[3], a[4], a[2], a[4], a[5]};
            float BA[9];
#pragma unroll
            for (int b = 0; b < 3; ++b)
#pragma unroll
              for (int cc = 0; cc < 3; ++cc)
                BA[3 * b + cc] = B[3 * b] * A[cc] + B[3 * b + 1] * A[3 + cc] + B[3 * b + 2] * A[6 + cc];
            const int ib[6] = {0, 0, 0, 1, 1, 2}, ic[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
            for (int e = 0; e < 6; ++e) {
              const int b = ib[e], cc = ic[e];
              S[e] = BA[3 * b] * B[3 * cc] + BA[3 * b + 1] * B[3 * cc + 1] + BA[3 * b + 2] * B[3 * cc + 2];
            }
          }
#pragma unroll
          for (int e = 0; e < 6; ++e) {
            lv[e] = fmaf(gsv, S[e], lv[e]);
            lv[6 + e] = fmaf(gzv, S[e], lv[6 + e]);
          }
        }
      }
    }
    if (!approx) {
      // exact frame: Gamma, and with alignment weights the centre term's sums
      float v[8] = {lv[12], lv[13], 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
      if (wa) {
        for (int j = tid; j < N; j += FB_THREADS) {
          const float wj = wts ? wts[j] : wuni;
#pragma unroll
          for (int b = 0; b < 3; ++b) {
            v[2 + b] = fmaf(wj, x[3 * j + b] - cx[b], v[2 + b]);
            v[5 + b] = fmaf(wj, gsp[3 * j + b], v[5 + b]);
          }
        }
      }
      fb_block_sums<8>(v, red, tot);
      const float Gs = Gsum ? Gsum[2 * f] : tot[0];
      const float Gz = Gsum ? Gsum[2 * f + 1] : tot[1];
      float Ss[3] = {0.0f, 0.0f, 0.0f}, Sz[3] = {0.0f, 0.0f, 0.0f};
      if (wa) {
        float xw[3], bws[3], vz[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
        for (int b = 0; b < 3; ++b) {
          xw[b] = tot[2 + b];
          bws[b] = tot[5 + b];
        }
        // beta^z's weighted sums: a second reduction (tot is rewritten after the barrier)
        for (int j = tid; j < N; j += FB_THREADS) {
          const float wj = wts ? wts[j] : wuni;
#pragma unroll
          for (int b = 0; b < 3; ++b) vz[b] = fmaf(wj, gzp[3 * j + b], vz[b]);
        }
        __syncthreads();  // every thread has read tot
        fb_block_sums<3>(vz, red, tot);
#pragma unroll
        for (int b = 0; b < 3; ++b) {
          Ss[b] = Gs * xw[b] - bws[b];
          Sz[b] = Gz * xw[b] - tot[b];
        }
      }
      for (int e = tid; e < N3; e += FB_THREADS) {
        const float wj = wts ? wts[e / 3] : wuni, w2 = wa ? wa[e / 3] : 0.0f;
        const int b = e - 3 * (e / 3);
        const float xv = x[e] - cx[b];
        gsp[e] = 2.0f * wj * (Gs * xv - gsp[e]) - 2.0f * w2 * Ss[b];
        gzp[e] = 2.0f * wj * (Gz * xv - gzp[e]) - 2.0f * w2 * Sz[b];
      }
      __syncthreads();  // tot is reused by the next frame
      continue;
    }
    const float* y = r >= 0 ? frames + (size_t)r * N3 : prior_coords;
    const float4 cyv = r >= 0 ? c32[r] : prior_c;
    const float cy[3] = {cyv.x, cyv.y, cyv.z};
    // pass 1: X = sum_j w x_j beta_j^T (s, z), H_xy = sum_j w y_j x_j^T, centred, true
    // weights; with alignment weights also X_w, Y_w and the weighted beta sums
    float v[FB_SUMS];
#pragma unroll
    for (int e = 0; e < FB_SUMS; ++e) v[e] = 0.0f;
#pragma unroll
    for (int e = 0; e < 12; ++e) v[27 + e] = lv[e];
#pragma unroll 2
    for (int j = tid; j < N; j += FB_THREADS) {
      const float wj = wts ? wts[j] : wuni;
      float xv[3], u[3], bs[3], bz[3];
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        xv[b] = x[3 * j + b] - cx[b];
        u[b] = y[3 * j + b] - cy[b];
        bs[b] = gsp[3 * j + b];
        bz[b] = gzp[3 * j + b];
      }
      if (wa) {
#pragma unroll
        for (int b = 0; b < 3; ++b) {
          v[39 + b] = fmaf(wj, xv[b], v[39 + b]);
          v[42 + b] = fmaf(wj, u[b], v[42 + b]);
          v[45 + b] = fmaf(wj, bs[b], v[45 + b]);
          v[48 + b] = fmaf(wj, bz[b], v[48 + b]);
        }
      }
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        const float wv = wj * xv[b], wu = wj * u[b];
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) {
          v[3 * b + cc] = fmaf(wv, bs[cc], v[3 * b + cc]);
          v[9 + 3 * b + cc] = fmaf(wv, bz[cc], v[9 + 3 * b + cc]);
          v[18 + 3 * b + cc] = fmaf(wu, xv[cc], v[18 + 3 * b + cc]);
        }
      }
    }
    fb_block_sums<FB_SUMS>(v, red, tot);
    if (!Gsum) {
      const float g2[2] = {lv[12], lv[13]};
      fb_block_sums<2>(g2, red, tot + FB_SUMS);
    }
    const float Gs = Gsum ? Gsum[2 * f] : tot[FB_SUMS];
    const float Gz = Gsum ? Gsum[2 * f + 1] : tot[FB_SUMS + 1];
    const double4 qq = rec.qxy[f];
    const float qxy[4] = {(float)qq.x, (float)qq.y, (float)qq.z, (float)qq.w};
    float R[9];
    quat_to_rot(qxy, R);
    if (tid == 0) {
      float acc[27], Ts[9], Tz[9];
#pragma unroll
      for (int e = 0; e < 27; ++e) acc[e] = tot[e];
      const float Ps[9] = {tot[27], tot[28], tot[29], tot[28], tot[30], tot[31], tot[29], tot[31], tot[32]};
      const float Pz[9] = {tot[33], tot[34], tot[35], tot[34], tot[36], tot[37], tot[35], tot[37], tot[38]};
      adjoint_rotation_terms2<float>(acc + 18, R, qxy, acc, acc + 9, Ps, Pz, Ts, Tz);
      float Cs[3] = {0.0f, 0.0f, 0.0f}, Cz[3] = {0.0f, 0.0f, 0.0f};
      if (wa) {
        // alignment weights: -w'_k (2 S + T^T Y_w), S = Gamma X_w - R sum_j w_j beta^y_j
        const float* xw = tot + 39;
        const float* yw = tot + 42;
        const float* bws = tot + 45;
        const float* bwz = tot + 48;
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) {
          const float Rbs = R[3 * cc] * bws[0] + R[3 * cc + 1] * bws[1] + R[3 * cc + 2] * bws[2];
          const float Rbz = R[3 * cc] * bwz[0] + R[3 * cc + 1] * bwz[1] + R[3 * cc + 2] * bwz[2];
          Cs[cc] = 2.0f * (Gs * xw[cc] - Rbs) + Ts[cc] * yw[0] + Ts[3 + cc] * yw[1] + Ts[6 + cc] * yw[2];
          Cz[cc] = 2.0f * (Gz * xw[cc] - Rbz) + Tz[cc] * yw[0] + Tz[3 + cc] * yw[1] + Tz[6 + cc] * yw[2];
        }
      }
#pragma unroll
      for (int e = 0; e < 9; ++e) {
        s_T[e] = Ts[e];
        s_T[9 + e] = Tz[e];
      }
#pragma unroll
      for (int e = 0; e < 3; ++e) {
        s_T[18 + e] = Cs[e];
        s_T[21 + e] = Cz[e];
      }
    }
    __syncthreads();
    float Ts[9], Tz[9], Cs[3], Cz[3];
#pragma unroll
    for (int e = 0; e < 9; ++e) {
      Ts[e] = s_T[e];
      Tz[e] = s_T[9 + e];
    }
#pragma unroll
    for (int e = 0; e < 3; ++e) {
      Cs[e] = s_T[18 + e];
      Cz[e] = s_T[21 + e];
    }
    // pass 2: the gradient rows over beta
#pragma unroll 2
    for (int j = tid; j < N; j += FB_THREADS) {
      const float wj = wts ? wts[j] : wuni, w2 = wa ? wa[j] : 0.0f;
      float xv[3], u[3], bsj[3], bzj[3];
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        xv[b] = x[3 * j + b] - cx[b];
        u[b] = y[3 * j + b] - cy[b];
        bsj[b] = gsp[3 * j + b];
        bzj[b] = gzp[3 * j + b];
      }
#pragma unroll
      for (int cc = 0; cc < 3; ++cc) {
        const float Rbs = R[3 * cc] * bsj[0] + R[3 * cc + 1] * bsj[1] + R[3 * cc + 2] * bsj[2];
        const float Rbz = R[3 * cc] * bzj[0] + R[3 * cc + 1] * bzj[1] + R[3 * cc + 2] * bzj[2];
        const float ts = Ts[cc] * u[0] + Ts[3 + cc] * u[1] + Ts[6 + cc] * u[2];
        const float tz = Tz[cc] * u[0] + Tz[3 + cc] * u[1] + Tz[6 + cc] * u[2];
        gsp[3 * j + cc] = 2.0f * wj * (Gs * xv[cc] - Rbs) + wj * ts - w2 * Cs[cc];
        gzp[3 * j + cc] = 2.0f * wj * (Gz * xv[cc] - Rbz) + wj * tz - w2 * Cz[cc];
      }
    }
    __syncthreads();  // red, tot and s_T are reused by the next frame
  }
}

// ---------------------------------------------------------------------------------------
// S_i = R_{a_i y} A_i R_{a_i y}^T (xx xy xz yy yz zz) for every landmark of the segments
// [seg_base, seg_base + nseg): the per-landmark part of Phi, shared by a segment's frames.
__global__ void seg_moments_kernel(int seg_base, int nseg, int M, const float* __restrict__ Bseg,
                                   const float* __restrict__ A32, float* __restrict__ S6) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nseg * M) return;
  const int slot = idx / M, i = idx - slot * M;
  const float* B = Bseg + ((size_t)(seg_base + slot) * M + i) * 9;
  const float* a = A32 + (size_t)i * 6;
  const float A[9] = {a[0], a[1], a[2], a[1], a[3], a[4], a[2], a[4], a[5]};
  float Bv[9], BA[9];
#pragma unroll
  for (int e = 0; e < 9; ++e) Bv[e] = B[e];
#pragma unroll
  for (int b = 0; b < 3; ++b)
#pragma unroll
    for (int c = 0; c < 3; ++c) BA[3 * b + c] = Bv[3 * b] * A[c] + Bv[3 * b + 1] * A[3 + c] + Bv[3 * b + 2] * A[6 + c];
  const int ib[6] = {0, 0, 0, 1, 1, 2}, ic[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
  for (int e = 0; e < 6; ++e) {
    const int b = ib[e], c = ic[e];
    S6[(size_t)idx * 6 + e] = BA[3 * b] * Bv[3 * c] + BA[3 * b + 1] * Bv[3 * c + 1] + BA[3 * b + 2] * Bv[3 * c + 2];
  }
}

// Per-frame finish for the FP32 modes, one warp per frame, the frame staged in shared
// memory: x - c, y - c_y, beta^s and beta^z are read from global memory once (coalesced)
// and both passes over the atoms run from shared memory.  Gamma comes from Gsum when the
// gamma kernel produced it (else from P), and Phi from the segment moments S6 when given
// (else from Bseg and A32), with the arithmetic of adjoint_finish_warp except that the top
// eigenvector of K(H_xy) is the stored alignment quaternion q_xy (adjoint_rotation_terms2).
template <bool ASYNC>
__global__ void __launch_bounds__(128)
adjoint_finish_staged(int F, int M, int N, const float* __restrict__ frames, const float4* __restrict__ c32,
                      const float* __restrict__ wts, const float* __restrict__ wa, float wuni,
                      const float* __restrict__ A32,
                      const float* __restrict__ q32, const float* __restrict__ P, const double* __restrict__ s,
                      float lambda, const float* __restrict__ Gsum, const float* __restrict__ S6, int seg_base,
                      const float* __restrict__ Bseg, const int* __restrict__ seg_of_frame, FrameRec rec,
                      const float* __restrict__ prior_coords, float4 prior_c, float* __restrict__ gs,
                      float* __restrict__ gz) {
  extern __shared__ float fsm[];
  const int wpb = blockDim.x >> 5, w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int f = blockIdx.x * wpb + w;
  if (f >= F) return;  // the whole warp leaves; only warp-level synchronisation below
  const int N3 = 3 * N;
  float* xv = fsm + (size_t)w * 4 * N3;  // x (minus c below)
  float* uv = xv + N3;                   // y (minus c_y below; approximate frames)
  float* bs = uv + N3;                   // beta^s
  float* bz = bs + N3;                   // beta^z
  const float4 c = c32[f];
  const float cx[3] = {c.x, c.y, c.z};
  const float* x = frames + (size_t)f * N3;
  float* gsp = gs + (size_t)f * N3;
  float* gzp = gz + (size_t)f * N3;
  // The frame and beta rows are copied first; the per-frame scalars are loaded next (the
  // staging's asm statements are compiler barriers: loads written after them start after
  // them), then the close structure's row once its index is known.
  if (ASYNC) {
    // rows are 16-byte aligned (3N % 4 == 0): every 16-byte piece is in flight at once
    const int n4 = N3 / 4;
    for (int e = lane; e < n4; e += 32) {
      const unsigned o = 16u * e;
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((unsigned)__cvta_generic_to_shared(xv) + o),
                   "l"(x + 4 * e) : "memory");
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((unsigned)__cvta_generic_to_shared(bs) + o),
                   "l"(gsp + 4 * e) : "memory");
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((unsigned)__cvta_generic_to_shared(bz) + o),
                   "l"(gzp + 4 * e) : "memory");
    }
  }
  const bool approx = rec.flag && rec.flag[f] == 0;
  const int r = rec.flag ? rec.ref[f] : 0;
  const float sf = (float)s[f], sl = s_low<float>(s[f], sf);
  float Gs = 0.0f, Gz = 0.0f;
  if (Gsum) {
    Gs = Gsum[2 * f];
    Gz = Gsum[2 * f + 1];
  }
  double4 qq = make_double4(1.0, 0.0, 0.0, 0.0);
  int seg = 0;
  if (rec.flag) {
    qq = rec.qxy[f];
    seg = seg_of_frame[f];
  }
  const float* y = r >= 0 ? frames + (size_t)r * N3 : prior_coords;
  if (ASYNC) {
    if (approx) {
      const int n4 = N3 / 4;
      for (int e = lane; e < n4; e += 32)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(
                         (unsigned)__cvta_generic_to_shared(uv) + 16u * e),
                     "l"(y + 4 * e) : "memory");
    }
  } else {
    for (int e = lane; e < N3; e += 32) {
      const int b = e - 3 * (e / 3);
      xv[e] = x[e] - cx[b];
      bs[e] = gsp[e];
      bz[e] = gzp[e];
      if (approx) uv[e] = y[e];
    }
  }
  const float4 cyv = approx && r >= 0 ? c32[r] : prior_c;
  // Over the landmarks while the copies are in flight (global loads only): Gamma when the
  // gamma kernel did not produce it, and at approximate frames Phi = sum_i gamma_i S_i (s, z)
  float ph[12];
#pragma unroll
  for (int e = 0; e < 12; ++e) ph[e] = 0.0f;
  if (approx || !Gsum) {
    constexpr int U = 4;  // landmarks per lane whose loads are in flight together
    for (int i0 = lane; i0 < M; i0 += 32 * U) {
      float pv[U], qv[U], S[U][6];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int i = i0 + 32 * u;
        const bool ok = i < M;
        pv[u] = ok ? P[(size_t)f * M + i] : 0.0f;
        qv[u] = ok ? q32[i] : 0.0f;
#pragma unroll
        for (int e = 0; e < 6; ++e) S[u][e] = 0.0f;
        if (ok && approx) {
          if (S6) {
            const float* sp = S6 + ((size_t)(seg - seg_base) * M + i) * 6;
#pragma unroll
            for (int e = 0; e < 6; ++e) S[u][e] = sp[e];
          } else {
            const float* B = Bseg + ((size_t)seg * M + i) * 9;
            const float* a = A32 + (size_t)i * 6;
            const float A[9] = {a[0], a[1], a[2], a[1], a[3], a[4], a[2], a[4], a[5]};
            float BA[9];
#pragma unroll
            for (int b = 0; b < 3; ++b)
#pragma unroll
              for (int cc = 0; cc < 3; ++cc)
                BA[3 * b + cc] = B[3 * b] * A[cc] + B[3 * b + 1] * A[3 + cc] + B[3 * b + 2] * A[6 + cc];
            const int ib[6] = {0, 0, 0, 1, 1, 2}, ic[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
            for (int e = 0; e < 6; ++e) {
              const int b = ib[e], cc = ic[e];
              S[u][e] = BA[3 * b] * B[3 * cc] + BA[3 * b + 1] * B[3 * cc + 1] + BA[3 * b + 2] * B[3 * cc + 2];
            }
          }
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        float gsv, gzv;
        gammas<float>(pv[u], lambda, qv[u], sf, sl, gsv, gzv);  // zero for i >= M (p = 0)
        if (!Gsum) {
          Gs += gsv;
          Gz += gzv;
        }
#pragma unroll
        for (int e = 0; e < 6; ++e) {
          ph[e] = fmaf(gsv, S[u][e], ph[e]);
          ph[6 + e] = fmaf(gzv, S[u][e], ph[6 + e]);
        }
      }
    }
    if (!Gsum) {
      Gs = wsum(Gs);
      Gz = wsum(Gz);
    }
  }
  if (ASYNC) {
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncwarp();
    for (int e = lane; e < N3; e += 32) xv[e] -= cx[e - 3 * (e / 3)];
  }
  if (!approx) {
    __syncwarp();
    float Ss[3] = {0.0f, 0.0f, 0.0f}, Sz[3] = {0.0f, 0.0f, 0.0f};  // centre term (alignment weights)
    if (wa) {
      float xw[3] = {0.0f, 0.0f, 0.0f}, bws[3] = {0.0f, 0.0f, 0.0f}, bwz[3] = {0.0f, 0.0f, 0.0f};
      for (int j = lane; j < N; j += 32) {
        const float wj = wts ? wts[j] : wuni;
#pragma unroll
        for (int b = 0; b < 3; ++b) {
          xw[b] = fmaf(wj, xv[3 * j + b], xw[b]);
          bws[b] = fmaf(wj, bs[3 * j + b], bws[b]);
          bwz[b] = fmaf(wj, bz[3 * j + b], bwz[b]);
        }
      }
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        xw[b] = wsum(xw[b]);
        Ss[b] = Gs * xw[b] - wsum(bws[b]);
        Sz[b] = Gz * xw[b] - wsum(bwz[b]);
      }
    }
    for (int e = lane; e < N3; e += 32) {
      const float wj = wts ? wts[e / 3] : wuni, w2 = wa ? wa[e / 3] : 0.0f;
      const int b = e - 3 * (e / 3);
      gsp[e] = 2.0f * wj * (Gs * xv[e] - bs[e]) - 2.0f * w2 * Ss[b];
      gzp[e] = 2.0f * wj * (Gz * xv[e] - bz[e]) - 2.0f * w2 * Sz[b];
    }
    return;
  }
  const float cy[3] = {cyv.x, cyv.y, cyv.z};
  for (int e = lane; e < N3; e += 32) uv[e] -= cy[e - 3 * (e / 3)];
  __syncwarp();
  float R[9], qxy[4];
  qxy[0] = (float)qq.x;
  qxy[1] = (float)qq.y;
  qxy[2] = (float)qq.z;
  qxy[3] = (float)qq.w;
  quat_to_rot(qxy, R);
  // X = sum_j w x_j beta_j^T (s, z) and H_xy = sum_j w y_j x_j^T, centred, true weights
  float acc[27];
#pragma unroll
  for (int e = 0; e < 27; ++e) acc[e] = 0.0f;
  float xw[3] = {0.0f, 0.0f, 0.0f}, yw[3] = {0.0f, 0.0f, 0.0f}, bws[3] = {0.0f, 0.0f, 0.0f},
        bwz[3] = {0.0f, 0.0f, 0.0f};  // alignment weights
#pragma unroll 2
  for (int j = lane; j < N; j += 32) {
    const float wj = wts ? wts[j] : wuni;
    float v[3], u[3];
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      v[b] = xv[3 * j + b];
      u[b] = uv[3 * j + b];
    }
    if (wa) {
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        xw[b] = fmaf(wj, v[b], xw[b]);
        yw[b] = fmaf(wj, u[b], yw[b]);
        bws[b] = fmaf(wj, bs[3 * j + b], bws[b]);
        bwz[b] = fmaf(wj, bz[3 * j + b], bwz[b]);
      }
    }
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const float wv = wj * v[b], wu = wj * u[b];
#pragma unroll
      for (int cc = 0; cc < 3; ++cc) {
        acc[3 * b + cc] = fmaf(wv, bs[3 * j + cc], acc[3 * b + cc]);
        acc[9 + 3 * b + cc] = fmaf(wv, bz[3 * j + cc], acc[9 + 3 * b + cc]);
        acc[18 + 3 * b + cc] = fmaf(wu, v[cc], acc[18 + 3 * b + cc]);
      }
    }
  }
#pragma unroll
  for (int e = 0; e < 27; ++e) acc[e] = wsum(acc[e]);
#pragma unroll
  for (int e = 0; e < 12; ++e) ph[e] = wsum(ph[e]);
  float Ts[9], Tz[9];
  {
    const float Ps[9] = {ph[0], ph[1], ph[2], ph[1], ph[3], ph[4], ph[2], ph[4], ph[5]};
    const float Pz[9] = {ph[6], ph[7], ph[8], ph[7], ph[9], ph[10], ph[8], ph[10], ph[11]};
    adjoint_rotation_terms2<float>(acc + 18, R, qxy, acc, acc + 9, Ps, Pz, Ts, Tz);
  }
  // alignment weights: -w'_k (2 S + T^T Y_w), S = Gamma X_w - R sum_j w_j beta^y_j
  float Cs[3] = {0.0f, 0.0f, 0.0f}, Cz[3] = {0.0f, 0.0f, 0.0f};
  if (wa) {
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      xw[b] = wsum(xw[b]);
      yw[b] = wsum(yw[b]);
      bws[b] = wsum(bws[b]);
      bwz[b] = wsum(bwz[b]);
    }
#pragma unroll
    for (int cc = 0; cc < 3; ++cc) {
      const float Rbs = R[3 * cc] * bws[0] + R[3 * cc + 1] * bws[1] + R[3 * cc + 2] * bws[2];
      const float Rbz = R[3 * cc] * bwz[0] + R[3 * cc + 1] * bwz[1] + R[3 * cc + 2] * bwz[2];
      Cs[cc] = 2.0f * (Gs * xw[cc] - Rbs) + Ts[cc] * yw[0] + Ts[3 + cc] * yw[1] + Ts[6 + cc] * yw[2];
      Cz[cc] = 2.0f * (Gz * xw[cc] - Rbz) + Tz[cc] * yw[0] + Tz[3 + cc] * yw[1] + Tz[6 + cc] * yw[2];
    }
  }
#pragma unroll 2
  for (int j = lane; j < N; j += 32) {
    const float wj = wts ? wts[j] : wuni, w2 = wa ? wa[j] : 0.0f;
    float v[3], u[3], bsj[3], bzj[3];
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      v[b] = xv[3 * j + b];
      u[b] = uv[3 * j + b];
      bsj[b] = bs[3 * j + b];
      bzj[b] = bz[3 * j + b];
    }
#pragma unroll
    for (int cc = 0; cc < 3; ++cc) {
      const float Rbs = R[3 * cc] * bsj[0] + R[3 * cc + 1] * bsj[1] + R[3 * cc + 2] * bsj[2];
      const float Rbz = R[3 * cc] * bzj[0] + R[3 * cc + 1] * bzj[1] + R[3 * cc + 2] * bzj[2];
      const float ts = Ts[cc] * u[0] + Ts[3 + cc] * u[1] + Ts[6 + cc] * u[2];
      const float tz = Tz[cc] * u[0] + Tz[3 + cc] * u[1] + Tz[6 + cc] * u[2];
      gsp[3 * j + cc] = 2.0f * wj * (Gs * v[cc] - Rbs) + wj * ts - w2 * Cs[cc];
      gzp[3 * j + cc] = 2.0f * wj * (Gz * v[cc] - Rbz) + wj * tz - w2 * Cz[cc];
    }
  }
}

}  // namespace

// ---------------------------------------------------------------------------------------
int beta_pair_split(Prec p, int F, int M, int N) {
  const int ctas = ((N + BP_TJ - 1) / BP_TJ) * ((F + BP_TF - 1) / BP_TF);
  if (ctas <= 0 || ctas >= 152) return 1;
  const int kl = p == P_F64 ? 4 : 8;
  const int want = (2 * 152 + ctas - 1) / ctas;     // about two CTAs per SM
  const int most = (M + 2 * kl - 1) / (2 * kl);     // at least two landmark chunks per range
  return want < 1 ? 1 : (want > most ? (most < 1 ? 1 : most) : want);
}

void launch_adjoint_beta(Prec p, int F, const LandmarkDev& L, const void* P, const double* s, double lambda,
                         const void* Rpair, const void* Bseg, const int* seg_of_frame, bool seg_form, void* gs,
                         void* gz, void* part, cudaStream_t st) {
  if (F <= 0) return;
  if (seg_form && p != P_F64) {
    dim3 grid((L.N + BS_TJ - 1) / BS_TJ, (F + BS_TF - 1) / BS_TF);
    if (p == P_F32)
      adjoint_beta_seg<float><<<grid, BS_THREADS, 0, st>>>(F, L.M, L.N, (const float*)L.coords, L.off, L.q32,
                                                           (const float*)P, s, (float)lambda, (const float*)Bseg,
                                                           seg_of_frame, (float*)gs, (float*)gz);
    else
      adjoint_beta_seg<__half><<<grid, BS_THREADS, 0, st>>>(F, L.M, L.N, (const __half*)L.coords, L.off, L.q32,
                                                            (const float*)P, s, (float)lambda, (const float*)Bseg,
                                                            seg_of_frame, (float*)gs, (float*)gz);
    note_launch();
    return;
  }
  const int nsplit = part ? beta_pair_split(p, F, L.M, L.N) : 1;
  void* out = nsplit > 1 ? part : nullptr;
  dim3 grid((L.N + BP_TJ - 1) / BP_TJ, (F + BP_TF - 1) / BP_TF, nsplit);
  switch (p) {
    case P_F64:
      adjoint_beta_pair<double, double><<<grid, BP_THREADS, 0, st>>>(
          F, L.M, L.N, (const double*)L.coords, nullptr, L.q, L.q32, (const double*)P, s, lambda, (const double*)Rpair,
          (const double*)Bseg, seg_of_frame, (double*)gs, (double*)gz, (double*)out);
      break;
    case P_F32:
      adjoint_beta_pair<float, float><<<grid, BP_THREADS, 0, st>>>(
          F, L.M, L.N, (const float*)L.coords, L.off, L.q, L.q32, (const float*)P, s, lambda, (const float*)Rpair,
          (const float*)Bseg, seg_of_frame, (float*)gs, (float*)gz, (float*)out);
      break;
    case P_F16:
      adjoint_beta_pair<float, __half><<<grid, BP_THREADS, 0, st>>>(
          F, L.M, L.N, (const __half*)L.coords, L.off, L.q, L.q32, (const float*)P, s, lambda, (const float*)Rpair,
          (const float*)Bseg, seg_of_frame, (float*)gs, (float*)gz, (float*)out);
      break;
  }
  note_launch();
  if (nsplit > 1) {
    const size_t total = (size_t)F * L.N * 6;
    const int blocks = (int)std::min<size_t>((total + 255) / 256, 152 * 4);
    if (p == P_F64)
      beta_pair_part_sum<double><<<blocks, 256, 0, st>>>(F, L.N, nsplit, (const double*)part, (double*)gs, (double*)gz);
    else
      beta_pair_part_sum<float><<<blocks, 256, 0, st>>>(F, L.N, nsplit, (const float*)part, (float*)gs, (float*)gz);
    note_launch();
  }
}

int nl_beta_split(int max_upd, int M, int N) {
  const int ctas = ((max_upd + BL_TF - 1) / BL_TF) * ((N + BL_TJ - 1) / BL_TJ);
  if (ctas <= 0) return 1;
  const int want = (2 * 152 * 4 + ctas - 1) / ctas;  // about two waves of 4 CTAs per SM
  const int most = (M + 8 * BL_KL - 1) / (8 * BL_KL);  // at least 64 landmarks per range
  return want < 1 ? 1 : (want > most ? (most < 1 ? 1 : most) : want);
}

void launch_nl_beta_tiles(Prec p, int max_upd, int max_tiles, const NlLists& nl, const NlTile* tiles, const int* NLtab,
                          int Mnl, const LandmarkDev& L, const void* P, const double* s, double lambda,
                          const void* Rupd, const void* Rnl, const void* Bseg, const int* segof, void* gs, void* gz,
                          float* part, cudaStream_t st) {
  if (p == P_F64) return;
  const unsigned gx = (unsigned)((L.N + BL_TJ - 1) / BL_TJ);
  const int nsplit = nl_beta_split(max_upd, L.M, L.N);
  for (int mode = 0; mode < 2; ++mode) {
    const int ny = mode == 0 ? (max_upd + BL_TF - 1) / BL_TF : max_tiles;
    if (ny <= 0) continue;
    dim3 grid(gx, ny, mode == 0 ? nsplit : 1);
    float* pt = mode == 0 ? part : nullptr;
    if (p == P_F32)
      adjoint_beta_list<float><<<grid, BL_THREADS, 0, st>>>(
          mode, tiles, nl.counts, nl.ulist, nl.nlist, NLtab, Mnl, L.M, L.N, (const float*)L.coords, L.off, L.q32,
          (const float*)P, s, (float)lambda, (const float*)Rupd, (const float*)Rnl, (const float*)Bseg, segof,
          (float*)gs, (float*)gz, pt);
    else
      adjoint_beta_list<__half><<<grid, BL_THREADS, 0, st>>>(
          mode, tiles, nl.counts, nl.ulist, nl.nlist, NLtab, Mnl, L.M, L.N, (const __half*)L.coords, L.off, L.q32,
          (const float*)P, s, (float)lambda, (const float*)Rupd, (const float*)Rnl, (const float*)Bseg, segof,
          (float*)gs, (float*)gz, pt);
    note_launch();
    if (mode == 0) {
      beta_part_sum<<<4 * 152, 256, 0, st>>>(nl.counts, nl.ulist, L.N, nsplit, part, (float*)gs, (float*)gz);
      note_launch();
    }
  }
}

void launch_seg_moments(int seg_base, int nseg, const LandmarkDev& L, const float* Bseg, float* S6, cudaStream_t st) {
  if (nseg <= 0 || L.M <= 0) return;
  const int n = nseg * L.M;
  seg_moments_kernel<<<(n + 255) / 256, 256, 0, st>>>(seg_base, nseg, L.M, Bseg, L.A32, S6);
  note_launch();
}

void launch_adjoint_finish(Prec p, int F, const void* frames, const LandmarkDev& L, FrameInfo fi, const void* P,
                           const double* s, double lambda, const void* Bseg, const int* seg_of_frame,
                           const FrameRec rec, const RefDesc& prior, void* gs, void* gz, cudaStream_t st,
                           const float* Gsum, const float* S6, int seg_base) {
  if (F <= 0) return;
  // FP32 modes: frames staged in shared memory (4 arrays of 3N floats per warp)
  const size_t per_warp = (size_t)12 * L.N * sizeof(float);
  if (p != P_F64 && per_warp <= 200 * 1024) {
    const bool async = (3 * L.N) % 4 == 0 && ((uintptr_t)frames % 16) == 0 && ((uintptr_t)gs % 16) == 0 &&
                       ((uintptr_t)gz % 16) == 0 && ((uintptr_t)prior.coords % 16) == 0;
    // warps per block: the most resident warps per SM (shared memory and registers both
    // limit them), larger blocks on ties
    thread_local size_t memo_bytes = 0;
    thread_local bool memo_async = false;
    thread_local int memo_wpb = 0;
    int wpb = 1, best = -1;
    if (memo_wpb > 0 && memo_bytes == per_warp && memo_async == async) {
      wpb = memo_wpb;
      best = 0;
    }
    for (int k = best < 0 ? 4 : 0; k >= 1; --k) {
      const size_t sm_k = per_warp * k;
      if (sm_k > 200 * 1024) continue;
      int nb = 0;
      if (async) {
        cudaFuncSetAttribute(adjoint_finish_staged<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_k);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, adjoint_finish_staged<true>, 32 * k, sm_k);
      } else {
        cudaFuncSetAttribute(adjoint_finish_staged<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_k);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, adjoint_finish_staged<false>, 32 * k, sm_k);
      }
      if (nb * k > best) {
        best = nb * k;
        wpb = k;
      }
    }
    memo_bytes = per_warp;
    memo_async = async;
    memo_wpb = wpb;
    const size_t smem = per_warp * wpb;
    const unsigned blocks = (unsigned)((F + wpb - 1) / wpb);
    if (async) {  // the attribute is set for every launch: the search above changed it
      cudaFuncSetAttribute(adjoint_finish_staged<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      adjoint_finish_staged<true><<<blocks, 32 * wpb, smem, st>>>(
          F, L.M, L.N, (const float*)frames, fi.c32, L.w, L.wa, (float)L.dscale, L.A32, L.q32, (const float*)P, s,
          (float)lambda, Gsum, S6, seg_base, (const float*)Bseg, seg_of_frame, rec, (const float*)prior.coords,
          prior.c32, (float*)gs, (float*)gz);
    } else {
      cudaFuncSetAttribute(adjoint_finish_staged<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      adjoint_finish_staged<false><<<blocks, 32 * wpb, smem, st>>>(
          F, L.M, L.N, (const float*)frames, fi.c32, L.w, L.wa, (float)L.dscale, L.A32, L.q32, (const float*)P, s,
          (float)lambda, Gsum, S6, seg_base, (const float*)Bseg, seg_of_frame, rec, (const float*)prior.coords,
          prior.c32, (float*)gs, (float*)gz);
    }
    note_launch();
    return;
  }
  if (p != P_F64) {  // too large to stage: a block per frame
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const unsigned blocks = (unsigned)std::min<long long>(F, (long long)FB_BLOCKS_PER_SM * std::max(sms, 1));
    adjoint_finish_block<<<blocks, FB_THREADS, 0, st>>>(
        F, L.M, L.N, (const float*)frames, fi.c32, L.w, L.wa, (float)L.dscale, L.A32, L.q32, (const float*)P, s,
        (float)lambda, Gsum, S6, seg_base, (const float*)Bseg, seg_of_frame, rec, (const float*)prior.coords,
        prior.c32, (float*)gs, (float*)gz);
    note_launch();
    return;
  }
  const unsigned blocks = (unsigned)((F + 3) / 4);  // FP64: a warp per frame
  adjoint_finish_warp<double, double><<<blocks, 128, 0, st>>>(
      F, L.M, L.N, (const double*)frames, fi.c32, fi.c64, L.w, L.w64, L.wa, L.wa64, L.A32, L.A, L.q, L.q32, L.dscale,
      (const double*)P, s, lambda, (const double*)Bseg, seg_of_frame, rec, (const double*)prior.coords, prior.c64,
      (double*)gs, (double*)gz);
  note_launch();
}

}  // namespace pcv

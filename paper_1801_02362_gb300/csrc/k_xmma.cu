// k_xmma.cu -- the approximate MSDs of Eq. (close_dist) on the tensor cores.
//
// On materialised deviations (see k_tile.cu) the approximate MSD of frame k and landmark i
// of the frame's segment is
//   D~_ki = (|dx_k|^2 + |d_i|^2 - 2 dx_k . d_i) / N,
// and the cross terms dx_k . d_i of a segment form a dense product: approximate frames x
// landmarks, contracted over K = 3 N16 deviation components.  It runs as tcgen05.mma
// kind::f16 with two measures for FP32 accuracy:
//   * split operands: every deviation v is scaled by 2^8 (exact) and split v' = h + l with
//     h = fp16(v') and l = fp16(v' - h), so h + l carries ~22 significant bits; the product
//     is h h' + h l' + l h' (three MMAs, products exact in the FP32 accumulator; the dropped
//     l l' is ~2^-22 relative).  With the 2^8 scale, h + l is within 2^-22 of v' for every
//     deviation of at least ~5e-4 nm (l is often subnormal there: the absolute spacing 2^-24
//     of FP16 subnormals is what bounds it), and deviations below ~255.9 nm stay finite
//     (2^8 v below 65504, the largest FP16);
//   * short accumulation chains: each accumulation into a tensor-memory accumulator
//     loses up to about one unit in the last place of the running sum, so the main
//     products h h' go to an accumulator that only ever sums a group of a few chunks of 16
//     components (one MMA each); then fold warps add it into Kahan-compensated FP32 totals
//     in registers (total and running correction, so the hundreds of folds of a long row
//     add no rounding of the running total) while the other accumulator buffer takes the
//     next group.  The correction products h l' + l h', 2^-11 of the main ones, go to a
//     third accumulator that sums the whole row and is folded once at the end: its
//     roundings are 2^-11 smaller, and the main accumulator takes one addition per chunk
//     instead of three, so a group can be three times as long for the same accuracy and
//     the fold (four FP32 operations per column) runs a third as often.  Two registers per
//     column limit a tile to 128 landmarks.
// Operands are packed once per step (pack_deviations_kernel writes the landmarks' operand
// together with the segment adjoint's, pack_frames_kernel the frames') in the canonical
// K-major layout without swizzling
// (core matrices of 8 rows x 8 halves = 128 contiguous bytes; LBO 128 B along K, SBO 256 B
// between 8-row groups): per chunk of 16 components a block of rows x 16 holding the h part
// then the l part.  A (approximate frames) is tiled per segment: the approximate frames of
// a segment (consecutive in the approximate list) fill tiles of up to 128 rows, listed by
// xmma_tiles_kernel; B (landmarks) per segment in column tiles of BN landmarks.  So every
// tile is one segment's product and takes one pass over K.  One thread moves a stage (A
// block and B block) with two cp.async.bulk copies counted on an mbarrier; one thread
// issues the MMAs; tcgen05.commit releases a stage, and marks an accumulator full.  Every
// wait is bounded by the context's
// clock budget; on expiry the kernel records STATUS_TIMEOUT, waits for its own copies and
// MMAs within the default budget, frees its tensor memory and returns.
#include <cuda_fp16.h>

#include <algorithm>
#include <cstdint>

#include "pcv_device.cuh"
#include "pcv_internal.h"
#include "tc_sm100.cuh"

namespace pcv {
namespace {

constexpr int XM_ROWS = 128;     // MMA M: approximate frames per tile
constexpr int XM_BN_MAX = 128;   // landmarks per tile (MMA N), multiple of 16
constexpr int XM_KC = 16;        // components per chunk: one MMA (K = 16) per product
constexpr int XM_STAGES = 12;    // 16 KB each: about 1.3 us of MMAs in flight
constexpr int XM_GROUP_MAX = 16;  // chunks summed in tensor memory before a fold (the
                                  // context's PCV_OPT_MMA_GROUP, 1..16)
constexpr int XM_FOLD_WARPS = 8;  // two per tensor-memory lane quarter (column halves)
constexpr int XM_THREADS = 32 * (XM_FOLD_WARPS + 2);  // + the copy warp and the MMA warp
constexpr int XM_TMEM_COLS = 4 * XM_BN_MAX;           // two main accumulators, the corrections'
                                                      // (and one unused: a power of two)
constexpr uint32_t XM_A_PART = XM_ROWS * XM_KC * 2;   // bytes of the h (or l) part of an A block
constexpr uint32_t XM_STAGE_BYTES = 2 * XM_A_PART + 2 * XM_BN_MAX * XM_KC * 2;
constexpr float XM_SCALE = 256.0f;              // 2^8 on every operand
constexpr float XM_UNSCALE2 = 1.0f / 65536.0f;  // 2^-16 on the products
constexpr long long XM_DRAIN_CYCLES = 4000000000LL;

// byte offset, inside the h part of a block, of row r and components 8 (p & 1) .. +7 of the
// block (a 16-byte core-matrix row)
__host__ __device__ __forceinline__ uint32_t xpiece_off(int r, int p) {
  return (uint32_t)((r >> 3) * 256 + (p & 1) * 128 + (r & 7) * 16);
}

// Tiles of the approximate frames, per segment: segment slot s holds the rows
// [first_s, first_s + n_s) of the approximate list (aseg is non-decreasing), which fill
// ceil(n_s / 128) tiles numbered from tile_start[s].  One block: binary searches for the
// ranges, then an exclusive scan of the tile counts over the slots.
constexpr int XT_THREADS = 1024;
__global__ void __launch_bounds__(XT_THREADS)
xmma_tiles_kernel(const int* __restrict__ acount, const int* __restrict__ aseg, int seg_base, int nseg,
                  int* __restrict__ seg_first, int* __restrict__ tile_start, XTile* __restrict__ tiles,
                  int* __restrict__ ntiles) {
  __shared__ int scan[XT_THREADS];
  __shared__ int s_carry;
  const int count = *acount, tid = threadIdx.x;
  if (tid == 0) s_carry = 0;
  __syncthreads();
  for (int s0 = 0; s0 < nseg; s0 += XT_THREADS) {
    const int slot = s0 + tid;
    int first = 0, n = 0;
    if (slot < nseg) {
      const int seg = seg_base + slot;
      int lo = 0, hi = count;  // lower bound of seg
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (aseg[mid] < seg) lo = mid + 1; else hi = mid;
      }
      first = lo;
      hi = count;  // lower bound of seg + 1
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (aseg[mid] < seg + 1) lo = mid + 1; else hi = mid;
      }
      n = lo - first;
    }
    const int nt = (n + XM_ROWS - 1) / XM_ROWS;
    scan[tid] = nt;
    __syncthreads();
    for (int off = 1; off < XT_THREADS; off <<= 1) {  // inclusive scan
      const int v = tid >= off ? scan[tid - off] : 0;
      __syncthreads();
      scan[tid] += v;
      __syncthreads();
    }
    const int t0 = s_carry + scan[tid] - nt;
    if (slot < nseg) {
      seg_first[slot] = first;
      tile_start[slot] = t0;
      for (int q = 0; q < nt; ++q) {
        XTile tl;
        tl.slot = slot;
        tl.k0 = first + q * XM_ROWS;
        tl.k1 = min(first + n, tl.k0 + XM_ROWS);
        tiles[t0 + q] = tl;
      }
    }
    __syncthreads();
    if (tid == XT_THREADS - 1) s_carry += scan[tid];
    __syncthreads();
  }
  if (tid == 0) *ntiles = s_carry;
}

// Frame deviations dx_k = R_xy^T (x_k - c) - y'(s) of the approximate frames (rows of the
// approximate list), scaled by 2^8 and split into FP16 h + l, in the tiles of their segments
// (xmma_tiles_kernel), with |dx_k|^2 in Nx[k].  A block takes 8 consecutive rows, one warp
// per row: per slice of 128 atoms each warp reads its frame's coordinates and its
// segment's y' coalesced, writes the 384 split values into shared memory, and then the
// block writes 16-byte core-matrix rows (8 components of one row), eight threads to a
// 128-byte core matrix.  Components beyond 3N up to 3 N16 are zeros.
constexpr int PF_ATOMS = 128, PF_COMP = 3 * PF_ATOMS, PF_LD = PF_COMP + 8;
__global__ void __launch_bounds__(256)
pack_frames_kernel(const int* __restrict__ acount, const int* __restrict__ alist, const int* __restrict__ aseg,
                   int seg_base, int N, int N16, const float* __restrict__ frames, const float4* __restrict__ c32,
                   const double4* __restrict__ qxy, const float* __restrict__ Yc, const int* __restrict__ seg_first,
                   const int* __restrict__ tile_start, uint8_t* __restrict__ Ap, float* __restrict__ Nx) {
  __shared__ __align__(16) __half sh[8][PF_LD], sl[8][PF_LD];
  __shared__ int s_ti[8], s_r[8];
  const int count = *acount;
  const int g = blockIdx.x;
  if (8 * g >= count) return;  // uniform over the block
  const int tid = threadIdx.x, u = tid >> 5, lane = tid & 31;
  const int k = 8 * g + u;
  const bool live = k < count;
  float R[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
  float4 c = make_float4(0.f, 0.f, 0.f, 0.f);
  const float* x = frames;
  const float* y = Yc;
  if (live) {
    const int f = alist[k];
    const double4 qq = qxy[f];
    const float qf[4] = {(float)qq.x, (float)qq.y, (float)qq.z, (float)qq.w};
    quat_to_rot(qf, R);
    c = c32[f];
    x = frames + (size_t)f * N * 3;
    y = Yc + (size_t)(aseg[k] - seg_base) * 3 * N;
  }
  if (lane == 0) {
    int ti = 0, r = 0;
    if (live) {
      const int slot = aseg[k] - seg_base, off = k - seg_first[slot];
      ti = tile_start[slot] + off / XM_ROWS;
      r = off % XM_ROWS;
    }
    s_ti[u] = live ? ti : -1;
    s_r[u] = r;
  }
  const int K = 3 * N16, nck = K / XM_KC;
  float nrm = 0.0f;
  __syncthreads();
  for (int c0 = 0; c0 < K; c0 += PF_COMP) {
    const int j0 = c0 / 3;
#pragma unroll
    for (int it = 0; it < PF_ATOMS / 32; ++it) {
      const int a = lane + 32 * it, j = j0 + a;
      float d[3] = {0.0f, 0.0f, 0.0f};
      if (live && j < N) {
        const float v0 = x[3 * j] - c.x, v1 = x[3 * j + 1] - c.y, v2 = x[3 * j + 2] - c.z;
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) d[cc] = (R[cc] * v0 + R[3 + cc] * v1 + R[6 + cc] * v2) - y[3 * j + cc];
      }
#pragma unroll
      for (int cc = 0; cc < 3; ++cc) {
        nrm = fmaf(d[cc], d[cc], nrm);
        const float v = d[cc] * XM_SCALE;
        const __half h = __float2half_rn(v);
        sh[u][3 * a + cc] = h;
        sl[u][3 * a + cc] = __float2half_rn(v - __half2float(h));
      }
    }
    __syncthreads();
    for (int e = tid; e < 8 * (PF_COMP / 8); e += 256) {
      const int rr = e & 7, pp = e >> 3, comp = c0 + 8 * pp;
      const int ti = s_ti[rr];
      if (comp >= K || ti < 0) continue;
      const int gp = comp / 8;  // global piece index of the row
      uint8_t* blk = Ap + ((size_t)ti * nck + gp / 2) * 2 * XM_A_PART;
      *reinterpret_cast<uint4*>(blk + xpiece_off(s_r[rr], gp)) = *reinterpret_cast<const uint4*>(&sh[rr][8 * pp]);
      *reinterpret_cast<uint4*>(blk + XM_A_PART + xpiece_off(s_r[rr], gp)) =
          *reinterpret_cast<const uint4*>(&sl[rr][8 * pp]);
    }
    __syncthreads();
  }
  nrm = warp_sum_float(nrm);
  if (lane == 0 && live) Nx[k] = nrm;
}

// Landmark deviations of every segment for both tensor-core products, computed once:
// d_i = R_{a_i y(s)} a_i - y'(s) of segment slot s = blockIdx.x (segment s0 + s; y is the
// prior structure for segment 0, else frame refresh_list[seg - 1]) for the landmarks
// 8 g .. 8 g + 7 (g = blockIdx.y), scaled by 2^8 and split into FP16 h + l, written as
//   * Bx, the approximate MSDs' landmark operand (rows landmarks, K components: column tile
//     i / BNx, row i % BNx), with |d_i|^2 in Nb[s * M + i];
//   * Ba (when not null), the adjoint's deviation operand (rows components, K landmarks:
//     column tile n / BNa, row n % BNa, K block i / 16);
// and y'(s) in Yc[s] (block g = 0).  Per slice of 128 atoms the block computes the 8 x 384
// values into shared memory, then writes the 16-byte core-matrix rows of both layouts (8
// components of one landmark; 8 landmarks of one component), eight threads to a 128-byte
// core matrix.  Landmarks >= M and components beyond 3N are written as zeros up to each
// layout's padded extent, so neither buffer needs clearing.  Segments are the fastest grid
// index, so the blocks resident together share one group's landmark rows.
// smem row stride 392 halves (784 B): 16-byte aligned rows, and the 8 rows of a column fall
// in 8 distinct banks
constexpr int PD_ATOMS = 128, PD_COMP = 3 * PD_ATOMS, PD_LD = PD_COMP + 8;
template <typename LT>
__global__ void __launch_bounds__(256)
pack_deviations_kernel(int s0, int M, int N, int N16, int BNx, int NTx, int BNa, int NTa, int Kpa,
                       const LT* __restrict__ lm, const float* __restrict__ lmoff, const float* __restrict__ Bseg,
                       const float* __restrict__ frames, const float4* __restrict__ c32,
                       const int* __restrict__ refresh_list, const float* __restrict__ prior, float4 prior_c,
                       uint8_t* __restrict__ Bx, float* __restrict__ Nb, uint8_t* __restrict__ Ba,
                       float* __restrict__ Yc) {
  __shared__ __align__(16) __half sh[8][PD_LD], sl[8][PD_LD];
  __shared__ float sR[8][9];
  __shared__ float red[8][8];
  const int slot = blockIdx.x, g = blockIdx.y, seg = s0 + slot;
  const int tid = threadIdx.x;
  const float* y;
  float4 c;
  if (seg == 0) {
    y = prior;
    c = prior_c;
  } else {
    const int f = refresh_list[seg - 1];
    y = frames + (size_t)f * 3 * N;
    c = c32[f];
  }
  if (tid < 72) {
    const int u = tid / 9, e = tid % 9, i = 8 * g + u;
    sR[u][e] = i < M ? Bseg[((size_t)seg * M + i) * 9 + e] : 0.0f;
  }
  const int Kx = 3 * N16, NRa = NTa * BNa;
  const int KX = max(Kx, Ba ? NRa : 0);  // components covered
  const bool wx = 8 * g < NTx * BNx, wa = Ba != nullptr && 8 * g < Kpa;
  const int nckx = Kx / XM_KC, nkba = Kpa / 16;
  const uint32_t bpx = (uint32_t)BNx * XM_KC * 2, bpa = (uint32_t)BNa * 16 * 2;  // bytes of one part of a block
  float nrm[4] = {0.0f, 0.0f, 0.0f, 0.0f};  // shares of |d|^2 of landmarks 2 it + (tid >> 7)
  __syncthreads();
  for (int c0 = 0; c0 < KX; c0 += PD_COMP) {
    const int j0 = c0 / 3;
    // 8 landmarks x 128 atoms: thread -> (landmark 2 it + (tid >> 7), atom tid & 127)
#pragma unroll
    for (int it = 0; it < 4; ++it) {
      const int u = 2 * it + (tid >> 7), a = tid & 127, j = j0 + a, i = 8 * g + u;
      float d[3] = {0.0f, 0.0f, 0.0f};
      if (j < N) {
        const float yv[3] = {y[3 * j] - c.x, y[3 * j + 1] - c.y, y[3 * j + 2] - c.z};
        if (g == 0 && u == 0 && Yc) {
#pragma unroll
          for (int cc = 0; cc < 3; ++cc) Yc[(size_t)slot * 3 * N + 3 * j + cc] = yv[cc];
        }
        if (i < M) {
          const float a0 = lm_coord<float, LT>(lm, lmoff, N, i, j, 0);
          const float a1 = lm_coord<float, LT>(lm, lmoff, N, i, j, 1);
          const float a2 = lm_coord<float, LT>(lm, lmoff, N, i, j, 2);
#pragma unroll
          for (int cc = 0; cc < 3; ++cc)
            d[cc] = (sR[u][3 * cc] * a0 + sR[u][3 * cc + 1] * a1 + sR[u][3 * cc + 2] * a2) - yv[cc];
        }
      }
#pragma unroll
      for (int cc = 0; cc < 3; ++cc) {
        nrm[it] = fmaf(d[cc], d[cc], nrm[it]);
        const float v = d[cc] * XM_SCALE;
        const __half h = __float2half_rn(v);
        sh[u][3 * a + cc] = h;
        sl[u][3 * a + cc] = __float2half_rn(v - __half2float(h));
      }
    }
    __syncthreads();
    // the approximate MSDs' layout: piece (landmark rr, 8 components pp of the slice)
    if (wx) {
      for (int e = tid; e < 8 * (PD_COMP / 8); e += 256) {
        const int rr = e & 7, pp = e >> 3, comp = c0 + 8 * pp;
        if (comp >= Kx) continue;
        const int i = 8 * g + rr, gp = comp / 8;  // global piece index of the row
        const uint4 hv = *reinterpret_cast<const uint4*>(&sh[rr][8 * pp]);
        const uint4 lv = *reinterpret_cast<const uint4*>(&sl[rr][8 * pp]);
        uint8_t* blk = Bx + (((size_t)slot * NTx + i / BNx) * nckx + gp / 2) * 2 * bpx;
        *reinterpret_cast<uint4*>(blk + xpiece_off(i % BNx, gp)) = hv;
        *reinterpret_cast<uint4*>(blk + bpx + xpiece_off(i % BNx, gp)) = lv;
      }
    }
    // the adjoint's layout: piece (component n, the 8 landmarks)
    if (wa) {
      for (int e = tid; e < PD_COMP; e += 256) {
        const int n = c0 + e;
        if (n >= NRa) continue;
        uint32_t hw[4], lw[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          hw[q] = (uint32_t)__half_as_ushort(sh[2 * q][e]) | ((uint32_t)__half_as_ushort(sh[2 * q + 1][e]) << 16);
          lw[q] = (uint32_t)__half_as_ushort(sl[2 * q][e]) | ((uint32_t)__half_as_ushort(sl[2 * q + 1][e]) << 16);
        }
        const int nt = n / BNa, r = n % BNa, kk0 = (8 * g) % 16;
        uint8_t* blk = Ba + (((size_t)slot * NTa + nt) * nkba + (8 * g) / 16) * 2 * bpa;
        const uint32_t off = (uint32_t)((r >> 3) * 256 + (kk0 >> 3) * 128 + (r & 7) * 16);
        *reinterpret_cast<uint4*>(blk + off) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
        *reinterpret_cast<uint4*>(blk + bpa + off) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
      }
    }
    __syncthreads();
  }
  // |d_i|^2: warps 0-3 held landmarks 0, 2, 4, 6 (one per it), warps 4-7 landmarks 1, 3, 5, 7
  const int w = tid >> 5, lane = tid & 31;
#pragma unroll
  for (int it = 0; it < 4; ++it) {
    const float v = warp_sum_float(nrm[it]);
    if (lane == 0) red[w][it] = v;
  }
  __syncthreads();
  if (tid < 8) {
    const int it = tid >> 1, hw = tid & 1, i = 8 * g + tid;
    float sum = 0.0f;
    for (int k = 0; k < 4; ++k) sum += red[4 * hw + k][it];
    if (i < M) Nb[(size_t)slot * M + i] = sum;
  }
}

struct XmmaArgs {
  const int* alist;
  const XTile* tiles;
  const int* ntiles;
  int M, nck, BN, NT;
  const uint8_t* Ap;
  const uint8_t* Bp;
  const float* Nx;
  const float* Nb;
  float dscale;
  float* Dout;
  unsigned* status;
  long long wait_cycles;
  int group;  // chunks per accumulator group (1..XM_GROUP_MAX)
};

// Tile (column tile blockIdx.x of BN landmarks, row tile blockIdx.y: entry blockIdx.y of
// the per-segment tile list, up to 128 approximate frames of one segment).  Warps 0-7 fold the accumulators and write D~ (warp w: tensor-memory lanes
// 32 (w & 3) .. + 31, i.e. those rows, and column half w >> 2); warp 8 lane 0 moves the
// operands; warp 9 lane 0 issues the MMAs.
__global__ void __launch_bounds__(XM_THREADS, 1) approx_cross_mma(XmmaArgs p) {
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ __align__(8) uint64_t full[XM_STAGES], empty[XM_STAGES], accf[2], acce[2], done;
  __shared__ uint32_t tmem_slot;
  __shared__ int s_frame[XM_ROWS];
  __shared__ int s_fail, s_fail_run, s_issued;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int n = blockIdx.x, t = blockIdx.y;
  if (t >= *p.ntiles) return;  // uniform over the block, before any allocation
  const XTile tl = p.tiles[t];
  const int row0 = tl.k0, nrows = tl.k1 - tl.k0;
  const int BN = p.BN, nck = p.nck;
  const int G = p.group;
  const int ngrp = (nck + G - 1) / G;
  const uint32_t b_part = (uint32_t)BN * XM_KC * 2;
  const uint32_t idesc = idesc_make(XM_ROWS, BN, 0u);  // kind::f16, F16 operands

  if (warp == 0) tmem_alloc(&tmem_slot, XM_TMEM_COLS);
  if (tid == 0) {
    for (int s = 0; s < XM_STAGES; ++s) {
      mbar_init(smem_u32(&full[s]), 1);
      mbar_init(smem_u32(&empty[s]), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_u32(&accf[b]), 1);
      mbar_init(smem_u32(&acce[b]), XM_FOLD_WARPS);
    }
    mbar_init(smem_u32(&done), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_fail = 0;
    s_issued = 0;
  }
  if (tid < XM_ROWS) s_frame[tid] = tid < nrows ? p.alist[row0 + tid] : -1;
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  const int nrun = 1;  // the tile's rows share one segment: one pass over K
  const uint32_t sbase = smem_u32(smem);
  const uint8_t* Ab = p.Ap + (size_t)t * nck * 2 * XM_A_PART;
  // fold warps: lane quarter and column range
  const int q = warp & 3;
  const int cw = ((BN / 2) + 15) / 16 * 16;
  const int col0 = (warp >> 2) ? cw : 0;
  const int ncol = (warp >> 2) ? BN - cw : cw;

  for (int run = 0; run < nrun; ++run) {
    const int k = 0, kend = nrows;
    const int slot = tl.slot;
    const uint8_t* Bb = p.Bp + (((size_t)slot * p.NT + n) * nck) * 2 * b_part;
    const int g0 = run * nck;    // chunks before this run (stage / phase bookkeeping)
    const int gg0 = run * ngrp;  // accumulator groups before this run
    if (warp == XM_FOLD_WARPS) {
      if (lane == 0) {  // copies
        for (int c = 0; c < nck; ++c) {
          const int g = g0 + c, st = g % XM_STAGES;
          if (g >= XM_STAGES &&
              !mbar_wait(smem_u32(&empty[st]), (uint32_t)((g / XM_STAGES - 1) & 1), p.wait_cycles)) {
            s_fail = 1;
            break;
          }
          const uint32_t dst = sbase + st * XM_STAGE_BYTES;
          mbar_expect_tx(smem_u32(&full[st]), 2 * XM_A_PART + 2 * b_part);
          bulk_g2s(dst, Ab + (size_t)c * 2 * XM_A_PART, 2 * XM_A_PART, smem_u32(&full[st]));
          bulk_g2s(dst + 2 * XM_A_PART, Bb + (size_t)c * 2 * b_part, 2 * b_part, smem_u32(&full[st]));
          s_issued = g + 1;
        }
      }
      __syncwarp();
    } else if (warp == XM_FOLD_WARPS + 1) {
      if (lane == 0) {  // MMA issue
        bool failed = false;
        const uint64_t dA0 = smem_desc(sbase, 128, 256);
        const uint32_t full_b = smem_u32(&full[0]);
        int st_m = g0 % XM_STAGES;  // stage and phase of the next chunk, counted as we go
        uint32_t ph_m = (uint32_t)((g0 / XM_STAGES) & 1);
        for (int gr = 0; gr < ngrp && !failed; ++gr) {
          const int gg = gg0 + gr, buf = gg & 1;
          // the fold of group gg - 2 has emptied this accumulator
          if (gg >= 2 && !mbar_wait(smem_u32(&acce[buf]), (uint32_t)(((gg >> 1) - 1) & 1), p.wait_cycles)) {
            s_fail = 1;
            break;
          }
          tc_fence_after();
          const uint32_t acc = tmem + (uint32_t)(buf * XM_BN_MAX), cacc = tmem + (uint32_t)(2 * XM_BN_MAX);
          const int c0 = gr * G, c1 = min(nck, c0 + G);
          for (int c = c0; c < c1; ++c) {
            if (!mbar_wait(full_b + 8u * (uint32_t)st_m, ph_m, p.wait_cycles)) {
              s_fail = 1;
              failed = true;
              break;
            }
            tc_fence_after();
            // descriptors of this stage: the stage-0 ones stepped by the stage offset (the
            // address field counts 16-byte units; shared addresses stay below 256 KB)
            const uint64_t dah = dA0 + (uint64_t)st_m * (XM_STAGE_BYTES >> 4), dal = dah + (XM_A_PART >> 4);
            const uint64_t dbh = dah + ((2 * XM_A_PART) >> 4), dbl = dbh + (b_part >> 4);
            const int st = st_m;
            if (++st_m == XM_STAGES) {
              st_m = 0;
              ph_m ^= 1u;
            }
            // the two small correction products into the row's correction accumulator, the
            // main product into the group's
            mma_f16(cacc, dah, dbl, idesc, c > 0 ? 1u : 0u);
            mma_f16(cacc, dal, dbh, idesc, 1u);
            mma_f16(acc, dah, dbh, idesc, c > c0 ? 1u : 0u);
            mma_commit(smem_u32(&empty[st]));
          }
          if (!failed) mma_commit(smem_u32(&accf[buf]));
        }
        mma_commit(smem_u32(&done));  // once every MMA issued so far is complete
      }
      __syncwarp();
    } else {  // fold warps
      // Kahan totals of column pairs: sum and the correction (minus the lost low part),
      // packed FP32 pairs so that each step of the fold is one instruction per two columns
      f2 ksum[XM_BN_MAX / 4], kcor[XM_BN_MAX / 4];
#pragma unroll
      for (int e = 0; e < XM_BN_MAX / 4; ++e) ksum[e] = kcor[e] = 0ull;
      const f2 one2 = f2_pack(1.0f, 1.0f), mone2 = f2_pack(-1.0f, -1.0f);
      for (int gr = 0; gr < ngrp; ++gr) {
        const int gg = gg0 + gr, buf = gg & 1;
        bool ok = mbar_wait(smem_u32(&accf[buf]), (uint32_t)((gg >> 1) & 1), p.wait_cycles);
        ok = __all_sync(0xffffffffu, ok);
        if (!ok) {
          if (lane == 0) s_fail = 1;
          break;
        }
        tc_fence_after();
        // the last group's commit also covers every correction MMA: fold that accumulator too
        for (int pass = 0; pass < (gr == ngrp - 1 ? 2 : 1); ++pass) {
        const uint32_t ta = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)((pass ? 2 : buf) * XM_BN_MAX + col0);
#pragma unroll
        for (int b = 0; b < XM_BN_MAX / 32; ++b) {
          if (b * 16 < ncol) {
            float v[16];
            tmem_ld16(ta + b * 16, v);
#pragma unroll
            for (int e = 0; e < 8; ++e) {
              // y = v - cor; t = sum + y; cor = (t - sum) - y; sum = t (a - b as fma(b, -1, a),
              // a + b as fma(a, 1, b): single roundings, as the scalar operations)
              f2& sum = ksum[b * 8 + e];
              f2& cor = kcor[b * 8 + e];
              const f2 y = f2_fma(cor, mone2, f2_pack(v[2 * e], v[2 * e + 1]));
              const f2 t2 = f2_fma(sum, one2, y);
              cor = f2_fma(y, mone2, f2_fma(sum, mone2, t2));
              sum = t2;
            }
          }
        }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&acce[buf]));
      }
      // rows of this run: D~ = (|dx|^2 + |d|^2 - 2 dx.d) / N (kernel units times dscale)
      const int rrow = q * 32 + lane;
      if (!s_fail && rrow >= k && rrow < kend) {
        const int f = s_frame[rrow];
        const float nx = p.Nx[row0 + rrow];  // rows of the approximate list
        const float* nb = p.Nb + (size_t)slot * p.M;
        float* out = p.Dout + (size_t)f * p.M;
        const int i0 = n * BN + col0;
#pragma unroll
        for (int e2 = 0; e2 < XM_BN_MAX / 4; ++e2) {
          float th[2], tl[2];
          f2_unpack(ksum[e2], th[0], th[1]);
          f2_unpack(kcor[e2], tl[0], tl[1]);
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int e = 2 * e2 + h, i = i0 + e;
            if (e < ncol && i < p.M)  // the compensated cross term sum - cor, its low part last
              out[i] = (((nx + nb[i]) - 2.0f * XM_UNSCALE2 * th[h]) + 2.0f * XM_UNSCALE2 * tl[h]) * p.dscale;
          }
        }
      }
    }
    const bool ok = mbar_wait(smem_u32(&done), (uint32_t)(run & 1), p.wait_cycles);
    if (!ok) s_fail = 1;
    __syncthreads();
    if (s_fail) {
      s_fail_run = run;  // every thread writes the same value
      break;
    }
  }
  if (s_fail) {
    // copies and MMAs already issued still land in this CTA's memory: wait for them within
    // the default budget before the tensor memory is released.  The MMA thread committed
    // `done` after its last MMA of the failed run whether its loop ended or broke off.
    if (tid == 0) atomicOr(p.status, STATUS_TIMEOUT);
    if (tid == XM_FOLD_WARPS * 32) {
      const int last = s_issued;
      for (int g = std::max(0, last - XM_STAGES); g < last; ++g)
        mbar_wait(smem_u32(&full[g % XM_STAGES]), (uint32_t)((g / XM_STAGES) & 1), XM_DRAIN_CYCLES);
    }
    mbar_wait(smem_u32(&done), (uint32_t)(s_fail_run & 1), XM_DRAIN_CYCLES);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, XM_TMEM_COLS);
  }
}

}  // namespace

// ---------------------------------------------------------------------------------------
XmmaShape xmma_shape(int M, int N) {
  XmmaShape s;
  const int K = 3 * round_up16(N);
  s.nck = K / XM_KC;
  s.NT = (M + XM_BN_MAX - 1) / XM_BN_MAX;
  s.BN = ((M + s.NT - 1) / s.NT + 15) / 16 * 16;
  s.a_bytes_per_tile = (size_t)s.nck * 2 * XM_A_PART;
  s.b_bytes_per_seg = (size_t)s.NT * s.nck * 2 * ((size_t)s.BN * XM_KC * 2);
  return s;
}

int xmma_max_tiles(int napp, int nseg) { return (napp + XM_ROWS - 1) / XM_ROWS + nseg; }

size_t xmma_a_bytes(const XmmaShape& sh, int napp, int nseg) {
  return (size_t)xmma_max_tiles(napp, nseg) * sh.a_bytes_per_tile;
}

void launch_xmma_tiles(const int* acount, const int* aseg, int seg_base, int nseg, int* seg_first, int* tile_start,
                       XTile* tiles, int* ntiles, cudaStream_t st) {
  xmma_tiles_kernel<<<1, XT_THREADS, 0, st>>>(acount, aseg, seg_base, nseg, seg_first, tile_start, tiles, ntiles);
  note_launch();
}

void launch_pack_deviations(Prec p, int s0, int ns, const LandmarkDev& L, const XmmaShape& xs, const MmaShape* ms,
                            const float* Bseg, const void* frames, FrameInfo fi, const int* refresh_list,
                            const RefDesc& prior, uint8_t* Bx, float* Nb, uint8_t* Ba, float* Yc, cudaStream_t st) {
  if (ns <= 0 || L.M <= 0) return;
  const int rows = std::max(xs.NT * xs.BN, ms ? ms->Kp : 0);  // landmark rows of the two layouts
  const dim3 grid(ns, (rows + 7) / 8);
  const int N16 = round_up16(L.N);
  const int BNa = ms ? ms->BN : 16, NTa = ms ? ms->NT : 1, Kpa = ms ? ms->Kp : 16;
  if (p == P_F16)
    pack_deviations_kernel<__half><<<grid, 256, 0, st>>>(s0, L.M, L.N, N16, xs.BN, xs.NT, BNa, NTa, Kpa,
                                                         (const __half*)L.coords, L.off, Bseg, (const float*)frames,
                                                         fi.c32, refresh_list, (const float*)prior.coords, prior.c32,
                                                         Bx, Nb, ms ? Ba : nullptr, Yc);
  else
    pack_deviations_kernel<float><<<grid, 256, 0, st>>>(s0, L.M, L.N, N16, xs.BN, xs.NT, BNa, NTa, Kpa,
                                                        (const float*)L.coords, L.off, Bseg, (const float*)frames,
                                                        fi.c32, refresh_list, (const float*)prior.coords, prior.c32,
                                                        Bx, Nb, ms ? Ba : nullptr, Yc);
  note_launch();
}

void launch_pack_frames(int napp, const int* acount, const int* alist, const int* aseg, int seg_base,
                        const LandmarkDev& L, const void* frames, FrameInfo fi, const double4* qxy, const float* Yc,
                        const int* seg_first, const int* tile_start, uint8_t* Ap, float* Nx, cudaStream_t st) {
  if (napp <= 0) return;
  pack_frames_kernel<<<(napp + 7) / 8, 256, 0, st>>>(acount, alist, aseg, seg_base, L.N, round_up16(L.N),
                                                     (const float*)frames, fi.c32, qxy, Yc, seg_first, tile_start,
                                                     Ap, Nx);
  note_launch();
}

void launch_approx_cross_mma(int napp, int nseg, const int* alist, const XTile* tiles, const int* ntiles,
                             const LandmarkDev& L, const XmmaShape& sh, const uint8_t* Ap, const uint8_t* Bp,
                             const float* Nx, const float* Nb, float* D, unsigned* status, cudaStream_t st) {
  if (napp <= 0 || L.M <= 0) return;
  XmmaArgs a;
  a.alist = alist;
  a.tiles = tiles;
  a.ntiles = ntiles;
  a.M = L.M;
  a.nck = sh.nck;
  a.BN = sh.BN;
  a.NT = sh.NT;
  a.Ap = Ap;
  a.Bp = Bp;
  a.Nx = Nx;
  a.Nb = Nb;
  a.dscale = (float)L.dscale;
  a.Dout = D;
  a.status = status;
  a.wait_cycles = L.wait_cycles;
  a.group = std::min(std::max(L.mma_group, 1), XM_GROUP_MAX);
  const size_t smem = (size_t)XM_STAGES * XM_STAGE_BYTES;
  cudaFuncSetAttribute(approx_cross_mma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  const dim3 grid(sh.NT, xmma_max_tiles(napp, nseg));
  approx_cross_mma<<<grid, XM_THREADS, smem, st>>>(a);
  note_launch();
}

}  // namespace pcv

// k_mma.cu -- the segment adjoint as a tensor-core GEMM (tcgen05, split FP16 operands).
//
// For frames sharing the close structure y of a segment, the adjoint needs
//   beta_f = sum_i gamma_fi b_i,   b_i = R_{a_i y} a_i  (3N values per landmark)
// for gamma^s and gamma^z (the derivatives of Eqs. 5-6 with respect to the MSDs).  Per
// segment this is a dense product: rows (frame, s|z) x K = landmarks x columns 3N.  It runs
// on the 5th-generation tensor cores (tcgen05.mma, kind::f16, accumulator in tensor
// memory) with two measures for FP32 accuracy:
//   * deviations: the product uses delta_i = b_i - y' (y' = the centred close structure),
//     and the epilogue adds Gamma_f y' (Gamma_f = sum_i gamma_fi).  The weights gamma are
//     concentrated on landmarks near the frame, hence near y, so the accumulated terms are
//     small compared with beta itself;
//   * split operands: every operand value is scaled by a power of two (2^8 for the
//     deviations; for each gamma row one that puts its largest entry in [2^13, 2^14)) and
//     split v = h + l with h = fp16(v), l = fp16(v - h); the product is h h' + h l' + l h'
//     (relative error about 2^-22 per product; FP16 products are exact in the accumulator).
//     The epilogue multiplies each row by its inverse scale.
//
// The producers write both operands pre-tiled in the canonical K-major shared-memory layout
// without swizzling: core matrices of 8 rows x 16 bytes (8 halves) stored as 128 contiguous
// bytes, the 2 core matrices of a 16-value K block 128 bytes apart (LBO) and the 8-row
// groups 256 bytes apart (SBO), the h part of a block followed by its l part.  So one stage
// (two K blocks) of operands is two contiguous runs moved by cp.async.bulk (one producer
// thread, completion counted in bytes on an mbarrier); one thread issues the MMAs and
// tcgen05.commit releases each stage when its MMAs are done.
// Every wait is bounded by a clock budget: on expiry the kernel records STATUS_TIMEOUT,
// waits for its copies and MMAs within a second budget, frees its tensor memory and returns.
#include <cuda_fp16.h>

#include <algorithm>
#include <cstdint>

#include "pcv_device.cuh"
#include "pcv_internal.h"
#include "tc_sm100.cuh"

namespace pcv {
namespace {

constexpr int MM_ROWS = 128;  // MMA M: 64 frames x {gamma^s, gamma^z}
constexpr int MM_FRAMES = 64;
constexpr int MM_KB = 16;       // K values (landmarks) per block: one MMA (K = 16) per product
constexpr int MM_KC = 32;       // K values per stage: two blocks
constexpr int MM_BN_MAX = 256;  // columns per CTA (MMA N), multiple of 16
constexpr int MM_THREADS = 128;
constexpr int MM_STAGES = 2;   // two CTAs per SM: one's epilogue overlaps the other's MMAs
constexpr int MM_TMEM_COLS = 256;
constexpr int MM_A_BYTES = MM_ROWS * MM_KB * 2;  // one part (h or l) of one A block
constexpr float MM_DSCALE = 256.0f;              // 2^8 on the deviations
constexpr int MM_GROUP_TILES = 16;  // frame tiles per group of the raster order
constexpr long long MM_WAIT_CYCLES = 4000000000LL;  // about 2 s at the maximum SM clock: the
                                                    // budget of the waits for copies and MMAs
                                                    // already issued after a failure

// byte offset of (row r, K value kk < 16) inside the h part of one canonical K-major block
// of FP16 values
__host__ __device__ __forceinline__ uint32_t canon_off(int r, int kk) {
  return (uint32_t)((r >> 3) * 256 + (kk >> 3) * 128 + (r & 7) * 16 + (kk & 7) * 2);
}

// a scaled value v (|v| < 65504) split into FP16 h + l
__device__ __forceinline__ void split_h(float v, __half& h, __half& l) {
  h = __float2half_rn(v);
  l = __float2half_rn(v - __half2float(h));
}
__device__ __forceinline__ uint32_t pack_h2(__half a, __half b) {
  return (uint32_t)__half_as_ushort(a) | ((uint32_t)__half_as_ushort(b) << 16);
}
// power of two putting the largest magnitude m of a row in [2^13, 2^14) (1 for m = 0)
__device__ __forceinline__ float row_scale(float m) {
  if (!(m > 0.0f)) return 1.0f;
  int e;
  frexpf(m, &e);  // m = f 2^e, f in [0.5, 1)
  return ldexpf(1.0f, 14 - e);
}

// ---------------------------------------------------------------------------------------
// gamma operand: for frame tile t (64 frames) and K block c (16 landmarks), blocks h | l of
// 128 rows x 16 values (rows 0..63 gamma^s of frames 64t + r, rows 64..127 gamma^z), each
// row scaled by its power of two (row_scale), zero for landmarks >= M and frames >= F;
// Gamma^s_f, Gamma^z_f in Gsum[2f], Gsum[2f + 1] and the rows' inverse scales (including the
// deviations' 2^-8) in Gsum[2Fp + 2f], Gsum[2Fp + 2f + 1].  One warp per 8 consecutive frames
// (a row group of the core matrices): lane = 4 (frame in the group) + (pair of landmarks in
// a group of 8), so every 4-byte store of the warp lands in one whole 128-byte core matrix.
__global__ void gamma_split_kernel(int F, int Fp, int M, int Kp, const float* __restrict__ P,
                                   const float* __restrict__ q32, const double* __restrict__ s, float lambda,
                                   uint8_t* __restrict__ A, float* __restrict__ Gsum) {
  const int lane = threadIdx.x & 31, rr = lane >> 2, kq = lane & 3;
  const int g = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (g * 8 >= Fp) return;  // uniform over the warp
  const int f = g * 8 + rr;
  const bool live = f < F;
  const float sf = live ? (float)s[f] : 0.0f, sl = live ? s_low<float>(s[f], sf) : 0.0f;
  const int nkb = Kp / MM_KB;
  const int t = f / MM_FRAMES, r = f % MM_FRAMES;
  uint8_t* tileA = A + (size_t)t * nkb * 2 * MM_A_BYTES;
  const float* prow = P + (size_t)(live ? f : 0) * M;
  auto gam = [&](int i, float& gs, float& gz) {
    gs = gz = 0.0f;
    if (live && i < M) {
      const float pv = prow[i];
      gz = pv;
      gs = -lambda * pv * ((q32[i] - sf) - sl);
    }
  };
  // pass 1: the rows' largest magnitudes (the 4 lanes of a frame)
  float ms = 0.0f, mz = 0.0f;
  for (int i0 = 0; i0 < Kp; i0 += 8) {
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      float gs, gz;
      gam(i0 + 2 * kq + u, gs, gz);
      ms = fmaxf(ms, fabsf(gs));
      mz = fmaxf(mz, fabsf(gz));
    }
  }
  ms = fmaxf(ms, __shfl_xor_sync(0xffffffffu, ms, 1));
  mz = fmaxf(mz, __shfl_xor_sync(0xffffffffu, mz, 1));
  ms = fmaxf(ms, __shfl_xor_sync(0xffffffffu, ms, 2));
  mz = fmaxf(mz, __shfl_xor_sync(0xffffffffu, mz, 2));
  const float scs = row_scale(ms), scz = row_scale(mz);
  // pass 2: sums and the split, scaled values
  float ss = 0.0f, sz = 0.0f;
#pragma unroll 2
  for (int i0 = 0; i0 < Kp; i0 += 8) {
    float gs[2], gz[2];
    __half hs[2], ls[2], hz[2], lz[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      gam(i0 + 2 * kq + u, gs[u], gz[u]);
      ss += gs[u];
      sz += gz[u];
      split_h(gs[u] * scs, hs[u], ls[u]);
      split_h(gz[u] * scz, hz[u], lz[u]);
    }
    const int c = i0 / MM_KB, kk = (i0 % MM_KB) + 2 * kq;
    uint8_t* blk = tileA + (size_t)c * 2 * MM_A_BYTES;
    *reinterpret_cast<uint32_t*>(blk + canon_off(r, kk)) = pack_h2(hs[0], hs[1]);
    *reinterpret_cast<uint32_t*>(blk + canon_off(r + MM_FRAMES, kk)) = pack_h2(hz[0], hz[1]);
    *reinterpret_cast<uint32_t*>(blk + MM_A_BYTES + canon_off(r, kk)) = pack_h2(ls[0], ls[1]);
    *reinterpret_cast<uint32_t*>(blk + MM_A_BYTES + canon_off(r + MM_FRAMES, kk)) = pack_h2(lz[0], lz[1]);
  }
  // sums over the 4 lanes of the frame
  ss += __shfl_xor_sync(0xffffffffu, ss, 1);
  sz += __shfl_xor_sync(0xffffffffu, sz, 1);
  ss += __shfl_xor_sync(0xffffffffu, ss, 2);
  sz += __shfl_xor_sync(0xffffffffu, sz, 2);
  if (kq == 0 && live) {
    Gsum[2 * f] = ss;
    Gsum[2 * f + 1] = sz;
    Gsum[2 * (size_t)Fp + 2 * f] = 1.0f / (scs * MM_DSCALE);
    Gsum[2 * (size_t)Fp + 2 * f + 1] = 1.0f / (scz * MM_DSCALE);
  }
}

// ---------------------------------------------------------------------------------------
// beta tile: rows 64 frames x {s, z}, columns [n0, n0 + BN) of 3N.  The tile's frames are
// taken in runs of equal segment; each run accumulates from zero over all K chunks with its
// segment's deviations and writes the rows of its own frames.
struct MmaArgs {
  int F, M, N, Kp, BN, NT, seg_base, ntiles;
  const uint8_t *A, *B;
  const float *Gsum, *Yc;
  const int* seg_of_frame;
  float *gs, *gz;
  unsigned* status;
  long long wait_cycles;  // budget of each wait of the pipeline (the context's option)
};

__global__ void __launch_bounds__(MM_THREADS, 2) adjoint_beta_mma(MmaArgs p) {
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ __align__(8) uint64_t full[MM_STAGES], empty[MM_STAGES], done;
  __shared__ uint32_t tmem_slot;
  __shared__ int s_seg[MM_FRAMES];
  __shared__ int s_run[MM_FRAMES + 1];
  __shared__ int s_nrun;
  __shared__ int s_fail;
  __shared__ int s_fail_run;
  __shared__ int s_issued;  // chunks whose copies the producer started (global counter)

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // grouped raster order: blocks take, group by group, MM_GROUP_TILES consecutive frame
  // tiles x all column tiles with the frame tiles fastest, so the resident blocks share one
  // group's gamma tiles (kept in L2 for the whole group) and each column tile's deviation
  // block of a segment is read once by the group's frame tiles of that segment
  const int gsz = MM_GROUP_TILES * p.NT;
  const int grp = (int)blockIdx.x / gsz, rem = (int)blockIdx.x - grp * gsz;
  const int g0t = grp * MM_GROUP_TILES, gtiles = min(MM_GROUP_TILES, p.ntiles - g0t);
  const int tile = g0t + rem % gtiles, ncol = rem / gtiles;
  const int f0 = tile * MM_FRAMES;
  const int n0 = ncol * p.BN;
  const int NB = 3 * p.N;
  const int nck = p.Kp / MM_KC;  // stages of two K blocks
  const uint32_t idesc = idesc_make(MM_ROWS, p.BN, 0u);  // kind::f16, F16 operands
  // bytes of one part of one block, and of a stage's A and B runs (two blocks, h and l)
  const uint32_t a_bytes = MM_A_BYTES, b_bytes = (uint32_t)p.BN * MM_KB * 2;
  const uint32_t a_stage = 2 * 2 * a_bytes, b_stage = 2 * 2 * b_bytes;
  const uint32_t stage_bytes = a_stage + 2 * 2 * (uint32_t)MM_BN_MAX * MM_KB * 2;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(MM_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int s = 0; s < MM_STAGES; ++s) {
      mbar_init(smem_u32(&full[s]), 1);
      mbar_init(smem_u32(&empty[s]), 1);
    }
    mbar_init(smem_u32(&done), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_fail = 0;
    s_issued = 0;
  }
  if (tid < MM_FRAMES) s_seg[tid] = f0 + tid < p.F ? p.seg_of_frame[f0 + tid] : -1;
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  if (tid == 0) {  // runs of equal segment among the tile's frames
    int n = 0, k = 0;
    while (k < MM_FRAMES && s_seg[k] >= 0) {
      s_run[n++] = k;
      int e = k;
      while (e < MM_FRAMES && s_seg[e] == s_seg[k]) ++e;
      k = e;
    }
    s_run[n] = k;
    s_nrun = n;
  }
  __syncthreads();
  const int nrun = s_nrun;
  const uint32_t sbase = smem_u32(smem);
  const uint8_t* Ab = p.A + (size_t)tile * nck * a_stage;

  for (int run = 0; run < nrun; ++run) {
    const int k = s_run[run], kend = s_run[run + 1];
    const int slot = s_seg[k] - p.seg_base;
    const uint8_t* Bb = p.B + (((size_t)slot * p.NT + ncol) * nck) * b_stage;
    const int g0 = run * nck;  // global chunk counter: stage and phase bookkeeping across runs
    if (warp == 1) {
      if (lane == 0) {  // producer
        for (int c = 0; c < nck; ++c) {
          const int g = g0 + c, st = g % MM_STAGES;
          if (g >= MM_STAGES &&
              !mbar_wait(smem_u32(&empty[st]), (uint32_t)((g / MM_STAGES - 1) & 1), p.wait_cycles)) {
            s_fail = 1;
            break;
          }
          const uint32_t dst = sbase + st * stage_bytes;
          mbar_expect_tx(smem_u32(&full[st]), a_stage + b_stage);
          bulk_g2s(dst, Ab + (size_t)c * a_stage, a_stage, smem_u32(&full[st]));
          bulk_g2s(dst + a_stage, Bb + (size_t)c * b_stage, b_stage, smem_u32(&full[st]));
          s_issued = g + 1;
        }
      }
      __syncwarp();
    } else if (warp == 0) {
      if (lane == 0) {  // MMA issuer
        for (int c = 0; c < nck; ++c) {
          const int g = g0 + c, st = g % MM_STAGES;
          if (!mbar_wait(smem_u32(&full[st]), (uint32_t)((g / MM_STAGES) & 1), p.wait_cycles)) {
            s_fail = 1;
            break;
          }
          tc_fence_after();
          const uint32_t a0 = sbase + st * stage_bytes, b0 = a0 + a_stage;
#pragma unroll
          for (int ks = 0; ks < MM_KC / MM_KB; ++ks) {  // one block of 16 K values per MMA
            const uint32_t ah = a0 + ks * 2 * a_bytes, al = ah + a_bytes;
            const uint32_t bh = b0 + ks * 2 * b_bytes, bl = bh + b_bytes;
            const uint64_t dah = smem_desc(ah, 128, 256), dal = smem_desc(al, 128, 256);
            const uint64_t dbh = smem_desc(bh, 128, 256), dbl = smem_desc(bl, 128, 256);
            // the two small correction products first, the main product last
            mma_f16(tmem, dah, dbl, idesc, (c > 0 || ks > 0) ? 1u : 0u);
            mma_f16(tmem, dal, dbh, idesc, 1u);
            mma_f16(tmem, dah, dbh, idesc, 1u);
          }
          mma_commit(smem_u32(&empty[st]));
        }
        mma_commit(smem_u32(&done));
      }
      __syncwarp();
    }
    // all warps: wait for the run's MMAs, then the epilogue beta = D + Gamma_f y'
    const bool ok = mbar_wait(smem_u32(&done), (uint32_t)(run & 1), p.wait_cycles);
    if (!ok) s_fail = 1;
    __syncthreads();
    if (s_fail) {
      s_fail_run = run;  // every thread writes the same value
      break;
    }
    tc_fence_after();
    // Each warp holds rows 32 warp + lane of the accumulator.  Columns are moved in halves
    // through shared memory (the operand stages are idle now) so that the global stores
    // run along rows: a warp writes 32 consecutive columns of one frame per instruction.
    const int r = warp * 32 + lane;
    const bool zrow = warp >= 2;  // rows 64..127: gamma^z
    const int ff = r & (MM_FRAMES - 1);
    const int f = f0 + ff;
    const int mine = (ff >= k && ff < kend && f < p.F) ? 1 : 0;
    const float Gam = mine ? p.Gsum[2 * f + (zrow ? 1 : 0)] : 0.0f;
    // the row's inverse scale (gamma row scale and the deviations' 2^8)
    const float usc = mine ? p.Gsum[2 * (size_t)p.ntiles * MM_FRAMES + 2 * f + (zrow ? 1 : 0)] : 0.0f;
    const float* yrow = p.Yc + (size_t)slot * NB;
    float* outb = zrow ? p.gz : p.gs;
    const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
    const int half = (p.BN / 2 + 15) / 16 * 16;  // columns per pass, multiple of 16
    const int ld = half + 1;                      // odd row stride: conflict-free scalar writes
    float* stg = reinterpret_cast<float*>(smem) + warp * 32 * ld;
    for (int c0 = 0; c0 < p.BN; c0 += half) {
      const int cn = min(half, p.BN - c0);
      for (int cb = 0; cb < cn; cb += 16) {
        float v[16];
        tmem_ld16(trow + c0 + cb, v);
#pragma unroll
        for (int e = 0; e < 16; ++e) stg[lane * ld + cb + e] = v[e] * usc;
      }
      __syncwarp();
      float yv[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int n = n0 + c0 + lane + 32 * q;
        yv[q] = (lane + 32 * q < cn && n < NB) ? yrow[n] : 0.0f;
      }
      for (int rr = 0; rr < 32; ++rr) {
        const int mr = __shfl_sync(0xffffffffu, mine, rr);
        const float G = __shfl_sync(0xffffffffu, Gam, rr);
        const int fr = __shfl_sync(0xffffffffu, f, rr);
        if (!mr) continue;
        float* orow = outb + (size_t)fr * NB;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int col = lane + 32 * q, n = n0 + c0 + col;
          if (col < cn && n < NB) orow[n] = fmaf(G, yv[q], stg[rr * ld + col]);
        }
      }
      __syncwarp();
    }
    tc_fence_before();
    __syncthreads();  // the accumulator is read before the next run overwrites it
  }
  if (s_fail) {
    // Copies and MMAs already issued still land in this CTA's memory: wait for them, within
    // the full budget MM_WAIT_CYCLES, before the tensor memory is released.  The MMA issuer
    // (thread 0) committed `done` after its last MMA of the failed run, whether its loop
    // ended or broke off, so that phase completes once every MMA issued is done; the
    // producer (thread 32) waits for the last copy into each stage.
    if (tid == 0) atomicOr(p.status, STATUS_TIMEOUT);
    if (tid == 32) {
      const int last = s_issued;
      for (int g = std::max(0, last - MM_STAGES); g < last; ++g)
        mbar_wait(smem_u32(&full[g % MM_STAGES]), (uint32_t)((g / MM_STAGES) & 1), MM_WAIT_CYCLES);
    }
    mbar_wait(smem_u32(&done), (uint32_t)(s_fail_run & 1), MM_WAIT_CYCLES);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(MM_TMEM_COLS) : "memory");
  }
}

}  // namespace

// ---------------------------------------------------------------------------------------
MmaShape mma_shape(int F, int M, int N) {
  MmaShape s;
  s.Kp = (M + MM_KC - 1) / MM_KC * MM_KC;
  s.Fp = (F + MM_FRAMES - 1) / MM_FRAMES * MM_FRAMES;
  const int NB = 3 * N;
  const int nt = (NB + MM_BN_MAX - 1) / MM_BN_MAX;
  s.BN = ((NB + nt - 1) / nt + 15) / 16 * 16;
  s.NT = (NB + s.BN - 1) / s.BN;
  s.a_bytes = (size_t)s.Fp * 2 * s.Kp * 2 * sizeof(__half);            // rows s, z; parts h, l
  s.b_bytes_per_seg = (size_t)s.NT * s.BN * s.Kp * 2 * sizeof(__half);  // parts h, l
  s.y_bytes_per_seg = (size_t)NB * sizeof(float);
  s.gsum_floats = 4 * (size_t)s.Fp;  // Gamma sums and the rows' inverse scales
  return s;
}

void launch_gamma_split(int F, const LandmarkDev& L, const MmaShape& sh, const float* P, const double* s,
                        double lambda, float* A, float* Gsum, cudaStream_t st) {
  if (F <= 0) return;
  gamma_split_kernel<<<sh.Fp / 64, 256, 0, st>>>(F, sh.Fp, L.M, sh.Kp, P, L.q32, s, (float)lambda,
                                                 reinterpret_cast<uint8_t*>(A), Gsum);
  note_launch();
}

void launch_adjoint_beta_mma(int F, const LandmarkDev& L, const MmaShape& sh, int seg_base, const float* A,
                             const float* Gsum, const float* B, const float* Yc, const int* seg_of_frame, float* gs,
                             float* gz, unsigned* status, cudaStream_t st) {
  if (F <= 0) return;
  MmaArgs a;
  a.F = F;
  a.M = L.M;
  a.N = L.N;
  a.Kp = sh.Kp;
  a.BN = sh.BN;
  a.NT = sh.NT;
  a.seg_base = seg_base;
  a.A = reinterpret_cast<const uint8_t*>(A);
  a.Gsum = Gsum;
  a.B = reinterpret_cast<const uint8_t*>(B);
  a.Yc = Yc;
  a.seg_of_frame = seg_of_frame;
  a.gs = gs;
  a.gz = gz;
  a.status = status;
  a.wait_cycles = L.wait_cycles;
  const size_t smem = (size_t)MM_STAGES * (2 * 2 * MM_A_BYTES + 2 * 2 * MM_BN_MAX * MM_KB * 2);
  cudaFuncSetAttribute(adjoint_beta_mma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  const int tiles = sh.Fp / MM_FRAMES;
  a.ntiles = tiles;
  // the last group may hold fewer frame tiles: exactly tiles x NT blocks in all
  adjoint_beta_mma<<<(unsigned)((size_t)tiles * sh.NT), MM_THREADS, smem, st>>>(a);
  note_launch();
}

}  // namespace pcv

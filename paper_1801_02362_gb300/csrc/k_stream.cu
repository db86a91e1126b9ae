// k_stream.cu -- landmark-parallel kernels for a few frames per call (FP32 modes).
//
// In molecular dynamics the path CVs are evaluated once per step: one frame per call
// (Algorithm 1 and 2 are written per step).  Then every call streams the whole landmark
// set (M x N x 3 values: 120 MB in FP32, 60 MB in FP16 storage for N = 5000, M = 2000) and
// the work is bound by memory bandwidth.  The frame-batch tiles of k_pair.cu would give
// one CTA per 32 landmarks; these kernels give one CTA per landmark instead:
//   exact_stream:  the landmark is staged in shared memory by asynchronous 16-byte copies,
//                  pass 1 forms H = sum_j w_j a_j x_j^T for each frame (Eq. corr), the top
//                  eigenvector of K(H) gives R_{a x} (FP32, as the batched kernel), and pass 2
//                  forms D = sum_j w_j |x_j - R a_j|^2 directly from the staged copy -- the
//                  landmark is read from memory once;
//   approx_stream: D~ = sum_j w_j |R_xy^T (x_j - c) - R_{a y} a_j|^2 (Eq. close_dist) in one
//                  pass over the landmark.
// exact_stream takes any number of frames, in groups of STREAM_FRAMES against the landmark
// staged once; the library sends it batches of up to STREAM_FRAMES (more groups per CTA
// were slower than the frame-batch tiles: 2.3 against 1.5 ms for 34 frames x 2000 landmarks
// of 5000 atoms).  approx_stream takes up to STREAM_FRAMES frames per launch.  Both use the
// same arithmetic and compensated sums as the batched kernels.
#include <cuda_fp16.h>

#include "pcv_device.cuh"
#include "pcv_internal.h"

namespace pcv {
namespace {

constexpr int ST_THREADS = 256;

template <typename LT>
__device__ __forceinline__ float ldf(const LT* p) {
  return (float)(*p);
}
template <>
__device__ __forceinline__ float ldf<__half>(const __half* p) {
  return __half2float(*p);
}

// stage landmark i (N*3 values of LT) into shared memory; 16-byte copies when aligned
template <typename LT>
__device__ __forceinline__ void stage_landmark(const LT* __restrict__ src, int n_vals, LT* dst, bool aligned) {
  if (aligned) {
    const int bytes = n_vals * (int)sizeof(LT);
    const int n16 = bytes / 16;
    const unsigned d0 = (unsigned)__cvta_generic_to_shared(dst);
    const char* s0 = reinterpret_cast<const char*>(src);
    for (int e = threadIdx.x; e < n16; e += blockDim.x)
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d0 + 16u * e), "l"(s0 + 16 * e) : "memory");
    asm volatile("cp.async.wait_all;" ::: "memory");
    for (int e = n16 * 16 / (int)sizeof(LT) + threadIdx.x; e < n_vals; e += blockDim.x) dst[e] = src[e];
  } else {
    for (int e = threadIdx.x; e < n_vals; e += blockDim.x) dst[e] = src[e];
  }
  __syncthreads();
}

// block sums of the NV floats of every thread: red[32 K + e] = sum over threads of v[e]
// (red holds 33 K floats, K >= NV; at most 32 warps)
template <int K, int NV>
__device__ __forceinline__ void block_reduce(const float* v, float* red) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int e = 0; e < NV; ++e) {
    const float t = warp_sum_float(v[e]);
    if (lane == 0) red[w * K + e] = t;
  }
  __syncthreads();
  if ((int)threadIdx.x < NV) {
    float t = 0.0f;
    for (int k = 0; k < nw; ++k) t += red[k * K + threadIdx.x];
    red[32 * K + threadIdx.x] = t;
  }
  __syncthreads();
}

template <typename LT>
__global__ void __launch_bounds__(ST_THREADS)
exact_stream_f32(int rows, const int* __restrict__ row_frame, const float* __restrict__ frames,
                 const float4* __restrict__ c32, const double* __restrict__ fG, const LT* __restrict__ lm,
                 const float* __restrict__ lmoff, const double* __restrict__ lG, const float* __restrict__ wts, int M, int N, double dscale,
                 bool aligned, float* __restrict__ Dout, float* __restrict__ Rout, unsigned* __restrict__ status,
                 int cap) {
  extern __shared__ __align__(16) unsigned char stream_sm[];
  LT* As = reinterpret_cast<LT*>(stream_sm);
  constexpr int K = STREAM_FRAMES * 9;
  __shared__ float red[33 * K];
  __shared__ float s_R[STREAM_FRAMES][9];
  __shared__ int s_f[STREAM_FRAMES];
  __shared__ float s_c[STREAM_FRAMES][3];
  const int i = blockIdx.x;
  // the frames in groups of STREAM_FRAMES against the landmark staged once
  for (int g0 = 0; g0 < rows; g0 += STREAM_FRAMES) {
    const int grows = min(rows - g0, STREAM_FRAMES);
    if (threadIdx.x < STREAM_FRAMES) {
      const int r = threadIdx.x;
      const int f = r < grows ? (row_frame ? row_frame[g0 + r] : g0 + r) : -1;
      s_f[r] = f;
      const float4 c = f >= 0 ? c32[f] : make_float4(0.f, 0.f, 0.f, 0.f);
      s_c[r][0] = c.x;
      s_c[r][1] = c.y;
      s_c[r][2] = c.z;
    }
    if (g0 == 0)
      stage_landmark<LT>(lm + (size_t)i * N * 3, 3 * N, As, aligned);  // ends with a barrier
    else
      __syncthreads();
    // pass 1: H_r = sum_j a_j (w_j x_j)^T
    float h[K];
#pragma unroll
    for (int e = 0; e < K; ++e) h[e] = 0.0f;
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
      const float a[3] = {lm_plus_off<LT>(ldf(As + 3 * j), lmoff, N, i, j, 0),
                          lm_plus_off<LT>(ldf(As + 3 * j + 1), lmoff, N, i, j, 1),
                          lm_plus_off<LT>(ldf(As + 3 * j + 2), lmoff, N, i, j, 2)};
      const float wj = wts ? wts[j] : 1.0f;
#pragma unroll
      for (int r = 0; r < STREAM_FRAMES; ++r) {
        if (r >= grows) break;
        const float* x = frames + ((size_t)s_f[r] * N + j) * 3;
        const float v[3] = {(x[0] - s_c[r][0]) * wj, (x[1] - s_c[r][1]) * wj, (x[2] - s_c[r][2]) * wj};
#pragma unroll
        for (int b = 0; b < 3; ++b)
#pragma unroll
          for (int c = 0; c < 3; ++c) h[9 * r + 3 * b + c] = fmaf(a[b], v[c], h[9 * r + 3 * b + c]);
      }
    }
    block_reduce<K, K>(h, red);
    if ((int)threadIdx.x < grows) {
      const int r = threadIdx.x;
      float H[9], q[4] = {1.0f, 0.0f, 0.0f, 0.0f}, R[9];
#pragma unroll
      for (int e = 0; e < 9; ++e) H[e] = red[32 * K + 9 * r + e];
      const float ub = (float)(0.5 * (fG[s_f[r]] + lG[i])) * 1.00001f + 1e-30f;
      if (!top_quat_f32(H, ub, q, cap)) atomicOr(status, STATUS_NOCONV);
      quat_to_rot(q, R);
#pragma unroll
      for (int e = 0; e < 9; ++e) s_R[r][e] = R[e];
    }
    __syncthreads();
    // pass 2: D_r = sum_j w_j |x_j - R a_j|^2 from the staged landmark, compensated
    float acc[STREAM_FRAMES], thi[STREAM_FRAMES], tlo[STREAM_FRAMES];
#pragma unroll
    for (int r = 0; r < STREAM_FRAMES; ++r) acc[r] = thi[r] = tlo[r] = 0.0f;
    int cnt = 0;
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
      const float a[3] = {lm_plus_off<LT>(ldf(As + 3 * j), lmoff, N, i, j, 0),
                          lm_plus_off<LT>(ldf(As + 3 * j + 1), lmoff, N, i, j, 1),
                          lm_plus_off<LT>(ldf(As + 3 * j + 2), lmoff, N, i, j, 2)};
      const float wj = wts ? wts[j] : 1.0f;
#pragma unroll
      for (int r = 0; r < STREAM_FRAMES; ++r) {
        if (r >= grows) break;
        const float* x = frames + ((size_t)s_f[r] * N + j) * 3;
        const float* Rr = s_R[r];
        const float d0 = (x[0] - s_c[r][0]) - fmaf(Rr[0], a[0], fmaf(Rr[1], a[1], Rr[2] * a[2]));
        const float d1 = (x[1] - s_c[r][1]) - fmaf(Rr[3], a[0], fmaf(Rr[4], a[1], Rr[5] * a[2]));
        const float d2 = (x[2] - s_c[r][2]) - fmaf(Rr[6], a[0], fmaf(Rr[7], a[1], Rr[8] * a[2]));
        acc[r] = fmaf(wj * d0, d0, fmaf(wj * d1, d1, fmaf(wj * d2, d2, acc[r])));
      }
      if (++cnt == 8) {
        cnt = 0;
#pragma unroll
        for (int r = 0; r < STREAM_FRAMES; ++r) {
          two_sum_acc(thi[r], tlo[r], acc[r]);
          acc[r] = 0.0f;
        }
      }
    }
    float part[2 * STREAM_FRAMES];
#pragma unroll
    for (int r = 0; r < STREAM_FRAMES; ++r) {
      two_sum_acc(thi[r], tlo[r], acc[r]);
      part[2 * r] = thi[r];
      part[2 * r + 1] = tlo[r];
    }
    __syncthreads();  // red is reused
    block_reduce<K, 2 * STREAM_FRAMES>(part, red);
    if ((int)threadIdx.x < grows) {
      const int r = threadIdx.x;
      Dout[(size_t)s_f[r] * M + i] = (red[32 * K + 2 * r] + red[32 * K + 2 * r + 1]) * (float)dscale;
      if (Rout) {
#pragma unroll
        for (int e = 0; e < 9; ++e) Rout[((size_t)(g0 + r) * M + i) * 9 + e] = s_R[r][e];
      }
    }
    __syncthreads();  // s_f, s_c, s_R and red are rewritten by the next group
  }
}

template <typename LT>
__global__ void __launch_bounds__(ST_THREADS)
approx_stream_f32(const int* __restrict__ alist, const int* __restrict__ aseg, const int* __restrict__ acount,
                  const float* __restrict__ frames, const float4* __restrict__ c32, const double4* __restrict__ qxy,
                  const LT* __restrict__ lm, const float* __restrict__ lmoff, const float* __restrict__ Bseg,
                  const float* __restrict__ wts, int M,
                  int N, double dscale, bool aligned, float* __restrict__ Dout) {
  extern __shared__ __align__(16) unsigned char stream_sm[];
  LT* As = reinterpret_cast<LT*>(stream_sm);
  constexpr int K = STREAM_FRAMES * 9;
  __shared__ float red[33 * K];
  __shared__ float s_Rt[STREAM_FRAMES][9];  // R_xy
  __shared__ float s_B[STREAM_FRAMES][9];   // R_{a_i y}
  __shared__ int s_f[STREAM_FRAMES];
  __shared__ float s_c[STREAM_FRAMES][3];
  const int rows = min(*acount, STREAM_FRAMES);
  if (rows <= 0) return;  // uniform over the grid
  const int i = blockIdx.x;
  if (threadIdx.x < STREAM_FRAMES) {
    const int r = threadIdx.x;
    const int f = r < rows ? alist[r] : -1;
    s_f[r] = f;
    float R[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1}, B[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    float4 c = make_float4(0.f, 0.f, 0.f, 0.f);
    if (f >= 0) {
      c = c32[f];
      const double4 qq = qxy[f];
      const float q[4] = {(float)qq.x, (float)qq.y, (float)qq.z, (float)qq.w};
      quat_to_rot(q, R);
      const float* Bp = Bseg + ((size_t)aseg[r] * M + i) * 9;
#pragma unroll
      for (int e = 0; e < 9; ++e) B[e] = Bp[e];
    }
#pragma unroll
    for (int e = 0; e < 9; ++e) {
      s_Rt[r][e] = R[e];
      s_B[r][e] = B[e];
    }
    s_c[r][0] = c.x;
    s_c[r][1] = c.y;
    s_c[r][2] = c.z;
  }
  stage_landmark<LT>(lm + (size_t)i * N * 3, 3 * N, As, aligned);
  float acc[STREAM_FRAMES], thi[STREAM_FRAMES], tlo[STREAM_FRAMES];
#pragma unroll
  for (int r = 0; r < STREAM_FRAMES; ++r) acc[r] = thi[r] = tlo[r] = 0.0f;
  int cnt = 0;
  for (int j = threadIdx.x; j < N; j += blockDim.x) {
    const float a[3] = {lm_plus_off<LT>(ldf(As + 3 * j), lmoff, N, i, j, 0),
                        lm_plus_off<LT>(ldf(As + 3 * j + 1), lmoff, N, i, j, 1),
                        lm_plus_off<LT>(ldf(As + 3 * j + 2), lmoff, N, i, j, 2)};
    const float wj = wts ? wts[j] : 1.0f;
#pragma unroll
    for (int r = 0; r < STREAM_FRAMES; ++r) {
      if (r >= rows) break;
      const float* x = frames + ((size_t)s_f[r] * N + j) * 3;
      const float v0 = x[0] - s_c[r][0], v1 = x[1] - s_c[r][1], v2 = x[2] - s_c[r][2];
      const float* R = s_Rt[r];
      const float* B = s_B[r];
      const float d0 = (R[0] * v0 + R[3] * v1 + R[6] * v2) - (B[0] * a[0] + B[1] * a[1] + B[2] * a[2]);
      const float d1 = (R[1] * v0 + R[4] * v1 + R[7] * v2) - (B[3] * a[0] + B[4] * a[1] + B[5] * a[2]);
      const float d2 = (R[2] * v0 + R[5] * v1 + R[8] * v2) - (B[6] * a[0] + B[7] * a[1] + B[8] * a[2]);
      acc[r] = fmaf(wj * d0, d0, fmaf(wj * d1, d1, fmaf(wj * d2, d2, acc[r])));
    }
    if (++cnt == 8) {
      cnt = 0;
#pragma unroll
      for (int r = 0; r < STREAM_FRAMES; ++r) {
        two_sum_acc(thi[r], tlo[r], acc[r]);
        acc[r] = 0.0f;
      }
    }
  }
  float part[2 * STREAM_FRAMES];
#pragma unroll
  for (int r = 0; r < STREAM_FRAMES; ++r) {
    two_sum_acc(thi[r], tlo[r], acc[r]);
    part[2 * r] = thi[r];
    part[2 * r + 1] = tlo[r];
  }
  block_reduce<K, 2 * STREAM_FRAMES>(part, red);
  if ((int)threadIdx.x < rows) {
    const int r = threadIdx.x;
    Dout[(size_t)s_f[r] * M + i] = (red[32 * K + 2 * r] + red[32 * K + 2 * r + 1]) * (float)dscale;
  }
}

// One frame (the per-step case): LPB landmarks per CTA, atoms in groups of APG (4 in FP32,
// 8 in FP16 storage) read as three 16-byte vectors of each landmark and of the frame; the
// frame is rotated once per group and serves the CTA's LPB landmarks.  No shared-memory
// staging, so many CTAs per SM keep enough loads in flight to stream the landmark set at
// the memory's rate.  Requires 16-byte aligned rows (N a multiple of APG).
template <typename LT, int LPB>
__global__ void __launch_bounds__(128)
approx_stream_vec(const int* __restrict__ alist, const int* __restrict__ aseg, const int* __restrict__ acount,
                  const float* __restrict__ frames, const float4* __restrict__ c32, const double4* __restrict__ qxy,
                  const LT* __restrict__ lm, const float* __restrict__ lmoff, const float* __restrict__ Bseg,
                  const float* __restrict__ wts, int M, int N, double dscale, float* __restrict__ Dout) {
  constexpr int APG = sizeof(LT) == 2 ? 8 : 4;
  __shared__ float red[32][LPB];
  if (*acount < 1) return;  // uniform over the grid
  const int f = alist[0], seg = aseg[0];
  const int i0 = blockIdx.x * LPB;
  float R[9];
  {
    const double4 qq = qxy[f];
    const float q[4] = {(float)qq.x, (float)qq.y, (float)qq.z, (float)qq.w};
    quat_to_rot(q, R);
  }
  const float4 c = c32[f];
  float B[LPB][9];
#pragma unroll
  for (int l = 0; l < LPB; ++l)
#pragma unroll
    for (int e = 0; e < 9; ++e) B[l][e] = i0 + l < M ? Bseg[((size_t)seg * M + i0 + l) * 9 + e] : 0.0f;
  float acc[LPB];
#pragma unroll
  for (int l = 0; l < LPB; ++l) acc[l] = 0.0f;
  const int ngroups = N / APG;
  const float* xf = frames + (size_t)f * N * 3;
  for (int g = threadIdx.x; g < ngroups; g += blockDim.x) {
    const int j0 = g * APG;
    float xr[APG][3];
    {
      const float4* xv = reinterpret_cast<const float4*>(xf + (size_t)j0 * 3);
      float xs[APG * 3];
#pragma unroll
      for (int q = 0; q < APG * 3 / 4; ++q) {
        const float4 t = xv[q];
        xs[4 * q] = t.x;
        xs[4 * q + 1] = t.y;
        xs[4 * q + 2] = t.z;
        xs[4 * q + 3] = t.w;
      }
#pragma unroll
      for (int a = 0; a < APG; ++a) {
        const float v0 = xs[3 * a] - c.x, v1 = xs[3 * a + 1] - c.y, v2 = xs[3 * a + 2] - c.z;
        xr[a][0] = R[0] * v0 + R[3] * v1 + R[6] * v2;
        xr[a][1] = R[1] * v0 + R[4] * v1 + R[7] * v2;
        xr[a][2] = R[2] * v0 + R[5] * v1 + R[8] * v2;
      }
    }
    float wv[APG];
#pragma unroll
    for (int a = 0; a < APG; ++a) wv[a] = wts ? wts[j0 + a] : 1.0f;
    // every landmark vector of the group is requested before any is used
    uint4 raw[LPB][3];
#pragma unroll
    for (int l = 0; l < LPB; ++l) {
      const int i = min(i0 + l, M - 1);  // rows beyond M repeat the last landmark; not written
      const uint4* src = reinterpret_cast<const uint4*>(lm + ((size_t)i * N + j0) * 3);
#pragma unroll
      for (int q = 0; q < 3; ++q) raw[l][q] = src[q];
    }
#pragma unroll
    for (int l = 0; l < LPB; ++l) {
      const int i = min(i0 + l, M - 1);
      float av[APG * 3];
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const unsigned u[4] = {raw[l][q].x, raw[l][q].y, raw[l][q].z, raw[l][q].w};
        if (sizeof(LT) == 2) {
#pragma unroll
          for (int h = 0; h < 4; ++h) {
            const __half2 hh = *reinterpret_cast<const __half2*>(&u[h]);
            const float2 ff = __half22float2(hh);
            av[8 * q + 2 * h] = ff.x;
            av[8 * q + 2 * h + 1] = ff.y;
          }
        } else {
#pragma unroll
          for (int h = 0; h < 4; ++h) av[4 * q + h] = __uint_as_float(u[h]);
        }
      }
      float o[3] = {0.0f, 0.0f, 0.0f};
      if (sizeof(LT) == 2) {  // one 16-atom block offset serves the group of 8
        const float* op = lmoff + ((size_t)i * ((N + 15) >> 4) + (j0 >> 4)) * 3;
        o[0] = op[0];
        o[1] = op[1];
        o[2] = op[2];
      }
      const float* Bl = B[l];
      float t = acc[l];
#pragma unroll
      for (int a = 0; a < APG; ++a) {
        const float a0 = av[3 * a] + o[0], a1 = av[3 * a + 1] + o[1], a2 = av[3 * a + 2] + o[2];
        const float d0 = xr[a][0] - (Bl[0] * a0 + Bl[1] * a1 + Bl[2] * a2);
        const float d1 = xr[a][1] - (Bl[3] * a0 + Bl[4] * a1 + Bl[5] * a2);
        const float d2 = xr[a][2] - (Bl[6] * a0 + Bl[7] * a1 + Bl[8] * a2);
        t = fmaf(wv[a] * d0, d0, fmaf(wv[a] * d1, d1, fmaf(wv[a] * d2, d2, t)));
      }
      acc[l] = t;
    }
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int l = 0; l < LPB; ++l) {
    const float t = warp_sum_float(acc[l]);
    if (lane == 0) red[w][l] = t;
  }
  __syncthreads();
  if ((int)threadIdx.x < LPB && i0 + (int)threadIdx.x < M) {
    float t = 0.0f;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[k][threadIdx.x];
    Dout[(size_t)f * M + i0 + threadIdx.x] = t * (float)dscale;
  }
}

template <typename K>
void allow_smem(K kernel, size_t bytes) {
  if (bytes > 48 * 1024) cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace

bool stream_fits(Prec p, int N) {
  if (p == P_F64) return false;
  const size_t bytes = (size_t)3 * N * (p == P_F16 ? sizeof(__half) : sizeof(float));
  return bytes <= 200 * 1024;
}

void launch_exact_stream(Prec p, int rows, const int* row_frame, const void* frames, const LandmarkDev& L,
                         FrameInfo fi, void* D, void* Rout, unsigned* status, cudaStream_t st) {
  if (rows <= 0 || L.M <= 0) return;
  const size_t es = p == P_F16 ? sizeof(__half) : sizeof(float);
  const size_t smem = (size_t)3 * L.N * es;
  const bool aligned = ((3 * (size_t)L.N * es) % 16 == 0) && ((uintptr_t)L.coords % 16 == 0);
  if (p == P_F16) {
    allow_smem(exact_stream_f32<__half>, smem);
    exact_stream_f32<__half><<<L.M, ST_THREADS, smem, st>>>(rows, row_frame, (const float*)frames, fi.c32, fi.G,
                                                            (const __half*)L.coords, L.off, L.G, L.w, L.M, L.N, L.dscale,
                                                            aligned, (float*)D, (float*)Rout, status,
                                                            L.newton_cap);
  } else {
    allow_smem(exact_stream_f32<float>, smem);
    exact_stream_f32<float><<<L.M, ST_THREADS, smem, st>>>(rows, row_frame, (const float*)frames, fi.c32, fi.G,
                                                           (const float*)L.coords, L.off, L.G, L.w, L.M, L.N, L.dscale,
                                                           aligned, (float*)D, (float*)Rout, status,
                                                           L.newton_cap);
  }
  note_launch();
}

void launch_approx_stream(Prec p, int max_rows, const int* approx_list, const int* approx_seg, const int* count,
                          const void* frames, const LandmarkDev& L, FrameInfo fi, const double4* qxy, const void* Bseg,
                          void* D, cudaStream_t st) {
  if (L.M <= 0) return;
  const int apg = p == P_F16 ? 8 : 4;
  if (max_rows == 1 && L.N % apg == 0 && (uintptr_t)L.coords % 16 == 0 && (uintptr_t)frames % 16 == 0) {
    // landmarks per 128-thread CTA (measured on the 5000-atom, 2000-landmark set): FP32 4 (the
    // frame is re-read and rotated once per CTA), FP16 2 (half the bytes per landmark: more
    // CTAs in flight cover the load latency better)
    if (p == P_F16)
      approx_stream_vec<__half, 2><<<(unsigned)((L.M + 1) / 2), 128, 0, st>>>(
          approx_list, approx_seg, count, (const float*)frames, fi.c32, qxy, (const __half*)L.coords, L.off,
          (const float*)Bseg, L.w, L.M, L.N, L.dscale, (float*)D);
    else
      approx_stream_vec<float, 4><<<(unsigned)((L.M + 3) / 4), 128, 0, st>>>(
          approx_list, approx_seg, count, (const float*)frames, fi.c32, qxy, (const float*)L.coords, L.off,
          (const float*)Bseg, L.w, L.M, L.N, L.dscale, (float*)D);
    note_launch();
    return;
  }
  const size_t es = p == P_F16 ? sizeof(__half) : sizeof(float);
  const size_t smem = (size_t)3 * L.N * es;
  const bool aligned = ((3 * (size_t)L.N * es) % 16 == 0) && ((uintptr_t)L.coords % 16 == 0);
  if (p == P_F16) {
    allow_smem(approx_stream_f32<__half>, smem);
    approx_stream_f32<__half><<<L.M, ST_THREADS, smem, st>>>(approx_list, approx_seg, count, (const float*)frames,
                                                             fi.c32, qxy, (const __half*)L.coords, L.off,
                                                             (const float*)Bseg, L.w, L.M, L.N, L.dscale, aligned,
                                                             (float*)D);
  } else {
    allow_smem(approx_stream_f32<float>, smem);
    approx_stream_f32<float><<<L.M, ST_THREADS, smem, st>>>(approx_list, approx_seg, count, (const float*)frames,
                                                            fi.c32, qxy, (const float*)L.coords, L.off, (const float*)Bseg,
                                                            L.w, L.M, L.N, L.dscale, aligned, (float*)D);
  }
  note_launch();
}

}  // namespace pcv

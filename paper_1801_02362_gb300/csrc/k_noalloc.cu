// k_noalloc.cu -- pcv_evaluate_exact_noalloc: exact-mode path CVs that never allocate.
//
// Some callers cannot call cudaMalloc: an MD engine that hands all device memory out of
// its own pool, or code running where a device allocation would stall or break the
// caller's timing.  This entry point keeps every intermediate in one fixed, file-scope
// device array (kScratchBytes), so it calls no cudaMalloc, cudaFree or allocating library
// routine.  The array exists on every GPU that loads the library until the process exits.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <mutex>

#include "../../include/pcv.h"
#include "pcv_internal.h"

namespace {

constexpr size_t kScratchBytes = (size_t)PCV_NOALLOC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;

// The shared scratch.  Host code must not pass `g_scratch` itself to a kernel: on the host
// this name is only a stand-in for the symbol.  Its device address comes from
// cudaGetSymbolAddress (see scratch_address).
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mu;
void* g_addr[kMaxDevices] = {nullptr};

// Device address of g_scratch on the current device, looked up once per device.
cudaError_t scratch_address(int device, void** out) {
  std::lock_guard<std::mutex> lock(g_mu);
  if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
  if (!g_addr[device]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return e;
    g_addr[device] = p;
  }
  *out = g_addr[device];
  return cudaSuccess;
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// Centre each landmark by its mean in FP64 and store the centred coordinates as FP32
// (the same rounding pcv_set_landmarks applies on the host), with G_a = sum_j |a_j|^2 of
// the stored values (uniform weights, kernel units) and q_i = i + 1 when no properties are
// given.  One warp per landmark.
__global__ void prep_landmarks_noalloc(int M, int N, const float* __restrict__ in, float* __restrict__ out,
                                       double* __restrict__ G, const double* __restrict__ q_in,
                                       double* __restrict__ q_out, float* __restrict__ q_out32) {
  const int i = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
  if (i >= M) return;
  const int lane = threadIdx.x & 31;
  const float* a = in + (size_t)i * N * 3;
  double c[3] = {0.0, 0.0, 0.0};
  for (int j = lane; j < N; j += 32)
    for (int k = 0; k < 3; ++k) c[k] += (double)a[3 * j + k];
  for (int k = 0; k < 3; ++k) {
    for (int off = 16; off > 0; off >>= 1) c[k] += __shfl_xor_sync(0xffffffffu, c[k], off);
    c[k] /= (double)N;
  }
  double g = 0.0;
  float* o = out + (size_t)i * N * 3;
  for (int j = lane; j < N; j += 32)
    for (int k = 0; k < 3; ++k) {
      const float v = (float)((double)a[3 * j + k] - c[k]);
      o[3 * j + k] = v;
      g += (double)v * (double)v;
    }
  for (int off = 16; off > 0; off >>= 1) g += __shfl_xor_sync(0xffffffffu, g, off);
  if (lane == 0) {
    G[i] = g;
    q_out[i] = q_in ? q_in[i] : (double)(i + 1);
    q_out32[i] = (float)q_out[i];
  }
}

}  // namespace

extern "C" PCV_API pcv_status pcv_evaluate_exact_noalloc(int F, int M, int N, const float* frames,
                                                         const float* landmarks, const double* q, double lambda,
                                                         double* s, double* z, double* msd, void* cuda_stream,
                                                         char* err, size_t err_len) {
  auto fail = [&](pcv_status st, const char* msg) {
    if (err && err_len > 0) {
      snprintf(err, err_len, "%s", msg);
    }
    return st;
  };
  if (F < 0 || M < 1 || N < 3) return fail(PCV_EINVAL, "need F >= 0, M >= 1, N >= 3");
  if (!(lambda > 0.0) || !std::isfinite(lambda)) return fail(PCV_EINVAL, "lambda must be > 0 and finite");
  if (F == 0) return PCV_OK;
  if (!frames || !landmarks || !s || !z) return fail(PCV_EINVAL, "frames, landmarks, s and z are required");
  // scratch layout, every piece 256-byte aligned
  const size_t b_lm = align256((size_t)M * N * 3 * sizeof(float));
  const size_t b_G = align256((size_t)M * sizeof(double));
  const size_t b_q = align256((size_t)M * sizeof(double));
  const size_t b_q32 = align256((size_t)M * sizeof(float));
  const size_t b_c32 = align256((size_t)F * sizeof(float4));
  const size_t b_c64 = align256((size_t)F * sizeof(double4));
  const size_t b_fG = align256((size_t)F * sizeof(double));
  const size_t b_D = align256((size_t)F * M * sizeof(float));
  const size_t b_ms = align256((size_t)F * 2 * sizeof(double));
  const size_t b_st = 256;
  const size_t need = b_lm + b_G + b_q + b_q32 + b_c32 + b_c64 + b_fG + b_D + b_ms + b_st;
  if (need > kScratchBytes) {
    char msg[160];
    snprintf(msg, sizeof(msg), "problem needs %zu bytes of scratch, more than the fixed %zu (reduce F or M)", need,
             kScratchBytes);
    return fail(PCV_EINVAL, msg);
  }
  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess) return fail(PCV_ECUDA, "cudaGetDevice failed");
  void* base = nullptr;
  cudaError_t e = scratch_address(device, &base);
  if (e != cudaSuccess) return fail(PCV_ECUDA, cudaGetErrorString(e));
  char* p = (char*)base;
  float* lm = (float*)p;
  p += b_lm;
  double* G = (double*)p;
  p += b_G;
  double* qs = (double*)p;
  p += b_q;
  float* qs32 = (float*)p;
  p += b_q32;
  pcv::FrameInfo fi;
  fi.c32 = (float4*)p;
  p += b_c32;
  fi.c64 = (double4*)p;
  p += b_c64;
  fi.G = (double*)p;
  p += b_fG;
  float* D = (float*)p;
  p += b_D;
  float* mstat = (float*)p;
  p += b_ms;
  unsigned* status = (unsigned*)p;

  cudaStream_t st = (cudaStream_t)cuda_stream;
  // the status word must start at zero: the scratch keeps the previous call's contents
  if ((e = cudaMemsetAsync(status, 0, sizeof(unsigned), st)) != cudaSuccess) return fail(PCV_ECUDA, cudaGetErrorString(e));
  prep_landmarks_noalloc<<<(unsigned)((M + 3) / 4), 128, 0, st>>>(M, N, landmarks, lm, G, q, qs, qs32);
  pcv::LandmarkDev L;
  L.M = M;
  L.N = N;
  L.coords = lm;
  L.G = G;
  L.q = qs;
  L.q32 = qs32;
  L.dscale = 1.0 / N;
  pcv::launch_frame_prep(pcv::P_F32, F, frames, L, fi, st);
  pcv::launch_exact_pairs(pcv::P_F32, F, nullptr, nullptr, frames, L, fi, D, nullptr, status, st);
  pcv::launch_finalize(pcv::P_F32, F, M, D, qs, qs32, lambda, s, z, mstat, nullptr, msd, false, st);
  if ((e = cudaGetLastError()) != cudaSuccess) return fail(PCV_ECUDA, cudaGetErrorString(e));
  unsigned h_status = 0;
  if ((e = cudaMemcpyAsync(&h_status, status, sizeof(unsigned), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
    return fail(PCV_ECUDA, cudaGetErrorString(e));
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return fail(PCV_ECUDA, cudaGetErrorString(e));
  if (h_status & pcv::STATUS_NOCONV) return fail(PCV_ENOCONV, "an eigen-solve reached its iteration cap");
  return PCV_OK;
}

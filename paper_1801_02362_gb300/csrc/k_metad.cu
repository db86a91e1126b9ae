// k_metad.cu -- Gaussian-hill metadynamics bias on the path CVs (Eq. vbias) and its force.
//
// The paper's metadynamics adds a Gaussian hill in (s, z) every tau_G steps at the current
// CV values; the bias of a step is the sum of the hills of the steps before it, and the
// bias force is its coordinate derivative through the CVs (Eq. vbias, Section 2).  The
// batched form evaluates F consecutive steps at once: this call's hills are known from its
// own s and z (deposited at the steps t' = tau_G, 2 tau_G, ... of Eq. vbias: step indices
// counted from 0 that are positive multiples of tau_G), so step t sums
// the hills held before the call plus this call's hills of steps before t -- a prefix of
// one hill array.  Kernels:
//   metad_deposit_kernel  appends this call's hills (s_t, z_t);
//   metad_bias_kernel     one thread per step, the hills staged in shared memory in tiles
//                         shared by a block of consecutive steps: V, -dV/ds, -dV/dz over
//                         the step's prefix of hills.  Positions are split into FP32
//                         (hi, lo) pairs, so each difference (s_hi - h_hi) + (s_lo - h_lo)
//                         is accurate to FP32 rounding of the difference itself (no FP64
//                         instruction per hill); the Gaussians are FP32; sums of 32 terms go
//                         into compensated (hi, lo) totals;
//   the force -(dV/ds ds/dx + dV/dz dz/dx) is the chain-rule kernel of pcv_combine_grad.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <string>

#include "../../include/pcv.h"
#include "pcv_device.cuh"
#include "pcv_internal.h"

struct pcv_metad {
  int device = 0;
  cudaStream_t stream = nullptr;
  double w = 0.0, sigma_s = 1.0, sigma_z = 1.0;
  int stride = 1, cap = 0, n_hills = 0;
  int64_t steps = 0;
  double* hills = nullptr;  // device, cap x (s_k, z_k)
  double* g = nullptr;      // device workspace: -dV/ds, -dV/dz of gcap frames
  size_t gcap = 0;
  std::string err = "no error";
};

namespace {

std::string g_metad_err = "no error";

pcv_status mfail(pcv_metad* m, pcv_status st, const char* fmt, ...) {
  char buf[256];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  (m ? m->err : g_metad_err) = buf;
  return st;
}

#define MCUDA(m, expr)                                                                        \
  do {                                                                                        \
    cudaError_t e_ = (expr);                                                                  \
    if (e_ != cudaSuccess) return mfail((m), PCV_ECUDA, "%s: %s", #expr, cudaGetErrorString(e_)); \
  } while (0)

// first step of the call that deposits a hill, and how many of the call's F steps do
void deposits(int64_t step0, int stride, int F, int* t0, int* nd) {
  // the smallest positive multiple of the stride at or after step0 (step 0 deposits nothing)
  const int64_t first = step0 == 0 ? (int64_t)stride : ((step0 + stride - 1) / stride) * stride;
  *t0 = (int)(first - step0);
  *nd = *t0 < F ? (F - 1 - *t0) / stride + 1 : 0;
}

__global__ void metad_deposit_kernel(int nd, int t0, int stride, int n_prev, const double* __restrict__ s,
                                     const double* __restrict__ z, double* __restrict__ hills) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nd) return;
  const int t = t0 + j * stride;
  hills[2 * (n_prev + j)] = s[t];
  hills[2 * (n_prev + j) + 1] = z[t];
}

constexpr int MD_THREADS = 256, MD_TILE = 1024;

__device__ __forceinline__ float2 split2(double v) {
  const float hi = (float)v;
  return make_float2(hi, (float)(v - (double)hi));
}

// hills of steps before step t: those held before the call and this call's deposits at
// steps t0, t0 + stride, ... below t
__device__ __forceinline__ int hills_before(int t, int t0, int stride, int n_prev) {
  return n_prev + (t > t0 ? (t - 1 - t0) / stride + 1 : 0);
}

__global__ void __launch_bounds__(MD_THREADS)
metad_bias_kernel(int F, int t0, int stride, int n_prev, const double* __restrict__ s, const double* __restrict__ z,
                  const double* __restrict__ hills, float w, float inv2ss, float inv2sz, float invss2, float invsz2,
                  double* __restrict__ V, double* __restrict__ g) {
  __shared__ float4 sh[MD_TILE];  // (s_hi, s_lo, z_hi, z_lo) of the hills of one tile
  const int t = blockIdx.x * MD_THREADS + threadIdx.x;
  const int t_last = min(F - 1, (int)(blockIdx.x * MD_THREADS + MD_THREADS - 1));
  const int n_max = hills_before(t_last, t0, stride, n_prev);  // the block's largest prefix
  const int n = t < F ? hills_before(t, t0, stride, n_prev) : 0;
  float2 sp = make_float2(0.0f, 0.0f), zp = make_float2(0.0f, 0.0f);
  if (t < F) {
    sp = split2(s[t]);
    zp = split2(z[t]);
  }
  float v = 0.0f, gs = 0.0f, gz = 0.0f;           // chunk partial sums
  float vh = 0.0f, vl = 0.0f, sh_ = 0.0f, sl_ = 0.0f, zh_ = 0.0f, zl_ = 0.0f;  // compensated totals
  for (int k0 = 0; k0 < n_max; k0 += MD_TILE) {
    const int kn = min(MD_TILE, n_max - k0);
    __syncthreads();  // the previous tile's readers are done
    for (int e = threadIdx.x; e < kn; e += MD_THREADS) {
      const float2 a = split2(hills[2 * (k0 + e)]), b = split2(hills[2 * (k0 + e) + 1]);
      sh[e] = make_float4(a.x, a.y, b.x, b.y);
    }
    __syncthreads();
    const int kend = min(kn, n - k0);  // this step's prefix within the tile
    for (int k = 0; k < kend; ++k) {
      const float4 h = sh[k];
      const float ds = (sp.x - h.x) + (sp.y - h.y), dz = (zp.x - h.z) + (zp.y - h.w);
      const float e = w * expf(-fmaf(ds * ds, inv2ss, dz * dz * inv2sz));
      v += e;
      gs = fmaf(e, ds, gs);  // -dV/ds = sum_k e_k ds_k / sigma_s^2 (scaled below)
      gz = fmaf(e, dz, gz);
      if ((k & 31) == 31) {
        pcv::two_sum_acc(vh, vl, v);
        pcv::two_sum_acc(sh_, sl_, gs);
        pcv::two_sum_acc(zh_, zl_, gz);
        v = gs = gz = 0.0f;
      }
    }
    pcv::two_sum_acc(vh, vl, v);
    pcv::two_sum_acc(sh_, sl_, gs);
    pcv::two_sum_acc(zh_, zl_, gz);
    v = gs = gz = 0.0f;
  }
  if (t < F) {
    V[t] = (double)vh + (double)vl;
    g[t] = ((double)sh_ + (double)sl_) * (double)invss2;
    g[F + t] = ((double)zh_ + (double)zl_) * (double)invsz2;
  }
}

}  // namespace

extern "C" {

pcv_status pcv_metad_create(pcv_metad** out, int device, void* cuda_stream, double height, double sigma_s,
                            double sigma_z, int stride, int max_hills) {
  if (!out) return mfail(nullptr, PCV_EINVAL, "out is NULL");
  *out = nullptr;
  if (!(std::isfinite(height)) || !(sigma_s > 0.0) || !(sigma_z > 0.0) || !std::isfinite(sigma_s) ||
      !std::isfinite(sigma_z))
    return mfail(nullptr, PCV_EINVAL, "height must be finite and the widths > 0");
  if (stride < 1 || max_hills < 1) return mfail(nullptr, PCV_EINVAL, "stride and max_hills must be >= 1");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
    return mfail(nullptr, PCV_EINVAL, "bad device %d", device);
  if (cudaSetDevice(device) != cudaSuccess) return mfail(nullptr, PCV_ECUDA, "cudaSetDevice failed");
  pcv_metad* m = new pcv_metad();
  m->device = device;
  m->stream = (cudaStream_t)cuda_stream;
  m->w = height;
  m->sigma_s = sigma_s;
  m->sigma_z = sigma_z;
  m->stride = stride;
  m->cap = max_hills;
  if (cudaMalloc(&m->hills, sizeof(double) * 2 * (size_t)max_hills) != cudaSuccess) {
    cudaGetLastError();
    delete m;
    return mfail(nullptr, PCV_ENOMEM, "cudaMalloc of %d hills failed", max_hills);
  }
  *out = m;
  return PCV_OK;
}

pcv_status pcv_metad_destroy(pcv_metad* m) {
  if (!m) return PCV_OK;
  cudaSetDevice(m->device);
  if (m->stream)
    cudaStreamSynchronize(m->stream);
  else
    cudaDeviceSynchronize();
  cudaFree(m->hills);
  cudaFree(m->g);
  delete m;
  return PCV_OK;
}

pcv_status pcv_metad_set_stream(pcv_metad* m, void* cuda_stream) {
  if (!m) return mfail(nullptr, PCV_EINVAL, "NULL metadynamics object");
  m->stream = (cudaStream_t)cuda_stream;
  return PCV_OK;
}

pcv_status pcv_metad_apply(pcv_metad* m, int precision, int F, int N, const double* s, const double* z,
                           const void* dsdx, const void* dzdx, double* bias, void* force) {
  if (!m) return mfail(nullptr, PCV_EINVAL, "NULL metadynamics object");
  if (F < 0 || N < 0) return mfail(m, PCV_EINVAL, "F and N must be >= 0");
  if (precision < PCV_FP64 || precision > PCV_FP16_STORAGE) return mfail(m, PCV_EINVAL, "bad precision");
  if (F == 0) return PCV_OK;
  if (!s || !z || !bias) return mfail(m, PCV_EINVAL, "s, z and bias are required");
  if (force && (!dsdx || !dzdx || N < 1)) return mfail(m, PCV_EINVAL, "a force needs dsdx, dzdx and N >= 1");
  int t0 = 0, nd = 0;
  deposits(m->steps, m->stride, F, &t0, &nd);
  if ((int64_t)m->n_hills + nd > m->cap)
    return mfail(m, PCV_EINVAL, "hill capacity %d exceeded (%d held, %d more)", m->cap, m->n_hills, nd);
  cudaSetDevice(m->device);
  if (m->gcap < (size_t)F) {
    cudaFree(m->g);
    m->g = nullptr;
    m->gcap = 0;
    if (cudaMalloc(&m->g, sizeof(double) * 2 * (size_t)F) != cudaSuccess) {
      cudaGetLastError();
      return mfail(m, PCV_ENOMEM, "cudaMalloc of the derivative workspace failed");
    }
    m->gcap = (size_t)F;
  }
  if (nd > 0) {
    metad_deposit_kernel<<<(nd + 127) / 128, 128, 0, m->stream>>>(nd, t0, m->stride, m->n_hills, s, z, m->hills);
    pcv::note_launch();
  }
  const float inv2ss = (float)(0.5 / (m->sigma_s * m->sigma_s)), inv2sz = (float)(0.5 / (m->sigma_z * m->sigma_z));
  const float invss2 = (float)(1.0 / (m->sigma_s * m->sigma_s)), invsz2 = (float)(1.0 / (m->sigma_z * m->sigma_z));
  const unsigned blocks = (unsigned)((F + MD_THREADS - 1) / MD_THREADS);
  metad_bias_kernel<<<blocks, MD_THREADS, 0, m->stream>>>(F, t0, m->stride, m->n_hills, s, z, m->hills, (float)m->w, inv2ss,
                                                   inv2sz, invss2, invsz2, bias, m->g);
  pcv::note_launch();
  if (force)
    pcv::launch_combine_grad((pcv::Prec)precision, F, 3 * N, m->g, m->g + F, dsdx, dzdx, force, m->stream);
  MCUDA(m, cudaGetLastError());
  m->n_hills += nd;
  m->steps += F;
  return PCV_OK;
}

pcv_status pcv_metad_get_hills(pcv_metad* m, double* hills, int cap, int* n_hills, int64_t* steps) {
  if (!m || !n_hills) return mfail(m, PCV_EINVAL, "NULL argument");
  *n_hills = m->n_hills;
  if (steps) *steps = m->steps;
  if (!hills) return PCV_OK;
  if (cap < m->n_hills) return mfail(m, PCV_EINVAL, "buffer holds %d hills, %d needed", cap, m->n_hills);
  cudaSetDevice(m->device);
  MCUDA(m, m->stream ? cudaStreamSynchronize(m->stream) : cudaDeviceSynchronize());
  if (m->n_hills > 0)
    MCUDA(m, cudaMemcpy(hills, m->hills, sizeof(double) * 2 * (size_t)m->n_hills, cudaMemcpyDeviceToHost));
  return PCV_OK;
}

pcv_status pcv_metad_set_hills(pcv_metad* m, const double* hills, int n_hills, int64_t steps) {
  if (!m) return mfail(nullptr, PCV_EINVAL, "NULL metadynamics object");
  if (n_hills < 0 || n_hills > m->cap || steps < 0 || (n_hills > 0 && !hills))
    return mfail(m, PCV_EINVAL, "bad hill count %d (capacity %d) or step count", n_hills, m->cap);
  for (int k = 0; k < 2 * n_hills; ++k)
    if (!std::isfinite(hills[k])) return mfail(m, PCV_EINVAL, "hill %d is not finite", k / 2);
  cudaSetDevice(m->device);
  MCUDA(m, m->stream ? cudaStreamSynchronize(m->stream) : cudaDeviceSynchronize());
  if (n_hills > 0)
    MCUDA(m, cudaMemcpy(m->hills, hills, sizeof(double) * 2 * (size_t)n_hills, cudaMemcpyHostToDevice));
  m->n_hills = n_hills;
  m->steps = steps;
  return PCV_OK;
}

const char* pcv_metad_last_error(const pcv_metad* m) { return m ? m->err.c_str() : g_metad_err.c_str(); }

}  // extern "C"

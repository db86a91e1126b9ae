// k_shard.cu -- merging path CVs computed on landmark shards.
//
// When the M landmarks are split into shards r (each with its landmarks' global properties
// q_i), every shard yields for each frame its own s_r, z_r (Eqs. 5-6 over its landmarks)
// and gradients.  Because z_r = -(1/lambda) ln sum_{i in r} exp(-lambda D_i), the whole-path
// values follow from the shard values alone:
//   z  = -(1/lambda) ln sum_r exp(-lambda z_r),
//   w_r = exp(-lambda (z_r - z)),  sum_r w_r = 1,
//   s  = sum_r w_r s_r,
//   dz = sum_r w_r dz_r,
//   ds = sum_r w_r (ds_r - lambda (s_r - s) dz_r).
// On several GPUs this is one MIN all-reduce of z_r (giving zmin) and one SUM all-reduce of
// the packed terms: with u_r = exp(-lambda (z_r - zmin)),
//   scalars  [u_r, u_r s_r]                 (2 per frame)
//   elements [u_r ds_r, u_r s_r dz_r, u_r dz_r]  (3 per coordinate)
// after which  W = sum u_r,  s = sum u_r s_r / W,  z = zmin - ln(W) / lambda,
//   dz = sum u_r dz_r / W,  ds = (sum u_r ds_r - lambda (sum u_r s_r dz_r - s sum u_r dz_r)) / W.
// Packed terms are FP64 so that the partial cancellation in the last line costs nothing.
// The same arithmetic runs on the host (pcv_shard_*_host) for callers and tests without a GPU.
#include <cmath>
#include <cstdint>

#include "../../include/pcv.h"
#include "pcv_internal.h"

namespace pcv {
namespace {

__host__ __device__ inline void pack_scalars(int f, double lambda, const double* zmin, const double* s,
                                             const double* z, double* scal) {
  const double u = exp(-lambda * (z[f] - zmin[f]));
  scal[2 * f] = u;
  scal[2 * f + 1] = u * s[f];
}

template <typename GT>
__host__ __device__ inline void pack_elem(size_t k, int f, double lambda, const double* zmin, const double* s,
                                          const double* z, const GT* dsdx, const GT* dzdx, double* elem) {
  const double u = exp(-lambda * (z[f] - zmin[f]));
  const double dz = (double)dzdx[k];
  elem[3 * k] = u * (double)dsdx[k];
  elem[3 * k + 1] = u * s[f] * dz;
  elem[3 * k + 2] = u * dz;
}

__host__ __device__ inline void unpack_scalars(int f, double lambda, const double* zmin, const double* scal,
                                               double* s, double* z) {
  const double W = scal[2 * f];
  s[f] = scal[2 * f + 1] / W;
  z[f] = zmin[f] - log(W) / lambda;
}

template <typename GT>
__host__ __device__ inline void unpack_elem(size_t k, int f, double lambda, const double* scal, const double* elem,
                                            GT* dsdx, GT* dzdx) {
  const double W = scal[2 * f];
  const double sf = scal[2 * f + 1] / W;
  const double A = elem[3 * k], B = elem[3 * k + 1], C = elem[3 * k + 2];
  dsdx[k] = (GT)((A - lambda * (B - sf * C)) / W);
  dzdx[k] = (GT)(C / W);
}

// one thread per (frame, coordinate); thread 0 of each frame also does the scalars
template <typename GT>
__global__ void pack_kernel(int F, int N3, double lambda, const double* zmin, const double* s, const double* z,
                            const GT* dsdx, const GT* dzdx, double* scal, double* elem) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  for (int f = blockIdx.y; f < F; f += gridDim.y) {
    if (e == 0) pack_scalars(f, lambda, zmin, s, z, scal);
    if (dsdx && e < N3) pack_elem<GT>((size_t)f * N3 + e, f, lambda, zmin, s, z, dsdx, dzdx, elem);
  }
}

template <typename GT>
__global__ void unpack_kernel(int F, int N3, double lambda, const double* zmin, const double* scal,
                              const double* elem, double* s, double* z, GT* dsdx, GT* dzdx) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  for (int f = blockIdx.y; f < F; f += gridDim.y) {
    if (e == 0) unpack_scalars(f, lambda, zmin, scal, s, z);
    if (dsdx && e < N3) unpack_elem<GT>((size_t)f * N3 + e, f, lambda, scal, elem, dsdx, dzdx);
  }
}

bool bad_args(int F, int N, double lambda, const void* zmin, const void* a, const void* b, const void* g1,
              const void* g2) {
  if (F < 0 || N < 1 || !(lambda > 0.0) || !std::isfinite(lambda)) return true;
  if (F > 0 && (!zmin || !a || !b)) return true;
  if ((g1 == nullptr) != (g2 == nullptr)) return true;
  return false;
}

}  // namespace
}  // namespace pcv

using namespace pcv;

extern "C" {

PCV_API pcv_status pcv_shard_pack(int precision, int F, int N, double lambda, const double* zmin, const double* s,
                                  const double* z, const void* dsdx, const void* dzdx, double* scalars,
                                  double* elements, void* stream) {
  if (bad_args(F, N, lambda, zmin, s, z, dsdx, dzdx) || !scalars || (dsdx && !elements) || precision < 0 ||
      precision > 2)
    return PCV_EINVAL;
  if (F == 0) return PCV_OK;
  const cudaStream_t st = (cudaStream_t)stream;
  const int N3 = 3 * N;
  const dim3 grid((N3 + 255) / 256, F < 65535 ? F : 65535);
  if (precision == PCV_FP64)
    pack_kernel<double><<<grid, 256, 0, st>>>(F, N3, lambda, zmin, s, z, (const double*)dsdx, (const double*)dzdx,
                                              scalars, elements);
  else
    pack_kernel<float><<<grid, 256, 0, st>>>(F, N3, lambda, zmin, s, z, (const float*)dsdx, (const float*)dzdx,
                                             scalars, elements);
  note_launch();
  return cudaGetLastError() == cudaSuccess ? PCV_OK : PCV_ECUDA;
}

PCV_API pcv_status pcv_shard_unpack(int precision, int F, int N, double lambda, const double* zmin,
                                    const double* scalars, const double* elements, double* s, double* z, void* dsdx,
                                    void* dzdx, void* stream) {
  if (bad_args(F, N, lambda, zmin, scalars, s, dsdx, dzdx) || !z || (dsdx && !elements) || precision < 0 ||
      precision > 2)
    return PCV_EINVAL;
  if (F == 0) return PCV_OK;
  const cudaStream_t st = (cudaStream_t)stream;
  const int N3 = 3 * N;
  const dim3 grid((N3 + 255) / 256, F < 65535 ? F : 65535);
  if (precision == PCV_FP64)
    unpack_kernel<double><<<grid, 256, 0, st>>>(F, N3, lambda, zmin, scalars, elements, s, z, (double*)dsdx,
                                                (double*)dzdx);
  else
    unpack_kernel<float><<<grid, 256, 0, st>>>(F, N3, lambda, zmin, scalars, elements, s, z, (float*)dsdx,
                                               (float*)dzdx);
  note_launch();
  return cudaGetLastError() == cudaSuccess ? PCV_OK : PCV_ECUDA;
}

PCV_API pcv_status pcv_shard_pack_host(int precision, int F, int N, double lambda, const double* zmin,
                                       const double* s, const double* z, const void* dsdx, const void* dzdx,
                                       double* scalars, double* elements) {
  if (bad_args(F, N, lambda, zmin, s, z, dsdx, dzdx) || !scalars || (dsdx && !elements) || precision < 0 ||
      precision > 2)
    return PCV_EINVAL;
  const int N3 = 3 * N;
  for (int f = 0; f < F; ++f) {
    pack_scalars(f, lambda, zmin, s, z, scalars);
    if (!dsdx) continue;
    for (int e = 0; e < N3; ++e) {
      const size_t k = (size_t)f * N3 + e;
      if (precision == PCV_FP64)
        pack_elem<double>(k, f, lambda, zmin, s, z, (const double*)dsdx, (const double*)dzdx, elements);
      else
        pack_elem<float>(k, f, lambda, zmin, s, z, (const float*)dsdx, (const float*)dzdx, elements);
    }
  }
  return PCV_OK;
}

PCV_API pcv_status pcv_shard_unpack_host(int precision, int F, int N, double lambda, const double* zmin,
                                         const double* scalars, const double* elements, double* s, double* z,
                                         void* dsdx, void* dzdx) {
  if (bad_args(F, N, lambda, zmin, scalars, s, dsdx, dzdx) || !z || (dsdx && !elements) || precision < 0 ||
      precision > 2)
    return PCV_EINVAL;
  const int N3 = 3 * N;
  for (int f = 0; f < F; ++f) {
    unpack_scalars(f, lambda, zmin, scalars, s, z);
    if (!dsdx) continue;
    for (int e = 0; e < N3; ++e) {
      const size_t k = (size_t)f * N3 + e;
      if (precision == PCV_FP64)
        unpack_elem<double>(k, f, lambda, scalars, elements, (double*)dsdx, (double*)dzdx);
      else
        unpack_elem<float>(k, f, lambda, scalars, elements, (float*)dsdx, (float*)dzdx);
    }
  }
  return PCV_OK;
}

}  // extern "C"

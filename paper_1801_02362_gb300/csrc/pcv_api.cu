// pcv_api.cu -- the C ABI (include/pcv.h): context, landmark preparation, the
// close-structure orchestration of Algorithm 2 over a batch of frames, and state I/O.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/pcv.h"
#include "pcv_internal.h"

using namespace pcv;

namespace {

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

// small device struct read back by the host during the refresh search
struct Small {
  ScanResult scan;
  int first;
  int refresh_count;
  int approx_count;
  int recheck_count;
  int last_refresh;
  int stop;  // first frame of the current chunk that definitely exceeds eps (launch_align_chunk)
  int nl_counts[4];  // neighbour list: updates, approximate updates, frames between updates
  float4 last_c32;
  double4 last_c64;
  double last_G;
};

// copy of the small struct into mapped host memory by the GPU's own stores: the host reads
// it after a stream synchronisation, and no copy engine is involved (a device-to-host copy
// here would queue behind large copies in flight on the same engine, e.g. the output copies
// of pcv_evaluate_host, and stall the refresh search)
__global__ void small_mirror_kernel(const Small* __restrict__ src, Small* __restrict__ dst) {
  const unsigned* a = reinterpret_cast<const unsigned*>(src);
  unsigned* b = reinterpret_cast<unsigned*>(dst);
  for (unsigned k = threadIdx.x; k < sizeof(Small) / sizeof(unsigned); k += blockDim.x) b[k] = a[k];
}

__global__ void small_tail_kernel(Small* sm, const int* refresh_list, const float4* c32, const double4* c64,
                                  const double* G) {
  const int n = sm->refresh_count;
  if (n > 0) {
    const int r = refresh_list[n - 1];
    sm->last_refresh = r;
    sm->last_c32 = c32[r];
    sm->last_c64 = c64[r];
    sm->last_G = G[r];
  } else {
    sm->last_refresh = -1;
  }
}

thread_local int64_t t_launches = 0;

// kernel families timed by the profiler
enum KernelId {
  K_PREP = 0, K_BAND, K_RECHECK, K_SCAN, K_CHUNK, K_FIRST, K_RECORDS, K_COMPACT, K_EXACT, K_APPROX,
  K_FINAL, K_ADJ_BETA, K_ADJ_FINISH, K_COMBINE, K_XY_REFINE, K_ADJ_BETA_SEG, K_MATERIALIZE, K_GAMMA, K_ADJ_MMA, K_SEG_MOMENTS,
  K_NL_SCHEDULE, K_NL_SELECT, K_NL_PAIR, K_NL_BETA, K_APPROX_MMA, K_COUNT
};
const char* const kKernelNames[PCV_PROFILE_KERNELS] = {
    "frame_prep", "align_band", "recheck_fp64", "band_scan", "align_chunk", "first_exceed", "records",
    "compact", "exact_pair", "approx_pair", "finalize", "adjoint_beta_pair", "adjoint_finish", "combine_grad", "xy_refine",
    "adjoint_beta_seg", "materialize", "gamma", "adjoint_beta_mma", "seg_moments", "nl_schedule", "nl_select",
    "nl_pair", "nl_beta", "approx_pair_mma"};
static_assert(K_COUNT <= PCV_PROFILE_KERNELS, "profiler table");

struct ProfEvent {
  int id;
  cudaEvent_t a, b;
};

}  // namespace

namespace pcv {
void note_launch(int n) { t_launches += n; }
}  // namespace pcv

struct pcv_ctx {
  int device = 0;
  int newton_cap = 60;                  // PCV_OPT_NEWTON_CAP
  int mma_group = 4;                    // PCV_OPT_MMA_GROUP
  int exact_tile = 0;                   // PCV_OPT_EXACT_TILE
  long long wait_cycles = 4000000000LL;  // PCV_OPT_WAIT_CYCLES
  cudaStream_t stream = nullptr;
  Prec prec = P_F32;
  // landmarks
  int M = 0, N = 0;
  bool have_lm = false;
  bool uniform = true;
  double dscale = 1.0;
  DevBuf lm, lmoff, lmG, lmA, lmA32, lmq, lmq32, w32, w64;
  bool split_w = false;  // alignment weights w' differ from the displacement weights w
  DevBuf wa32, wa64;
  double lambda = 0.0;
  bool have_lambda = false;
  double eps = -1.0;
  int band_W = 2;
  int min_chunk = 4096;
  int64_t mat_cap = int64_t(16) << 30;  // bytes of materialised operands allowed (PCV_OPT_MATERIALIZE)
  bool tensor_cores = true;             // segment adjoint on the tensor cores (PCV_OPT_TENSOR_CORES)
  double gap_estimate = 0.0;
  // neighbour list: size M_nl (0 = none) and update stride L; the list held between calls
  int nl_size = 0, nl_stride = 1;
  bool has_nl = false;
  DevBuf nl_keep;
  DevBuf nlSlot, nlUpd, nlU, nlUA, nlUAseg, nlN, NLtab, Rupd, Rnl, nlTiles, nlPart;
  DevBuf betaPart;  // landmark-range partial sums of the adjoint beta at small F
  // close state
  bool has_y = false;
  DevBuf y, Bprior;
  float4 y_c32 = {0, 0, 0, 0};
  double4 y_c64 = {0, 0, 0, 0};
  double y_G = 0.0;
  // workspace
  DevBuf c32, c64, fG, bandD, bandQ, bandF, chD, chQ, chF, rlist, rcount, recF, recRef, recD, recQ, reflist,
      segof, alist, aseg, Dbuf, Rpair, Bseg, mstat, status, nrecheck, small;
  DevBuf rcScr;  // the FP64 re-check's partial sums and completion counts
  DevBuf exSplit;  // partial sums of the exact pairs split over atom slices
  DevBuf Xr, Bm, GSb, GZb;  // materialised x', b and the gamma rows
  DevBuf Apk, Bpk;          // the same deviations packed for the tensor cores (FP16 h + l)
  DevBuf xtiles;            // their per-segment tile list, first rows, first tiles, count
  DevBuf Nx, Nb, Yc, Gsum;       // |dx|^2, |d|^2, centred close structures, Gamma sums
  DevBuf Amma, Bmma;              // tensor-core adjoint operands
  DevBuf S6;                      // per-segment landmark moments R A R^T of the finish
  DevBuf h_frames, h_s, h_z, h_gs, h_gz, h_msd, h_ref;  // device staging for pcv_evaluate_host
  cudaStream_t h2d_stream = nullptr, d2h_stream = nullptr;  // copy streams of pcv_evaluate_host
  int host_chunks = 0, host_end_share = 25;                  // its chunk plan (PCV_OPT_HOST_*)
  std::vector<cudaEvent_t> h_events;                        // its chunk events
  Small* small_host = nullptr;      // mapped pinned host memory
  Small* small_host_dev = nullptr;  // its device-side address
  // state of group evaluations led by this context (pcv_evaluate_group with it first)
  DevBuf grp_inst, grp_tiles;
  std::vector<uint64_t> grp_sig;       // what the captured graph was built for
  cudaGraphExec_t grp_exec = nullptr;
  cudaStream_t grp_stream = nullptr;   // the library's own stream: graphs cannot be captured on stream 0
  cudaEvent_t grp_ev[2] = {nullptr, nullptr};
  int grp_blocks = 0;                  // persistent grid chosen by the autotuner
  int grp_shape = 0;                   // exact tile shape chosen by the autotuner
  int grp_ntiles = 0;                  // tiles of that shape
  pcv_stats stats{};
  std::string err;
  // profiler
  bool prof_on = false;
  std::vector<ProfEvent> prof_pending;
  std::vector<cudaEvent_t> prof_pool;
  double prof_ms[PCV_PROFILE_KERNELS] = {0};
  int64_t prof_launches[PCV_PROFILE_KERNELS] = {0};
};

namespace {
cudaEvent_t prof_event(pcv_ctx* c) {
  if (!c->prof_pool.empty()) {
    cudaEvent_t e = c->prof_pool.back();
    c->prof_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// times the launches issued during its lifetime when the profiler is on
struct ProfScope {
  pcv_ctx* c;
  ProfEvent ev;
  ProfScope(pcv_ctx* ctx, int id) : c(ctx) {
    ev.id = id;
    ev.a = ev.b = nullptr;
    if (c->prof_on) {
      ev.a = prof_event(c);
      ev.b = prof_event(c);
      cudaEventRecord(ev.a, c->stream);
    }
  }
  ~ProfScope() {
    if (c->prof_on && ev.a) {
      cudaEventRecord(ev.b, c->stream);
      c->prof_pending.push_back(ev);
    }
  }
};
#define PROF(ctx, id) ProfScope prof_scope_##id(ctx, id)
}  // namespace

namespace {

std::string g_err = "no error";

pcv_status fail(pcv_ctx* c, pcv_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (c)
    c->err = buf;
  else
    g_err = buf;
  return st;
}

#define CUDA_TRY(c, expr)                                                                    \
  do {                                                                                       \
    cudaError_t e_ = (expr);                                                                 \
    if (e_ != cudaSuccess) return fail((c), PCV_ECUDA, "%s: %s", #expr, cudaGetErrorString(e_)); \
  } while (0)

pcv_status ensure(pcv_ctx* c, DevBuf& b, size_t bytes) {
  if (bytes == 0) bytes = 16;
  if (b.bytes >= bytes) return PCV_OK;
  // a launch error still pending is reported here: a failed allocation below clears the
  // runtime's error state, which would hide it from the caller's final check
  const cudaError_t pending = cudaGetLastError();
  if (pending != cudaSuccess) return fail(c, PCV_ECUDA, "kernel launch: %s", cudaGetErrorString(pending));
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.bytes = 0;
  cudaError_t e = cudaMalloc(&b.p, bytes);
  if (e != cudaSuccess) {
    b.p = nullptr;
    cudaGetLastError();
    return fail(c, PCV_ENOMEM, "cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
  }
  b.bytes = bytes;
  return PCV_OK;
}

void release(DevBuf& b) {
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.bytes = 0;
}

size_t frame_elem(Prec p) { return p == P_F64 ? sizeof(double) : sizeof(float); }
size_t store_elem(Prec p) { return p == P_F64 ? sizeof(double) : (p == P_F16 ? sizeof(__half) : sizeof(float)); }
size_t work_elem(Prec p) { return p == P_F64 ? sizeof(double) : sizeof(float); }

LandmarkDev lm_view(const pcv_ctx* c) {
  LandmarkDev L;
  L.M = c->M;
  L.N = c->N;
  L.coords = c->lm.p;
  L.G = (const double*)c->lmG.p;
  L.A = (const double*)c->lmA.p;
  L.A32 = (const float*)c->lmA32.p;
  L.q = (const double*)c->lmq.p;
  L.q32 = (const float*)c->lmq32.p;
  L.w = c->uniform ? nullptr : (const float*)c->w32.p;
  L.w64 = c->uniform ? nullptr : (const double*)c->w64.p;
  L.dscale = c->dscale;
  L.off = c->prec == P_F16 ? (const float*)c->lmoff.p : nullptr;
  L.wa = c->split_w ? (const float*)c->wa32.p : nullptr;
  L.wa64 = c->split_w ? (const double*)c->wa64.p : nullptr;
  L.newton_cap = c->newton_cap;
  L.wait_cycles = c->wait_cycles;
  L.mma_group = c->mma_group;
  L.exact_tile = c->exact_tile;
  return L;
}

RefDesc prior_view(const pcv_ctx* c) {
  RefDesc r;
  r.coords = c->y.p;
  r.c32 = c->y_c32;
  r.c64 = c->y_c64;
  r.G = c->y_G;
  return r;
}

pcv_status sync_small(pcv_ctx* c) {
  small_mirror_kernel<<<1, 64, 0, c->stream>>>((const Small*)c->small.p, c->small_host_dev);
  note_launch();
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  c->stats.host_syncs += 1;
  return PCV_OK;
}

}  // namespace

// =======================================================================================
extern "C" {

pcv_status pcv_create(pcv_ctx** out, int device, void* cuda_stream, int precision) {
  if (!out) return fail(nullptr, PCV_EINVAL, "pcv_create: out is NULL");
  *out = nullptr;
  if (precision < PCV_FP64 || precision > PCV_FP16_STORAGE)
    return fail(nullptr, PCV_EINVAL, "pcv_create: bad precision %d", precision);
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess) return fail(nullptr, PCV_ECUDA, "cudaGetDeviceCount: %s", cudaGetErrorString(e));
  if (device < 0 || device >= ndev) return fail(nullptr, PCV_EINVAL, "pcv_create: bad device %d", device);
  e = cudaSetDevice(device);
  if (e != cudaSuccess) return fail(nullptr, PCV_ECUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
  pcv_ctx* c = new pcv_ctx();
  c->device = device;
  c->stream = (cudaStream_t)cuda_stream;
  c->prec = (Prec)precision;
  pcv_status st = ensure(c, c->small, sizeof(Small));
  if (st == PCV_OK) st = ensure(c, c->status, 16);
  if (st == PCV_OK) st = ensure(c, c->nrecheck, 16);
  if (st == PCV_OK) st = ensure(c, c->rcScr, recheck_scratch_bytes());
  if (st == PCV_OK && (cudaHostAlloc((void**)&c->small_host, sizeof(Small), cudaHostAllocMapped) != cudaSuccess ||
                       cudaHostGetDevicePointer((void**)&c->small_host_dev, c->small_host, 0) != cudaSuccess))
    st = fail(nullptr, PCV_ENOMEM, "cudaHostAlloc (mapped) failed");
  if (st == PCV_OK && (cudaMemset(c->status.p, 0, 16) != cudaSuccess || cudaMemset(c->nrecheck.p, 0, 16) != cudaSuccess ||
                       cudaMemset(c->rcScr.p, 0, recheck_scratch_bytes()) != cudaSuccess))
    st = fail(nullptr, PCV_ECUDA, "cudaMemset failed");
  if (st != PCV_OK) {
    g_err = c->err.empty() ? g_err : c->err;
    pcv_destroy(c);
    return st;
  }
  c->err = "no error";
  *out = c;
  return PCV_OK;
}

pcv_status pcv_destroy(pcv_ctx* c) {
  if (!c) return PCV_OK;
  cudaSetDevice(c->device);
  if (c->stream) cudaStreamSynchronize(c->stream);
  else cudaDeviceSynchronize();
  DevBuf* bufs[] = {&c->lm, &c->lmoff, &c->lmG, &c->lmA, &c->lmA32, &c->lmq, &c->lmq32, &c->w32, &c->w64, &c->wa32,
                    &c->wa64, &c->y, &c->Bprior, &c->c32, &c->c64,
                    &c->fG, &c->bandD, &c->bandQ, &c->bandF, &c->chD, &c->chQ, &c->chF, &c->rlist, &c->rcount,
                    &c->recF, &c->recRef, &c->recD, &c->recQ, &c->reflist, &c->segof, &c->alist, &c->aseg,
                    &c->Dbuf, &c->Rpair, &c->Bseg, &c->Xr, &c->Bm, &c->Apk, &c->Bpk, &c->xtiles, &c->GSb, &c->GZb, &c->Nx, &c->Nb, &c->Yc, &c->Gsum, &c->Amma, &c->Bmma, &c->S6, &c->mstat, &c->status, &c->nrecheck, &c->rcScr, &c->exSplit, &c->small, &c->h_frames,
                    &c->h_s, &c->h_z, &c->h_gs, &c->h_gz, &c->h_msd, &c->h_ref, &c->grp_inst, &c->grp_tiles,
                    &c->nl_keep, &c->nlSlot, &c->nlUpd, &c->nlU, &c->nlUA, &c->nlUAseg, &c->nlN, &c->NLtab,
                    &c->Rupd, &c->Rnl, &c->nlTiles, &c->nlPart, &c->betaPart};
  if (c->grp_stream) cudaStreamSynchronize(c->grp_stream);
  for (DevBuf* b : bufs) release(*b);
  if (c->grp_exec) cudaGraphExecDestroy(c->grp_exec);
  for (cudaEvent_t e : c->grp_ev)
    if (e) cudaEventDestroy(e);
  if (c->grp_stream) cudaStreamDestroy(c->grp_stream);
  for (cudaStream_t hs : {c->h2d_stream, c->d2h_stream})
    if (hs) {
      cudaStreamSynchronize(hs);
      cudaStreamDestroy(hs);
    }
  for (cudaEvent_t e : c->h_events) cudaEventDestroy(e);
  for (const ProfEvent& e : c->prof_pending) {
    cudaEventDestroy(e.a);
    cudaEventDestroy(e.b);
  }
  for (cudaEvent_t e : c->prof_pool) cudaEventDestroy(e);
  if (c->small_host) cudaFreeHost(c->small_host);
  delete c;
  return PCV_OK;
}

pcv_status pcv_set_stream(pcv_ctx* c, void* cuda_stream) {
  if (!c) return fail(nullptr, PCV_EINVAL, "NULL context");
  c->stream = (cudaStream_t)cuda_stream;
  return PCV_OK;
}

const char* pcv_last_error(const pcv_ctx* c) { return c ? c->err.c_str() : g_err.c_str(); }

pcv_status pcv_set_lambda(pcv_ctx* c, double lambda) {
  if (!c) return fail(nullptr, PCV_EINVAL, "NULL context");
  if (!(lambda > 0.0) || !std::isfinite(lambda)) return fail(c, PCV_EINVAL, "lambda must be > 0 and finite");
  c->lambda = lambda;
  c->have_lambda = true;
  return PCV_OK;
}

pcv_status pcv_set_close_threshold(pcv_ctx* c, double eps) {
  if (!c) return fail(nullptr, PCV_EINVAL, "NULL context");
  if (std::isnan(eps)) return fail(c, PCV_EINVAL, "eps is NaN");
  c->eps = eps;
  return PCV_OK;
}

pcv_status pcv_set_option(pcv_ctx* c, int key, int64_t value) {
  if (!c) return fail(nullptr, PCV_EINVAL, "NULL context");
  switch (key) {
    case PCV_OPT_BAND:
      if (value < 1 || value > 6) return fail(c, PCV_EINVAL, "band must be in 1..6");
      c->band_W = (int)value;
      return PCV_OK;
    case PCV_OPT_CHUNK:
      if (value < 1 || value > (1 << 30)) return fail(c, PCV_EINVAL, "chunk must be in 1..2^30");
      c->min_chunk = (int)value;
      return PCV_OK;
    case PCV_OPT_PROFILE:
      c->prof_on = value != 0;
      return PCV_OK;
    case PCV_OPT_MATERIALIZE:
      if (value < 0) return fail(c, PCV_EINVAL, "materialise cap must be >= 0");
      c->mat_cap = value;
      return PCV_OK;
    case PCV_OPT_TENSOR_CORES:
      c->tensor_cores = value != 0;
      return PCV_OK;
    case PCV_OPT_HOST_CHUNKS:
      if (value < 0 || value > 64) return fail(c, PCV_EINVAL, "host chunks must be in 0..64");
      c->host_chunks = (int)value;
      return PCV_OK;
    case PCV_OPT_HOST_END_SHARE:
      if (value < 1 || value > 100) return fail(c, PCV_EINVAL, "host end share must be in 1..100");
      c->host_end_share = (int)value;
      return PCV_OK;
    case PCV_OPT_NEWTON_CAP:
      if (value < 1 || value > 60) return fail(c, PCV_EINVAL, "Newton cap must be in 1..60");
      c->newton_cap = (int)value;
      return PCV_OK;
    case PCV_OPT_WAIT_CYCLES:
      if (value < 0 || value > 4000000000LL) return fail(c, PCV_EINVAL, "wait budget must be in 0..4e9 cycles");
      c->wait_cycles = value == 0 ? 4000000000LL : (long long)value;
      return PCV_OK;
    case PCV_OPT_MMA_GROUP:
      if (value < 1 || value > 16) return fail(c, PCV_EINVAL, "MMA group must be in 1..16");
      c->mma_group = (int)value;
      return PCV_OK;
    case PCV_OPT_EXACT_TILE:
      if (value < 0 || value > EXACT_SHAPES) return fail(c, PCV_EINVAL, "exact tile shape must be in 0..%d", EXACT_SHAPES);
      c->exact_tile = (int)value;
      return PCV_OK;
    case PCV_OPT_APPROX_TILE:
      if (value != 0) return fail(c, PCV_EINVAL, "only tile variant 0 is built");
      return PCV_OK;
    default:
      return fail(c, PCV_EINVAL, "unknown option %d", key);
  }
}

pcv_status pcv_set_neighbor_list(pcv_ctx* c, int size, int stride) {
  if (!c) return fail(nullptr, PCV_EINVAL, "NULL context");
  if (size < 0) return fail(c, PCV_EINVAL, "neighbour-list size must be >= 0");
  if (stride < 1) return fail(c, PCV_EINVAL, "neighbour-list stride must be >= 1");
  c->nl_size = size;
  c->nl_stride = stride;
  c->has_nl = false;
  return PCV_OK;
}

pcv_status pcv_reset_close_state(pcv_ctx* c) {
  if (!c) return fail(nullptr, PCV_EINVAL, "NULL context");
  c->has_y = false;  // the gap estimate is a tuning statistic and survives the reset
  c->has_nl = false;
  const int64_t syncs = c->stats.host_syncs, launches = c->stats.kernel_launches;
  c->stats = pcv_stats{};
  c->stats.host_syncs = syncs;  // cumulative over the context's lifetime
  c->stats.kernel_launches = launches;
  cudaSetDevice(c->device);
  CUDA_TRY(c, cudaMemsetAsync(c->nrecheck.p, 0, 16, c->stream));
  return PCV_OK;
}

// ---------------------------------------------------------------------------------------
// Landmark preparation (row "a1"): FP64 centring by the weighted centre, rounding to the
// storage type, then G_a, A_i = sum_j w_j a_j a_j^T from the stored (rounded) values.
pcv_status pcv_set_landmarks(pcv_ctx* c, int M, int N, const double* coords, const double* w, const double* q) {
  return pcv_set_landmarks_weighted(c, M, N, coords, w, nullptr, q);
}

pcv_status pcv_set_landmarks_weighted(pcv_ctx* c, int M, int N, const double* coords, const double* w,
                                      const double* w_align, const double* q) {
  if (!c) return fail(nullptr, PCV_EINVAL, "NULL context");
  if (M < 1 || N < 3) return fail(c, PCV_EINVAL, "need M >= 1 and N >= 3 (got M=%d N=%d)", M, N);
  if (!coords) return fail(c, PCV_EINVAL, "coords is NULL");
  if ((size_t)M * N > ((size_t)1 << 31) / 3) return fail(c, PCV_EINVAL, "M*N*3 exceeds 2^31");
  std::vector<double> wn(N, 1.0 / N);
  bool uniform = true;
  if (w) {
    double sum = 0.0;
    for (int j = 0; j < N; ++j) {
      if (!(w[j] > 0.0) || !std::isfinite(w[j])) return fail(c, PCV_EINVAL, "weight %d not > 0", j);
      sum += w[j];
    }
    for (int j = 0; j < N; ++j) wn[j] = w[j] / sum;
    uniform = false;
  }
  // alignment weights w' (Section 3.1): they set the centres; equal to w unless given and
  // different
  std::vector<double> wan(wn);
  if (w_align) {
    double sum = 0.0;
    for (int j = 0; j < N; ++j) {
      if (!(w_align[j] > 0.0) || !std::isfinite(w_align[j]))
        return fail(c, PCV_EINVAL, "alignment weight %d not > 0", j);
      sum += w_align[j];
    }
    for (int j = 0; j < N; ++j) wan[j] = w_align[j] / sum;
  }
  bool split = false;
  for (int j = 0; j < N; ++j) split = split || wan[j] != wn[j];
  const size_t n3 = (size_t)N * 3;
  for (size_t k = 0; k < (size_t)M * n3; ++k)
    if (!std::isfinite(coords[k])) return fail(c, PCV_EINVAL, "non-finite landmark coordinate at %zu", k);
  std::vector<double> qv(M);
  for (int i = 0; i < M; ++i) {
    qv[i] = q ? q[i] : (double)(i + 1);
    if (!std::isfinite(qv[i])) return fail(c, PCV_EINVAL, "non-finite property q[%d]", i);
  }
  const Prec p = c->prec;
  std::vector<double> G(M), A((size_t)M * 6);
  std::vector<unsigned char> store((size_t)M * n3 * store_elem(p));
  // FP16 storage: per block of 16 atoms an FP32 offset (the block mean of the centred
  // coordinates) and FP16 residuals; the device reads offset + residual in FP32
  const int NB = (N + 15) / 16;
  std::vector<float> off(p == P_F16 ? (size_t)M * NB * 3 : 0);
  std::vector<float> w32(N);
  for (int j = 0; j < N; ++j) w32[j] = (float)wn[j];
  for (int i = 0; i < M; ++i) {
    const double* a = coords + (size_t)i * n3;
    double cen[3] = {0, 0, 0};  // the alignment-weighted centre
    for (int j = 0; j < N; ++j)
      for (int k = 0; k < 3; ++k) cen[k] += wan[j] * a[3 * j + k];
    double g = 0.0, Ai[6] = {0, 0, 0, 0, 0, 0};
    if (p == P_F16) {
      for (int b = 0; b < NB; ++b) {
        double m3[3] = {0, 0, 0};
        const int j1 = std::min(N, 16 * b + 16);
        for (int j = 16 * b; j < j1; ++j)
          for (int k = 0; k < 3; ++k) m3[k] += a[3 * j + k] - cen[k];
        for (int k = 0; k < 3; ++k) off[((size_t)i * NB + b) * 3 + k] = (float)(m3[k] / (j1 - 16 * b));
      }
    }
    for (int j = 0; j < N; ++j) {
      double v[3];
      for (int k = 0; k < 3; ++k) {
        const double cv = a[3 * j + k] - cen[k];
        const size_t idx = (size_t)i * n3 + 3 * j + k;
        if (p == P_F64) {
          ((double*)store.data())[idx] = cv;
          v[k] = cv;
        } else if (p == P_F32) {
          const float f = (float)cv;
          ((float*)store.data())[idx] = f;
          v[k] = f;
        } else {
          const float o = off[((size_t)i * NB + j / 16) * 3 + k];
          const __half h = __float2half_rn((float)(cv - (double)o));
          ((__half*)store.data())[idx] = h;
          v[k] = (double)(__half2float(h) + o);  // the device's FP32 reconstruction
        }
      }
      const double wk = uniform ? 1.0 : (p == P_F64 ? wn[j] : (double)w32[j]);
      g += wk * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
      Ai[0] += wn[j] * v[0] * v[0];
      Ai[1] += wn[j] * v[0] * v[1];
      Ai[2] += wn[j] * v[0] * v[2];
      Ai[3] += wn[j] * v[1] * v[1];
      Ai[4] += wn[j] * v[1] * v[2];
      Ai[5] += wn[j] * v[2] * v[2];
    }
    G[i] = g;
    for (int e = 0; e < 6; ++e) A[(size_t)i * 6 + e] = Ai[e];
  }
  cudaSetDevice(c->device);
  pcv_status st;
  if ((st = ensure(c, c->lm, store.size())) != PCV_OK) return st;
  if (p == P_F16 && (st = ensure(c, c->lmoff, sizeof(float) * off.size())) != PCV_OK) return st;
  if ((st = ensure(c, c->lmG, sizeof(double) * M)) != PCV_OK) return st;
  if ((st = ensure(c, c->lmA, sizeof(double) * 6 * M)) != PCV_OK) return st;
  if ((st = ensure(c, c->lmA32, sizeof(float) * 6 * M)) != PCV_OK) return st;
  if ((st = ensure(c, c->lmq, sizeof(double) * M)) != PCV_OK) return st;
  if ((st = ensure(c, c->lmq32, sizeof(float) * M)) != PCV_OK) return st;
  if ((st = ensure(c, c->w32, sizeof(float) * N)) != PCV_OK) return st;
  if ((st = ensure(c, c->w64, sizeof(double) * N)) != PCV_OK) return st;
  if (split && (st = ensure(c, c->wa32, sizeof(float) * N)) != PCV_OK) return st;
  if (split && (st = ensure(c, c->wa64, sizeof(double) * N)) != PCV_OK) return st;
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  CUDA_TRY(c, cudaMemcpy(c->lm.p, store.data(), store.size(), cudaMemcpyHostToDevice));
  if (p == P_F16)
    CUDA_TRY(c, cudaMemcpy(c->lmoff.p, off.data(), sizeof(float) * off.size(), cudaMemcpyHostToDevice));
  CUDA_TRY(c, cudaMemcpy(c->lmG.p, G.data(), sizeof(double) * M, cudaMemcpyHostToDevice));
  CUDA_TRY(c, cudaMemcpy(c->lmA.p, A.data(), sizeof(double) * 6 * M, cudaMemcpyHostToDevice));
  std::vector<float> A32(A.begin(), A.end());
  CUDA_TRY(c, cudaMemcpy(c->lmA32.p, A32.data(), sizeof(float) * 6 * M, cudaMemcpyHostToDevice));
  CUDA_TRY(c, cudaMemcpy(c->lmq.p, qv.data(), sizeof(double) * M, cudaMemcpyHostToDevice));
  std::vector<float> q32(qv.begin(), qv.end());
  CUDA_TRY(c, cudaMemcpy(c->lmq32.p, q32.data(), sizeof(float) * M, cudaMemcpyHostToDevice));
  CUDA_TRY(c, cudaMemcpy(c->w32.p, w32.data(), sizeof(float) * N, cudaMemcpyHostToDevice));
  CUDA_TRY(c, cudaMemcpy(c->w64.p, wn.data(), sizeof(double) * N, cudaMemcpyHostToDevice));
  if (split) {
    std::vector<float> wa32(wan.begin(), wan.end());
    CUDA_TRY(c, cudaMemcpy(c->wa32.p, wa32.data(), sizeof(float) * N, cudaMemcpyHostToDevice));
    CUDA_TRY(c, cudaMemcpy(c->wa64.p, wan.data(), sizeof(double) * N, cudaMemcpyHostToDevice));
  }
  c->M = M;
  c->N = N;
  c->uniform = uniform;
  c->split_w = split;
  c->dscale = uniform ? 1.0 / N : 1.0;
  c->have_lm = true;
  return pcv_reset_close_state(c);
}

// ---------------------------------------------------------------------------------------
namespace {

// workspace of the adjoint beta's landmark-range split (few frames); *part null: no split
pcv_status beta_part_workspace(pcv_ctx* c, int F, void** part) {
  *part = nullptr;
  const int k = beta_pair_split(c->prec, F, c->M, c->N);
  if (k <= 1) return PCV_OK;
  const pcv_status ps = ensure(c, c->betaPart, work_elem(c->prec) * 6 * (size_t)k * F * c->N);
  if (ps == PCV_OK) *part = c->betaPart.p;
  return ps;
}

pcv_status ensure_frame_workspace(pcv_ctx* c, int F, bool close, bool grads) {
  const size_t M = c->M, W = c->band_W;
  pcv_status st;
#define ENS(buf, bytes) \
  if ((st = ensure(c, c->buf, (bytes))) != PCV_OK) return st
  ENS(c32, sizeof(float4) * F);
  ENS(c64, sizeof(double4) * F);
  ENS(fG, sizeof(double) * F);
  ENS(Dbuf, work_elem(c->prec) * (size_t)F * M);
  ENS(mstat, sizeof(double) * 2 * F);
  if (close) {
    ENS(bandD, sizeof(double) * F * W);
    ENS(bandQ, sizeof(double4) * F * W);
    ENS(bandF, F * W);
    ENS(chD, sizeof(double) * F);
    ENS(chQ, sizeof(double4) * F);
    ENS(chF, F);
    ENS(rlist, sizeof(int) * (F * (W + 1) + 1));
    ENS(recF, F);
    ENS(recRef, sizeof(int) * F);
    ENS(recD, sizeof(double) * F);
    ENS(recQ, sizeof(double4) * F);
    ENS(reflist, sizeof(int) * F);
    ENS(segof, sizeof(int) * F);
    ENS(alist, sizeof(int) * F);
    ENS(aseg, sizeof(int) * F);
    ENS(rcount, 64);
  } else if (grads) {
    ENS(Rpair, work_elem(c->prec) * 9 * (size_t)F * M);
  }
#undef ENS
  return PCV_OK;
}

FrameInfo frame_info(pcv_ctx* c) {
  FrameInfo fi;
  fi.c32 = (float4*)c->c32.p;
  fi.c64 = (double4*)c->c64.p;
  fi.G = (double*)c->fG.p;
  return fi;
}

FrameRec frame_rec(pcv_ctx* c) {
  FrameRec r;
  r.flag = (uint8_t*)c->recF.p;
  r.ref = (int*)c->recRef.p;
  r.dxy = (double*)c->recD.p;
  r.qxy = (double4*)c->recQ.p;
  return r;
}

// Neighbour list in force: a size strictly between 0 and M (otherwise every landmark is
// evaluated at every step).
bool nl_active(const pcv_ctx* c) { return c->nl_size > 0 && c->nl_size < c->M; }

pcv_status ensure_nl_workspace(pcv_ctx* c, int F, bool exact_grads) {
  const size_t Mnl = c->nl_size;
  pcv_status st;
  if ((st = ensure(c, c->nl_keep, sizeof(int) * Mnl)) != PCV_OK) return st;
  if ((st = ensure(c, c->nlSlot, sizeof(int) * F)) != PCV_OK) return st;
  if ((st = ensure(c, c->nlUpd, F)) != PCV_OK) return st;
  if ((st = ensure(c, c->nlU, sizeof(int) * F)) != PCV_OK) return st;
  if ((st = ensure(c, c->nlUA, sizeof(int) * F)) != PCV_OK) return st;
  if ((st = ensure(c, c->nlUAseg, sizeof(int) * F)) != PCV_OK) return st;
  if ((st = ensure(c, c->nlN, sizeof(int) * F)) != PCV_OK) return st;
  if ((st = ensure(c, c->NLtab, sizeof(int) * Mnl * ((size_t)F + 1))) != PCV_OK) return st;
  if ((st = ensure(c, c->nlTiles, sizeof(NlTile) * ((size_t)F + F / NL_TILE_F + 4))) != PCV_OK) return st;
  if (exact_grads && (st = ensure(c, c->Rnl, work_elem(c->prec) * 9 * Mnl * (size_t)F)) != PCV_OK) return st;
  return PCV_OK;
}

NlLists nl_lists(pcv_ctx* c) {
  NlLists nl;
  nl.slot = (int*)c->nlSlot.p;
  nl.upd = (uint8_t*)c->nlUpd.p;
  nl.ulist = (int*)c->nlU.p;
  nl.uapp_list = (int*)c->nlUA.p;
  nl.uapp_seg = (int*)c->nlUAseg.p;
  nl.nlist = (int*)c->nlN.p;
  nl.counts = ((Small*)c->small.p)->nl_counts;
  return nl;
}

// the carried-over list is slot 0 of the table
pcv_status nl_stage_carried(pcv_ctx* c) {
  if (!c->has_nl) return PCV_OK;
  launch_dev_copy(c->NLtab.p, c->nl_keep.p, sizeof(int) * c->nl_size, c->stream);
  return PCV_OK;
}

// Algorithm 2 over F frames: decide every frame (reassignment / approximate and its close
// structure), then evaluate reassignment frames exactly and the rest approximately.
RecheckScratch rc_scratch(pcv_ctx* c) { return recheck_scratch_at(c->rcScr.p); }

// scratch for the exact pairs of `rows` frames split over atom slices (none when they do not split)
pcv_status exact_split_scratch(pcv_ctx* c, int rows, ScratchView& scr) {
  scr = ScratchView{nullptr, 0};
  if (c->prec == P_F64 || rows <= 0 || c->exact_tile != 0) return PCV_OK;
  const int k = exact_split_count(rows, c->M, c->N);
  if (k <= 1) return PCV_OK;
  const size_t bytes = exact_split_bytes(rows, c->M, k);
  const pcv_status st = ensure(c, c->exSplit, bytes);
  if (st != PCV_OK) return st;
  scr = ScratchView{c->exSplit.p, c->exSplit.bytes};
  return PCV_OK;
}

pcv_status evaluate_close(pcv_ctx* c, int F, const void* frames, double* s, double* z, void* gs, void* gz,
                          double* msd, uint8_t* refreshed) {
  const cudaStream_t st = c->stream;
  const LandmarkDev L = lm_view(c);
  const FrameInfo fi = frame_info(c);
  const FrameRec rec = frame_rec(c);
  const RefDesc prior = prior_view(c);
  const int W = c->band_W;
  const int M = c->M;
  Small* sm = (Small*)c->small.p;
  AlignOut band{(double*)c->bandD.p, (double4*)c->bandQ.p, (uint8_t*)c->bandF.p};
  AlignOut chunk{(double*)c->chD.p, (double4*)c->chQ.p, (uint8_t*)c->chF.p};
  int* rl = (int*)c->rlist.p;  // recheck list
  int* rc = &sm->recheck_count;
  const bool had_prior = c->has_y;

  {
    PROF(c, K_PREP);
    launch_frame_prep(c->prec, F, frames, L, fi, st);
  }
  // The band pays off when reassignments come every few frames; with long observed gaps the
  // search uses speculative chunks only.  Band rows are computed lazily from the first frame
  // that needs them (band_from: rows [band_from, F) are ready).
  int band_from = F;
  auto want_band = [&]() { return F > 1 && !(c->gap_estimate > 8.0 * W); };
  auto ensure_band = [&](int from) {
    from = from < 1 ? 1 : from;
    if (from >= band_from) return;
    launch_set_int(rc, 0, st);
    {
      PROF(c, K_BAND);
      launch_align_band(c->prec, F, W, from, band_from, frames, L, fi, c->eps, band, rl, rc, st);
    }
    PROF(c, K_RECHECK);
    launch_recheck(c->prec, (band_from - from) * W, rl, rc, W, frames, L, fi.c32, prior, -1, c->eps, band, chunk,
                   (unsigned long long*)c->nrecheck.p, rc_scratch(c), st);
    band_from = from;
  };
  // host-driven refresh search
  int t = 0, ref = -1, o = 0;
  bool band_mode = false;
  if (!had_prior) {
    launch_initial_record(rec, st);
    t = 1;
    ref = 0;
    o = 0;
    band_mode = want_band();
  }
  long long guard = 0;
  while (t < F) {
    if (++guard > 4LL * F + 16) return fail(c, PCV_ESTATE, "refresh search did not terminate");
    if (band_mode) {
      ensure_band(t);
      {
        PROF(c, K_SCAN);
        launch_band_scan(F, W, t, o, band, rec, &sm->scan, st);
      }
      pcv_status ps = sync_small(c);
      if (ps != PCV_OK) return ps;
      const int ts = c->small_host->scan.t_stop;
      const int nr = c->small_host->scan.nref;
      if (nr > 0) {
        const double gap = (double)((ts < F ? ts : F) - t) / nr;
        c->gap_estimate = c->gap_estimate > 0.0 ? 0.5 * (c->gap_estimate + gap) : gap;
      }
      if (ts >= F) break;
      if (ts < t) return fail(c, PCV_ESTATE, "band scan went backwards");
      t = ts;
      ref = c->small_host->scan.ref;
      band_mode = false;
      continue;
    }
    // speculative chunk of frames aligned onto the close structure `ref`
    int B = c->min_chunk;
    // the chunk kernel stops at its first definite exceed, so a long chunk costs only the
    // frames in flight beyond it: four times the observed gap makes a second round rare
    if (c->gap_estimate > 0.0) B = (int)std::fmin(std::fmax((double)B, 4.0 * c->gap_estimate), 1e9);
    const int t1 = (int)std::min<long long>((long long)F, (long long)t + B);
    launch_chunk_round_init(rc, &sm->stop, &sm->first, t1, st);
    {
      PROF(c, K_CHUNK);
      launch_align_chunk(c->prec, t, t1, frames, L, fi, ref, prior, c->eps, chunk, rl, rc, &sm->stop, st);
    }
    {
      PROF(c, K_RECHECK);
      launch_recheck(c->prec, t1 - t, rl, rc, W, frames, L, fi.c32, prior, ref, c->eps, band, chunk,
                     (unsigned long long*)c->nrecheck.p, rc_scratch(c), st);
    }
    {
      PROF(c, K_FIRST);
      launch_first_exceed(t, t1, chunk.flag, &sm->stop, &sm->first, st);
    }
    if (t1 == F && t1 - t == 1) {
      // the batch's last frame in a search round of its own (every call of one frame): the
      // search ends with this round whatever the frame's decision, so its records take the
      // first exceed from the device and the host does not wait for it
      PROF(c, K_RECORDS);
      launch_chunk_records_dev(t, &sm->first, t1, ref, chunk, rec, st);
      break;
    }
    pcv_status ps = sync_small(c);
    if (ps != PCV_OK) return ps;
    const int first = c->small_host->first;
    {
      PROF(c, K_RECORDS);
      launch_chunk_records(t, first, t1, ref, chunk, rec, st);
    }
    if (first < t1) {
      const double gap = (double)(first - (ref >= 0 ? ref : first - 1));
      c->gap_estimate = c->gap_estimate > 0.0 ? 0.5 * (c->gap_estimate + gap) : gap;
      t = first + 1;
      ref = first;
      o = 0;
      band_mode = want_band();
    } else {
      t = t1;
    }
  }
  // compaction and per-segment work
  {
    PROF(c, K_COMPACT);
    launch_compact(F, rec, (int*)c->reflist.p, &sm->refresh_count, (int*)c->segof.p, (int*)c->alist.p,
                   &sm->approx_count, (int*)c->aseg.p, 0, st);
  }
  small_tail_kernel<<<1, 1, 0, st>>>(sm, (const int*)c->reflist.p, fi.c32, fi.c64, fi.G);
  // neighbour list: update frames are the reassignments and every L-th step
  const bool nl = nl_active(c);
  const int Mnl = c->nl_size;
  pcv_status ps;
  if (nl && (ps = ensure_nl_workspace(c, F, false)) != PCV_OK) return ps;
  const NlLists nll = nl ? nl_lists(c) : NlLists{};  // after the workspace exists
  if (nl) {
    PROF(c, K_NL_SCHEDULE);
    launch_nl_schedule(F, (long long)c->stats.frames, c->nl_stride, c->has_nl, rec.flag, (const int*)c->segof.p, nll,
                       st);
  }
  ps = sync_small(c);
  if (ps != PCV_OK) return ps;
  const int nref = c->small_host->refresh_count;
  const int napp = c->small_host->approx_count;
  const int nl_upd = nl ? c->small_host->nl_counts[0] : 0;
  const int nl_uapp = nl ? c->small_host->nl_counts[1] : 0;
  const int nl_between = nl ? c->small_host->nl_counts[2] : 0;
  if (nl && gs && gz && c->prec != P_F64 &&
      (ps = ensure(c, c->nlPart, sizeof(float) * 6 * (size_t)nl_beta_split(nl_upd, M, c->N) * nl_upd * c->N)) !=
          PCV_OK)
    return ps;
  const size_t seg_bytes = work_elem(c->prec) * 9 * (size_t)M;
  if ((ps = ensure(c, c->Bseg, seg_bytes * (size_t)(nref + 1))) != PCV_OK) return ps;
  if (had_prior) launch_dev_copy(c->Bseg.p, c->Bprior.p, seg_bytes, st);
  void* Bseg1 = (char*)c->Bseg.p + seg_bytes;
  // Frames sharing close structures (segments of 16 frames or more on average): the
  // segment GEMM form of the adjoint, and with FP32 arithmetic and uniform weights the
  // materialised operands x' and b when they fit the cap.
  const bool grads = gs && gz;
  const bool seg_form = (int64_t)(nref + 1) * 16 <= (int64_t)F && !nl;
  const int seg_base = had_prior ? 0 : 1;  // without a prior structure segment 0 is empty
  const int nseg = nref + 1 - seg_base;
  bool tiled = false, mma = false, xmma = false;
  const MmaShape msh = mma_shape(F, M, c->N);
  const XmmaShape xsh = xmma_shape(M, c->N);
  if (c->prec != P_F64 && c->uniform && !c->split_w && seg_form && nseg > 0) {
    // with the tensor cores the deviations are packed for the MMAs (FP16 h + l), else
    // stored as FP32 rows for the CUDA-core tiles
    xmma = c->tensor_cores;
    const size_t xb = xmma ? xmma_a_bytes(xsh, napp, nseg) : tile_bytes_frames(napp, c->N);
    const size_t bb = xmma ? xsh.b_bytes_per_seg * (size_t)nseg : tile_bytes_landmarks(nseg, M, c->N);
    const size_t nb = sizeof(float) * ((size_t)napp + (size_t)nseg * M + (size_t)nseg * 3 * c->N + 2 * (size_t)F);
    const size_t gb = grads ? tile_bytes_gamma(F, M) : 0;  // per gamma kind
    const size_t mb = msh.a_bytes + msh.b_bytes_per_seg * nseg;
    mma = grads && c->tensor_cores;
    if ((int64_t)(xb + bb + nb + (mma ? mb : 2 * gb)) <= c->mat_cap) {
      // the materialised operands are an optimisation: when the device cannot hold them the
      // kernels that rotate while staging take over
      DevBuf& xbuf = xmma ? c->Apk : c->Xr;
      DevBuf& bbuf = xmma ? c->Bpk : c->Bm;
      bool ok = ensure(c, xbuf, xb) == PCV_OK && ensure(c, bbuf, bb) == PCV_OK &&
                ensure(c, c->Nx, sizeof(float) * (size_t)napp) == PCV_OK &&
                ensure(c, c->Nb, sizeof(float) * (size_t)nseg * M) == PCV_OK &&
                ensure(c, c->Yc, sizeof(float) * 3 * (size_t)c->N * nseg) == PCV_OK &&
                (!grads || ensure(c, c->Gsum, sizeof(float) * std::max(2 * (size_t)F, msh.gsum_floats)) == PCV_OK);
      if (ok && xmma)
        ok = ensure(c, c->xtiles, sizeof(int) * (2 * (size_t)nseg + 3 * (size_t)xmma_max_tiles(napp, nseg) + 1)) ==
             PCV_OK;
      if (ok && mma)
        ok = ensure(c, c->Amma, msh.a_bytes) == PCV_OK && ensure(c, c->Bmma, msh.b_bytes_per_seg * nseg) == PCV_OK;
      else if (ok && grads)
        ok = ensure(c, c->GSb, gb) == PCV_OK && ensure(c, c->GZb, gb) == PCV_OK;
      if (ok) {
        tiled = true;
      } else {
        for (DevBuf* b : {&c->Xr, &c->Bm, &c->Apk, &c->Bpk, &c->xtiles, &c->Amma, &c->Bmma, &c->GSb, &c->GZb})
          release(*b);
        c->err = "no error";
        mma = false;
        xmma = false;
      }
    } else {
      mma = false;
      xmma = false;
    }
  }
  {
    ScratchView scr{nullptr, 0};
    if ((ps = exact_split_scratch(c, nref, scr)) != PCV_OK) return ps;
    PROF(c, K_EXACT);
    launch_exact_pairs(c->prec, nref, (const int*)c->reflist.p, nullptr, frames, L, fi, c->Dbuf.p, Bseg1,
                       (unsigned*)c->status.p, st, &scr);
  }
  // per-segment tile list of the tensor-core MSDs: [seg_first | tile_start | tiles | count]
  int *xt_first = nullptr, *xt_start = nullptr, *xt_count = nullptr;
  XTile* xt_tiles = nullptr;
  if (tiled && xmma) {
    xt_first = (int*)c->xtiles.p;
    xt_start = xt_first + nseg;
    xt_tiles = (XTile*)(xt_start + nseg);
    xt_count = (int*)(xt_tiles + xmma_max_tiles(napp, nseg));
  }
  if (tiled && xmma) {
    PROF(c, K_MATERIALIZE);
    launch_xmma_tiles(&sm->approx_count, (const int*)c->aseg.p, seg_base, nseg, xt_first, xt_start, xt_tiles, xt_count,
                      st);
    launch_pack_deviations(c->prec, seg_base, nseg, L, xsh, mma ? &msh : nullptr, (const float*)c->Bseg.p, frames,
                           fi, (const int*)c->reflist.p, prior, (uint8_t*)c->Bpk.p, (float*)c->Nb.p,
                           (uint8_t*)c->Bmma.p, (float*)c->Yc.p, st);
    launch_xy_refine(c->prec, F, frames, L, fi, prior, rec, st);
    launch_pack_frames(napp, &sm->approx_count, (const int*)c->alist.p, (const int*)c->aseg.p, seg_base, L, frames,
                       fi, rec.qxy, (const float*)c->Yc.p, xt_first, xt_start, (uint8_t*)c->Apk.p, (float*)c->Nx.p,
                       st);
  } else if (tiled) {
    PROF(c, K_MATERIALIZE);
    launch_materialize_landmarks(c->prec, seg_base, nseg, L, (const float*)c->Bseg.p, frames, fi,
                                 (const int*)c->reflist.p, prior, (float*)c->Bm.p, (float*)c->Nb.p, (float*)c->Yc.p, st);
    // the accurate R_xy of the approximate frames is formed while their deviations are
    // materialised (one read of each frame)
    launch_materialize_frames(napp, &sm->approx_count, (const int*)c->alist.p, (const int*)c->aseg.p, seg_base, L,
                              frames, fi, rec.qxy, (const float*)c->Yc.p, (float*)c->Xr.p, (float*)c->Nx.p, rec.ref,
                              prior, st);
  } else {
    PROF(c, K_XY_REFINE);
    launch_xy_refine(c->prec, F, frames, L, fi, prior, rec, st);
  }
  // FP32 / FP16 storage: tiles of up to 16 frames sharing a list (and a close structure)
  const bool nl_tiled = nl && c->prec != P_F64;
  const int nl_max_tiles = (nl_between + NL_TILE_F - 1) / NL_TILE_F + nl_upd + 1;
  NlTile* tl = (NlTile*)c->nlTiles.p;
  if (nl_tiled) {
    {
      PROF(c, K_NL_SCHEDULE);
      launch_nl_tiles(F, nll, tl, st);
    }
    {  // all-landmark approximate distances of the update frames that are not reassignments
      PROF(c, K_APPROX);
      launch_nl_approx_tiles(c->prec, nl_uapp, 0, nll, tl, (const int*)c->NLtab.p, Mnl, frames, L, fi, rec.qxy,
                             c->Bseg.p, (const int*)c->segof.p, c->Dbuf.p, st);
    }
    {
      PROF(c, K_NL_SELECT);
      launch_nl_select(c->prec, nl_upd, nll, M, Mnl, c->Dbuf.p, (int*)c->NLtab.p, st);
    }
    if ((ps = nl_stage_carried(c)) != PCV_OK) return ps;
    PROF(c, K_NL_PAIR);
    launch_nl_fill_inf(c->prec, nl_between, nll, M, c->Dbuf.p, st);
    launch_nl_approx_tiles(c->prec, 0, nl_max_tiles, nll, tl, (const int*)c->NLtab.p, Mnl, frames, L, fi, rec.qxy,
                           c->Bseg.p, (const int*)c->segof.p, c->Dbuf.p, st);
  } else if (nl) {
    {  // all-landmark approximate distances of the update frames that are not reassignments
      PROF(c, K_APPROX);
      launch_approx_pairs(c->prec, nl_uapp, nll.uapp_list, nll.uapp_seg, &nll.counts[1], frames, L, fi, rec.qxy,
                          c->Bseg.p, c->Dbuf.p, st);
    }
    {
      PROF(c, K_NL_SELECT);
      launch_nl_select(c->prec, nl_upd, nll, M, Mnl, c->Dbuf.p, (int*)c->NLtab.p, st);
    }
    if ((ps = nl_stage_carried(c)) != PCV_OK) return ps;
    PROF(c, K_NL_PAIR);
    launch_nl_approx(c->prec, nl_between, nll, (const int*)c->NLtab.p, Mnl, frames, L, fi, rec.qxy, c->Bseg.p,
                     (const int*)c->segof.p, c->Dbuf.p, st);
  } else if (xmma) {
    PROF(c, K_APPROX_MMA);
    launch_approx_cross_mma(napp, nseg, (const int*)c->alist.p, xt_tiles, xt_count, L, xsh, (const uint8_t*)c->Apk.p,
                            (const uint8_t*)c->Bpk.p, (const float*)c->Nx.p, (const float*)c->Nb.p, (float*)c->Dbuf.p,
                            (unsigned*)c->status.p, st);
  } else {
    PROF(c, K_APPROX);
    if (tiled)
      launch_approx_pairs_tile(napp, (const int*)c->alist.p, (const int*)c->aseg.p, &sm->approx_count, seg_base, L,
                               (const float*)c->Xr.p, (const float*)c->Bm.p, (const float*)c->Nx.p,
                               (const float*)c->Nb.p, (float*)c->Dbuf.p, st);
    else
      launch_approx_pairs(c->prec, napp, (const int*)c->alist.p, (const int*)c->aseg.p, &sm->approx_count, frames,
                          L, fi, rec.qxy, c->Bseg.p, c->Dbuf.p, st);
  }
  {
    PROF(c, K_FINAL);
    launch_finalize(c->prec, F, M, c->Dbuf.p, L.q, L.q32, c->lambda, s, z, (float*)c->mstat.p, (double*)c->mstat.p, msd,
                    gs != nullptr, st);
  }
  if (refreshed) launch_dev_copy(refreshed, rec.flag, F, st);
  if (grads && nl) {
    {
      PROF(c, K_NL_BETA);
      if (nl_tiled)
        launch_nl_beta_tiles(c->prec, nl_upd, nl_max_tiles, nll, tl, (const int*)c->NLtab.p, Mnl, L, c->Dbuf.p, s,
                             c->lambda, nullptr, nullptr, c->Bseg.p, (const int*)c->segof.p, gs, gz,
                             (float*)c->nlPart.p, st);
      else
        launch_nl_beta(c->prec, F, nll, (const int*)c->NLtab.p, Mnl, L, c->Dbuf.p, s, c->lambda, nullptr, nullptr,
                       c->Bseg.p, (const int*)c->segof.p, gs, gz, st);
    }
    PROF(c, K_ADJ_FINISH);
    launch_adjoint_finish(c->prec, F, frames, L, fi, c->Dbuf.p, s, c->lambda, c->Bseg.p, (const int*)c->segof.p, rec,
                          prior, gs, gz, st);
  } else if (grads) {
    if (mma) {
      {
        PROF(c, K_GAMMA);
        launch_gamma_split(F, L, msh, (const float*)c->Dbuf.p, s, c->lambda, (float*)c->Amma.p, (float*)c->Gsum.p, st);
      }
      PROF(c, K_ADJ_MMA);
      launch_adjoint_beta_mma(F, L, msh, seg_base, (const float*)c->Amma.p, (const float*)c->Gsum.p,
                              (const float*)c->Bmma.p, (const float*)c->Yc.p, (const int*)c->segof.p, (float*)gs,
                              (float*)gz, (unsigned*)c->status.p, st);
    } else if (tiled) {
      {
        PROF(c, K_GAMMA);
        launch_gamma(F, L, (const float*)c->Dbuf.p, s, c->lambda, (float*)c->GSb.p, (float*)c->GZb.p,
                     (float*)c->Gsum.p, st);
      }
      PROF(c, K_ADJ_BETA_SEG);
      launch_adjoint_beta_tile(F, L, seg_base, (const float*)c->GSb.p, (const float*)c->GZb.p, (const float*)c->Bm.p,
                               (const float*)c->Gsum.p, (const float*)c->Yc.p, (const int*)c->segof.p, (float*)gs,
                               (float*)gz, st);
    } else {
      void* part = nullptr;
      if (!(seg_form && c->prec != P_F64)) {
        const pcv_status pw = beta_part_workspace(c, F, &part);
        if (pw != PCV_OK) return pw;
      }
      ProfScope ps(c, seg_form && c->prec != P_F64 ? K_ADJ_BETA_SEG : K_ADJ_BETA);
      launch_adjoint_beta(c->prec, F, L, c->Dbuf.p, s, c->lambda, nullptr, c->Bseg.p, (const int*)c->segof.p,
                          seg_form, gs, gz, part, st);
    }
    // segment moments for Phi when frames share close structures (FP32 modes)
    const bool moments = c->prec != P_F64 && seg_form && nseg > 0;
    if (moments) {
      if ((ps = ensure(c, c->S6, sizeof(float) * 6 * (size_t)nseg * M)) != PCV_OK) return ps;
      PROF(c, K_SEG_MOMENTS);
      launch_seg_moments(seg_base, nseg, L, (const float*)c->Bseg.p, (float*)c->S6.p, st);
    }
    PROF(c, K_ADJ_FINISH);
    launch_adjoint_finish(c->prec, F, frames, L, fi, c->Dbuf.p, s, c->lambda, c->Bseg.p, (const int*)c->segof.p, rec,
                          prior, gs, gz, st, tiled ? (const float*)c->Gsum.p : nullptr,
                          moments ? (const float*)c->S6.p : nullptr, seg_base);
  }
  // carry the close structure over to the next call
  const int last = c->small_host->last_refresh;
  if (nref > 0 && last >= 0) {
    const size_t ybytes = frame_elem(c->prec) * 3 * (size_t)c->N;
    if ((ps = ensure(c, c->y, ybytes)) != PCV_OK) return ps;
    if ((ps = ensure(c, c->Bprior, seg_bytes)) != PCV_OK) return ps;
    launch_dev_copy(c->y.p, (const char*)frames + ybytes * (size_t)last, ybytes, st);
    launch_dev_copy(c->Bprior.p, (char*)c->Bseg.p + seg_bytes * (size_t)nref, seg_bytes, st);
    c->y_c32 = c->small_host->last_c32;
    c->y_c64 = c->small_host->last_c64;
    c->y_G = c->small_host->last_G;
    c->has_y = true;
  }
  if (nl) {
    launch_nl_carry(nll, (const int*)c->NLtab.p, Mnl, (int*)c->nl_keep.p, st);
    c->has_nl = true;
  }
  c->stats.frames += F;
  c->stats.xy_alignments += had_prior ? F : F - 1;
  c->stats.landmark_alignments += (int64_t)M * nref;
  c->stats.approx_msds += nl ? (int64_t)M * nl_uapp + (int64_t)Mnl * nl_between : (int64_t)M * napp;
  c->stats.refreshes_initial += had_prior ? 0 : 1;
  c->stats.refreshes_threshold += nref - (had_prior ? 0 : 1);
  return PCV_OK;
}

// Original method with a neighbour list (Section 6.2): all M landmarks at every L-th step,
// the M_nl listed ones in between.  The update frames follow from the step counter alone,
// so the host knows their number without a device round trip.
pcv_status evaluate_exact_nl(pcv_ctx* c, int F, const void* frames, double* s, double* z, void* gs, void* gz,
                             double* msd, uint8_t* refreshed) {
  const cudaStream_t st = c->stream;
  const LandmarkDev L = lm_view(c);
  const FrameInfo fi = frame_info(c);
  const bool grads = gs && gz;
  const int M = c->M, Mnl = c->nl_size, Ls = c->nl_stride;
  const long long step0 = (long long)c->stats.frames;
  int nupd = 0;
  for (int t = 0; t < F; ++t)
    if ((step0 + t) % Ls == 0 || (t == 0 && !c->has_nl)) ++nupd;
  pcv_status ps = ensure_nl_workspace(c, F, grads);
  if (ps != PCV_OK) return ps;
  if (grads && (ps = ensure(c, c->Rupd, work_elem(c->prec) * 9 * (size_t)M * nupd)) != PCV_OK) return ps;
  if (grads && c->prec != P_F64 &&
      (ps = ensure(c, c->nlPart, sizeof(float) * 6 * (size_t)nl_beta_split(nupd, M, c->N) * nupd * c->N)) != PCV_OK)
    return ps;
  const NlLists nll = nl_lists(c);
  {
    PROF(c, K_PREP);
    launch_frame_prep(c->prec, F, frames, L, fi, st);
  }
  {
    PROF(c, K_NL_SCHEDULE);
    launch_nl_schedule(F, step0, Ls, c->has_nl, nullptr, nullptr, nll, st);
  }
  {
    PROF(c, K_EXACT);
    launch_exact_pairs(c->prec, nupd, nll.ulist, nullptr, frames, L, fi, c->Dbuf.p, grads ? c->Rupd.p : nullptr,
                       (unsigned*)c->status.p, st);
  }
  {
    PROF(c, K_NL_SELECT);
    launch_nl_select(c->prec, nupd, nll, M, Mnl, c->Dbuf.p, (int*)c->NLtab.p, st);
  }
  if ((ps = nl_stage_carried(c)) != PCV_OK) return ps;
  // FP32 / FP16 storage: tiles of up to 16 frames sharing a list x 32 listed landmarks
  const bool tiles = c->prec != P_F64;
  const int max_tiles = (F - nupd + NL_TILE_F - 1) / NL_TILE_F + nupd + 1;
  NlTile* tl = (NlTile*)c->nlTiles.p;
  {
    PROF(c, K_NL_PAIR);
    if (tiles) {
      launch_nl_tiles(F, nll, tl, st);
      launch_nl_fill_inf(c->prec, F - nupd, nll, M, c->Dbuf.p, st);
      launch_nl_exact_tiles(c->prec, max_tiles, nll, tl, (const int*)c->NLtab.p, Mnl, frames, L, fi, c->Dbuf.p,
                            grads ? c->Rnl.p : nullptr, (unsigned*)c->status.p, st);
    } else {
      launch_nl_exact(c->prec, F - nupd, nll, (const int*)c->NLtab.p, Mnl, frames, L, fi, c->Dbuf.p,
                      grads ? c->Rnl.p : nullptr, (unsigned*)c->status.p, st);
    }
  }
  {
    PROF(c, K_FINAL);
    launch_finalize(c->prec, F, M, c->Dbuf.p, L.q, L.q32, c->lambda, s, z, (float*)c->mstat.p, (double*)c->mstat.p,
                    msd, grads, st);
  }
  if (refreshed) launch_fill_u8(refreshed, 1, (size_t)F, st);
  if (grads) {
    {
      PROF(c, K_NL_BETA);
      if (tiles)
        launch_nl_beta_tiles(c->prec, nupd, max_tiles, nll, tl, (const int*)c->NLtab.p, Mnl, L, c->Dbuf.p, s,
                             c->lambda, c->Rupd.p, c->Rnl.p, nullptr, nullptr, gs, gz, (float*)c->nlPart.p, st);
      else
        launch_nl_beta(c->prec, F, nll, (const int*)c->NLtab.p, Mnl, L, c->Dbuf.p, s, c->lambda, c->Rupd.p,
                       c->Rnl.p, nullptr, nullptr, gs, gz, st);
    }
    PROF(c, K_ADJ_FINISH);
    FrameRec none;
    RefDesc nop;
    launch_adjoint_finish(c->prec, F, frames, L, fi, c->Dbuf.p, s, c->lambda, nullptr, nullptr, none, nop, gs, gz, st);
  }
  launch_nl_carry(nll, (const int*)c->NLtab.p, Mnl, (int*)c->nl_keep.p, st);
  c->has_nl = true;
  c->stats.frames += F;
  c->stats.landmark_alignments += (int64_t)M * nupd + (int64_t)Mnl * (F - nupd);
  return PCV_OK;
}

pcv_status evaluate_exact(pcv_ctx* c, int F, const void* frames, double* s, double* z, void* gs, void* gz,
                          double* msd, uint8_t* refreshed) {
  const cudaStream_t st = c->stream;
  const LandmarkDev L = lm_view(c);
  const FrameInfo fi = frame_info(c);
  const bool grads = gs && gz;
  {
    PROF(c, K_PREP);
    launch_frame_prep(c->prec, F, frames, L, fi, st);
  }
  {
    ScratchView scr{nullptr, 0};
    const pcv_status ps = exact_split_scratch(c, F, scr);
    if (ps != PCV_OK) return ps;
    PROF(c, K_EXACT);
    launch_exact_pairs(c->prec, F, nullptr, nullptr, frames, L, fi, c->Dbuf.p, grads ? c->Rpair.p : nullptr,
                       (unsigned*)c->status.p, st, &scr);
  }
  {
    PROF(c, K_FINAL);
    launch_finalize(c->prec, F, c->M, c->Dbuf.p, L.q, L.q32, c->lambda, s, z, (float*)c->mstat.p, (double*)c->mstat.p,
                    msd, grads, st);
  }
  if (refreshed) launch_fill_u8(refreshed, 1, (size_t)F, st);
  if (grads) {
    {
      void* part = nullptr;
      const pcv_status pw = beta_part_workspace(c, F, &part);
      if (pw != PCV_OK) return pw;
      PROF(c, K_ADJ_BETA);
      launch_adjoint_beta(c->prec, F, L, c->Dbuf.p, s, c->lambda, c->Rpair.p, nullptr, nullptr, false, gs, gz, part,
                          st);
    }
    PROF(c, K_ADJ_FINISH);
    FrameRec none;
    RefDesc nop;
    launch_adjoint_finish(c->prec, F, frames, L, fi, c->Dbuf.p, s, c->lambda, nullptr, nullptr, none, nop, gs, gz, st);
  }
  c->stats.frames += F;
  c->stats.landmark_alignments += (int64_t)c->M * F;
  return PCV_OK;
}

}  // namespace

pcv_status pcv_evaluate(pcv_ctx* c, int F, const void* frames, double* s, double* z, void* dsdx, void* dzdx,
                        double* msd, uint8_t* refreshed) {
  if (!c) return fail(nullptr, PCV_EINVAL, "NULL context");
  if (!c->have_lm) return fail(c, PCV_ESTATE, "landmarks not set");
  if (!c->have_lambda) return fail(c, PCV_ESTATE, "lambda not set");
  if (F < 0) return fail(c, PCV_EINVAL, "F < 0");
  if (F == 0) return PCV_OK;
  if (!frames || !s || !z) return fail(c, PCV_EINVAL, "frames, s and z are required");
  if ((dsdx == nullptr) != (dzdx == nullptr)) return fail(c, PCV_EINVAL, "pass both dsdx and dzdx or neither");
  if ((size_t)F * c->M > ((size_t)1 << 40)) return fail(c, PCV_EINVAL, "F*M too large");
  cudaSetDevice(c->device);
  const bool close = c->eps >= 0.0;
  pcv_status st = ensure_frame_workspace(c, F, close, dsdx != nullptr && !nl_active(c));
  if (st != PCV_OK) return st;
  const int64_t launches0 = t_launches;
  st = close ? evaluate_close(c, F, frames, s, z, dsdx, dzdx, msd, refreshed)
             : (nl_active(c) ? evaluate_exact_nl(c, F, frames, s, z, dsdx, dzdx, msd, refreshed)
                             : evaluate_exact(c, F, frames, s, z, dsdx, dzdx, msd, refreshed));
  c->stats.kernel_launches += t_launches - launches0;
  if (st != PCV_OK) return st;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(c, PCV_ECUDA, "kernel launch: %s", cudaGetErrorString(e));
  return PCV_OK;
}

// ---------------------------------------------------------------------------------------
// Group evaluation (multiple walkers / ragged instances): one persistent launch per step of
// the exact path over every instance, replayed from a captured CUDA graph.
pcv_status pcv_evaluate_group(pcv_ctx* const* ctxs, int n, const pcv_batch_io* io, void* stream) {
  if (n < 1 || !ctxs || !io) return fail(nullptr, PCV_EINVAL, "need n >= 1 contexts and as many io entries");
  pcv_ctx* lead = ctxs[0];
  if (!lead) return fail(nullptr, PCV_EINVAL, "NULL context 0");
  bool persistent = true;
  for (int k = 0; k < n; ++k) {
    pcv_ctx* c = ctxs[k];
    if (!c) return fail(lead, PCV_EINVAL, "NULL context %d", k);
    for (int j = 0; j < k; ++j)
      if (ctxs[j] == c) return fail(lead, PCV_EINVAL, "context %d appears twice (entries %d and %d)", k, j, k);
    if (!c->have_lm || !c->have_lambda) return fail(lead, PCV_ESTATE, "context %d: landmarks or lambda not set", k);
    if (c->device != lead->device) return fail(lead, PCV_EINVAL, "context %d is on another device", k);
    const pcv_batch_io& b = io[k];
    if (b.F < 0) return fail(lead, PCV_EINVAL, "entry %d: F < 0", k);
    if (b.F > 0 && (!b.frames || !b.s || !b.z)) return fail(lead, PCV_EINVAL, "entry %d: frames, s, z required", k);
    if ((b.dsdx == nullptr) != (b.dzdx == nullptr)) return fail(lead, PCV_EINVAL, "entry %d: dsdx and dzdx", k);
    if ((size_t)b.F * c->M > ((size_t)1 << 40)) return fail(lead, PCV_EINVAL, "entry %d: F*M too large", k);
    // the persistent path covers exact mode without gradients in the FP32 modes, one storage type
    if (c->eps >= 0.0 || b.dsdx || c->prec == P_F64 || c->prec != lead->prec || nl_active(c) || c->split_w)
      persistent = false;
  }
  cudaSetDevice(lead->device);
  const cudaStream_t user = (cudaStream_t)stream;
  if (!persistent) {  // one evaluation per instance, in order, on the caller's stream
    for (int k = 0; k < n; ++k) {
      pcv_ctx* c = ctxs[k];
      const cudaStream_t old = c->stream;
      c->stream = user;
      const pcv_batch_io& b = io[k];
      const pcv_status r = pcv_evaluate(c, b.F, b.frames, b.s, b.z, b.dsdx, b.dzdx, b.msd, b.refreshed);
      c->stream = old;
      if (r != PCV_OK) {
        if (c != lead) fail(lead, r, "entry %d: %s", k, c->err.c_str());
        return r;
      }
    }
    return PCV_OK;
  }
  // workspaces and descriptors
  std::vector<GroupInst> inst(n);
  std::vector<GroupTile> tiles_of[EXACT_SHAPES];  // the tile list of every shape
  int Ftot = 0;
  std::vector<uint64_t> sig = {(uint64_t)n};
  for (int k = 0; k < n; ++k) {
    pcv_ctx* c = ctxs[k];
    const pcv_batch_io& b = io[k];
    pcv_status r = ensure_frame_workspace(c, b.F > 0 ? b.F : 1, false, false);
    if (r != PCV_OK) return r;
    const LandmarkDev L = lm_view(c);
    GroupInst& t = inst[k];
    t.frames = (const float*)b.frames;
    t.lm = L.coords;
    t.lmoff = L.off;
    t.lG = L.G;
    t.w = L.w;
    t.dscale = L.dscale;
    t.q32 = L.q32;
    t.lambda = (float)c->lambda;
    t.M = c->M;
    t.N = c->N;
    t.F = b.F;
    t.fbase = Ftot;
    t.c32 = (float4*)c->c32.p;
    t.fG = (double*)c->fG.p;
    t.D = (float*)c->Dbuf.p;
    t.mstat = (float*)c->mstat.p;
    t.s = b.s;
    t.z = b.z;
    t.msd = b.msd;
    t.status = (unsigned*)c->status.p;
    for (int sh = 0; sh < EXACT_SHAPES; ++sh)
      for (int r0 = 0; r0 < b.F; r0 += kExactShape[sh].tf)
        for (int i0 = 0; i0 < c->M; i0 += kExactShape[sh].tm) tiles_of[sh].push_back(GroupTile{k, r0, i0, 0});
    Ftot += b.F;
    const uint64_t lam_bits = *reinterpret_cast<const uint64_t*>(&c->lambda);
    for (uint64_t v : {(uint64_t)(uintptr_t)c, (uint64_t)b.F, (uint64_t)(uintptr_t)b.frames, (uint64_t)(uintptr_t)b.s,
                       (uint64_t)(uintptr_t)b.z, (uint64_t)(uintptr_t)b.msd, (uint64_t)(uintptr_t)L.coords,
                       (uint64_t)(uintptr_t)c->Dbuf.p, (uint64_t)(uintptr_t)c->c32.p, lam_bits,
                       (uint64_t)c->M, (uint64_t)c->N})
      sig.push_back(v);
  }
  if (!lead->grp_stream) {
    CUDA_TRY(lead, cudaStreamCreateWithFlags(&lead->grp_stream, cudaStreamNonBlocking));
    CUDA_TRY(lead, cudaEventCreateWithFlags(&lead->grp_ev[0], cudaEventDisableTiming));
    CUDA_TRY(lead, cudaEventCreateWithFlags(&lead->grp_ev[1], cudaEventDisableTiming));
  }
  const cudaStream_t gs = lead->grp_stream;
  const bool fp16 = lead->prec == P_F16;
  size_t max_tiles = 1;
  for (int sh = 0; sh < EXACT_SHAPES; ++sh) max_tiles = std::max(max_tiles, tiles_of[sh].size());
  sig.push_back((uint64_t)lead->exact_tile);
  // order the group's work after the caller's earlier work
  CUDA_TRY(lead, cudaEventRecord(lead->grp_ev[0], user));
  CUDA_TRY(lead, cudaStreamWaitEvent(gs, lead->grp_ev[0], 0));
  if (sig != lead->grp_sig) {
    pcv_status r;
    if ((r = ensure(lead, lead->grp_inst, sizeof(GroupInst) * n)) != PCV_OK) return r;
    if ((r = ensure(lead, lead->grp_tiles, sizeof(GroupTile) * max_tiles)) != PCV_OK) return r;
    CUDA_TRY(lead, cudaMemcpyAsync(lead->grp_inst.p, inst.data(), sizeof(GroupInst) * n, cudaMemcpyHostToDevice, gs));
    const GroupInst* I = (const GroupInst*)lead->grp_inst.p;
    const GroupTile* T = (const GroupTile*)lead->grp_tiles.p;
    launch_frame_prep_group(I, n, Ftot, gs);
    // autotuner: for every tile shape (or the one PCV_OPT_EXACT_TILE fixes on ctxs[0]), its
    // tile list, then persistent grids of 1, 2, 3, 4 and 8 CTAs per SM and one CTA per tile,
    // each timed once after a first run of the shape has warmed the caches; the fastest
    // (shape, grid) is kept for this group
    int sms = 152;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, lead->device);
    float best = 3.4e38f;
    int best_blocks = 4 * sms, best_shape = lead->exact_tile > 0 ? lead->exact_tile - 1 : 0;
    {  // the timing events live for the search only (released on every return, before any capture)
      struct Events {
        cudaEvent_t a = nullptr, b = nullptr;
        ~Events() {
          if (a) cudaEventDestroy(a);
          if (b) cudaEventDestroy(b);
        }
      } ev;
      CUDA_TRY(lead, cudaEventCreate(&ev.a));
      CUDA_TRY(lead, cudaEventCreate(&ev.b));
      const cudaEvent_t t0 = ev.a, t1 = ev.b;
      for (int sh = 0; sh < EXACT_SHAPES; ++sh) {
        if (lead->exact_tile > 0 && sh != lead->exact_tile - 1) continue;
        const std::vector<GroupTile>& tl = tiles_of[sh];
        const int ntiles = (int)tl.size();
        if (ntiles == 0) continue;
        CUDA_TRY(lead, cudaMemcpyAsync(lead->grp_tiles.p, tl.data(), sizeof(GroupTile) * ntiles,
                                       cudaMemcpyHostToDevice, gs));
        launch_exact_group(fp16, sh, I, T, ntiles, 4 * sms, gs);
        const int cands[] = {sms, 2 * sms, 3 * sms, 4 * sms, 8 * sms, ntiles};
        for (int cand : cands) {
          const int blocks = cand < 1 ? 1 : (cand > ntiles ? ntiles : cand);
          CUDA_TRY(lead, cudaEventRecord(t0, gs));
          launch_exact_group(fp16, sh, I, T, ntiles, blocks, gs);
          CUDA_TRY(lead, cudaEventRecord(t1, gs));
          CUDA_TRY(lead, cudaEventSynchronize(t1));  // a failed run must not count as a fast one
          float ms = 0.0f;
          CUDA_TRY(lead, cudaEventElapsedTime(&ms, t0, t1));
          if (ms < best) {
            best = ms;
            best_blocks = blocks;
            best_shape = sh;
          }
        }
      }
    }
    lead->grp_blocks = best_blocks;
    lead->grp_shape = best_shape;
    const int ntiles = (int)tiles_of[best_shape].size();
    if (ntiles > 0)
      CUDA_TRY(lead, cudaMemcpyAsync(lead->grp_tiles.p, tiles_of[best_shape].data(), sizeof(GroupTile) * ntiles,
                                     cudaMemcpyHostToDevice, gs));
    CUDA_TRY(lead, cudaStreamSynchronize(gs));  // the host vectors are released on return
    lead->grp_ntiles = ntiles;
    // capture the step: frame preparation, exact tiles, path CVs
    if (lead->grp_exec) {
      cudaGraphExecDestroy(lead->grp_exec);
      lead->grp_exec = nullptr;
    }
    cudaGraph_t graph = nullptr;
    CUDA_TRY(lead, cudaStreamBeginCapture(gs, cudaStreamCaptureModeThreadLocal));
    launch_frame_prep_group(I, n, Ftot, gs);
    launch_exact_group(fp16, lead->grp_shape, I, T, ntiles, lead->grp_blocks, gs);
    launch_finalize_group(I, n, Ftot, gs);
    CUDA_TRY(lead, cudaStreamEndCapture(gs, &graph));
    const cudaError_t ie = cudaGraphInstantiate(&lead->grp_exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) return fail(lead, PCV_ECUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(ie));
    lead->grp_sig = sig;
  }
  CUDA_TRY(lead, cudaGraphLaunch(lead->grp_exec, gs));
  CUDA_TRY(lead, cudaEventRecord(lead->grp_ev[1], gs));
  CUDA_TRY(lead, cudaStreamWaitEvent(user, lead->grp_ev[1], 0));
  for (int k = 0; k < n; ++k) {
    pcv_ctx* c = ctxs[k];
    c->stats.frames += io[k].F;
    c->stats.landmark_alignments += (int64_t)c->M * io[k].F;
    if (io[k].refreshed) launch_fill_u8(io[k].refreshed, 1, (size_t)io[k].F, user);
  }
  lead->stats.kernel_launches += 3;
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(lead, PCV_ECUDA, "group launch: %s", cudaGetErrorString(e));
  return PCV_OK;
}

pcv_status pcv_group_tuning(const pcv_ctx* ctx, int* tile_frames, int* tile_landmarks, int* blocks) {
  if (!ctx || !tile_frames || !tile_landmarks || !blocks) return fail(nullptr, PCV_EINVAL, "NULL argument");
  const bool tuned = ctx->grp_blocks > 0;
  *tile_frames = tuned ? kExactShape[ctx->grp_shape].tf : 0;
  *tile_landmarks = tuned ? kExactShape[ctx->grp_shape].tm : 0;
  *blocks = ctx->grp_blocks;
  return PCV_OK;
}

// Chunk sizes of pcv_evaluate_host: n chunks (0: about one per 16k frames, between 1 and 8)
// whose first and last hold end_share percent of a middle one; at least 2048 frames each.
std::vector<int> host_chunk_plan(int F, int n, int end_share) {
  if (n <= 0) n = std::min(8, std::max(1, (F + 16383) / 16384));
  n = std::min(n, std::max(1, F / 2048));
  if (n <= 1) return {F};
  if (n == 2) return {F / 2, F - F / 2};  // no middle chunk to scale the ends by
  const double we = end_share / 100.0;
  const double unit = F / ((n - 2) + 2.0 * we);  // a middle chunk
  const int e = std::max(2048, (int)(unit * we));
  std::vector<int> plan(n, 0);
  plan[0] = plan[n - 1] = e;
  const int rest = F - 2 * e, mid = n - 2;
  for (int k = 0; k < mid; ++k) plan[1 + k] = rest / mid + (k < rest % mid ? 1 : 0);
  return plan;
}

pcv_status pcv_host_chunk_plan(int F, int n, int end_share, int* sizes, int cap, int* count) {
  if (F < 0 || n < 0 || n > 64 || end_share < 1 || end_share > 100 || !count || (cap > 0 && !sizes))
    return fail(nullptr, PCV_EINVAL, "bad chunk-plan arguments");
  if (F == 0) {
    *count = 0;
    return PCV_OK;
  }
  const std::vector<int> plan = host_chunk_plan(F, n, end_share);
  *count = (int)plan.size();
  for (int k = 0; k < (int)plan.size() && k < cap; ++k) sizes[k] = plan[k];
  return PCV_OK;
}

pcv_status pcv_evaluate_host(pcv_ctx* c, int F, const void* frames, double* s, double* z, void* dsdx, void* dzdx,
                             double* msd, uint8_t* refreshed) {
  if (!c) return fail(nullptr, PCV_EINVAL, "NULL context");
  if (!c->have_lm) return fail(c, PCV_ESTATE, "landmarks not set");
  if (F < 0) return fail(c, PCV_EINVAL, "F < 0");
  if (F == 0) return PCV_OK;
  if (!frames || !s || !z) return fail(c, PCV_EINVAL, "frames, s and z are required");
  if ((dsdx == nullptr) != (dzdx == nullptr)) return fail(c, PCV_EINVAL, "pass both dsdx and dzdx or neither");
  cudaSetDevice(c->device);
  const size_t fbytes = frame_elem(c->prec) * 3 * (size_t)c->N * F;
  pcv_status st;
  if ((st = ensure(c, c->h_frames, fbytes)) != PCV_OK) return st;
  if ((st = ensure(c, c->h_s, sizeof(double) * F)) != PCV_OK) return st;
  if ((st = ensure(c, c->h_z, sizeof(double) * F)) != PCV_OK) return st;
  if (dsdx) {
    if ((st = ensure(c, c->h_gs, fbytes)) != PCV_OK) return st;
    if ((st = ensure(c, c->h_gz, fbytes)) != PCV_OK) return st;
  }
  if (msd && (st = ensure(c, c->h_msd, sizeof(double) * (size_t)F * c->M)) != PCV_OK) return st;
  if (refreshed && (st = ensure(c, c->h_ref, F)) != PCV_OK) return st;
  // The batch is evaluated in chunks of consecutive frames (the close-structure state and
  // the neighbour list carry over between chunks exactly as between calls): the frames of
  // later chunks are copied in on one copy stream, and the outputs of earlier chunks copied
  // out on another, while a chunk is evaluated on the context's stream.  The first and the
  // last chunk are smaller than the others: nothing overlaps the first chunk's copy-in or
  // the last chunk's copy-out.
  // automatic: the frame rule of host_chunk_plan, or one chunk per 128 MiB of frame
  // coordinates when that gives more (large structures: 10k frames of 5000 atoms are 600 MB
  // whose copy-in would otherwise precede the whole evaluation)
  int nchunks = c->host_chunks;
  if (nchunks == 0)
    nchunks = std::max((int)host_chunk_plan(F, 0, c->host_end_share).size(),
                       (int)std::min<size_t>(8, (fbytes + ((size_t)128 << 20) - 1) >> 27));
  const std::vector<int> plan = host_chunk_plan(F, nchunks, c->host_end_share);
  const int nchunk = (int)plan.size();
  std::vector<size_t> first(nchunk + 1, 0);
  for (int k = 0; k < nchunk; ++k) first[k + 1] = first[k] + (size_t)plan[k];
  for (cudaStream_t* hs : {&c->h2d_stream, &c->d2h_stream})
    if (!*hs) CUDA_TRY(c, cudaStreamCreateWithFlags(hs, cudaStreamNonBlocking));
  while ((int)c->h_events.size() < 2 * nchunk + 1) {
    cudaEvent_t e;
    CUDA_TRY(c, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    c->h_events.push_back(e);
  }
  cudaEvent_t* ev_in = c->h_events.data();            // frames of chunk k are on the device
  cudaEvent_t* ev_done = c->h_events.data() + nchunk;  // chunk k is evaluated
  cudaEvent_t ev_start = c->h_events[2 * nchunk];
  const size_t fstride = frame_elem(c->prec) * 3 * (size_t)c->N;  // bytes per frame
  // the copies start after the context's earlier work (the staging buffers may be in use)
  CUDA_TRY(c, cudaEventRecord(ev_start, c->stream));
  CUDA_TRY(c, cudaStreamWaitEvent(c->h2d_stream, ev_start, 0));
  CUDA_TRY(c, cudaStreamWaitEvent(c->d2h_stream, ev_start, 0));
  for (int k = 0; k < nchunk; ++k) {
    const size_t f0 = first[k], nf = (size_t)plan[k];
    CUDA_TRY(c, cudaMemcpyAsync((char*)c->h_frames.p + fstride * f0, (const char*)frames + fstride * f0, fstride * nf,
                                cudaMemcpyHostToDevice, c->h2d_stream));
    CUDA_TRY(c, cudaEventRecord(ev_in[k], c->h2d_stream));
  }
  for (int k = 0; k < nchunk; ++k) {
    const size_t f0 = first[k], nf = (size_t)plan[k];
    CUDA_TRY(c, cudaStreamWaitEvent(c->stream, ev_in[k], 0));
    st = pcv_evaluate(c, (int)nf, (char*)c->h_frames.p + fstride * f0, (double*)c->h_s.p + f0,
                      (double*)c->h_z.p + f0, dsdx ? (char*)c->h_gs.p + fstride * f0 : nullptr,
                      dsdx ? (char*)c->h_gz.p + fstride * f0 : nullptr,
                      msd ? (double*)c->h_msd.p + f0 * c->M : nullptr, refreshed ? (uint8_t*)c->h_ref.p + f0 : nullptr);
    if (st != PCV_OK) {
      cudaStreamSynchronize(c->h2d_stream);
      cudaStreamSynchronize(c->d2h_stream);
      return st;
    }
    CUDA_TRY(c, cudaEventRecord(ev_done[k], c->stream));
    CUDA_TRY(c, cudaStreamWaitEvent(c->d2h_stream, ev_done[k], 0));
    const cudaStream_t o = c->d2h_stream;
    CUDA_TRY(c, cudaMemcpyAsync(s + f0, (double*)c->h_s.p + f0, sizeof(double) * nf, cudaMemcpyDeviceToHost, o));
    CUDA_TRY(c, cudaMemcpyAsync(z + f0, (double*)c->h_z.p + f0, sizeof(double) * nf, cudaMemcpyDeviceToHost, o));
    if (dsdx) {
      CUDA_TRY(c, cudaMemcpyAsync((char*)dsdx + fstride * f0, (char*)c->h_gs.p + fstride * f0, fstride * nf,
                                  cudaMemcpyDeviceToHost, o));
      CUDA_TRY(c, cudaMemcpyAsync((char*)dzdx + fstride * f0, (char*)c->h_gz.p + fstride * f0, fstride * nf,
                                  cudaMemcpyDeviceToHost, o));
    }
    if (msd)
      CUDA_TRY(c, cudaMemcpyAsync(msd + f0 * c->M, (double*)c->h_msd.p + f0 * c->M, sizeof(double) * nf * c->M,
                                  cudaMemcpyDeviceToHost, o));
    if (refreshed)
      CUDA_TRY(c, cudaMemcpyAsync(refreshed + f0, (uint8_t*)c->h_ref.p + f0, nf, cudaMemcpyDeviceToHost, o));
  }
  CUDA_TRY(c, cudaStreamSynchronize(c->d2h_stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return PCV_OK;
}

pcv_status pcv_combine_grad(pcv_ctx* c, int F, const double* g_s, const double* g_z, const void* dsdx,
                            const void* dzdx, void* out) {
  if (!c) return fail(nullptr, PCV_EINVAL, "NULL context");
  if (!c->have_lm) return fail(c, PCV_ESTATE, "landmarks not set");
  if (F < 0) return fail(c, PCV_EINVAL, "F < 0");
  if (F == 0) return PCV_OK;
  if (!dsdx || !dzdx || !out) return fail(c, PCV_EINVAL, "dsdx, dzdx and out are required");
  cudaSetDevice(c->device);
  const int64_t launches0 = t_launches;
  {
    PROF(c, K_COMBINE);
    launch_combine_grad(c->prec, F, 3 * c->N, g_s, g_z, dsdx, dzdx, out, c->stream);
  }
  c->stats.kernel_launches += t_launches - launches0;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(c, PCV_ECUDA, "kernel launch: %s", cudaGetErrorString(e));
  return PCV_OK;
}

pcv_status pcv_sync(pcv_ctx* c) {
  if (!c) return fail(nullptr, PCV_EINVAL, "NULL context");
  cudaSetDevice(c->device);
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  unsigned status = 0;
  CUDA_TRY(c, cudaMemcpy(&status, c->status.p, sizeof(unsigned), cudaMemcpyDeviceToHost));
  if (status) {
    CUDA_TRY(c, cudaMemset(c->status.p, 0, sizeof(unsigned)));
    if (status & STATUS_TIMEOUT)
      return fail(c, PCV_ETIMEOUT, "a device-side wait exceeded its time limit; the batch's results are invalid");
    if (status & STATUS_NOCONV) return fail(c, PCV_ENOCONV, "an eigen-solve reached its iteration cap");
  }
  return PCV_OK;
}

pcv_status pcv_get_profile(pcv_ctx* c, int n, double* ms, int64_t* launches) {
  if (!c) return fail(nullptr, PCV_EINVAL, "NULL context");
  if (n < 0 || n > PCV_PROFILE_KERNELS || (n > 0 && (!ms || !launches))) return fail(c, PCV_EINVAL, "bad arrays");
  cudaSetDevice(c->device);
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  for (const ProfEvent& e : c->prof_pending) {
    float t = 0.0f;
    if (cudaEventElapsedTime(&t, e.a, e.b) == cudaSuccess) {
      c->prof_ms[e.id] += t;
      c->prof_launches[e.id] += 1;
    }
    c->prof_pool.push_back(e.a);
    c->prof_pool.push_back(e.b);
  }
  c->prof_pending.clear();
  for (int k = 0; k < n; ++k) {
    ms[k] = c->prof_ms[k];
    launches[k] = c->prof_launches[k];
  }
  for (int k = 0; k < PCV_PROFILE_KERNELS; ++k) {
    c->prof_ms[k] = 0.0;
    c->prof_launches[k] = 0;
  }
  return PCV_OK;
}

const char* pcv_profile_name(int id) { return (id >= 0 && id < PCV_PROFILE_KERNELS) ? kKernelNames[id] : ""; }

pcv_status pcv_get_stats(pcv_ctx* c, pcv_stats* out) {
  if (!c || !out) return fail(c, PCV_EINVAL, "NULL argument");
  cudaSetDevice(c->device);
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  unsigned long long n = 0;
  CUDA_TRY(c, cudaMemcpy(&n, c->nrecheck.p, sizeof(n), cudaMemcpyDeviceToHost));
  c->stats.fp64_rechecks = (int64_t)n;
  *out = c->stats;
  return PCV_OK;
}

// state blob: header, then y (N*3 frame type), B (M*9 work type), the neighbour list
// (nl_size ints)
namespace {
struct StateHeader {
  char magic[8];
  int32_t version, prec, M, N, has_y, pad;
  int32_t nl_size, has_nl;
  float4 y_c32;
  double4 y_c64;
  double y_G;
  double gap_estimate;
  pcv_stats stats;
};
}  // namespace

pcv_status pcv_save_state(pcv_ctx* c, void* buf, size_t* len) {
  if (!c || !len) return fail(c, PCV_EINVAL, "NULL argument");
  if (!c->have_lm) return fail(c, PCV_ESTATE, "landmarks not set");
  const size_t ybytes = frame_elem(c->prec) * 3 * (size_t)c->N;
  const size_t bbytes = work_elem(c->prec) * 9 * (size_t)c->M;
  const size_t lbytes = sizeof(int) * (size_t)c->nl_size;
  const size_t need = sizeof(StateHeader) + ybytes + bbytes + lbytes;
  if (!buf) {
    *len = need;
    return PCV_OK;
  }
  if (*len < need) return fail(c, PCV_EINVAL, "buffer too small (%zu < %zu)", *len, need);
  pcv_stats stt;
  pcv_status st = pcv_get_stats(c, &stt);
  if (st != PCV_OK) return st;
  StateHeader h{};
  memcpy(h.magic, "PCVSTAT", 8);
  h.version = 2;
  h.prec = (int)c->prec;
  h.nl_size = c->nl_size;
  h.has_nl = c->has_nl ? 1 : 0;
  h.M = c->M;
  h.N = c->N;
  h.has_y = c->has_y ? 1 : 0;
  h.y_c32 = c->y_c32;
  h.y_c64 = c->y_c64;
  h.y_G = c->y_G;
  h.gap_estimate = c->gap_estimate;
  h.stats = stt;
  char* out = (char*)buf;
  memcpy(out, &h, sizeof(h));
  if (c->has_y) {
    CUDA_TRY(c, cudaMemcpy(out + sizeof(h), c->y.p, ybytes, cudaMemcpyDeviceToHost));
    CUDA_TRY(c, cudaMemcpy(out + sizeof(h) + ybytes, c->Bprior.p, bbytes, cudaMemcpyDeviceToHost));
  } else {
    memset(out + sizeof(h), 0, ybytes + bbytes);
  }
  if (c->has_nl)
    CUDA_TRY(c, cudaMemcpy(out + sizeof(h) + ybytes + bbytes, c->nl_keep.p, lbytes, cudaMemcpyDeviceToHost));
  else
    memset(out + sizeof(h) + ybytes + bbytes, 0, lbytes);
  *len = need;
  return PCV_OK;
}

pcv_status pcv_load_state(pcv_ctx* c, const void* buf, size_t len) {
  if (!c || !buf) return fail(c, PCV_EINVAL, "NULL argument");
  if (!c->have_lm) return fail(c, PCV_ESTATE, "landmarks not set");
  const size_t ybytes = frame_elem(c->prec) * 3 * (size_t)c->N;
  const size_t bbytes = work_elem(c->prec) * 9 * (size_t)c->M;
  if (len < sizeof(StateHeader) + ybytes + bbytes) return fail(c, PCV_ESTATE, "state blob too short");
  StateHeader h;
  memcpy(&h, buf, sizeof(h));
  if (memcmp(h.magic, "PCVSTAT", 8) != 0 || h.version != 2) return fail(c, PCV_ESTATE, "not a state blob");
  if (h.prec != (int)c->prec || h.M != c->M || h.N != c->N) return fail(c, PCV_ESTATE, "state blob does not match");
  if (h.nl_size != c->nl_size) return fail(c, PCV_ESTATE, "state blob has another neighbour-list size");
  const size_t lbytes = sizeof(int) * (size_t)h.nl_size;
  if (len < sizeof(StateHeader) + ybytes + bbytes + lbytes) return fail(c, PCV_ESTATE, "state blob too short");
  if (h.has_nl && h.nl_size > 0) {
    const int* lst = (const int*)((const char*)buf + sizeof(h) + ybytes + bbytes);
    for (int r = 0; r < h.nl_size; ++r)
      if (lst[r] < 0 || lst[r] >= c->M) return fail(c, PCV_ESTATE, "state blob holds a bad neighbour list");
  }
  cudaSetDevice(c->device);
  pcv_status st;
  if ((st = ensure(c, c->y, ybytes)) != PCV_OK) return st;
  if ((st = ensure(c, c->Bprior, bbytes)) != PCV_OK) return st;
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  const char* in = (const char*)buf;
  CUDA_TRY(c, cudaMemcpy(c->y.p, in + sizeof(h), ybytes, cudaMemcpyHostToDevice));
  CUDA_TRY(c, cudaMemcpy(c->Bprior.p, in + sizeof(h) + ybytes, bbytes, cudaMemcpyHostToDevice));
  c->has_nl = false;
  if (h.has_nl && h.nl_size > 0) {
    if ((st = ensure(c, c->nl_keep, lbytes)) != PCV_OK) return st;
    CUDA_TRY(c, cudaMemcpy(c->nl_keep.p, in + sizeof(h) + ybytes + bbytes, lbytes, cudaMemcpyHostToDevice));
    c->has_nl = true;
  }
  c->has_y = h.has_y != 0;
  c->y_c32 = h.y_c32;
  c->y_c64 = h.y_c64;
  c->y_G = h.y_G;
  c->gap_estimate = h.gap_estimate;
  c->stats = h.stats;
  unsigned long long n = (unsigned long long)h.stats.fp64_rechecks;
  CUDA_TRY(c, cudaMemcpy(c->nrecheck.p, &n, sizeof(n), cudaMemcpyHostToDevice));
  return PCV_OK;
}

}  // extern "C"

/*
 * pcv.h -- C ABI of the GB300 path-CV / MSD library.
 *
 * Batched mean-square-distance (MSD) evaluation behind property-map / path collective
 * variables in metadynamics, with the floating close-structure approximation, after
 * Pazurikova, Olha, Krenek, Spiwok, "Acceleration of Mean Square Distance Calculations
 * with Floating Close Structure in Metadynamics Simulations" (arXiv:1801.02362).
 *
 * Notation: M landmark (reference) structures a_i, N atoms, F frames x_t per call.
 * (The paper writes N for the number of reference structures; here that is M.)
 *
 * Conventions for every call:
 *  - Plain pointers and sizes only.  "device" pointers are CUDA device memory of the
 *    context's device; "host" pointers are ordinary CPU memory.  The caller owns every
 *    buffer it passes; the library never frees or retains caller pointers after a call
 *    returns.  Device work is enqueued on the context's stream and is asynchronous
 *    unless a call says otherwise.
 *  - Coordinates are row-major (structure, atom, xyz), in nm.
 *  - Every call returns a pcv_status.  Argument errors are detected on the host before
 *    any work is enqueued and leave the context unchanged.  pcv_last_error() returns a
 *    one-line description of the last failure on the context.
 *  - Precision modes fix the element types:
 *      PCV_FP64          frames double, landmarks double, all arithmetic FP64,
 *                        gradients double;
 *      PCV_FP32          frames float, landmarks float (centred); correlation sums in
 *                        FP32, the 4x4 eigen-solve in FP32 for the rotation only, and the
 *                        MSD summed directly as sum_j w_j |x_j - R a_j|^2 in compensated
 *                        FP32 (it is stationary in R, so a rotation accurate to FP32 gives
 *                        an MSD accurate to FP32); close-structure decisions within the
 *                        FP32 rounding window of the threshold are re-checked in FP64;
 *                        gradients float;
 *      PCV_FP16_STORAGE  as PCV_FP32 but landmarks stored as FP16 residuals about an
 *                        FP32 offset per landmark and block of 16 consecutive atoms (the
 *                        block mean of the centred coordinates): 6 bytes per atom plus
 *                        12 bytes per block, with the rounding error of a block's extent
 *                        rather than of the whole structure's.
 *  - The library allocates its own device workspace (cudaMalloc, grow-only) on first
 *    use of a size; it is freed by pcv_destroy.
 */
#ifndef PCV_H
#define PCV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PCV_API_VERSION 1

#if defined(__GNUC__)
#define PCV_API __attribute__((visibility("default")))
#else
#define PCV_API
#endif

typedef struct pcv_ctx pcv_ctx;

typedef enum {
  PCV_OK = 0,
  PCV_EINVAL = -1,  /* invalid argument (sizes, NULL where required, NaN, lambda <= 0) */
  PCV_ECUDA = -2,   /* a CUDA runtime call failed; see pcv_last_error()                */
  PCV_ENOMEM = -3,  /* device or host allocation failed                                 */
  PCV_ENOCONV = -4, /* an eigen-solve hit its iteration cap (reported at pcv_sync)      */
  PCV_ESTATE = -5,  /* call out of order (no landmarks, bad saved state, ...)           */
  PCV_ETIMEOUT = -6 /* a bounded device-side wait expired (reported at pcv_sync); the
                       results of the batches since the previous pcv_sync are invalid */
} pcv_status;

typedef enum { PCV_FP64 = 0, PCV_FP32 = 1, PCV_FP16_STORAGE = 2 } pcv_precision;

/* Counters of the work done since the last pcv_reset_close_state (or creation).  The
 * "expensive" distance computations of the paper's cost model (Section "Theoretical
 * Speedup": M + (N-M)/L per step originally, 1 + N/K with the close structure) are
 * xy_alignments + landmark_alignments. */
typedef struct {
  int64_t frames;              /* frames evaluated                                        */
  int64_t xy_alignments;       /* exact alignments of a frame onto the close structure y  */
  int64_t landmark_alignments; /* exact (eigen-solved) frame-landmark MSDs                */
  int64_t approx_msds;         /* approximate MSDs, Eq. (close_dist)                      */
  int64_t refreshes_threshold; /* close-structure reassignments with D(x,y) > eps        */
  int64_t refreshes_initial;   /* initial close-structure assignments                     */
  int64_t fp64_rechecks;       /* refresh decisions re-evaluated in full FP64             */
  int64_t host_syncs;          /* host round trips of the refresh search                  */
  int64_t kernel_launches;     /* CUDA kernels this context launched                      */
} pcv_stats;

/* Create a context on CUDA device `device`, enqueueing on `cuda_stream` (a cudaStream_t;
 * NULL = legacy default stream), in precision mode `precision` (pcv_precision).
 * Errors: PCV_EINVAL (bad device / precision), PCV_ECUDA, PCV_ENOMEM. */
PCV_API pcv_status pcv_create(pcv_ctx** out, int device, void* cuda_stream, int precision);

/* Free every device and host resource of the context.  Synchronises its stream. */
PCV_API pcv_status pcv_destroy(pcv_ctx* ctx);

/* Replace the stream the context enqueues on (a cudaStream_t). */
PCV_API pcv_status pcv_set_stream(pcv_ctx* ctx, void* cuda_stream);

/* Set the landmark (reference) structures a_i of Eq. (property_map_cv).
 *   coords  host, M*N*3 doubles, landmark-major; each landmark is centred here by its
 *           weighted centre (Section "Floating Close Structure": both structures are
 *           shifted to the same location before fitting) and stored in the mode's
 *           storage type;
 *   w       host, N doubles > 0, or NULL for uniform weights; normalised to sum 1.  One
 *           weight set serves as displacement weights w and alignment weights w'
 *           (Eq. der_dist; pcv_set_landmarks_weighted takes separate sets);
 *   q       host, M doubles, the property q_i of each landmark, or NULL for q_i = i
 *           (1-based index: the path CV s).
 * Resets the close-structure state.  Synchronous with respect to the host buffers.
 * Errors: PCV_EINVAL (M < 1, N < 3, NULL coords, non-finite values, w <= 0). */
PCV_API pcv_status pcv_set_landmarks(pcv_ctx* ctx, int M, int N, const double* coords, const double* w,
                             const double* q);

/* As pcv_set_landmarks, with separate alignment weights (Section 3.1 after Eq. der_dist):
 *   w        displacement weights: each atom's contribution to the distance
 *            D = sum_j w_j |x_j - R a_j|^2 (host, N doubles > 0, or NULL for uniform);
 *   w_align  alignment weights: each atom's contribution to the centre of mass, which sets
 *            the translation (host, N doubles > 0, or NULL for w_align = w).
 * Frames, landmarks and close structures are centred by their w_align-weighted centres;
 * the rotation minimises the w-weighted distance.  The derivatives of Eq. (der_dist) and
 * Eq. (close_der_dist) then carry the centre term w'_k sum_j (-2 w_j d_j), and in close mode
 * the rotation term's dependence of the fit on the centre of x.  With different sets the
 * materialised-operand and tensor-core paths and the persistent group launch are not used
 * (the kernels that rotate while staging are).  Both sets are normalised to sum 1.
 * Errors: as pcv_set_landmarks, and PCV_EINVAL for w_align entries <= 0. */
PCV_API pcv_status pcv_set_landmarks_weighted(pcv_ctx* ctx, int M, int N, const double* coords, const double* w,
                                              const double* w_align, const double* q);

/* Set lambda of Eq. (property_map_cv), in nm^-2.  Errors: PCV_EINVAL unless lambda > 0
 * and finite. */
PCV_API pcv_status pcv_set_lambda(pcv_ctx* ctx, double lambda);

/* Set the close-structure threshold eps in nm^2 (Algorithm 2: reassign when
 * D(x, y) > eps, strictly; the paper uses 0.01).  eps < 0 selects exact mode
 * (Algorithm 1 for every frame).  Changing eps keeps the current close structure. */
PCV_API pcv_status pcv_set_close_threshold(pcv_ctx* ctx, double eps);

/* Neighbour list (Section 2; Section 3.1 after Eq. der_dist; end of Section 3.2; the cost
 * model of Section 6.2).  size = M_nl landmarks kept, stride = L steps between updates.
 * Steps are counted from the last pcv_reset_close_state / pcv_set_landmarks (the
 * `frames` counter of pcv_stats).  A step is an update step when its index is a multiple
 * of L, when no list is held yet, and, in close mode, at every close-structure
 * reassignment.  At an update step the distances to all M landmarks are computed (exact
 * mode and reassignments: exactly; other close-mode steps: the approximate distances of
 * Eq. close_dist), s and z use all of them, and the list becomes the M_nl landmarks with
 * the smallest distances (ties to the lower index).  Between updates only the listed
 * landmarks are evaluated and the sums of Eq. (property_map_cv), z and the derivatives run
 * over them; the other entries of msd are +infinity.  size = 0 or size >= M evaluates
 * every landmark at every step (the default).  Setting the list drops the list held (the
 * next step is an update).  In FP32 / FP16 storage the choice is made on the FP32
 * distances, so a landmark whose distance ties the M_nl-th smallest within FP32 rounding
 * may be chosen differently from an FP64 evaluation.
 * Errors: PCV_EINVAL (size < 0, stride < 1). */
PCV_API pcv_status pcv_set_neighbor_list(pcv_ctx* ctx, int size, int stride);

/* Evaluate F frames (time-ordered consecutive MD steps in close mode).
 *   frames     device, F*N*3 (double in PCV_FP64, else float), uncentred;
 *   s, z       device, F doubles each, required: the path CV s of Eq. (property_map_cv)
 *              and z = -(1/lambda) ln sum_i exp(-lambda D_i) (Branduardi et al. 2007,
 *              cited in Section 2);
 *   dsdx,dzdx  device, F*N*3 (double in PCV_FP64, else float), or NULL: ds/dx and dz/dx
 *              from Eq. (der_dist) (exact and reassignment frames) and
 *              Eq. (close_der_dist) (approximate frames);
 *   msd        device, F*M doubles, or NULL: D(x_t, a_i) (Eq. dist) or its close-structure
 *              approximation (Eq. close_dist); +infinity for landmarks outside the
 *              neighbour list between list updates (pcv_set_neighbor_list);
 *   refreshed  device, F bytes, or NULL: 0 approximate frame, 1 close structure reassigned
 *              because D(x, y) > eps, 2 initial assignment (exact mode: all 1).
 * In close mode the close structure y and the rotations R_{a_i y} carry over between
 * calls.  The call blocks the host only for the refresh search (a few small device-to-
 * host reads per reassignment); all other work is asynchronous.
 * Errors: PCV_EINVAL (F < 0, NULL s/z/frames with F > 0), PCV_ESTATE (no landmarks or
 * lambda), PCV_ECUDA, PCV_ENOMEM. */
PCV_API pcv_status pcv_evaluate(pcv_ctx* ctx, int F, const void* frames, double* s, double* z, void* dsdx,
                        void* dzdx, double* msd, uint8_t* refreshed);

/* As pcv_evaluate, with every buffer in host memory (pageable or pinned).  The frames are
 * copied to the device, evaluated, and the requested outputs copied back; the call
 * returns when the outputs are in host memory. */
PCV_API pcv_status pcv_evaluate_host(pcv_ctx* ctx, int F, const void* frames, double* s, double* z,
                             void* dsdx, void* dzdx, double* msd, uint8_t* refreshed);

/* Chunk plan of pcv_evaluate_host for F frames with the options PCV_OPT_HOST_CHUNKS = n
 * (0: the frame rule, about one chunk per 16k frames, 1..8; pcv_evaluate_host raises the
 * automatic count to one chunk per 128 MiB of frames when that gives more, and a plan for
 * that count is this function with n set to it) and PCV_OPT_HOST_END_SHARE =
 * end_share (1..100): the chunk sizes in order, first and last end_share percent of a middle
 * one, every chunk at least 2048 frames (the number of chunks is lowered to F / 2048 when
 * needed).  Writes min(count, cap) sizes into sizes (host array; may be NULL with cap 0) and
 * the number of chunks into *count.  Pure host computation, no device needed.
 * Errors: PCV_EINVAL (F < 0, n outside 0..64, end_share outside 1..100, count NULL, or
 * sizes NULL with cap > 0). */
PCV_API pcv_status pcv_host_chunk_plan(int F, int n, int end_share, int* sizes, int cap, int* count);

/* Chain rule for a scalar loss L(s, z): out[t] = g_s[t] * dsdx[t] + g_z[t] * dzdx[t] for
 * every frame t (device buffers; element type of dsdx/dzdx/out as in pcv_evaluate; g_s,
 * g_z device doubles, either may be NULL for zero). */
PCV_API pcv_status pcv_combine_grad(pcv_ctx* ctx, int F, const double* g_s, const double* g_z,
                            const void* dsdx, const void* dzdx, void* out);

/* Forget the close structure and the neighbour list: the next frame is an initial
 * assignment and a list update, and the step count restarts at 0.  Clears the counters
 * except host_syncs and kernel_launches, which count over the context's life. */
PCV_API pcv_status pcv_reset_close_state(pcv_ctx* ctx);

/* Serialise the close-structure state (y, R_{a_i y}, counters including the step count,
 * the neighbour list held) into host memory.
 * If buf is NULL, *len receives the size needed.  Errors: PCV_EINVAL if *len is too
 * small. */
PCV_API pcv_status pcv_save_state(pcv_ctx* ctx, void* buf, size_t* len);

/* Restore a state written by pcv_save_state for the same landmarks, N, M, precision and
 * neighbour-list size.  Errors: PCV_ESTATE if the blob does not match. */
PCV_API pcv_status pcv_load_state(pcv_ctx* ctx, const void* buf, size_t len);

/* Copy the counters.  Synchronises the context's stream. */
PCV_API pcv_status pcv_get_stats(pcv_ctx* ctx, pcv_stats* out);

/* Wait for the context's work and report deferred device errors since the last pcv_sync:
 * PCV_ETIMEOUT when a kernel's bounded wait expired, PCV_ENOCONV when an eigen-solve hit
 * its iteration cap. */
PCV_API pcv_status pcv_sync(pcv_ctx* ctx);

/* Tuning knobs (pcv_set_option keys). */
enum {
  PCV_OPT_BAND = 1,        /* frames compared with each of the previous BAND frames
                              ahead of the refresh search (1..6, default 2)           */
  PCV_OPT_CHUNK = 2,       /* minimum frames per speculative x-y alignment chunk       */
  PCV_OPT_EXACT_TILE = 3,  /* shape of the exact pair kernel's tile (FP32 / FP16 storage):
                              0 = automatic (16 frames x 32 landmarks per CTA; the group
                              launch's autotuner tries every shape), 1 = 16 x 32,
                              2 = 32 x 16, 3 = 8 x 64.  On ctxs[0] of pcv_evaluate_group a
                              nonzero value fixes the shape the autotuner uses.           */
  PCV_OPT_APPROX_TILE = 4, /* tile variant index of the approximate pair kernel        */
  PCV_OPT_PROFILE = 5,     /* 1: time every kernel launch with CUDA events on the
                              context's stream (see pcv_get_profile), 0: off (default)  */
  PCV_OPT_MATERIALIZE = 6, /* byte cap (default 2^34) on the device buffers of the
                              materialised close-structure operands: rotated frames
                              x' = R_xy^T (x - c), rotated landmarks b = R_{a_i y} a per
                              segment, and the gamma rows of the adjoint.  Used in the
                              FP32 and FP16-storage modes with uniform weights when
                              segments average 16 frames or more; 0 turns them off (the
                              kernels then rotate while staging; so they also do when the
                              device cannot allocate the operands).  Results agree within
                              the mode's tolerance either way.                          */
  PCV_OPT_TENSOR_CORES = 7, /* 1 (default): with materialised operands, the approximate MSDs'
                              cross terms dx . d_i run on the tensor cores (FP16 operands
                              split h + l after a 2^8 scale, three products per term, FP32
                              accumulation in short groups) and so does the segment adjoint
                              beta = sum_i gamma_i (R_{a_i y} a_i) (TF32 operands split hi +
                              lo, three products per term, on deviations from the close
                              structure); 0: FP32 CUDA cores for both.                    */
  PCV_OPT_HOST_CHUNKS = 8,  /* pcv_evaluate_host: number of chunks the batch is split into
                              so that copies overlap evaluation (0 = automatic, default:
                              one per 16k frames or per 128 MiB of frames, whichever gives
                              more, at most 8; 1 = no overlap; at most 64)               */
  PCV_OPT_HOST_END_SHARE = 9, /* pcv_evaluate_host: size of the first and the last chunk in
                              percent of a middle chunk (1..100; default 25): a small first
                              chunk starts the evaluation early and a small last chunk
                              shortens the copy-out that follows it                     */
  PCV_OPT_NEWTON_CAP = 10,  /* iteration cap of the Newton eigen-solves in the exact pair
                              kernels (1..60, default 60).  A pair that reaches the cap sets
                              the status word: pcv_sync then returns PCV_ENOCONV.  Lower
                              values exist to exercise that report.                      */
  PCV_OPT_WAIT_CYCLES = 11, /* clock budget (SM cycles) of each bounded wait inside the
                              tensor-core kernels (0 = default, 4e9, about 2 s at the maximum
                              clock; else 1..4e9).  A wait that runs out sets the status
                              word, the kernel waits for its own copies and MMAs within the
                              default budget, frees its tensor memory and returns; pcv_sync
                              then returns PCV_ETIMEOUT.  Small values exist to exercise
                              that report.                                                */
  PCV_OPT_MMA_GROUP = 12    /* tensor-core approximate MSDs (PCV_OPT_TENSOR_CORES = 1): chunks
                              of 16 deviation components whose main products are summed in
                              tensor memory before the partial sums are added into FP32
                              totals (1..16, default 4).  Each accumulation step can lose
                              about one unit in the last place of the running sum, so
                              shorter groups are more accurate and cost more folding work.  */
};
PCV_API pcv_status pcv_set_option(pcv_ctx* ctx, int key, int64_t value);

/* Kernel timings collected while PCV_OPT_PROFILE is on, per kernel family id
 * 0..PCV_PROFILE_KERNELS-1 (names from pcv_profile_name): total milliseconds of device time
 * between events recorded around each launch on the context's stream, and launch counts.
 * ms and launches are host arrays of n entries (n <= PCV_PROFILE_KERNELS).  Synchronises
 * the stream, then clears the collected timings. */
#define PCV_PROFILE_KERNELS 25
PCV_API pcv_status pcv_get_profile(pcv_ctx* ctx, int n, double* ms, int64_t* launches);

/* Name of kernel family `id` ("" outside 0..PCV_PROFILE_KERNELS-1). */
PCV_API const char* pcv_profile_name(int id);

/* Many walkers or instances in one call (multiple-walker metadynamics: each walker has its
 * own landmark path, sizes N and M, lambda and frames).
 *
 * io[k] is the batch of context ctxs[k] with the meaning of pcv_evaluate's arguments
 * (frames, s, z, dsdx, dzdx, msd, refreshed; device pointers; F may differ per entry and may
 * be 0).  The contexts must be distinct and on one device.  Work is ordered after the work
 * already enqueued on `stream` (a cudaStream_t; NULL = the default stream) and later work on
 * `stream` waits for it.
 *
 * When every context is in exact mode (threshold < 0) with FP32 or FP16 storage (all the
 * same), without a neighbour list and with one weight set (w' = w), and no entry asks for
 * gradients, the step runs as three launches over all
 * instances: frame preparation (one warp per frame), the exact pair tiles of every instance
 * in one persistent kernel, and the path CVs (one warp per frame).  The first call with a
 * given set of contexts, sizes and buffers runs the autotuner: for each exact tile shape
 * (16 x 32, 32 x 16, 8 x 64 frames x landmarks; or the one PCV_OPT_EXACT_TILE sets on
 * ctxs[0]) it lists the instances' tiles and times persistent grids of 1, 2, 3, 4 and 8
 * CTAs per SM and one CTA per tile, keeps the fastest shape and grid (pcv_group_tuning),
 * and captures the three launches in a CUDA graph on a stream the first context owns; later
 * calls with the same contexts, sizes, buffers, lambdas and shape option replay the graph.  Otherwise the batches are evaluated one after
 * another with pcv_evaluate.  Errors: PCV_EINVAL / PCV_ESTATE as pcv_evaluate, reported on
 * ctxs[0] (pcv_last_error(ctxs[0])); device-side failures are reported by pcv_sync of the
 * context concerned.  The paper evaluates one structure per call; this is the batched
 * form of its per-step evaluation. */
typedef struct pcv_batch_io {
  int F;
  const void* frames;
  double* s;
  double* z;
  void* dsdx;
  void* dzdx;
  double* msd;
  uint8_t* refreshed;
} pcv_batch_io;
PCV_API pcv_status pcv_evaluate_group(pcv_ctx* const* ctxs, int n, const pcv_batch_io* io, void* stream);
/* What the group launch's autotuner chose for the groups whose first context is ctx: the
 * exact tile (frames x landmarks) and the persistent grid's CTAs, from the last call that
 * tuned (zeros before any).  Errors: PCV_EINVAL for a NULL pointer. */
PCV_API pcv_status pcv_group_tuning(const pcv_ctx* ctx, int* tile_frames, int* tile_landmarks, int* blocks);

/* Landmark shards (one GPU per shard, or several contexts on one GPU).
 *
 * Eqs. 5-6 are a log-sum-exp over the landmarks, so path CVs computed by contexts that
 * each hold a subset of the landmarks (with the landmarks' global properties q_i) combine
 * exactly into the whole-path values: with w_r = exp(-lambda (z_r - z)) over shards r,
 *   z = -(1/lambda) ln sum_r exp(-lambda z_r),  s = sum_r w_r s_r,  dz = sum_r w_r dz_r,
 *   ds = sum_r w_r (ds_r - lambda (s_r - s) dz_r).
 * The combine is one MIN reduction of z_r over the shards (zmin, F values) and one SUM
 * reduction of packed terms:
 *   pcv_shard_pack:   shard values -> scalars (F x 2 doubles) and, when gradients are
 *                     given, elements (F x N x 3 x 3 doubles);
 *   (sum scalars and elements over the shards: an all-reduce, or a host/device sum)
 *   pcv_shard_unpack: summed terms -> s, z (F doubles) and dsdx, dzdx (F x N x 3).
 * precision selects the gradient type: double for PCV_FP64, float otherwise.  dsdx and
 * dzdx are both given or both NULL (then elements may be NULL).  zmin[f] must be <= z_r[f]
 * for every shard (the MIN over shards is exact and keeps every exp <= 1).
 * Device versions: all pointers are device memory, work is enqueued on `stream` (a
 * cudaStream_t, NULL = default stream), and the output of pack may alias nothing of its
 * input.  Host versions: all pointers are host memory; no GPU is needed.
 * Returns PCV_EINVAL on F < 0, N < 1, lambda <= 0 or missing arrays, PCV_ECUDA when the
 * launch fails.  The paper shards landmarks over MPI ranks in its implementation; this is
 * the same reduction written for exact reassembly. */
PCV_API pcv_status pcv_shard_pack(int precision, int F, int N, double lambda, const double* zmin, const double* s,
                                  const double* z, const void* dsdx, const void* dzdx, double* scalars,
                                  double* elements, void* stream);
PCV_API pcv_status pcv_shard_unpack(int precision, int F, int N, double lambda, const double* zmin,
                                    const double* scalars, const double* elements, double* s, double* z, void* dsdx,
                                    void* dzdx, void* stream);
PCV_API pcv_status pcv_shard_pack_host(int precision, int F, int N, double lambda, const double* zmin,
                                       const double* s, const double* z, const void* dsdx, const void* dzdx,
                                       double* scalars, double* elements);
PCV_API pcv_status pcv_shard_unpack_host(int precision, int F, int N, double lambda, const double* zmin,
                                         const double* scalars, const double* elements, double* s, double* z,
                                         void* dsdx, void* dzdx);

/* Exact-mode path CVs for callers that cannot allocate device memory.
 *
 * The paper has no counterpart; this is a deployment aid.  Some callers cannot call
 * cudaMalloc: an MD engine that hands out all device memory from its own pool, or code
 * where a device allocation would stall or break the caller's timing.  This call needs no
 * context and allocates nothing.  Its intermediates live in one fixed device array of
 * PCV_NOALLOC_SCRATCH_BYTES that every GPU loading the library holds until the process
 * exits.
 *
 * It computes the same s, z and MSDs as pcv_evaluate in exact mode with uniform weights
 * and FP32 storage (Algorithm 1 for every frame; no close structure, no gradients):
 *   frames     device, F*N*3 floats, uncentred;
 *   landmarks  device, M*N*3 floats, uncentred (centred here, in FP64, then stored FP32);
 *   q          device, M doubles, or NULL for q_i = i (1-based);
 *   lambda     > 0, nm^-2;
 *   s, z       device, F doubles each; msd device, F*M doubles, or NULL;
 *   cuda_stream  the stream to run on (NULL = legacy default stream), on the current device;
 *   err, err_len  optional host buffer that receives a one-line message on failure.
 * Limits and behaviour:
 *   - the problem must fit the fixed scratch: about 12*M*N + 4*F*M + 72*F + 20*M bytes
 *     (plus alignment) <= PCV_NOALLOC_SCRATCH_BYTES; larger problems return PCV_EINVAL
 *     with a message, before any GPU work;
 *   - the first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) and keeps it for later calls;
 *   - every call shares the one array, which keeps the previous call's contents: calls that
 *     overlap on the GPU (different streams, threads or processes on the same device)
 *     race and must be serialised by the caller;
 *   - the call waits for its own stream and reports PCV_ENOCONV if an eigen-solve hit its
 *     iteration cap; other errors: PCV_EINVAL, PCV_ECUDA;
 *   - the coordinates are not checked for NaN or infinity (pcv_set_landmarks checks its
 *     landmarks; here they arrive in device memory): non-finite inputs give non-finite or
 *     meaningless outputs, with no error status. */
#define PCV_NOALLOC_SCRATCH_BYTES (16u << 20)
PCV_API pcv_status pcv_evaluate_exact_noalloc(int F, int M, int N, const float* frames, const float* landmarks,
                                              const double* q, double lambda, double* s, double* z, double* msd,
                                              void* cuda_stream, char* err, size_t err_len);

/* Gaussian-hill metadynamics on the path CVs (Eq. vbias, Section 2): the consumer of s, z
 * and their derivatives that turns them into a bias potential and a bias force.
 *
 * A hill of height `height` and widths sigma_s, sigma_z (in s and z units) is deposited at
 * (s_t, z_t) at the steps t' = tau_G, 2 tau_G, ... (tau_G = `stride`; steps are numbered
 * from 0, so the first hill lands at step tau_G).  The bias of a step sums the hills of the
 * steps before it:
 *   V_t = sum_k height exp(-(s_t - s_k)^2 / (2 sigma_s^2) - (z_t - z_k)^2 / (2 sigma_z^2)),
 * and its force is F_t = -dV_t/dx = -(dV/ds ds/dx + dV/dz dz/dx).  Steps are counted from
 * creation (or pcv_metad_set_hills) across calls; each call evaluates F consecutive steps.
 * The hills live in device memory of the object (capacity max_hills, fixed at creation).
 * The Gaussians are evaluated in FP32 from FP64 differences (relative error ~1e-6).
 *
 * pcv_metad_create: device, stream (cudaStream_t, NULL = legacy default), height (finite;
 *   negative gives a well), sigma_s, sigma_z > 0, stride >= 1, max_hills >= 1.  Errors:
 *   PCV_EINVAL, PCV_ECUDA, PCV_ENOMEM.
 * pcv_metad_apply: s, z device, F doubles (e.g. from pcv_evaluate); dsdx, dzdx device,
 *   F*N*3 (double in PCV_FP64 `precision`, else float), may be NULL when force is NULL;
 *   bias device, F doubles (out); force device, F*N*3 of the same type (out) or NULL.
 *   Asynchronous on the object's stream.  Errors: PCV_EINVAL (sizes, NULL inputs, hill
 *   capacity exceeded -- checked before any work), PCV_ECUDA.
 * pcv_metad_get_hills: copies the n_hills hills (s_k, z_k) to host memory (hills may be
 *   NULL to query the count) and the step count; synchronises the stream.
 * pcv_metad_set_hills: replaces the hills (host memory, n_hills pairs) and the step count
 *   (restart).  Synchronises the stream.
 * The paper accumulates the hills on a grid to bound the cost of long runs; the GPU sums
 * them directly (frames x hills, one warp per frame). */
typedef struct pcv_metad pcv_metad;
PCV_API pcv_status pcv_metad_create(pcv_metad** out, int device, void* cuda_stream, double height, double sigma_s,
                                    double sigma_z, int stride, int max_hills);
PCV_API pcv_status pcv_metad_destroy(pcv_metad* m);
PCV_API pcv_status pcv_metad_set_stream(pcv_metad* m, void* cuda_stream);
PCV_API pcv_status pcv_metad_apply(pcv_metad* m, int precision, int F, int N, const double* s, const double* z,
                                   const void* dsdx, const void* dzdx, double* bias, void* force);
PCV_API pcv_status pcv_metad_get_hills(pcv_metad* m, double* hills, int cap, int* n_hills, int64_t* steps);
PCV_API pcv_status pcv_metad_set_hills(pcv_metad* m, const double* hills, int n_hills, int64_t steps);
PCV_API const char* pcv_metad_last_error(const pcv_metad* m);

/* One-line description of the last error on ctx (never NULL). */
PCV_API const char* pcv_last_error(const pcv_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* PCV_H */

// pcv_internal.h -- host-side launcher interface between the C-ABI layer (pcv_api.cu)
// and the kernel translation units (k_pair.cu, k_aux.cu).  Not part of the public ABI.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace pcv {

enum Prec { P_F64 = 0, P_F32 = 1, P_F16 = 2 };

// counts kernel launches of the calling host thread (defined in pcv_api.cu)
void note_launch(int n = 1);

// status bits written to the context's device status word
constexpr unsigned STATUS_NOCONV = 1, STATUS_TIMEOUT = 2u;

// Landmark set resident on the device (written by pcv_set_landmarks).
struct LandmarkDev {
  int M = 0, N = 0;
  const void* coords = nullptr;  // M*N*3, centred, storage type of the mode
  const double* G = nullptr;     // M: sum_j wk_j |a_j|^2 in kernel units (see below)
  const double* A = nullptr;     // M*6: sum_j w_j a_j a_j^T (true weights, xx xy xz yy yz zz)
  const float* A32 = nullptr;    // the same in FP32
  const double* q = nullptr;     // M: property q_i
  const float* q32 = nullptr;    // M: the same in FP32
  const float* w = nullptr;      // N: true weights (normalised), or nullptr when uniform
  const double* w64 = nullptr;   // N: the same weights in FP64, or nullptr when uniform
  double dscale = 1.0;           // kernel units -> true: 1/N for uniform weights, else 1
  const float* off = nullptr;    // FP16 storage: M*ceil(N/16)*3 block offsets (else nullptr)
  // alignment weights w' (normalised; they set the centres), or nullptr when w' = w
  const float* wa = nullptr;
  const double* wa64 = nullptr;
  // per-context solver limits, carried with the landmark view to the launches: the Newton
  // iteration cap of the exact pair kernels' eigen-solves, and the clock budget of each
  // bounded wait in the tensor-core kernels (cycles)
  int newton_cap = 60;
  int exact_tile = 0;  // exact tile shape: 0 the default, k > 0 kExactShape[k - 1]
  long long wait_cycles = 4000000000LL;
  // chunks of 16 deviation components the tensor-core MSD kernel sums in tensor memory
  // before folding them into its FP32 totals
  int mma_group = 4;
};
// FP16 storage keeps, per landmark and block of 16 consecutive atoms, an FP32 offset (the
// block's mean centred coordinate) and the FP16 residuals: coordinate = offset + residual
// (see lm_coord).  Residuals span a block (~1 nm), not the structure, so the rounding error
// stays far below what a single centroid shift would give for large structures.
// "Kernel units": with uniform weights the kernels sum unweighted products and the
// results are scaled by dscale = 1/N in FP64 at the end; with explicit weights the
// weights are applied inside the sums and dscale = 1.

// Per-frame quantities from frame_prep: centre (as float for the FP32 path, double for
// FP64 mode) and G_x = sum_j wk_j |x_j - c|^2 of the values the pair kernels stage.
struct FrameInfo {
  float4* c32 = nullptr;   // F: (cx, cy, cz, 0) FP32 modes
  double4* c64 = nullptr;  // F: FP64 mode centres
  double* G = nullptr;     // F
};

// A reference structure for frame-vs-structure alignment: either frame `index` of the
// batch or (index < 0) the stored close structure.
struct RefDesc {
  const void* coords = nullptr;  // N*3, frame type
  float4 c32;
  double4 c64;
  double G = 0.0;
};

// results of frame-vs-structure alignments
struct AlignOut {
  double* D = nullptr;   // D(x_t, ref) in true units
  double4* q = nullptr;  // quaternion of R_{x ref}: rotation fitting ref onto x_t
  uint8_t* flag = nullptr;  // bit0: D > eps, bit1: ambiguous (needs FP64 re-check)
};

// ---- k_aux.cu ----
void launch_frame_prep(Prec p, int F, const void* frames, const LandmarkDev& L, FrameInfo fi,
                       cudaStream_t st);
// band: for t in [max(t_lo,1), t_hi) and k = 1..W with t-k >= 0: D(x_t, x_{t-k}) -> out[t*W + k-1]
void launch_align_band(Prec p, int F, int W, int t_lo, int t_hi, const void* frames, const LandmarkDev& L,
                       FrameInfo fi, double eps, AlignOut out, int* recheck_list, int* recheck_count,
                       cudaStream_t st);
// chunk: for t in [t0, t1): D(x_t, ref) -> out[t]; ref_index >= 0 is a frame of the batch.
// *stop (device int, t1 on entry: launch_chunk_round_init) ends at the first frame that
// definitely exceeds eps; frames past it may be left unaligned.
void launch_align_chunk(Prec p, int t0, int t1, const void* frames, const LandmarkDev& L,
                        FrameInfo fi, int ref_index, const RefDesc& prior, double eps,
                        AlignOut out, int* recheck_list, int* recheck_count, int* stop, cudaStream_t st);
// FP64 re-check of the ambiguous alignments listed in `list` (entries encode slot kind).
// Scratch: the blocks' partial sums of the shared entries and their completion counts
// (recheck_scratch_bytes(); the counts zero on first use, and every launch leaves them zero).
struct RecheckScratch {
  double* part;
  int* done;
};
size_t recheck_scratch_bytes();
RecheckScratch recheck_scratch_at(void* base);  // views of a buffer of that size
void launch_recheck(Prec p, int max_entries, const int* list, const int* count, int W,
                    const void* frames, const LandmarkDev& L, const float4* c32, const RefDesc& prior,
                    int chunk_ref, double eps, AlignOut band, AlignOut chunk, unsigned long long* n_rechecks,
                    RecheckScratch scr, cudaStream_t st);
// recheck list entries: (slot << 1) | kind, kind 0 = band slot t*W + k-1, 1 = chunk slot t
// accurate quaternions of R_xy for the approximate frames (FP32 modes; FP64 mode keeps the
// FP64 band / chunk quaternions)
struct FrameRec;
void launch_xy_refine(Prec p, int F, const void* frames, const LandmarkDev& L, FrameInfo fi, const RefDesc& prior,
                      FrameRec rec, cudaStream_t st);
// first t in [t0, min(t1, *stop + 1)) with chunk flag bit0 set -> *first (t1 on entry:
// launch_chunk_round_init; stop may be null)
void launch_first_exceed(int t0, int t1, const uint8_t* flag, const int* stop, int* first, cudaStream_t st);
// start of a speculative chunk [.., t1): recheck count 0, stop and first t1 (one launch)
void launch_chunk_round_init(int* recheck_count, int* stop, int* first, int t1, cudaStream_t st);

// per-frame decision records
struct FrameRec {
  uint8_t* flag = nullptr;  // 0 approx, 1 refresh, 2 initial
  int* ref = nullptr;       // frame index of the close structure used (-1: stored y)
  double* dxy = nullptr;    // D(x_t, y) that decided the frame (-1 at initial)
  double4* qxy = nullptr;   // quaternion of R_{x y} (approximate frames)
};
struct ScanResult {
  int t_stop;  // first frame the band could not decide (F if none)
  int ref;     // close-structure frame index in force at t_stop
  int nref;    // reassignments among the decided frames
  int pad;
};
// decide frames [t0, F) from the band with the state `o_init` (offset of frame t0-1 from
// its close structure, 0..W); writes records and *res (device)
void launch_band_scan(int F, int W, int t0, int o_init, const AlignOut band, FrameRec rec,
                      ScanResult* res, cudaStream_t st);
// frames [t0, t_end) approximate w.r.t. ref (chunk results), and frame t_end (if < t1) a
// refresh
void launch_chunk_records(int t0, int t_end, int t1, int ref, const AlignOut chunk, FrameRec rec,
                          cudaStream_t st);
// the same with the first exceeding frame read on the device (t_end_dev; t1 = none)
void launch_chunk_records_dev(int t0, const int* t_end_dev, int t1, int ref, const AlignOut chunk, FrameRec rec,
                              cudaStream_t st);
void launch_initial_record(FrameRec rec, cudaStream_t st);

// compaction of refresh / approximate frames (device lists, counts returned on device)
void launch_compact(int F, const FrameRec rec, int* refresh_list, int* refresh_count,
                    int* seg_of_frame, int* approx_list, int* approx_count, int* approx_seg,
                    int prior_seg, cudaStream_t st);

// softmax finalisation: s, z per frame from the F x M distances (float in FP32 modes,
// double in FP64 mode); mstat[f] = (m, l) with m = min_i D_i, l = sum_i exp(-lambda(D_i-m));
// msd_out (optional) receives the distances as doubles; want_p overwrites D with the
// weights p_i = exp(-lambda (D_i - m)) / l used by the adjoint
void launch_finalize(Prec p, int F, int M, void* D, const double* q, const float* q32, double lambda, double* s,
                     double* z, float* mstat, double* mstat64, double* msd_out, bool want_p, cudaStream_t st);

// adjoint (k_adjoint.cu): beta = sum_i gamma_i Rot_fi a_i written into gs/gz, then the
// per-frame finish.  P holds the softmax weights p (launch_finalize with want_p).  Rpair
// (exact mode): F*M*9 rotations; otherwise Bseg[seg_of_frame[f]*M + i].  seg_form: frames
// share their segment's rotations (close structure, few segments).  part: workspace of
// beta_pair_split(p, F, M, N) * F * N * 6 elements of the storage type (double in FP64
// mode), used when the split is above 1 (the frames give less than a wave of CTAs and the
// landmarks are divided into ranges whose partial sums are added by a second kernel); null:
// no split.
int beta_pair_split(Prec p, int F, int M, int N);
void launch_adjoint_beta(Prec p, int F, const LandmarkDev& L, const void* P, const double* s, double lambda,
                         const void* Rpair, const void* Bseg, const int* seg_of_frame, bool seg_form, void* gs,
                         void* gz, void* part, cudaStream_t st);
// rec.flag == nullptr: exact mode (no rotation term)
// Gsum (Gamma^s_f, Gamma^z_f) and S6 (segment moments of segments from seg_base) are
// optional inputs of the FP32 finish; null: computed from P and from Bseg, A32
void launch_adjoint_finish(Prec p, int F, const void* frames, const LandmarkDev& L, FrameInfo fi, const void* P,
                           const double* s, double lambda, const void* Bseg, const int* seg_of_frame,
                           const FrameRec rec, const RefDesc& prior, void* gs, void* gz, cudaStream_t st,
                           const float* Gsum = nullptr, const float* S6 = nullptr, int seg_base = 0);
// S_i = R_{a_i y} A_i R_{a_i y}^T (6 floats) of segments [seg_base, seg_base + nseg)
void launch_seg_moments(int seg_base, int nseg, const LandmarkDev& L, const float* Bseg, float* S6, cudaStream_t st);
void launch_combine_grad(Prec p, int F, int N3, const double* g_s, const double* g_z,
                         const void* gs, const void* gz, void* out, cudaStream_t st);
void launch_fill_u8(uint8_t* p, uint8_t v, size_t n, cudaStream_t st);
// device-to-device copy by a kernel (not a copy engine)
void launch_dev_copy(void* dst, const void* src, size_t bytes, cudaStream_t st);
void launch_set_int(int* p, int v, cudaStream_t st);

// ---- k_pair.cu ----
// device scratch handed to a launcher: ptr and its size in bytes
struct ScratchView {
  void* ptr;
  size_t bytes;
};
// exact pairs: rows r in [0, rows) are frames row_frame[r] (or r if null); D -> D[f*M+i]
// (float in FP32 modes, double in FP64 mode); R (optional) -> Rout[(r*M + i)*9].  With
// scratch of exact_split_bytes(rows, M, exact_split_count(rows, M, N)) bytes, batches whose
// tiles would not fill two waves of the GPU split the atoms over several CTAs per tile.
int exact_split_count(int rows, int M, int N);  // 1: no split
size_t exact_split_bytes(int rows, int M, int nsplit);
void launch_exact_pairs(Prec p, int rows, const int* row_frame, const int* rows_dev, const void* frames,
                        const LandmarkDev& L, FrameInfo fi, void* D, void* Rout, unsigned* status,
                        cudaStream_t st, const ScratchView* scr = nullptr);
// approximate pairs (form A): list entries k < *count: frame approx_list[k] of segment
// approx_seg[k]; rotations Bseg[seg*M + i] (9 floats each), R_{x y} from rec.qxy
void launch_approx_pairs(Prec p, int max_rows, const int* approx_list, const int* approx_seg,
                         const int* count, const void* frames, const LandmarkDev& L, FrameInfo fi,
                         const double4* qxy, const void* Bseg, void* D, cudaStream_t st);

// ---------------------------------------------------------------------------------------
// group evaluation (many instances, exact mode, FP32 / FP16 storage): one descriptor per
// instance in device memory; work items are global frames or (instance, frame tile,
// landmark tile) triples
struct GroupInst {
  const float* frames;  // F x N x 3
  const void* lm;       // landmarks (float or __half storage), lmoff the FP16 block offsets
  const float* lmoff;
  const double* lG;
  const float* w;       // weights or nullptr (uniform)
  double dscale;
  const float* q32;
  float lambda;
  int M, N, F, fbase;   // fbase: global index of the instance's first frame
  float4* c32;          // workspace of the instance's context
  double* fG;
  float* D;
  float* mstat;
  double* s;            // outputs
  double* z;
  double* msd;          // optional
  unsigned* status;
};
struct GroupTile {
  int inst, row0, i0, pad;
};
// shapes of the exact tile (frames x landmarks, 128 threads of 2 x 2 pairs; k_pair.cu):
// index 0 is the default; the group launch's autotuner times all of them
struct ExactShape {
  int tf, tm;
};
constexpr int EXACT_SHAPES = 3;
constexpr ExactShape kExactShape[EXACT_SHAPES] = {{16, 32}, {32, 16}, {8, 64}};
void launch_frame_prep_group(const GroupInst* I, int n, int Ftot, cudaStream_t st);
void launch_finalize_group(const GroupInst* I, int n, int Ftot, cudaStream_t st);
// persistent grid of `blocks` CTAs over the tiles; fp16: landmarks in FP16 storage
void launch_exact_group(bool fp16, int shape, const GroupInst* I, const GroupTile* tiles, int ntiles, int blocks,
                        cudaStream_t st);

// ---------------------------------------------------------------------------------------
// landmark-parallel kernels for up to STREAM_FRAMES frames per call (k_stream.cu; FP32
// and FP16-storage modes; one CTA per landmark, the landmark staged in shared memory)
constexpr int STREAM_FRAMES = 4;
bool stream_fits(Prec p, int N);  // the staged landmark fits in shared memory
void launch_exact_stream(Prec p, int rows, const int* row_frame, const void* frames, const LandmarkDev& L,
                         FrameInfo fi, void* D, void* Rout, unsigned* status, cudaStream_t st);
void launch_approx_stream(Prec p, int max_rows, const int* approx_list, const int* approx_seg, const int* count,
                          const void* frames, const LandmarkDev& L, FrameInfo fi, const double4* qxy, const void* Bseg,
                          void* D, cudaStream_t st);

// ---------------------------------------------------------------------------------------
// materialised-operand path (k_tile.cu; FP32 and FP16-storage modes, uniform weights).
// Rows padded to round_up16(N) atoms; segment slots s = seg - seg_base in [0, ns).
inline int round_up16(int n) { return (n + 15) & ~15; }
size_t tile_bytes_frames(int napp, int N);
size_t tile_bytes_landmarks(int nseg, int M, int N);
size_t tile_bytes_gamma(int F, int M);
// d_i = R_{a_i y} a_i - y' per segment (Bm), |d_i|^2 (Nb, ns*M floats), y' (Yc, ns*3N floats);
// y is the prior structure for segment 0, else frame refresh_list[seg - 1]
void launch_materialize_landmarks(Prec p, int s0, int ns, const LandmarkDev& L, const float* Bseg, const void* frames,
                                  FrameInfo fi, const int* refresh_list, const RefDesc& prior, float* Bm, float* Nb,
                                  float* Yc, cudaStream_t st);
// dx_k = R_xy^T (x - c) - y' for approximate frames k < *acount (Xr), |dx_k|^2 (Nx); after
// launch_materialize_landmarks.  refine_ref (the frames' close-structure index, FrameRec.ref)
// non-null: R_xy is formed here from the frame and its close structure (prior: the stored
// one) and its quaternion written to qxy, in place of launch_xy_refine; null: qxy is read.
void launch_materialize_frames(int napp, const int* acount, const int* alist, const int* aseg, int seg_base,
                               const LandmarkDev& L, const void* frames, FrameInfo fi, double4* qxy,
                               const float* Yc, float* Xr, float* Nx, const int* refine_ref, const RefDesc& prior,
                               cudaStream_t st);
// gamma^s, gamma^z rows (round_up16(M) entries each, tile_bytes_gamma bytes per kind) from
// the softmax weights P, and Gamma^s_f, Gamma^z_f (Gsum, 2F floats)
void launch_gamma(int F, const LandmarkDev& L, const float* P, const double* s, double lambda, float* GS, float* GZ,
                  float* Gsum, cudaStream_t st);
void launch_approx_pairs_tile(int napp, const int* alist, const int* aseg, const int* acount, int seg_base,
                              const LandmarkDev& L, const float* Xr, const float* Bm, const float* Nx, const float* Nb,
                              float* D, cudaStream_t st);
void launch_adjoint_beta_tile(int F, const LandmarkDev& L, int seg_base, const float* GS, const float* GZ,
                              const float* Bm, const float* Gsum, const float* Yc, const int* seg_of_frame, float* gs,
                              float* gz, cudaStream_t st);

// ---------------------------------------------------------------------------------------
// approximate MSDs on the tensor cores (k_xmma.cu; FP32 and FP16-storage modes, uniform
// weights, materialised deviations): packed FP16 h + l operands, kind::f16 MMAs.
struct XmmaShape {
  int nck = 0, BN = 0, NT = 0;   // chunks of 16 components, landmark tile width, landmark tiles
  size_t a_bytes_per_tile = 0;   // packed frames, per tile of 128 approximate frames
  size_t b_bytes_per_seg = 0;    // packed landmarks, per segment
};
XmmaShape xmma_shape(int M, int N);
// a tile of up to 128 approximate frames of one segment: rows [k0, k1) of the approximate
// list, segment slot `slot`
struct XTile {
  int slot, k0, k1;
};
int xmma_max_tiles(int napp, int nseg);
size_t xmma_a_bytes(const XmmaShape& sh, int napp, int nseg);
// the per-segment tile list (*ntiles entries, at most xmma_max_tiles), each slot's first
// row in the approximate list and first tile
void launch_xmma_tiles(const int* acount, const int* aseg, int seg_base, int nseg, int* seg_first, int* tile_start,
                       XTile* tiles, int* ntiles, cudaStream_t st);
struct MmaShape;
// d_i = R_{a_i y} a_i - y' of segment slots [0, ns) (segments s0 + slot), computed once and
// packed for the approximate MSDs (Bx, with |d_i|^2 in Nb, ns*M floats) and, when ms is not
// null, for the segment adjoint (Ba); y' in Yc (ns*3N floats)
void launch_pack_deviations(Prec p, int s0, int ns, const LandmarkDev& L, const XmmaShape& xs, const MmaShape* ms,
                            const float* Bseg, const void* frames, FrameInfo fi, const int* refresh_list,
                            const RefDesc& prior, uint8_t* Bx, float* Nb, uint8_t* Ba, float* Yc, cudaStream_t st);
// dx_k = R_xy^T (x - c) - y' of approximate frames k < *acount packed into Ap, |dx_k|^2 (Nx);
// after launch_pack_deviations (y') and with the frames' R_xy in qxy
void launch_pack_frames(int napp, const int* acount, const int* alist, const int* aseg, int seg_base,
                        const LandmarkDev& L, const void* frames, FrameInfo fi, const double4* qxy, const float* Yc,
                        const int* seg_first, const int* tile_start, uint8_t* Ap, float* Nx, cudaStream_t st);
// D~ of every approximate frame and landmark from the packed operands (STATUS_TIMEOUT in
// *status if a bounded wait expired)
void launch_approx_cross_mma(int napp, int nseg, const int* alist, const XTile* tiles, const int* ntiles,
                             const LandmarkDev& L, const XmmaShape& sh, const uint8_t* Ap, const uint8_t* Bp,
                             const float* Nx, const float* Nb, float* D, unsigned* status, cudaStream_t st);

// ---------------------------------------------------------------------------------------
// tensor-core segment adjoint (k_mma.cu; FP32 and FP16-storage modes, uniform weights)
struct MmaShape {
  int Kp = 0, Fp = 0, BN = 0, NT = 0;  // landmarks / frames padded, column tile, column tiles
  size_t a_bytes = 0;                  // gamma operand (hi and lo, s and z) for Fp frames
  size_t b_bytes_per_seg = 0;          // deviation operand per segment
  size_t y_bytes_per_seg = 0;          // centred close structure per segment
  size_t gsum_floats = 0;              // Gamma sums and the gamma rows' inverse scales
};
MmaShape mma_shape(int F, int M, int N);
// gamma operand pre-tiled for the MMA, and Gamma^s_f, Gamma^z_f (Gsum, 2F floats)
void launch_gamma_split(int F, const LandmarkDev& L, const MmaShape& sh, const float* P, const double* s,
                        double lambda, float* A, float* Gsum, cudaStream_t st);
// beta^s, beta^z for all F frames into gs, gz (STATUS_TIMEOUT in *status if a wait expired)
void launch_adjoint_beta_mma(int F, const LandmarkDev& L, const MmaShape& sh, int seg_base, const float* A,
                             const float* Gsum, const float* B, const float* Yc, const int* seg_of_frame, float* gs,
                             float* gz, unsigned* status, cudaStream_t st);

// ---------------------------------------------------------------------------------------
// neighbour list (k_nl.cu): frame schedule of one call, list table NLtab (slot 0: the list
// carried over from the previous call; slot k+1: the list chosen at the k-th update frame)
struct NlLists {
  int* slot = nullptr;       // F: list slot used by each frame (its own at update frames)
  uint8_t* upd = nullptr;    // F: 1 at update frames
  int* ulist = nullptr;      // update frames in time order
  int* uapp_list = nullptr;  // update frames evaluated approximately (close mode) and
  int* uapp_seg = nullptr;   //   their close-structure segment
  int* nlist = nullptr;      // frames between updates
  int* counts = nullptr;     // device ints: [0] updates, [1] approximate updates, [2] between
};
// update frames: (step0 + t) % L == 0, t == 0 without a carried list, flag[t] != 0 (close
// mode reassignments; flag may be null)
void launch_nl_schedule(int F, long long step0, int L, bool have_list, const uint8_t* flag, const int* segof,
                        const NlLists& nl, cudaStream_t st);
// list of every update frame from its row of D (all M distances), into NLtab slots 1..
void launch_nl_select(Prec p, int max_upd, const NlLists& nl, int M, int Mnl, const void* D, int* NLtab,
                      cudaStream_t st);
// distances of the frames between updates to their listed landmarks (+inf elsewhere in the
// row): exact (rotations -> Rnl[(f*Mnl + r)*9] when Rnl is given) or approximate
void launch_nl_exact(Prec p, int max_rows, const NlLists& nl, const int* NLtab, int Mnl, const void* frames,
                     const LandmarkDev& L, FrameInfo fi, void* D, void* Rnl, unsigned* status, cudaStream_t st);
void launch_nl_approx(Prec p, int max_rows, const NlLists& nl, const int* NLtab, int Mnl, const void* frames,
                      const LandmarkDev& L, FrameInfo fi, const double4* qxy, const void* Bseg, const int* segof,
                      void* D, cudaStream_t st);
// beta of the adjoint over each frame's landmarks; rotations from Bseg[segof[f]] (close
// mode) or Rupd rows (update frames) and Rnl (between updates) in exact mode
void launch_nl_beta(Prec p, int F, const NlLists& nl, const int* NLtab, int Mnl, const LandmarkDev& L, const void* P,
                    const double* s, double lambda, const void* Rupd, const void* Rnl, const void* Bseg,
                    const int* segof, void* gs, void* gz, cudaStream_t st);
// the list of this call's last update frame -> keep (unchanged without an update)
void launch_nl_carry(const NlLists& nl, const int* NLtab, int Mnl, int* keep, cudaStream_t st);

// Tiles of frames between updates for the tiled FP32 / FP16 kernels: `rows` (<= NL_TILE_F)
// consecutive entries of nlist from position p0, all on the list `slot`.  nl_tiles writes
// them and their number to counts[3]; at most (frames between) / NL_TILE_F + updates + 2.
struct NlTile {
  int p0, rows, slot, pad;
};
constexpr int NL_TILE_F = 16;
void launch_nl_tiles(int F, const NlLists& nl, NlTile* tiles, cudaStream_t st);
// +inf over the MSD rows of the frames between updates (before their listed entries are written)
void launch_nl_fill_inf(Prec p, int max_between, const NlLists& nl, int M, void* D, cudaStream_t st);
// exact MSDs of the frames between updates to their listed landmarks, tiled (FP32 / FP16
// storage; rotations -> Rnl[(f*Mnl + column)*9] when Rnl is given) (k_pair.cu)
void launch_nl_exact_tiles(Prec p, int max_tiles, const NlLists& nl, const NlTile* tiles, const int* NLtab, int Mnl,
                           const void* frames, const LandmarkDev& L, FrameInfo fi, void* D, void* Rnl,
                           unsigned* status, cudaStream_t st);
// exact-mode beta of the adjoint, tiled (FP32 / FP16 storage) (k_adjoint.cu): the update
// frames over every landmark (rotations Rupd, row = position in ulist; the landmarks split
// into nl_beta_split ranges whose partial sums go to part, nl_beta_split * max_upd * N * 6
// floats), then the frames in between over their lists (rotations Rnl)
int nl_beta_split(int max_upd, int M, int N);
// (close mode: Bseg and segof given, rotations R_{a_i y} of each frame's segment)
void launch_nl_beta_tiles(Prec p, int max_upd, int max_tiles, const NlLists& nl, const NlTile* tiles, const int* NLtab,
                          int Mnl, const LandmarkDev& L, const void* P, const double* s, double lambda,
                          const void* Rupd, const void* Rnl, const void* Bseg, const int* segof, void* gs, void* gz,
                          float* part, cudaStream_t st);
// close mode, FP32 / FP16 storage: Eq. (close_dist) for every landmark of the approximate
// update frames (uapp_list) and for the listed landmarks of the tiles (k_pair.cu)
void launch_nl_approx_tiles(Prec p, int max_uapp, int max_tiles, const NlLists& nl, const NlTile* tiles,
                            const int* NLtab, int Mnl, const void* frames, const LandmarkDev& L, FrameInfo fi,
                            const double4* qxy, const void* Bseg, const int* segof, void* D, cudaStream_t st);

}  // namespace pcv

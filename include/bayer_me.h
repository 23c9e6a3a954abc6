/*
 * bayer_me.h -- C ABI of the B300 (sm_103a) Bayer-domain block motion
 * estimation and motion-vector feature propagation library (libbayer_me.so).
 *
 * Method: arXiv 2508.05990, "Efficient Bayer-Domain Video Computer Vision with
 * Fast Motion Estimation and Learned Perception Residual".
 *   Sec. 2.2 "Definition":   MV = ME(F_R, F_C)
 *   Sec. 3.2 "Fast Motion Estimation": block pyramid, coarse-to-fine stages,
 *                            SAD matching criterion, argmin = MV
 *   Sec. 3.3 equation:       z_pred = Warp(z_R, MV)
 *   Sec. 4.1 "CUDA Settings": (2R+1)^2 candidates per block per stage; the MV
 *                            field is h x w; a Batch dimension of frame pairs.
 *
 * Conventions (all entry points)
 *   Frames: uint16 row-major H x W (row pitch in elements), RGGB mosaic with
 *     R at (0, 0), values 0..4095 (12 bit).  Larger values give undefined MVs.
 *   MV sign: the current block at (x, y) matches the reference block at
 *     (x + dx, y + dy).
 *   MV field: h = ceil(H / block) rows x w = ceil(W / block) columns of
 *     bayer_mv_t (8 bytes, row-major), one field per frame pair.
 *   Candidate set of a stage centred on p with radius R (in steps) and step s:
 *     { p + (u*s, v*s) : u, v in [-R, R] }; a candidate whose displaced block
 *     leaves the frame is skipped; partial edge blocks are clipped to the frame.
 *   Tie-break: lexicographic minimum of (sad, |dx|+|dy|, dy, dx).
 *   Phase: EVEN uses even offsets only (same-colour CFA samples); RAW uses all.
 *   |dx|, |dy| of any MV are at most 511.
 *
 * Ownership: every frame, feature, proposal and MV buffer is owned by the
 *   caller and is a DEVICE pointer unless the entry point's name ends in _host.
 *   The handle owns only its workspace.  All device entry points are
 *   asynchronous on the caller's CUDA stream (NULL = legacy default stream);
 *   the caller keeps buffers alive until the stream reaches the call.
 *
 * Errors: argument errors are returned synchronously and launch nothing.
 *   BAYER_ERR_CUDA reports a failed launch or CUDA runtime call; device-side
 *   conditions are read back with bayer_me_sync_status.  One handle per host
 *   thread; the library keeps no global mutable state.
 */
#ifndef BAYER_ME_H
#define BAYER_ME_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bayer_me_s* bayer_me_t;

/* One motion vector record: 8 bytes. */
typedef struct {
  int16_t dx;
  int16_t dy;
  uint32_t sad;
} bayer_mv_t;

typedef enum {
  BAYER_OK = 0,
  BAYER_ERR_INVALID_ARG = 1,
  BAYER_ERR_UNSUPPORTED = 2,
  BAYER_ERR_CUDA = 3,
  BAYER_ERR_OOM = 4,
  BAYER_ERR_TIMEOUT = 5
} bayer_status_t;

enum { BAYER_MODE_FULL = 0, BAYER_MODE_C2F = 1, BAYER_MODE_SEEDED = 2 };
enum { BAYER_PHASE_EVEN = 0, BAYER_PHASE_RAW = 1 };
enum { BAYER_INTERP_NEAREST = 0, BAYER_INTERP_BILINEAR = 1 };
enum { BAYER_LAYOUT_NCHW = 0, BAYER_LAYOUT_NHWC = 1 };

#define BAYER_MAX_LEVELS 4
#define BAYER_MAX_STAGES 4

/* Search parameters for bayer_me_estimate_ex.
 *   mode FULL:   exhaustive search |dx|, |dy| <= range around the zero MV
 *                (EVEN: step 2, RAW: step 1) -- the plain definition of block
 *                matching (Sec. 2.2, "Block Matching-based ME").
 *   mode C2F:    the paper's block pyramid (Sec. 3.2): levels[0..n_levels-1]
 *                block sizes, large to small; every level runs the stages
 *                (stage_radius[k], stage_step[k]) in order, each centred on
 *                the previous stage's best; level 0 starts at the zero MV,
 *                level l > 0 at the MV of the level l-1 block holding the
 *                child's top-left pixel.  Standard setting: levels {64, 32},
 *                stages (8, 8), (4, 4), (2, 1) (FME-settings table).  In EVEN
 *                phase an odd step s becomes s + 1 with radius R*s/(s+1)
 *                (integer division).  The output is the last level's field.
 *   mode SEEDED: per block, confidence < conf_thresh -> FULL search with
 *                `range`; otherwise the proposal (dx, dy) is rounded to the
 *                nearest even integer (half away from zero), clamped to
 *                [-range, range] and to the block's valid displacements, and
 *                one stage R = 2, step 2 (+-4) is searched around it with
 *                |dx|, |dy| <= range.  EVEN phase only.
 * batch pairs are processed in one launch: pair b uses ref + b*ref_batch_stride
 * and cur + b*cur_batch_stride (elements, >= 0; frames may overlap, they are
 * only read) and writes field b of mv_out. */
typedef struct {
  int mode;          /* BAYER_MODE_* */
  int phase;         /* BAYER_PHASE_* */
  int block;         /* FULL, SEEDED: block size, one of 8, 16, 32, 64 */
  int range;         /* FULL, SEEDED: maximum |dx|, |dy| in pixels (EVEN: even) */
  int n_levels;      /* C2F: 1..BAYER_MAX_LEVELS */
  int levels[BAYER_MAX_LEVELS];
  int n_stages;      /* C2F: 1..BAYER_MAX_STAGES */
  int stage_radius[BAYER_MAX_STAGES];
  int stage_step[BAYER_MAX_STAGES];
  float conf_thresh; /* SEEDED: confidence threshold (0.5 by default) */
  int batch;         /* number of frame pairs, >= 1 */
  long long ref_batch_stride; /* elements between reference frames of consecutive pairs */
  long long cur_batch_stride; /* elements between current frames of consecutive pairs */
} bayer_me_params_t;

/* Create a handle bound to CUDA device `device` (makes it current).
 * *out receives the handle.  Returns BAYER_ERR_CUDA if the device cannot be
 * used, BAYER_ERR_OOM if the workspace cannot be allocated. */
bayer_status_t bayer_me_init(bayer_me_t* out, int device);

/* Release the handle and its workspace (synchronises the device first). */
bayer_status_t bayer_me_destroy(bayer_me_t h);

/* Static, NUL-terminated description of a status code. */
const char* bayer_status_string(bayer_status_t s);

/* Exhaustive EVEN-phase block matching of one frame pair (Sec. 2.2, Sec. 3.2
 * "Matching Criterion"): for every block, the SAD of every candidate offset
 * (dx, dy) with even |dx|, |dy| <= range, argmin by the tie-break above.
 *   ref, cur: device frames H x W, pitch W.  block in {8, 16, 32, 64};
 *   W, H even and >= block; range even, 0 <= range <= 510.
 *   mv_out: device array of ceil(H/block) * ceil(W/block) records. */
bayer_status_t bayer_me_estimate(bayer_me_t h, const uint16_t* ref, const uint16_t* cur, int W, int H,
                                 int block, int range, bayer_mv_t* mv_out, void* stream);

/* General form: FULL / C2F / SEEDED, EVEN or RAW, batched pairs, row pitch.
 *   pitch: elements per frame row (>= W).
 *   prop_dxdy: SEEDED only, device float array [batch][h][w][2] (dx, dy);
 *   conf: SEEDED only, device float array [batch][h][w].
 *   mv_out: device array [batch][h][w] for the output level's block size.
 *   fallback_out: optional (SEEDED), device uint8 [batch][h][w], 1 where the
 *     full search was used.
 * Workspace for C2F's intermediate levels is taken from the handle. */
bayer_status_t bayer_me_estimate_ex(bayer_me_t h, const uint16_t* ref, const uint16_t* cur, int W, int H,
                                    int pitch, const bayer_me_params_t* params, const float* prop_dxdy,
                                    const float* conf, bayer_mv_t* mv_out, uint8_t* fallback_out,
                                    void* stream);

/* Motion-vector feature propagation z_pred = Warp(z_R, MV) (Sec. 3.3).
 * Feature cell (fy, fx) takes the MV of block (fy*stride/block, fx*stride/block)
 * and samples z_R at (fy + dy/stride, fx + dx/stride):
 *   NEAREST: offsets dy/stride, dx/stride rounded half away from zero; a copy.
 *   BILINEAR: y0 = floor, wy = fraction (likewise x);
 *     out = (1-wy)*((1-wx)*a + wx*b) + wy*((1-wx)*c + wx*d), each product and
 *     sum rounded to float in this order (no fused multiply-add).
 *   Indices are clamped to the map.
 *   feat: device float32, n maps of C x Hf x Wf (NCHW) or Hf x Wf x C (NHWC),
 *     contiguous; out: same shape, must not overlap feat.
 *   mv: device, n fields of mv_h x mv_w; stride divides block;
 *     mv_h == ceil(Hf*stride/block), mv_w == ceil(Wf*stride/block). */
bayer_status_t bayer_feat_propagate(bayer_me_t h, const float* feat, int n, int C, int Hf, int Wf, int layout,
                                    int interp, const bayer_mv_t* mv, int mv_h, int mv_w, int block, int stride,
                                    float* out, void* stream);

/* The whole per-clip path with HOST buffers (the end-to-end form of
 * Sec. 3.1's inference: ME of each consecutive frame pair (F_{t-1}, F_t),
 * then propagation of that pair's reference features):
 *   frames: host uint16 [n_frames][H][W]; feats: host float32
 *   [n_frames-1][C][Hf][Wf] (NCHW); mv_out: host [n_frames-1][h][w];
 *   feat_out: host float32 like feats.  Full EVEN search with block, range;
 *   interp as in bayer_feat_propagate.  Copies run on the handle's streams,
 *   overlapped with compute across pairs; returns after the last copy
 *   completes.  Page-locked host buffers give full copy bandwidth. */
bayer_status_t bayer_clip_process_host(bayer_me_t h, const uint16_t* frames, int n_frames, int W, int H,
                                       int block, int range, const float* feats, int C, int Hf, int Wf,
                                       int stride, int interp, bayer_mv_t* mv_out, float* feat_out);

/* Read and clear the handle's device status word after synchronising
 * `stream`: BAYER_OK, or the first device-side error raised since the last
 * call (e.g. BAYER_ERR_TIMEOUT from a bounded wait). */
bayer_status_t bayer_me_sync_status(bayer_me_t h, void* stream);

/* Failure-path self-test of the device-side bounded wait (not in the paper).
 * Every tensor-core kernel of this library waits on mbarriers with an
 * iteration limit; when the limit runs out the kernel records
 * BAYER_ERR_TIMEOUT in the handle's status word and finishes instead of
 * hanging.  This entry point runs that wait in a one-CTA kernel on `stream`:
 * with arrive != 0 the barrier's phase completes and the wait succeeds; with
 * arrive == 0 nothing arrives and the wait gives up after `limit` polls
 * (limit >= 1), leaving BAYER_ERR_TIMEOUT for bayer_me_sync_status to return.
 * No fault, trap or unbounded loop is involved either way. */
bayer_status_t bayer_me_selftest_wait(bayer_me_t h, int arrive, unsigned limit, void* stream);

/* Test hook (not in the paper): the next n workspace growths of the handle
 * (C2F levels, learned search, refine activations, host pipeline buffers)
 * fail with BAYER_ERR_OOM without allocating; the call that hits one returns
 * that status and launches nothing, and later calls allocate normally.
 * n = 0 clears the hook.  Lets tests exercise the out-of-memory path. */
bayer_status_t bayer_me_debug_fail_allocs(bayer_me_t h, int n);

/* Roofline probe: throughput of the exact SAD primitive on this device.
 * Runs a register-only loop of `variant` (0 = sad.u32 integer, 1 = float
 * subtract + absolute add, 2 = both interleaved, 3 = packed pixel pairs:
 * min.u16x2 + dp2a, two pixel-candidates per pair) on every SM and returns the
 * pixel-candidates per clock per SM and the SM clock (MHz) seen during the
 * run.  Synchronous. */
bayer_status_t bayer_probe_alu(bayer_me_t h, int variant, double* pc_per_clk_per_sm, double* sm_mhz,
                               int* sm_count);

/* ---------------------------------------------------------------------------
 * Learned-seeded search (not in the paper).  A small CNN proposes an MV and a
 * confidence per 16x16 block; confident blocks are refined by one +-4 stage
 * (R = 2, step 2) around the proposal, the others fall back to the exhaustive
 * +-range search -- the SEEDED mode of bayer_me_estimate_ex with the proposals
 * computed on the device.  The network follows the paper's recipe for its own
 * learned module where one exists: AdamW with a cosine schedule (Sec. 4.1
 * "Training Details") and the BerHu loss (Sec. 3.3).
 *
 * Network, parameters as one flat vector (float32 master, bfloat16 copy, both
 * caller-owned device arrays of BAYER_CNN_NPARAMS elements, the bf16 copy
 * passed as uint16_t):
 *   x0 = 8 channels: the R, G (R row), G (B row), B planes of ref, then of cur,
 *        at half resolution, each sample v / 2048 - 1
 *   x_l = ReLU(conv3x3(x_{l-1}, stride 2, zero pad 1) + b_l), 32 channels,
 *        l = 1..4; weights w_l[co][ci][ky][kx]
 *   z = head 1x1 conv 32 -> 12 + bias; channel 3*(2*sy + sx) + q of L4 cell
 *       (i, k) is quantity q of block (2i + sy, 2k + sx)
 *   dx = range * tanh(z_0), dy = range * tanh(z_1), conf = sigmoid(z_2)
 * Activations are bfloat16, accumulation float32.  Each layer has its natural
 * size ceil(n / 2) of its input's n (the last row or column may read the zero
 * pad), so the depth-to-space output has 2 * ceil(H / 32) block rows; the
 * block grid is its top ceil(H / 16) rows (one fewer where ceil(H / 16) is
 * odd, e.g. H = 720 or 2160).  W must be a multiple of 32; H a multiple of 8
 * for the forward and the learned search (1080 included, whose last block row
 * is 8 rows high), of 32 for the loss (BAYER_ERR_UNSUPPORTED otherwise).
 * Loss (mean over the blocks of the batch): BerHu_4(dx - dx*) +
 * BerHu_4(dy - dy*) - t log(conf) - w_neg (1 - t) log(1 - conf), with
 * BerHu_c(e) = |e| for |e| <= c, else (e^2 + c^2) / (2c); t = 1 where the
 * proposal rounded to the nearest even integer lies within +-4 of the label
 * (dx*, dy*) in both components (then the +-4 refine reaches the label).
 * w_neg > 1 makes a confidence >= 0.5 mean P(t = 1) >= w_neg / (1 + w_neg). */
#define BAYER_CNN_W1 0
#define BAYER_CNN_B1 2304
#define BAYER_CNN_W2 2336
#define BAYER_CNN_B2 11552
#define BAYER_CNN_W3 11584
#define BAYER_CNN_B3 20800
#define BAYER_CNN_W4 20832
#define BAYER_CNN_B4 30048
#define BAYER_CNN_WH 30080
#define BAYER_CNN_BH 30464
#define BAYER_CNN_NPARAMS 30476

/* Network forward on `batch` frame pairs (strides as in bayer_me_params_t):
 * prop_dxdy [batch][h][W/16][2] and conf [batch][h][W/16], h = ceil(H / 16)
 * (device float32).  Activations use the handle's workspace. */
bayer_status_t bayer_cnn_forward(bayer_me_t h, const uint16_t* ref, const uint16_t* cur, int W, int H, int pitch,
                                 int batch, long long ref_batch_stride, long long cur_batch_stride,
                                 const uint16_t* w_bf16, int range, float* prop_dxdy, float* conf, void* stream);

/* Loss (neg_weight = w_neg > 0) and its gradient w.r.t. all parameters on
 * `batch` pairs labelled by `labels` [batch][H/16][W/16] (the exhaustive-search fields): grad
 * [BAYER_CNN_NPARAMS] and loss [1], device float32, overwritten.  The backward
 * runs on the tensor cores with bfloat16 operands (the forward's activations
 * and weights, each layer's pre-activation gradient rounded to bfloat16) and
 * float32 accumulation; gradients are summed with atomics, so their last bits
 * vary from call to call. */
bayer_status_t bayer_cnn_loss_grad(bayer_me_t h, const uint16_t* ref, const uint16_t* cur, int W, int H, int pitch,
                                   int batch, long long ref_batch_stride, long long cur_batch_stride,
                                   const uint16_t* w_bf16, const bayer_mv_t* labels, int range, float neg_weight,
                                   float* grad, float* loss, void* stream);

/* One AdamW step (decoupled weight decay, bias-corrected moments) on the
 * float32 master w, refreshing the bfloat16 copy; step counts from 1. */
bayer_status_t bayer_cnn_adamw(bayer_me_t h, float* w, uint16_t* w_bf16, const float* grad, float* m, float* v,
                               int step, float lr, float beta1, float beta2, float eps, float weight_decay,
                               void* stream);

/* Learned-seeded search: network forward, +-4 refine of the blocks with
 * conf >= conf_thresh, exhaustive +-range search of the others (block 16,
 * EVEN phase, range in {8, 16, 24, 32}).  mv_out [batch][ceil(H/16)][W/16]
 * (a last block row clipped by the frame is searched over its rows in the
 * frame, as in the exhaustive search);
 * fallback_out (optional) 1 where the full search ran; n_fallback (optional,
 * device int) the number of such blocks.  The result is exactly the SEEDED
 * mode of bayer_me_estimate_ex given the network's proposals. */
bayer_status_t bayer_me_estimate_learned(bayer_me_t h, const uint16_t* ref, const uint16_t* cur, int W, int H,
                                         int pitch, int batch, long long ref_batch_stride,
                                         long long cur_batch_stride, const uint16_t* w_bf16, int range,
                                         float conf_thresh, bayer_mv_t* mv_out, uint8_t* fallback_out,
                                         int* n_fallback, void* stream);

/* ---------------------------------------------------------------------------
 * Refine convolution of propagated features.  The paper corrects the
 * propagated features z_pred with a learned residual (Sec. 3.3: z_C = z_pred +
 * z_Res, PRNet); its dense-convolution core is reduced here to three 3x3
 * convolutions (stride 1, zero pad 1): C -> hidden (ReLU) -> hidden (ReLU) ->
 * C (linear), biases added, on NHWC float32 maps.
 *   precision BAYER_PREC_BF16: inputs, weights and the two hidden activations
 *     rounded to bfloat16, products accumulated in float32 on the tensor cores
 *     (tcgen05, accumulators in TMEM); output float32.
 *   precision BAYER_PREC_FP32: everything in float32 on the SIMT cores.
 * Supported: C = 128, hidden = 64.  feat, out: device float32
 * [n][Hf][Wf][C] (must not overlap); w1 [hidden][C][3][3], b1 [hidden],
 * w2 [hidden][hidden][3][3], b2 [hidden], w3 [C][hidden][3][3], b3 [C]:
 * device float32.  Hidden activations use the handle's workspace. */
enum { BAYER_PREC_BF16 = 0, BAYER_PREC_FP32 = 1 };
bayer_status_t bayer_refine_conv(bayer_me_t h, const float* feat, int n, int Hf, int Wf, int C, int hidden,
                                 const float* w1, const float* b1, const float* w2, const float* b2, const float* w3,
                                 const float* b3, int precision, float* out, void* stream);

/* ---------------------------------------------------------------------------
 * Many camera streams at once (not in the paper; its batch dimension, Sec. 4.1
 * "CUDA Settings", extended to frame pairs of different sizes).  One frame pair
 * per entry: exhaustive EVEN search (block 16, +-range, range in
 * {8, 16, 24, 32}; W a multiple of 16, H even: a last block row clipped by
 * the frame, e.g. H = 1080, is searched over its rows in the frame), then,
 * where feat is not NULL, propagation of that pair's NCHW feature map as in
 * bayer_feat_propagate (stride divides 16; Wf == W / stride and
 * Hf == ceil(H / stride)).  mv_out holds ceil(H/16) x W/16 records.
 * The searches run in one launch (one CTA per strip of blocks of any pair)
 * and the propagations in a second one, or, smallest frames first, per class
 * of frame size a search launch followed by that class's propagation launch;
 * the launches are captured as a CUDA graph and replayed on later calls with
 * the same set of sizes.  A pair with 16-byte aligned frame rows can have its
 * search windows staged by TMA tile loads, and a bilinear propagation with
 * stride < 16 whose feat is 16-byte aligned and Wf a multiple of 4 can be
 * staged through shared memory by TMA tile loads (tensor maps per pair,
 * encoded on every call); the schedule decides; other pairs are read with
 * plain loads.  Either way the result is the same bit for bit.  The first
 * call for a set of sizes also runs an autotuner: it times each launch
 * schedule (blocks per strip 4 or 8; pairs as given or largest first; the
 * per-size launches smallest first), then, for the best of them, plain-load
 * search windows and global-memory propagation items in place of TMA tiles,
 * and keeps, among those within 3 % of the fastest step, the one with the
 * lowest median per-pair completion time (the handle's autotune table).  A TMA wait that expires
 * records BAYER_ERR_TIMEOUT in the handle's status word
 * (bayer_me_sync_status).
 *   pairs: HOST array of n descriptors of device buffers (caller-owned).
 *   end_ns: optional device int64 [n]: per pair, nanoseconds from the start
 *     of the search launch until that pair's output (propagated features, or
 *     the MV field without features) was complete.
 *   schedule: optional host int.  In: 0 to let the autotuner choose, or a
 *     schedule code to run that schedule instead (40, 41, 80, 81, 142 or 182,
 *     plus 1000 for plain-load search windows and/or 2000 for global-memory
 *     propagation items; any other value returns BAYER_ERR_INVALID_ARG).
 *     Out: the schedule run, 1000 * (plain windows + 2 * global-memory
 *     propagation) + 100 * (per-size launches) + 10 * blocks per strip +
 *     order (0 as given, 1 largest first, 2 smallest first).
 * The first call synchronises the device (autotuning); later calls are
 * asynchronous on `stream`. */
typedef struct {
  const uint16_t* ref; /* device frame, H rows of `pitch` elements */
  const uint16_t* cur;
  int W, H, pitch;
  bayer_mv_t* mv_out;  /* device [ceil(H/16)][W/16] */
  const float* feat;   /* device NCHW [C][Hf][Wf], or NULL */
  float* feat_out;     /* device, like feat */
  int C, Hf, Wf, stride;
} bayer_pair_t;

bayer_status_t bayer_me_multi_stream(bayer_me_t h, const bayer_pair_t* pairs, int n, int range, int interp,
                                     long long* end_ns, int* schedule, void* stream);

/* Allocation-free coarse-to-fine search.  The paper has no counterpart: this
 * entry point serves callers that cannot call cudaMalloc -- for example a
 * real-time frame loop, where an allocation can synchronise the device and
 * stall every stream, or a host that commits all device memory to a fixed
 * budget at start-up and forbids later allocations.  It takes no handle (a
 * handle allocates its workspace) and runs the same search, on the same
 * kernels, as bayer_me_estimate_ex with mode BAYER_MODE_C2F.
 *   Device: it launches on the CURRENT device; the caller makes the device
 *     that holds ref, cur and mv_out current (cudaSetDevice) before the call.
 *   Scratch: the intermediate pyramid fields live in one static device array
 *     of BAYER_NOALLOC_SCRATCH_BYTES (1 MiB), which every GPU that loads the
 *     library holds until the process exits.  2 x the largest intermediate
 *     field (batch x h x w records of every level but the last) must fit in
 *     it; larger requests return BAYER_ERR_UNSUPPORTED and launch nothing.
 *   Set-up: the first call on a device looks the array's device address up
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before any stream capture.  With CUDA's lazy module loading, that first
 *     call is also when the driver loads the kernels it launches, so make it
 *     at start-up, where the driver may still take device memory.
 *   Sharing: all calls share the array, which keeps the last call's contents.
 *     Every intermediate field is written before it is read, so nothing needs
 *     clearing; calls whose work overlaps on the GPU (several streams or host
 *     threads) race on the array and must be serialised by the caller.
 *   Calls no cudaMalloc, cudaFree or other allocating routine.
 *   Arguments as in bayer_me_estimate_ex (params->mode must be C2F). */
#define BAYER_NOALLOC_SCRATCH_BYTES (1u << 20)
bayer_status_t bayer_me_estimate_c2f_noalloc(const uint16_t* ref, const uint16_t* cur, int W, int H, int pitch,
                                             const bayer_me_params_t* params, bayer_mv_t* mv_out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* BAYER_ME_H */

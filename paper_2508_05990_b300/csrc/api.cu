// C ABI of libbayer_me.so (declarations and contracts in include/bayer_me.h).
//
// Host-side argument validation (no launch on error), kernel selection, the
// handle's workspace (coarse-to-fine intermediate fields, host-pipeline
// staging buffers, the device status word) and the host-buffer clip pipeline.
#include <cstdio>
#include <cstring>
#include <new>

#include <nvtx3/nvToolsExt.h>

#include "common.cuh"
#include "kernels.cuh"

struct bayer_me_s {
  int device = 0;
  int* d_status = nullptr;       // device status word (bayer_status_t)
  void* scratch = nullptr;       // coarse-to-fine intermediate fields
  size_t scratch_bytes = 0;
  // host pipeline (bayer_clip_process_host)
  cudaStream_t s_in = nullptr, s_comp = nullptr, s_out = nullptr;
  uint16_t* d_frames = nullptr;
  size_t frames_bytes = 0;
  float* d_feat = nullptr;
  size_t feat_bytes = 0;
  float* d_fout = nullptr;
  size_t fout_bytes = 0;
  bayer_mv_t* d_mv = nullptr;
  size_t mv_bytes = 0;
  // learned proposal network and seeded search
  void* cnn_acts = nullptr;
  size_t cnn_acts_bytes = 0;
  void* cnn_dpre = nullptr;
  size_t cnn_dpre_bytes = 0;
  float* prop = nullptr;  // [blocks][2] proposals, then [blocks] confidences
  size_t prop_bytes = 0;
  int* list = nullptr;    // [2 + 2 blocks]: two counts, then the two fallback lists
  size_t list_bytes = 0;
  // refine convolution
  void* ref_w = nullptr;  // bf16 weights and biases
  size_t ref_w_bytes = 0;
  void* ref_act = nullptr;  // two hidden activation maps
  size_t ref_act_bytes = 0;
  bme::MultiStream* ms = nullptr;  // multi-stream tables, autotune table, graphs
  int fail_allocs = 0;             // test hook: the next n workspace allocations report BAYER_ERR_OOM
};

namespace {

using bme::GenericArgs;

bool is_block(int b) { return b == 8 || b == 16 || b == 32 || b == 64; }

bayer_status_t cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return BAYER_OK;
  if (e == cudaErrorMemoryAllocation) return BAYER_ERR_OOM;
  return BAYER_ERR_CUDA;
}

// Grow a device buffer of the handle to at least `bytes` (contents not kept).
// Synchronises the device first, because work queued earlier may still use
// the old buffer.  While the handle's fail_allocs test hook is positive, a
// growth that would allocate fails with BAYER_ERR_OOM instead (no allocation,
// the old buffer is kept).
template <typename T>
bayer_status_t grow(bayer_me_s* h, T** p, size_t* cap, size_t bytes) {
  if (*cap >= bytes) return BAYER_OK;
  if (h->fail_allocs > 0) {
    --h->fail_allocs;
    return BAYER_ERR_OOM;
  }
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_status(e);
  if (*p) cudaFree(*p);
  *p = nullptr;
  *cap = 0;
  e = cudaMalloc(reinterpret_cast<void**>(p), bytes);
  if (e != cudaSuccess) return cuda_status(e);
  *cap = bytes;
  return BAYER_OK;
}

// NVTX range around each entry point (visible in Nsight timelines; free when
// no tool is attached).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int now = -1;
    if (prev >= 0 && cudaGetDevice(&now) == cudaSuccess && now != prev) cudaSetDevice(prev);
  }
};

bayer_status_t check_frames(const void* ref, const void* cur, int W, int H, int pitch, int block) {
  if (!ref || !cur) return BAYER_ERR_INVALID_ARG;
  if (!is_block(block)) return BAYER_ERR_INVALID_ARG;
  if (W <= 0 || H <= 0 || (W & 1) || (H & 1)) return BAYER_ERR_INVALID_ARG;
  if (W < block || H < block) return BAYER_ERR_INVALID_ARG;
  if (pitch < W) return BAYER_ERR_INVALID_ARG;
  if (W > 32767 || H > 32767) return BAYER_ERR_INVALID_ARG;
  return BAYER_OK;
}

// Full search dispatch: the specialised 16x16 EVEN kernel where it applies
// (W a multiple of 16; a last block row clipped by the frame height is served
// by the same kernel); else the packed C2F level kernel running the search as
// one stage (step 2 for EVEN, 1 for RAW, centre 0: the same candidates, limit
// and key); the generic stage kernel where neither applies.
bayer_status_t full_search(const uint16_t* ref, const uint16_t* cur, int W, int H, int pitch, long long rbs,
                           long long cbs, int batch, int block, int range, int phase, bayer_mv_t* out, int* status,
                           cudaStream_t st) {
  const int h = (H + block - 1) / block, w = (W + block - 1) / block;
  if (phase == BAYER_PHASE_EVEN && block == 16 && (W % 16) == 0 && bme::full16_even_supported(range)) {
    return cuda_status(bme::launch_full16_even(ref, cur, W, H, pitch, rbs, cbs, batch, range, out, status, st));
  }
  GenericArgs a{};
  a.ref = ref;
  a.cur = cur;
  a.W = W;
  a.H = H;
  a.pitch = pitch;
  a.ref_bs = rbs;
  a.cur_bs = cbs;
  a.B = block;
  a.h = h;
  a.w = w;
  a.nst = 1;
  a.S[0] = phase == BAYER_PHASE_EVEN ? 2 : 1;
  a.R[0] = range / a.S[0];
  a.lim = range;
  a.center_mode = 0;
  a.out = out;
  cudaError_t e = bme::launch_c2f_level(a, batch, st);
  if (e == cudaErrorNotSupported) e = bme::launch_generic(a, batch, st);
  return cuda_status(e);
}

bool seeded16_fast(int block, int phase, int W, int H, int range) {
  return block == 16 && phase == BAYER_PHASE_EVEN && (W % 16) == 0 && bme::full16_even_supported(range);
}

// Seeded refine on the fast kernels: warp-per-block +-4 refine, compacted list
// of low-confidence blocks, list-mode exhaustive search of that list.
// The fallback lists for nblk blocks: two counters, then the block indices
// of every fallback block, then those of the clipped last block row (frames
// whose height is no multiple of 16) again.
bayer_status_t fallback_list_space(bayer_me_s* h, long long nblk) {
  return grow(h, &h->list, &h->list_bytes, (size_t)(2 * nblk + 2) * sizeof(int));
}

// The same, its counters zeroed on st.
bayer_status_t fallback_list(bayer_me_s* h, long long nblk, cudaStream_t st) {
  bayer_status_t s = fallback_list_space(h, nblk);
  if (s != BAYER_OK) return s;
  return cuda_status(cudaMemsetAsync(h->list, 0, 2 * sizeof(int), st));
}

// The +-4 refine and the fallback searches; list_ready: the list has room and
// its counter is zeroed earlier on st (by the network's first launch), so
// that the refine kernel follows the network's last layer directly, as its
// dependent launch.
bayer_status_t seeded_fast(bayer_me_s* h, const uint16_t* ref, const uint16_t* cur, int W, int H, int pitch,
                           long long rbs, long long cbs, int batch, int range, const float* prop, const float* conf,
                           float thresh, bayer_mv_t* out, uint8_t* fallback, int* n_fallback, cudaStream_t st,
                           bool list_ready = false) {
  const int hb = (H + 15) / 16, wb = W / 16;  // a last block row clipped by the frame counts
  const long long nblk = (long long)batch * hb * wb;
  if (!list_ready) {
    bayer_status_t s = fallback_list(h, nblk, st);
    if (s != BAYER_OK) return s;
  }
  cudaError_t e = cudaSuccess;
  bme::Seeded16Args a{};
  a.ref = ref;
  a.cur = cur;
  a.W = W;
  a.H = H;
  a.pitch = pitch;
  a.ref_bs = rbs;
  a.cur_bs = cbs;
  a.h = hb;
  a.w = wb;
  a.batch = batch;
  a.prop = prop;
  a.conf = conf;
  a.thresh = thresh;
  a.range = range;
  a.out = out;
  a.fallback = fallback;
  a.count = h->list;
  a.count2 = h->list + 1;
  a.list = h->list + 2;
  a.list2 = h->list + 2 + nblk;
  if (e == cudaSuccess) e = bme::launch_seeded16(a, st);
  // every fallback block as 16 rows (the clipped row's results are then
  // replaced), then the clipped row's over its rows in the frame: the clipped
  // form of the list kernel is slower for every block, so it runs only there
  if (e == cudaSuccess)
    e = bme::launch_full16_list(ref, cur, W, H, pitch, rbs, cbs, batch, hb, wb, range, a.list, a.count, (int)nblk,
                                false, out, h->d_status, st);
  if (e == cudaSuccess && H % 16)
    e = bme::launch_full16_list(ref, cur, W, H, pitch, rbs, cbs, batch, hb, wb, range, a.list2, a.count2,
                                batch * wb, true, out, h->d_status, st);
  if (e == cudaSuccess && n_fallback)
    e = cudaMemcpyAsync(n_fallback, a.count, sizeof(int), cudaMemcpyDeviceToDevice, st);
  return cuda_status(e);
}

// Frames for the network: W a multiple of 32; H a multiple of 32 for training
// (the loss covers the network's whole 2 H4 x 2 W4 block grid), of 8 for
// inference (the layers take their natural sizes, the proposals are cropped
// to the ceil(H / 16) block rows).
bayer_status_t check_cnn_frames(const void* ref, const void* cur, int W, int H, int pitch, int batch, long long rbs,
                                long long cbs, bool infer) {
  bayer_status_t s = check_frames(ref, cur, W, H, pitch, 16);
  if (s != BAYER_OK) return s;
  if ((W % 32) != 0 || (H % (infer ? 8 : 32)) != 0) return BAYER_ERR_UNSUPPORTED;
  if (batch < 1 || batch > 65535 || rbs < 0 || cbs < 0) return BAYER_ERR_INVALID_ARG;
  return BAYER_OK;
}

}  // namespace

extern "C" {

const char* bayer_status_string(bayer_status_t s) {
  switch (s) {
    case BAYER_OK: return "ok";
    case BAYER_ERR_INVALID_ARG: return "invalid argument";
    case BAYER_ERR_UNSUPPORTED: return "unsupported configuration";
    case BAYER_ERR_CUDA: return "CUDA error";
    case BAYER_ERR_OOM: return "out of device memory";
    case BAYER_ERR_TIMEOUT: return "device-side wait timed out";
  }
  return "unknown status";
}

bayer_status_t bayer_me_init(bayer_me_t* out, int device) {
  if (!out) return BAYER_ERR_INVALID_ARG;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return BAYER_ERR_CUDA;
  cudaError_t e = cudaSetDevice(device);
  if (e != cudaSuccess) return cuda_status(e);
  bayer_me_s* h = new (std::nothrow) bayer_me_s();
  if (!h) return BAYER_ERR_OOM;
  h->device = device;
  e = bme::configure_full16();
  if (e == cudaSuccess) e = bme::configure_full16_list();
  if (e == cudaSuccess) e = bme::configure_seeded16();
  if (e == cudaSuccess) e = bme::configure_conv_tc();
  if (e == cudaSuccess) e = bme::configure_conv_s2_rows_tc();
  if (e == cudaSuccess) e = bme::configure_conv_rows_tc();
  if (e == cudaSuccess) e = bme::configure_conv_bwd_tc();
  if (e == cudaSuccess) e = cudaMalloc(&h->d_status, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(h->d_status, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->s_in, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->s_comp, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->s_out, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    bayer_me_destroy(h);
    return cuda_status(e);
  }
  *out = h;
  return BAYER_OK;
}

bayer_status_t bayer_me_destroy(bayer_me_t h) {
  if (!h) return BAYER_ERR_INVALID_ARG;
  DeviceGuard g(h->device);
  cudaDeviceSynchronize();
  if (h->d_status) cudaFree(h->d_status);
  if (h->scratch) cudaFree(h->scratch);
  if (h->d_frames) cudaFree(h->d_frames);
  if (h->d_feat) cudaFree(h->d_feat);
  if (h->d_fout) cudaFree(h->d_fout);
  if (h->d_mv) cudaFree(h->d_mv);
  if (h->cnn_acts) cudaFree(h->cnn_acts);
  if (h->cnn_dpre) cudaFree(h->cnn_dpre);
  if (h->prop) cudaFree(h->prop);
  if (h->list) cudaFree(h->list);
  if (h->ref_w) cudaFree(h->ref_w);
  if (h->ref_act) cudaFree(h->ref_act);
  if (h->ms) bme::ms_destroy(h->ms);
  if (h->s_in) cudaStreamDestroy(h->s_in);
  if (h->s_comp) cudaStreamDestroy(h->s_comp);
  if (h->s_out) cudaStreamDestroy(h->s_out);
  delete h;
  return BAYER_OK;
}

bayer_status_t bayer_me_estimate(bayer_me_t h, const uint16_t* ref, const uint16_t* cur, int W, int H, int block,
                                 int range, bayer_mv_t* mv_out, void* stream) {
  NvtxRange nvtx_range("bayer_me_estimate");
  if (!h || !mv_out) return BAYER_ERR_INVALID_ARG;
  bayer_status_t s = check_frames(ref, cur, W, H, W, block);
  if (s != BAYER_OK) return s;
  if (range < 0 || (range & 1) || range > 510) return BAYER_ERR_INVALID_ARG;
  DeviceGuard g(h->device);
  return full_search(ref, cur, W, H, W, 0, 0, 1, block, range, BAYER_PHASE_EVEN, mv_out, h->d_status,
                     static_cast<cudaStream_t>(stream));
}

bayer_status_t bayer_me_estimate_ex(bayer_me_t h, const uint16_t* ref, const uint16_t* cur, int W, int H,
                                    int pitch, const bayer_me_params_t* p, const float* prop_dxdy,
                                    const float* conf, bayer_mv_t* mv_out, uint8_t* fallback_out, void* stream) {
  NvtxRange nvtx_range("bayer_me_estimate_ex");
  if (!h || !p || !mv_out) return BAYER_ERR_INVALID_ARG;
  if (p->batch < 1 || p->batch > 65535) return BAYER_ERR_INVALID_ARG;
  if (p->phase != BAYER_PHASE_EVEN && p->phase != BAYER_PHASE_RAW) return BAYER_ERR_INVALID_ARG;
  if (p->ref_batch_stride < 0 || p->cur_batch_stride < 0) return BAYER_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  DeviceGuard g(h->device);

  if (p->mode == BAYER_MODE_FULL) {
    bayer_status_t s = check_frames(ref, cur, W, H, pitch, p->block);
    if (s != BAYER_OK) return s;
    if (p->range < 0 || p->range > 510) return BAYER_ERR_INVALID_ARG;
    if (p->phase == BAYER_PHASE_EVEN && (p->range & 1)) return BAYER_ERR_INVALID_ARG;
    return full_search(ref, cur, W, H, pitch, p->ref_batch_stride, p->cur_batch_stride, p->batch, p->block,
                       p->range, p->phase, mv_out, h->d_status, st);
  }

  if (p->mode == BAYER_MODE_SEEDED) {
    bayer_status_t s = check_frames(ref, cur, W, H, pitch, p->block);
    if (s != BAYER_OK) return s;
    if (p->phase != BAYER_PHASE_EVEN) return BAYER_ERR_UNSUPPORTED;
    if (p->range < 4 || p->range > 510 || (p->range & 1)) return BAYER_ERR_INVALID_ARG;
    if (!prop_dxdy || !conf) return BAYER_ERR_INVALID_ARG;
    if (seeded16_fast(p->block, p->phase, W, H, p->range))
      return seeded_fast(h, ref, cur, W, H, pitch, p->ref_batch_stride, p->cur_batch_stride, p->batch, p->range,
                         prop_dxdy, conf, p->conf_thresh, mv_out, fallback_out, nullptr, st);
    GenericArgs a{};
    a.ref = ref;
    a.cur = cur;
    a.W = W;
    a.H = H;
    a.pitch = pitch;
    a.ref_bs = p->ref_batch_stride;
    a.cur_bs = p->cur_batch_stride;
    a.B = p->block;
    a.h = (H + p->block - 1) / p->block;
    a.w = (W + p->block - 1) / p->block;
    a.nst = 1;
    a.lim = p->range;
    a.center_mode = 2;
    a.prop = prop_dxdy;
    a.conf = conf;
    a.thresh = p->conf_thresh;
    a.range = p->range;
    a.fallback = fallback_out;
    a.out = mv_out;
    return cuda_status(bme::launch_generic(a, p->batch, st));
  }

  if (p->mode == BAYER_MODE_C2F) {
    if (p->n_levels < 1 || p->n_levels > BAYER_MAX_LEVELS) return BAYER_ERR_INVALID_ARG;
    if (p->n_stages < 1 || p->n_stages > BAYER_MAX_STAGES) return BAYER_ERR_INVALID_ARG;
    int R[BAYER_MAX_STAGES], S[BAYER_MAX_STAGES];
    int reach = 0;
    for (int k = 0; k < p->n_stages; ++k) {
      R[k] = p->stage_radius[k];
      S[k] = p->stage_step[k];
      if (R[k] < 0 || S[k] < 1 || R[k] > 64 || S[k] > 64) return BAYER_ERR_INVALID_ARG;
      if (p->phase == BAYER_PHASE_EVEN && (S[k] & 1)) {
        R[k] = (R[k] * S[k]) / (S[k] + 1);
        S[k] = S[k] + 1;
      }
      reach += R[k] * S[k];
    }
    for (int l = 0; l < p->n_levels; ++l) {
      bayer_status_t s = check_frames(ref, cur, W, H, pitch, p->levels[l]);
      if (s != BAYER_OK) return s;
      if (l > 0 && p->levels[l] > p->levels[l - 1]) return BAYER_ERR_INVALID_ARG;
    }
    if (reach * p->n_levels > 511) return BAYER_ERR_INVALID_ARG;  // |dx|, |dy| <= 511
    // two intermediate fields, ping-pong
    size_t need = 0;
    for (int l = 0; l + 1 < p->n_levels; ++l) {
      const int B = p->levels[l];
      const size_t n = (size_t)p->batch * ((H + B - 1) / B) * ((W + B - 1) / B) * sizeof(bayer_mv_t);
      need = n > need ? n : need;
    }
    if (need) {
      bayer_status_t s = grow(h, reinterpret_cast<char**>(&h->scratch), &h->scratch_bytes, 2 * need);
      if (s != BAYER_OK) return s;
    }
    bayer_mv_t* buf[2] = {static_cast<bayer_mv_t*>(h->scratch),
                          reinterpret_cast<bayer_mv_t*>(static_cast<char*>(h->scratch) + need)};
    const bayer_mv_t* parent = nullptr;
    int parent_B = 0;
    for (int l = 0; l < p->n_levels; ++l) {
      const int B = p->levels[l];
      GenericArgs a{};
      a.ref = ref;
      a.cur = cur;
      a.W = W;
      a.H = H;
      a.pitch = pitch;
      a.ref_bs = p->ref_batch_stride;
      a.cur_bs = p->cur_batch_stride;
      a.B = B;
      a.h = (H + B - 1) / B;
      a.w = (W + B - 1) / B;
      a.nst = p->n_stages;
      for (int k = 0; k < p->n_stages; ++k) {
        a.R[k] = R[k];
        a.S[k] = S[k];
      }
      a.lim = 1 << 20;
      a.center_mode = parent ? 1 : 0;
      a.parent = parent;
      a.parent_B = parent_B;
      a.parent_h = parent ? (H + parent_B - 1) / parent_B : 0;
      a.parent_w = parent ? (W + parent_B - 1) / parent_B : 0;
      a.out = (l == p->n_levels - 1) ? mv_out : buf[l & 1];
      cudaError_t e = bme::launch_c2f_level(a, p->batch, st);
      if (e == cudaErrorNotSupported) e = bme::launch_generic(a, p->batch, st);
      if (e != cudaSuccess) return cuda_status(e);
      parent = a.out;
      parent_B = B;
    }
    return BAYER_OK;
  }
  return BAYER_ERR_INVALID_ARG;
}

bayer_status_t bayer_feat_propagate(bayer_me_t h, const float* feat, int n, int C, int Hf, int Wf, int layout,
                                    int interp, const bayer_mv_t* mv, int mv_h, int mv_w, int block, int stride,
                                    float* out, void* stream) {
  NvtxRange nvtx_range("bayer_feat_propagate");
  if (!h || !feat || !mv || !out) return BAYER_ERR_INVALID_ARG;
  if (n < 1 || C < 1 || Hf < 1 || Wf < 1) return BAYER_ERR_INVALID_ARG;
  if (layout != BAYER_LAYOUT_NCHW && layout != BAYER_LAYOUT_NHWC) return BAYER_ERR_INVALID_ARG;
  if (interp != BAYER_INTERP_NEAREST && interp != BAYER_INTERP_BILINEAR) return BAYER_ERR_INVALID_ARG;
  if (!is_block(block) || stride < 1 || stride > block || block % stride != 0) return BAYER_ERR_INVALID_ARG;
  const long long eh = ((long long)Hf * stride + block - 1) / block;
  const long long ew = ((long long)Wf * stride + block - 1) / block;
  if (mv_h != eh || mv_w != ew) return BAYER_ERR_INVALID_ARG;
  const size_t bytes = (size_t)n * C * Hf * Wf * sizeof(float);
  const char* fb = reinterpret_cast<const char*>(feat);
  const char* ob = reinterpret_cast<const char*>(out);
  if (ob < fb + bytes && fb < ob + bytes) return BAYER_ERR_INVALID_ARG;  // out overlaps feat
  DeviceGuard g(h->device);
  bme::PropArgs a{feat, out, n, C, Hf, Wf, mv, mv_h, mv_w, block / stride, stride};
  a.status = h->d_status;
  return cuda_status(bme::launch_propagate(a, layout, interp, static_cast<cudaStream_t>(stream)));
}

bayer_status_t bayer_clip_process_host(bayer_me_t h, const uint16_t* frames, int n_frames, int W, int H, int block,
                                       int range, const float* feats, int C, int Hf, int Wf, int stride, int interp,
                                       bayer_mv_t* mv_out, float* feat_out) {
  NvtxRange nvtx_range("bayer_clip_process_host");
  if (!h || !frames || !feats || !mv_out || !feat_out || n_frames < 2) return BAYER_ERR_INVALID_ARG;
  bayer_status_t s = check_frames(frames, frames, W, H, W, block);
  if (s != BAYER_OK) return s;
  if (range < 0 || (range & 1) || range > 510) return BAYER_ERR_INVALID_ARG;
  if (interp != BAYER_INTERP_NEAREST && interp != BAYER_INTERP_BILINEAR) return BAYER_ERR_INVALID_ARG;
  if (C < 1 || Hf < 1 || Wf < 1 || stride < 1 || block % stride != 0) return BAYER_ERR_INVALID_ARG;
  const int h_ = (H + block - 1) / block, w_ = (W + block - 1) / block;
  if (((long long)Hf * stride + block - 1) / block != h_ || ((long long)Wf * stride + block - 1) / block != w_)
    return BAYER_ERR_INVALID_ARG;
  DeviceGuard g(h->device);
  const int npairs = n_frames - 1;
  const size_t frame_elems = (size_t)W * H;
  const size_t map_elems = (size_t)C * Hf * Wf;
  const size_t field = (size_t)h_ * w_;
  if ((s = grow(h, &h->d_frames, &h->frames_bytes, frame_elems * n_frames * sizeof(uint16_t))) != BAYER_OK) return s;
  if ((s = grow(h, &h->d_feat, &h->feat_bytes, map_elems * npairs * sizeof(float))) != BAYER_OK) return s;
  if ((s = grow(h, &h->d_fout, &h->fout_bytes, map_elems * npairs * sizeof(float))) != BAYER_OK) return s;
  if ((s = grow(h, &h->d_mv, &h->mv_bytes, field * npairs * sizeof(bayer_mv_t))) != BAYER_OK) return s;

  // Stream plan: s_in copies the frames, then each pair's features; s_comp
  // runs the batched search once the frames are in, then each pair's
  // propagation once its features are in; s_out returns the MV fields and
  // each propagated map as soon as it is done.
  cudaEvent_t ev_frames, ev_me;
  cudaEventCreateWithFlags(&ev_frames, cudaEventDisableTiming);
  cudaEventCreateWithFlags(&ev_me, cudaEventDisableTiming);
  cudaEvent_t* ev_in = new cudaEvent_t[npairs];
  cudaEvent_t* ev_done = new cudaEvent_t[npairs];
  for (int t = 0; t < npairs; ++t) {
    cudaEventCreateWithFlags(&ev_in[t], cudaEventDisableTiming);
    cudaEventCreateWithFlags(&ev_done[t], cudaEventDisableTiming);
  }
  cudaError_t e = cudaMemcpyAsync(h->d_frames, frames, frame_elems * n_frames * sizeof(uint16_t),
                                  cudaMemcpyHostToDevice, h->s_in);
  if (e == cudaSuccess) e = cudaEventRecord(ev_frames, h->s_in);
  for (int t = 0; t < npairs && e == cudaSuccess; ++t) {
    e = cudaMemcpyAsync(h->d_feat + map_elems * t, feats + map_elems * t, map_elems * sizeof(float),
                        cudaMemcpyHostToDevice, h->s_in);
    if (e == cudaSuccess) e = cudaEventRecord(ev_in[t], h->s_in);
  }
  if (e == cudaSuccess) e = cudaStreamWaitEvent(h->s_comp, ev_frames, 0);
  if (e == cudaSuccess) {
    s = full_search(h->d_frames, h->d_frames + frame_elems, W, H, W, (long long)frame_elems,
                    (long long)frame_elems, npairs, block, range, BAYER_PHASE_EVEN, h->d_mv, h->d_status, h->s_comp);
    if (s != BAYER_OK) e = cudaErrorLaunchFailure;
  }
  if (e == cudaSuccess) e = cudaEventRecord(ev_me, h->s_comp);
  for (int t = 0; t < npairs && e == cudaSuccess; ++t) {
    e = cudaStreamWaitEvent(h->s_comp, ev_in[t], 0);
    bme::PropArgs a{h->d_feat + map_elems * t, h->d_fout + map_elems * t, 1, C, Hf, Wf, h->d_mv + field * t,
                    h_, w_, block / stride, stride};
    a.status = h->d_status;
    if (e == cudaSuccess) e = bme::launch_propagate(a, BAYER_LAYOUT_NCHW, interp, h->s_comp);
    if (e == cudaSuccess) e = cudaEventRecord(ev_done[t], h->s_comp);
  }
  if (e == cudaSuccess) e = cudaStreamWaitEvent(h->s_out, ev_me, 0);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(mv_out, h->d_mv, field * npairs * sizeof(bayer_mv_t), cudaMemcpyDeviceToHost, h->s_out);
  for (int t = 0; t < npairs && e == cudaSuccess; ++t) {
    e = cudaStreamWaitEvent(h->s_out, ev_done[t], 0);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(feat_out + map_elems * t, h->d_fout + map_elems * t, map_elems * sizeof(float),
                          cudaMemcpyDeviceToHost, h->s_out);
  }
  cudaError_t e2 = cudaStreamSynchronize(h->s_in);
  cudaError_t e3 = cudaStreamSynchronize(h->s_comp);
  cudaError_t e4 = cudaStreamSynchronize(h->s_out);
  if (e == cudaSuccess) e = e2 != cudaSuccess ? e2 : (e3 != cudaSuccess ? e3 : e4);
  cudaEventDestroy(ev_frames);
  cudaEventDestroy(ev_me);
  for (int t = 0; t < npairs; ++t) {
    cudaEventDestroy(ev_in[t]);
    cudaEventDestroy(ev_done[t]);
  }
  delete[] ev_in;
  delete[] ev_done;
  return cuda_status(e);
}

bayer_status_t bayer_cnn_forward(bayer_me_t h, const uint16_t* ref, const uint16_t* cur, int W, int H, int pitch,
                                 int batch, long long ref_bs, long long cur_bs, const uint16_t* w_bf16, int range,
                                 float* prop_dxdy, float* conf, void* stream) {
  NvtxRange nvtx_range("bayer_cnn_forward");
  if (!h || !w_bf16 || !prop_dxdy || !conf || range < 1 || range > 510) return BAYER_ERR_INVALID_ARG;
  bayer_status_t s = check_cnn_frames(ref, cur, W, H, pitch, batch, ref_bs, cur_bs, true);
  if (s != BAYER_OK) return s;
  DeviceGuard g(h->device);
  if ((s = grow(h, reinterpret_cast<char**>(&h->cnn_acts), &h->cnn_acts_bytes, bme::cnn_act_bytes(W, H, batch))) !=
      BAYER_OK)
    return s;
  bme::CnnFrames fr{ref, cur, W, H, pitch, ref_bs, cur_bs};
  return cuda_status(bme::cnn_forward(fr, batch, w_bf16, range, h->cnn_acts, prop_dxdy, conf, h->d_status,
                                      static_cast<cudaStream_t>(stream)));
}

bayer_status_t bayer_cnn_loss_grad(bayer_me_t h, const uint16_t* ref, const uint16_t* cur, int W, int H, int pitch,
                                   int batch, long long ref_bs, long long cur_bs, const uint16_t* w_bf16,
                                   const bayer_mv_t* labels, int range, float neg_weight, float* grad, float* loss,
                                   void* stream) {
  NvtxRange nvtx_range("bayer_cnn_loss_grad");
  if (!h || !w_bf16 || !labels || !grad || !loss || range < 1 || range > 510) return BAYER_ERR_INVALID_ARG;
  if (!(neg_weight > 0.f)) return BAYER_ERR_INVALID_ARG;
  bayer_status_t s = check_cnn_frames(ref, cur, W, H, pitch, batch, ref_bs, cur_bs, false);
  if (s != BAYER_OK) return s;
  DeviceGuard g(h->device);
  if ((s = grow(h, reinterpret_cast<char**>(&h->cnn_acts), &h->cnn_acts_bytes, bme::cnn_act_bytes(W, H, batch))) !=
      BAYER_OK)
    return s;
  if ((s = grow(h, reinterpret_cast<char**>(&h->cnn_dpre), &h->cnn_dpre_bytes, bme::cnn_grad_bytes(W, H, batch))) !=
      BAYER_OK)
    return s;
  bme::CnnFrames fr{ref, cur, W, H, pitch, ref_bs, cur_bs};
  return cuda_status(bme::cnn_loss_grad(fr, batch, w_bf16, labels, range, neg_weight, h->cnn_acts, h->cnn_dpre, grad,
                                        loss, h->d_status, static_cast<cudaStream_t>(stream)));
}

bayer_status_t bayer_cnn_adamw(bayer_me_t h, float* w, uint16_t* w_bf16, const float* grad, float* m, float* v,
                               int step, float lr, float beta1, float beta2, float eps, float weight_decay,
                               void* stream) {
  NvtxRange nvtx_range("bayer_cnn_adamw");
  if (!h || !w || !w_bf16 || !grad || !m || !v || step < 1) return BAYER_ERR_INVALID_ARG;
  if (!(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f) || !(eps > 0.f)) return BAYER_ERR_INVALID_ARG;
  DeviceGuard g(h->device);
  return cuda_status(bme::cnn_adamw(w, w_bf16, grad, m, v, BAYER_CNN_NPARAMS, step, lr, beta1, beta2, eps,
                                    weight_decay, static_cast<cudaStream_t>(stream)));
}

bayer_status_t bayer_me_estimate_learned(bayer_me_t h, const uint16_t* ref, const uint16_t* cur, int W, int H,
                                         int pitch, int batch, long long ref_bs, long long cur_bs,
                                         const uint16_t* w_bf16, int range, float conf_thresh, bayer_mv_t* mv_out,
                                         uint8_t* fallback_out, int* n_fallback, void* stream) {
  NvtxRange nvtx_range("bayer_me_estimate_learned");
  if (!h || !w_bf16 || !mv_out) return BAYER_ERR_INVALID_ARG;
  bayer_status_t s = check_cnn_frames(ref, cur, W, H, pitch, batch, ref_bs, cur_bs, true);
  if (s != BAYER_OK) return s;
  if (!bme::full16_even_supported(range)) return BAYER_ERR_UNSUPPORTED;
  DeviceGuard g(h->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t nblk = (size_t)batch * ((H + 15) / 16) * (W / 16);
  if ((s = grow(h, reinterpret_cast<char**>(&h->cnn_acts), &h->cnn_acts_bytes, bme::cnn_act_bytes(W, H, batch))) !=
      BAYER_OK)
    return s;
  if ((s = grow(h, reinterpret_cast<char**>(&h->prop), &h->prop_bytes, nblk * 3 * sizeof(float))) != BAYER_OK) return s;
  float* prop = h->prop;
  float* conf = h->prop + 2 * nblk;
  // the network's first launch zeroes the fallback list's counter
  if ((s = fallback_list_space(h, (long long)nblk)) != BAYER_OK) return s;
  bme::CnnFrames fr{ref, cur, W, H, pitch, ref_bs, cur_bs};
  cudaError_t e = bme::cnn_forward(fr, batch, w_bf16, range, h->cnn_acts, prop, conf, h->d_status, st, h->list);
  if (e != cudaSuccess) return cuda_status(e);
  return seeded_fast(h, ref, cur, W, H, pitch, ref_bs, cur_bs, batch, range, prop, conf, conf_thresh, mv_out,
                     fallback_out, n_fallback, st, true);
}

bayer_status_t bayer_refine_conv(bayer_me_t h, const float* feat, int n, int Hf, int Wf, int C, int hidden,
                                 const float* w1, const float* b1, const float* w2, const float* b2, const float* w3,
                                 const float* b3, int precision, float* out, void* stream) {
  NvtxRange nvtx_range("bayer_refine_conv");
  if (!h || !feat || !out || !w1 || !b1 || !w2 || !b2 || !w3 || !b3) return BAYER_ERR_INVALID_ARG;
  if (n < 1 || Hf < 1 || Wf < 1) return BAYER_ERR_INVALID_ARG;
  if (precision != BAYER_PREC_BF16 && precision != BAYER_PREC_FP32) return BAYER_ERR_INVALID_ARG;
  if (C != 128 || hidden != 64) return BAYER_ERR_UNSUPPORTED;
  const size_t bytes = (size_t)n * Hf * Wf * C * sizeof(float);
  const char* fb = reinterpret_cast<const char*>(feat);
  const char* ob = reinterpret_cast<const char*>(out);
  if (ob < fb + bytes && fb < ob + bytes) return BAYER_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(feat) | reinterpret_cast<uintptr_t>(out)) & 15) return BAYER_ERR_INVALID_ARG;
  DeviceGuard g(h->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t pix = (size_t)n * Hf * Wf;
  const size_t esz = precision == BAYER_PREC_BF16 ? 2 : 4;
  bayer_status_t s = grow(h, reinterpret_cast<char**>(&h->ref_act), &h->ref_act_bytes, 2 * pix * hidden * esz);
  if (s != BAYER_OK) return s;
  cudaError_t e;
  if (precision == BAYER_PREC_FP32) {
    float* a1 = static_cast<float*>(h->ref_act);
    float* a2 = a1 + pix * hidden;
    e = bme::launch_conv3x3_f32(feat, n, Hf, Wf, C, w1, b1, hidden, true, a1, st);
    if (e == cudaSuccess) e = bme::launch_conv3x3_f32(a1, n, Hf, Wf, hidden, w2, b2, hidden, true, a2, st);
    if (e == cudaSuccess) e = bme::launch_conv3x3_f32(a2, n, Hf, Wf, hidden, w3, b3, C, false, out, st);
    return cuda_status(e);
  }
  // weights packed into the row-stream kernel's shared-memory image (bf16), each 256-byte aligned
  const int cins[3] = {C, hidden, hidden}, couts[3] = {hidden, hidden, C};
  const float* ws[3] = {w1, w2, w3};
  size_t off[3], total = 0;
  for (int i = 0; i < 3; ++i) {
    off[i] = total;
    total += (bme::conv_rows_weight_bytes(cins[i], couts[i]) + 255) / 256 * 256;
  }
  if ((s = grow(h, reinterpret_cast<char**>(&h->ref_w), &h->ref_w_bytes, total)) != BAYER_OK) return s;
  char* wb = static_cast<char*>(h->ref_w);
  for (int i = 0; i < 3; ++i) {
    e = bme::pack_conv_rows_weights(ws[i], couts[i], cins[i], reinterpret_cast<uint16_t*>(wb + off[i]), st);
    if (e != cudaSuccess) return cuda_status(e);
  }
  __nv_bfloat16* a1 = static_cast<__nv_bfloat16*>(h->ref_act);
  __nv_bfloat16* a2 = a1 + pix * hidden;
  bme::ConvRowsArgs c{};
  c.H = Hf;
  c.W = Wf;
  c.batch = n;
  c.status = h->d_status;
  c.in_f32 = feat;
  c.wimg = reinterpret_cast<const uint4*>(wb + off[0]);
  c.bias = b1;
  c.out = a1;
  e = bme::launch_conv_rows_tc(c, C, hidden, 2, 0, true, st);
  if (e != cudaSuccess) return cuda_status(e);
  c.in = a1;
  c.wimg = reinterpret_cast<const uint4*>(wb + off[1]);
  c.bias = b2;
  c.out = a2;
  e = bme::launch_conv_rows_tc(c, hidden, hidden, 0, 0, true, st);
  if (e != cudaSuccess) return cuda_status(e);
  c.in = a2;
  c.wimg = reinterpret_cast<const uint4*>(wb + off[2]);
  c.bias = b3;
  c.out = nullptr;
  c.out_f32 = out;
  e = bme::launch_conv_rows_tc(c, hidden, C, 0, 1, false, st);
  return cuda_status(e);
}

bayer_status_t bayer_me_multi_stream(bayer_me_t h, const bayer_pair_t* pairs, int n, int range, int interp,
                                     long long* end_ns, int* schedule, void* stream) {
  NvtxRange nvtx_range("bayer_me_multi_stream");
  if (!h || !pairs || n < 1) return BAYER_ERR_INVALID_ARG;
  if (!bme::full16_even_supported(range)) return BAYER_ERR_UNSUPPORTED;
  if (interp != BAYER_INTERP_NEAREST && interp != BAYER_INTERP_BILINEAR) return BAYER_ERR_INVALID_ARG;
  for (int i = 0; i < n; ++i) {
    const bayer_pair_t& q = pairs[i];
    if (!q.ref || !q.cur || !q.mv_out) return BAYER_ERR_INVALID_ARG;
    if (q.W < 16 || q.H < 16 || (q.W % 16) || (q.H & 1) || q.pitch < q.W || q.W > 32767 || q.H > 32767)
      return BAYER_ERR_INVALID_ARG;
    if (q.feat) {
      if (!q.feat_out || q.C < 1 || q.stride < 1 || 16 % q.stride) return BAYER_ERR_INVALID_ARG;
      // the map covers the frame: Wf = W / stride, Hf = ceil(H / stride)
      if ((long long)q.Wf * q.stride != q.W || q.Hf != (q.H + q.stride - 1) / q.stride) return BAYER_ERR_INVALID_ARG;
      const size_t bytes = (size_t)q.C * q.Hf * q.Wf * sizeof(float);
      const char* fb = reinterpret_cast<const char*>(q.feat);
      const char* ob = reinterpret_cast<const char*>(q.feat_out);
      if (ob < fb + bytes && fb < ob + bytes) return BAYER_ERR_INVALID_ARG;
    }
  }
  const int force = schedule ? *schedule : 0;
  if (force != 0 && !bme::ms_schedule_valid(force)) return BAYER_ERR_INVALID_ARG;
  DeviceGuard g(h->device);
  if (!h->ms) {
    h->ms = bme::ms_create(h->device, h->d_status);
    if (!h->ms) return BAYER_ERR_CUDA;
  }
  cudaError_t e = bme::ms_run(h->ms, pairs, n, range, interp, end_ns, force, static_cast<cudaStream_t>(stream));
  if (e == cudaSuccess && schedule) *schedule = bme::ms_config_nw(h->ms, pairs, n, range, interp, force);
  return cuda_status(e);
}

bayer_status_t bayer_me_selftest_wait(bayer_me_t h, int arrive, unsigned limit, void* stream) {
  if (!h || limit == 0) return BAYER_ERR_INVALID_ARG;
  DeviceGuard g(h->device);
  return cuda_status(bme::launch_wait_selftest(h->d_status, arrive != 0, limit, static_cast<cudaStream_t>(stream)));
}

bayer_status_t bayer_me_debug_fail_allocs(bayer_me_t h, int n) {
  if (!h || n < 0) return BAYER_ERR_INVALID_ARG;
  h->fail_allocs = n;
  return BAYER_OK;
}

bayer_status_t bayer_me_sync_status(bayer_me_t h, void* stream) {
  if (!h) return BAYER_ERR_INVALID_ARG;
  DeviceGuard g(h->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int v = 0;
  cudaError_t e = cudaMemcpyAsync(&v, h->d_status, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->d_status, 0, sizeof(int), st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_status(e);
  return static_cast<bayer_status_t>(v);
}

bayer_status_t bayer_probe_alu(bayer_me_t h, int variant, double* pc_per_clk_per_sm, double* sm_mhz,
                               int* sm_count) {
  NvtxRange nvtx_range("bayer_probe_alu");
  if (!h || !pc_per_clk_per_sm || !sm_mhz || !sm_count || variant < 0 || variant > 3)
    return BAYER_ERR_INVALID_ARG;
  DeviceGuard g(h->device);
  return cuda_status(bme::run_probe_alu(variant, pc_per_clk_per_sm, sm_mhz, sm_count));
}

}  // extern "C"

// Allocation-free coarse-to-fine search (bayer_me_estimate_c2f_noalloc).
//
// For callers that cannot call cudaMalloc: the pyramid's intermediate MV
// fields live in a file-scope device array instead of handle workspace.  The
// array is part of the library image, so every GPU that loads the library
// holds it until the process exits; it is kept small (1 MiB).
//
// Host code cannot use the array's name as a device address (there it names a
// host-side stand-in), so the first call on each device looks the address up
// with cudaGetSymbolAddress, with that device current, and caches it per
// device.  The kernels then receive that pointer like any other buffer.
#include <mutex>

#include "common.cuh"
#include "kernels.cuh"

namespace {

constexpr size_t kScratchRecords = (size_t)BAYER_NOALLOC_SCRATCH_BYTES / sizeof(bayer_mv_t);

static __device__ __align__(256) bayer_mv_t g_c2f_scratch[kScratchRecords];

constexpr int kMaxDevices = 64;
std::mutex g_addr_mu;
bayer_mv_t* g_addr[kMaxDevices] = {};  // device address of g_c2f_scratch, per device

// Device address of the scratch array on the current device (looked up once).
cudaError_t scratch_address(bayer_mv_t** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_addr_mu);
  if (g_addr[dev] == nullptr) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_c2f_scratch);
    if (e != cudaSuccess) return e;
    g_addr[dev] = static_cast<bayer_mv_t*>(p);
  }
  *out = g_addr[dev];
  return cudaSuccess;
}

bool is_block(int b) { return b == 8 || b == 16 || b == 32 || b == 64; }

}  // namespace

extern "C" bayer_status_t bayer_me_estimate_c2f_noalloc(const uint16_t* ref, const uint16_t* cur, int W, int H,
                                                        int pitch, const bayer_me_params_t* p, bayer_mv_t* mv_out,
                                                        void* stream) {
  if (!ref || !cur || !p || !mv_out) return BAYER_ERR_INVALID_ARG;
  if (p->mode != BAYER_MODE_C2F) return BAYER_ERR_INVALID_ARG;
  if (p->batch < 1 || p->batch > 65535) return BAYER_ERR_INVALID_ARG;
  if (p->phase != BAYER_PHASE_EVEN && p->phase != BAYER_PHASE_RAW) return BAYER_ERR_INVALID_ARG;
  if (p->ref_batch_stride < 0 || p->cur_batch_stride < 0) return BAYER_ERR_INVALID_ARG;
  if (p->n_levels < 1 || p->n_levels > BAYER_MAX_LEVELS) return BAYER_ERR_INVALID_ARG;
  if (p->n_stages < 1 || p->n_stages > BAYER_MAX_STAGES) return BAYER_ERR_INVALID_ARG;
  if (W <= 0 || H <= 0 || (W & 1) || (H & 1) || pitch < W || W > 32767 || H > 32767) return BAYER_ERR_INVALID_ARG;
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
    const int B = p->levels[l];
    if (!is_block(B) || W < B || H < B) return BAYER_ERR_INVALID_ARG;
    if (l > 0 && B > p->levels[l - 1]) return BAYER_ERR_INVALID_ARG;
  }
  if (reach * p->n_levels > 511) return BAYER_ERR_INVALID_ARG;

  // both halves of the ping-pong must fit in the static array
  size_t half = 0;
  for (int l = 0; l + 1 < p->n_levels; ++l) {
    const int B = p->levels[l];
    const size_t n = (size_t)p->batch * ((H + B - 1) / B) * ((W + B - 1) / B);
    half = n > half ? n : half;
  }
  if (2 * half > kScratchRecords) return BAYER_ERR_UNSUPPORTED;

  bayer_mv_t* scratch = nullptr;
  cudaError_t e = scratch_address(&scratch);
  if (e != cudaSuccess) return BAYER_ERR_CUDA;
  bayer_mv_t* buf[2] = {scratch, scratch + half};

  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const bayer_mv_t* parent = nullptr;
  int parent_B = 0;
  for (int l = 0; l < p->n_levels; ++l) {
    const int B = p->levels[l];
    bme::GenericArgs a{};
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
    // the packed level kernel where it applies (it only sets a kernel
    // attribute, no allocation), else the generic one: the same kernels, in
    // the same order, as the handle path
    e = bme::launch_c2f_level(a, p->batch, st);
    if (e == cudaErrorNotSupported) e = bme::launch_generic(a, p->batch, st);
    if (e != cudaSuccess) return BAYER_ERR_CUDA;
    parent = a.out;
    parent_B = B;
  }
  return BAYER_OK;
}

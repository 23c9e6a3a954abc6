// Generic block-matching stage kernel (Sec. 3.2 "Parallel Coarse-to-fine
// Block Matching", "Matching Criterion"; Sec. 4.1 "CUDA Settings").
//
// Serves every search the specialised 16x16 EVEN kernel does not: RAW phase,
// block sizes 8/32/64, partial edge blocks, the paper's coarse-to-fine levels
// (all stages of one level fused in one CTA, each stage centred on the
// previous stage's best, held in shared memory) and the learned-seeded refine
// (proposal rounded to an even centre, or full search below the confidence
// threshold).
//
// Mapping: one CTA (4 warps) per block; the current block is staged in shared
// memory once; warps take candidates round-robin, the 32 lanes of a warp split
// the block's pixels (min(B, 32) columns x 32/min(B, 32) rows per step),
// read the reference through the read-only cache (frames are L2-resident),
// accumulate with sad.u32, and sum with one warp reduction per candidate.
#include "common.cuh"
#include "kernels.cuh"

namespace bme {

namespace {

constexpr int kGW = 4;  // warps per CTA

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

__global__ void __launch_bounds__(kGW * 32) me_generic_kernel(const GenericArgs a) {
  extern __shared__ __align__(16) uint32_t cb[];  // current block, B x B
  __shared__ uint64_t wbest[kGW];
  __shared__ uint64_t s_key;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int bx = blockIdx.x, by = blockIdx.y, pair = blockIdx.z;
  const int B = a.B;
  const uint16_t* ref = a.ref + (long long)pair * a.ref_bs;
  const uint16_t* cur = a.cur + (long long)pair * a.cur_bs;
  const int x0 = bx * B, y0 = by * B;
  const int bw = min(B, a.W - x0), bh = min(B, a.H - y0);
  const long long bidx = ((long long)pair * a.h + by) * a.w + bx;

  for (int e = threadIdx.x; e < B * B; e += blockDim.x) {
    const int y = e / B, x = e - y * B;
    uint32_t v = 0;
    if (y < bh && x < bw) v = __ldg(cur + (long long)(y0 + y) * a.pitch + x0 + x);
    cb[e] = v;
  }

  // ---- centre and stage list
  int cx = 0, cy = 0, nst = a.nst, lim = a.lim;
  int Rs[BAYER_MAX_STAGES], Ss[BAYER_MAX_STAGES];
#pragma unroll
  for (int k = 0; k < BAYER_MAX_STAGES; ++k) {
    Rs[k] = a.R[k];
    Ss[k] = a.S[k];
  }
  if (a.center_mode == 1) {
    // level l > 0 of the pyramid: the parent block holds the child's top-left pixel
    const int pi = y0 / a.parent_B, pj = x0 / a.parent_B;
    const bayer_mv_t p = a.parent[((long long)pair * a.parent_h + pi) * a.parent_w + pj];
    cx = p.dx;
    cy = p.dy;
  } else if (a.center_mode == 2) {
    const bool fb = !(a.conf[bidx] >= a.thresh);
    nst = 1;
    lim = a.range;
    if (fb) {
      Rs[0] = a.range / 2;
      Ss[0] = 2;
    } else {
      Rs[0] = 2;
      Ss[0] = 2;
      const float px = fminf(fmaxf(a.prop[2 * bidx], -1024.f), 1024.f);
      const float py = fminf(fmaxf(a.prop[2 * bidx + 1], -1024.f), 1024.f);
      cx = 2 * (int)roundf(px * 0.5f);
      cy = 2 * (int)roundf(py * 0.5f);
      cx = clampi(clampi(cx, -a.range, a.range), -x0, a.W - bw - x0);
      cy = clampi(clampi(cy, -a.range, a.range), -y0, a.H - bh - y0);
    }
    if (a.fallback != nullptr && threadIdx.x == 0) a.fallback[bidx] = fb ? 1 : 0;
  }
  __syncthreads();

  const int LPR = B < 32 ? B : 32;  // lanes per block row
  const int RPI = 32 / LPR;         // block rows per step
  const int ly = lane / LPR, lx = lane - ly * LPR;

  for (int k = 0; k < nst; ++k) {
    const int R = Rs[k], s = Ss[k], n = 2 * R + 1, ncand = n * n;
    uint64_t best = kInvalidKey;
    for (int c = warp; c < ncand; c += kGW) {
      const int vv = c / n, uu = c - vv * n;
      const int dx = cx + (uu - R) * s, dy = cy + (vv - R) * s;
      if (abs(dx) > lim || abs(dy) > lim) continue;
      if (x0 + dx < 0 || x0 + dx + bw > a.W || y0 + dy < 0 || y0 + dy + bh > a.H) continue;
      const uint16_t* rb = ref + (long long)(y0 + dy) * a.pitch + (x0 + dx);
      uint32_t part = 0;
      for (int y = ly; y < bh; y += RPI) {
        const uint16_t* rrow = rb + (long long)y * a.pitch;
        const uint32_t* crow = cb + y * B;
        for (int x = lx; x < bw; x += LPR) part = sad_u32(__ldg(rrow + x), crow[x], part);
      }
      const uint32_t sad = __reduce_add_sync(0xffffffffu, part);
      const uint64_t key = make_key(sad, dx, dy);
      best = key < best ? key : best;
    }
    if (lane == 0) wbest[warp] = best;
    __syncthreads();
    if (threadIdx.x == 0) {
      uint64_t b = wbest[0];
#pragma unroll
      for (int i = 1; i < kGW; ++i) b = wbest[i] < b ? wbest[i] : b;
      s_key = b;
    }
    __syncthreads();
    const uint64_t b = s_key;
    if (b != kInvalidKey) {
      const bayer_mv_t m = key_to_mv(b);
      cx = m.dx;
      cy = m.dy;
    }
  }
  if (threadIdx.x == 0) {
    bayer_mv_t m;
    if (s_key == kInvalidKey) {
      // no valid candidate (cannot happen for the searches the ABI exposes)
      m.dx = 0;
      m.dy = 0;
      m.sad = 0xFFFFFFFFu;
    } else {
      m = key_to_mv(s_key);
    }
    a.out[bidx] = m;
  }
}

}  // namespace

cudaError_t launch_generic(const GenericArgs& a, int batch, cudaStream_t st) {
  dim3 grid(a.w, a.h, batch);
  const size_t smem = (size_t)a.B * a.B * sizeof(uint32_t);
  me_generic_kernel<<<grid, kGW * 32, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace bme

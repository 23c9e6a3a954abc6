// Seeded +-4 refine of 16x16 blocks (the learned-seeded search; not in the
// paper).  One warp per block: a block whose confidence is below the
// threshold is appended to a device list for the exhaustive search (see
// me_full16.cu, list mode); otherwise the proposal is limited to +-1024,
// rounded to the nearest even integer (half away from zero), clamped to
// [-range, range] and to the block's valid displacements, and the 25
// candidates centre + (2u, 2v), u, v in [-2, 2], with |dx|, |dy| <= range and
// the displaced block inside the frame are evaluated from a 24x24 window and
// the current block staged in the warp's shared memory: lane (v, g) holds the
// five candidates of row v over column quarter g (each 128-bit window load
// feeds five accumulators), and two shuffles sum the quarters.
// Argmin with the (sad, |dx|+|dy|, dy, dx) key as everywhere else.
#include "common.cuh"
#include "kernels.cuh"

namespace bme {

namespace {

constexpr int kSW = 8;     // warps per CTA
constexpr int kWin = 24;   // window side (16 + 2 * 4)
constexpr int kWP = 24;    // window pitch (words)

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

__global__ void __launch_bounds__(kSW * 32) seeded16_kernel(const Seeded16Args a) {
  __shared__ __align__(16) uint32_t win_all[kSW][kWin * kWP];
  __shared__ __align__(16) uint32_t cur_all[kSW][256];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long nblk = (long long)a.batch * a.h * a.w;
  const long long gb = (long long)blockIdx.x * kSW + warp;
  if (gb >= nblk) return;
  const int pair = (int)(gb / ((long long)a.h * a.w));
  const int rem = (int)(gb - (long long)pair * a.h * a.w);
  const int by = rem / a.w, bx = rem - by * a.w;
  const int x0 = bx * 16, y0 = by * 16;
  if (!(a.conf[gb] >= a.thresh)) {
    if (lane == 0) {
      a.list[atomicAdd(a.count, 1)] = (int)gb;
      if (a.fallback) a.fallback[gb] = 1;
    }
    return;
  }
  const float px = fminf(fmaxf(a.prop[2 * gb], -1024.f), 1024.f);
  const float py = fminf(fmaxf(a.prop[2 * gb + 1], -1024.f), 1024.f);
  int cx = 2 * (int)roundf(px * 0.5f);
  int cy = 2 * (int)roundf(py * 0.5f);
  cx = clampi(clampi(cx, -a.range, a.range), -x0, a.W - 16 - x0);
  cy = clampi(clampi(cy, -a.range, a.range), -y0, a.H - 16 - y0);

  const uint16_t* ref = a.ref + (long long)pair * a.ref_bs;
  const uint16_t* cur = a.cur + (long long)pair * a.cur_bs;
  uint32_t* win = win_all[warp];
  uint32_t* cb = cur_all[warp];
  const int wx0 = x0 + cx - 4, wy0 = y0 + cy - 4;
  if (a.vec2) {
    // pairs of samples: the window starts at an even column (even centre, block
    // origin a multiple of 16) and W is even, so a pair is wholly in or out
    uint32_t rw[9], rc[4];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      const int e = lane + 32 * i, ry = e / 12, px = e - ry * 12;
      const int gy = wy0 + ry, gx = wx0 + 2 * px;
      rw[i] = (gy >= 0 && gy < a.H && gx >= 0 && gx < a.W)
                  ? __ldg(reinterpret_cast<const uint32_t*>(ref + (long long)gy * a.pitch + gx)) : 0u;
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int e = lane + 32 * i;
      rc[i] = __ldg(reinterpret_cast<const uint32_t*>(cur + (long long)(y0 + (e >> 3)) * a.pitch + x0 + 2 * (e & 7)));
    }
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      const int e = lane + 32 * i, ry = e / 12, px = e - ry * 12;
      win[ry * kWP + 2 * px] = pix_lo(rw[i]);
      win[ry * kWP + 2 * px + 1] = pix_hi(rw[i]);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int e = lane + 32 * i;
      cb[(e >> 3) * 16 + 2 * (e & 7)] = pix_lo(rc[i]);
      cb[(e >> 3) * 16 + 2 * (e & 7) + 1] = pix_hi(rc[i]);
    }
  } else {
    for (int e = lane; e < kWin * kWin; e += 32) {
      const int ry = e / kWin, rx = e - ry * kWin;
      const int gy = wy0 + ry, gx = wx0 + rx;
      uint32_t v = 0;
      if (gy >= 0 && gy < a.H && gx >= 0 && gx < a.W) v = __ldg(ref + (long long)gy * a.pitch + gx);
      win[ry * kWP + rx] = pix_word(v);
    }
    for (int e = lane; e < 256; e += 32)
      cb[e] = pix_word(__ldg(cur + (long long)(y0 + (e >> 4)) * a.pitch + x0 + (e & 15)));
  }
  __syncwarp();

  // lane = 4 * v + g (v: candidate row, g: column quarter), 20 lanes: each
  // 128-bit window load (4 samples) feeds the 5 candidates of the row.
  uint64_t key = kInvalidKey;
  const int v = lane >> 2, g = lane & 3;
  uint32_t acc[5] = {0, 0, 0, 0, 0};
  if (lane < 20) {
    const uint32_t* wr = win + (2 * v) * kWP + 4 * g;
    const uint32_t* cr = cb + 4 * g;
#pragma unroll 4
    for (int r = 0; r < 16; ++r) {
      const uint4 w0 = *reinterpret_cast<const uint4*>(wr + r * kWP);
      const uint4 w1 = *reinterpret_cast<const uint4*>(wr + r * kWP + 4);
      const uint4 w2 = *reinterpret_cast<const uint4*>(wr + r * kWP + 8);
      const uint4 c4 = *reinterpret_cast<const uint4*>(cr + r * 16);
      const uint32_t wv[12] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w, w2.x, w2.y, w2.z, w2.w};
      const uint32_t cv[4] = {c4.x, c4.y, c4.z, c4.w};
#pragma unroll
      for (int u = 0; u < 5; ++u)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[u] = sad_u32(wv[2 * u + c], cv[c], acc[u]);
    }
  }
#pragma unroll
  for (int u = 0; u < 5; ++u) {
    acc[u] += __shfl_xor_sync(0xffffffffu, acc[u], 1);
    acc[u] += __shfl_xor_sync(0xffffffffu, acc[u], 2);
  }
  if (lane < 20 && g == 0) {
#pragma unroll
    for (int u = 0; u < 5; ++u) {
      const int dx = cx + 2 * (u - 2), dy = cy + 2 * (v - 2);
      const bool ok = abs(dx) <= a.range && abs(dy) <= a.range && x0 + dx >= 0 && x0 + dx + 16 <= a.W &&
                      y0 + dy >= 0 && y0 + dy + 16 <= a.H;
      const uint64_t k = ok ? make_key(acc[u], dx, dy) : kInvalidKey;
      key = k < key ? k : key;
    }
  }
  key = warp_min_u64(key);
  if (lane == 0) {
    a.out[gb] = key_to_mv(key);
    if (a.fallback) a.fallback[gb] = 0;
  }
}

}  // namespace

cudaError_t launch_seeded16(const Seeded16Args& in, cudaStream_t st) {
  Seeded16Args a = in;
  a.vec2 = (reinterpret_cast<uintptr_t>(a.ref) % 4) == 0 && (reinterpret_cast<uintptr_t>(a.cur) % 4) == 0 &&
           a.pitch % 2 == 0 && a.ref_bs % 2 == 0 && a.cur_bs % 2 == 0;
  const long long nblk = (long long)a.batch * a.h * a.w;
  seeded16_kernel<<<(unsigned)((nblk + kSW - 1) / kSW), kSW * 32, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace bme

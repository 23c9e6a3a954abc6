// Seeded +-4 refine of 16x16 blocks (the learned-seeded search; not in the
// paper).  A block whose confidence is below the threshold goes to a device
// list for the exhaustive search (me_full16.cu, list mode); otherwise the
// proposal is limited to +-1024, rounded to the nearest even integer (half
// away from zero), clamped to [-range, range] and to the block's valid
// displacements, and the 25 candidates centre + (2u, 2v), u, v in [-2, 2],
// with |dx|, |dy| <= range and the displaced block inside the frame are
// evaluated.  Argmin with the (sad, |dx|+|dy|, dy, dx) key as everywhere else.
//
// Frames whose height is no multiple of 16 (the CLIP instance): the last
// block row is clipped to its rows in the frame; its fallback blocks are also
// appended to a second list, which a list search in the clipped form runs
// after the list search of the first (whose 16-row results for those blocks
// it overwrites).
//
// Mapping: one warp per three consecutive blocks, 10 lanes per block.
// Lanes 0-2 read the blocks' confidences and proposals; low-confidence
// blocks are appended to the fallback list (one atomic per warp).  For the
// confident blocks the warp stages the 24 x 24 windows and the current
// blocks in its shared memory as packed pixel pairs (the centre is even, so
// the window starts on a pair; with 16-byte aligned frame rows by 16-byte
// chunks realigned across lanes, else every pair load of the three blocks in
// flight at once), then lane 10 j + 5 half + v owns candidate row v (5 candidates)
// of block j over one half of its columns: 30 of 32 lanes carry SADs.  As in
// the exhaustive search (full16.cuh), SAD = sum(cur) + sum(win) -
// 2 sum min(cur, win) with min.u16x2 + dp2a per pixel pair; each lane keeps
// the column sums of the 8 window words and 4 current words it loads per row,
// so the two halves' partial SADs add up exactly.  A block's minimum is
// gathered from its five row lanes.
#include "common.cuh"
#include "kernels.cuh"
#include "tc_common.cuh"

namespace bme {

namespace {

constexpr int kSW = 4;            // warps per CTA
constexpr int kPer = 3;           // blocks per warp
constexpr int kWin = 24;          // window side (16 + 2 * 4)
constexpr int kWP = 12;           // window pitch (words): dense pixel pairs
constexpr int kCurOff = kWin * kWP;          // current block: 16 rows of 8 words
constexpr int kSlot = kCurOff + 128 + 8;     // words per block slot; with this lane order the search's
                                             // 128-bit loads take 14 (window) + 4 (current) wavefronts
                                             // per row (36 with 32-bit pixel words)
constexpr int kPairsWin = kWin * kWin / 2;  // sample pairs of a window (288 = 9 * 32)
constexpr int kPairsCur = 128;              // sample pairs of a current block (4 * 32)
constexpr size_t kSmem = (size_t)kSW * kPer * kSlot * sizeof(uint32_t);

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

// CLIP: the frame height is no multiple of 16, so the last block row is
// clipped to bh = H - y0 rows: its current rows below the frame stay zero
// (min(win, 0) adds nothing), its window sums weigh only rows < bh, and its
// candidates are valid while y0 + dy + bh <= H.
template <bool CLIP>
__global__ void __launch_bounds__(kSW * 32) seeded16_kernel(const Seeded16Args a) {
  extern __shared__ __align__(16) uint32_t smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long nblk = (long long)a.batch * a.h * a.w;
  const long long gb0 = ((long long)blockIdx.x * kSW + warp) * kPer;
  if (gb0 >= nblk) return;

  // geometry of the warp's three blocks (warp-uniform; consecutive block indices)
  int bp[kPer], bxy[kPer];
  {
    const long long hw = (long long)a.h * a.w;
    int p = (int)(gb0 / hw);
    const int rem = (int)(gb0 - (long long)p * hw);
    int by = rem / a.w, bx = rem - by * a.w;
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
      bp[k] = p;
      bxy[k] = (bx * 16) | ((by * 16) << 16);
      if (++bx == a.w) {
        bx = 0;
        if (++by == a.h) {
          by = 0;
          ++p;
        }
      }
    }
  }
  const bool vec = a.vec2;
  const bool vec16 = a.vec16;
  // launched as a dependent of the network's last layer: its proposals are
  // read only after this wait (the fallback list's counter was zeroed before
  // the network ran)
  tc::grid_dep_wait();
  tc::grid_dep_launch();

  // ---- lanes 0..2 load block gb0 + lane's confidence and proposal while
  // every lane loads its samples of the three current blocks
  float cf = 0.f, px = 0.f, py = 0.f;
  const bool mine = lane < kPer && gb0 + lane < nblk;
  if (mine) {
    const long long gb = gb0 + lane;
    cf = a.conf[gb];
    px = a.prop[2 * gb];
    py = a.prop[2 * gb + 1];
  }
  uint32_t rc[kPer][kPairsCur / 32];
  uint4 rc16[kPer];
  if (vec16) {
    // 16-byte loads: lane = (row lane / 2, half lane % 2) of each current block
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
      const int x0 = bxy[k] & 0xFFFF, y0 = bxy[k] >> 16;
      const uint16_t* cur = a.cur + (long long)bp[k] * a.cur_bs + (long long)(y0 + (lane >> 1)) * a.pitch + x0;
      const bool in = gb0 + k < nblk && (!CLIP || y0 + (lane >> 1) < a.H);
      rc16[k] = in ? __ldg(reinterpret_cast<const uint4*>(cur) + (lane & 1)) : make_uint4(0, 0, 0, 0);
    }
  } else if (vec) {
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
      const int x0 = bxy[k] & 0xFFFF, y0 = bxy[k] >> 16;
      const uint16_t* cur = a.cur + (long long)bp[k] * a.cur_bs + (long long)y0 * a.pitch + x0;
#pragma unroll
      for (int i = 0; i < kPairsCur / 32; ++i) {
        const int f = lane + 32 * i;
        const bool in = gb0 + k < nblk && (!CLIP || y0 + (f >> 3) < a.H);
        rc[k][i] = in ? __ldg(reinterpret_cast<const uint32_t*>(cur + (f >> 3) * a.pitch + 2 * (f & 7))) : 0u;
      }
    }
  }

  // ---- confidence test and search centre (lanes 0..2)
  bool confident = false, fb = false;
  int cpk = 0;
  if (mine) {
    const long long gb = gb0 + lane;
    fb = !(cf >= a.thresh);
    if (a.fallback) a.fallback[gb] = fb ? 1 : 0;
  }
  {
    // lane k < 3 handles block k; select its geometry without dynamic indexing
    const int mxy = lane == 0 ? bxy[0] : (lane == 1 ? bxy[1] : bxy[2]);
    const int x0 = mxy & 0xFFFF, y0 = mxy >> 16;
    if (mine && !fb) {
      const float qx = fminf(fmaxf(px, -1024.f), 1024.f);
      const float qy = fminf(fmaxf(py, -1024.f), 1024.f);
      int cx = 2 * (int)roundf(qx * 0.5f);
      int cy = 2 * (int)roundf(qy * 0.5f);
      cx = clampi(clampi(cx, -a.range, a.range), -x0, a.W - 16 - x0);
      const int bh = CLIP && y0 + 16 > a.H ? a.H - y0 : 16;
      cy = clampi(clampi(cy, -a.range, a.range), -y0, a.H - bh - y0);
      cpk = (int)(((unsigned)cx & 0xFFFFu) | ((unsigned)cy << 16));
      confident = true;
    }
  }
  const unsigned m = __ballot_sync(0xffffffffu, fb);
  if (m) {
    int base = 0;
    if (lane == 0) base = atomicAdd(a.count, __popc(m));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (fb) a.list[base + __popc(m & ((1u << lane) - 1u))] = (int)(gb0 + lane);
    if constexpr (CLIP) {
      // fallback blocks of the clipped last block row go to the second list as
      // well: the list search runs them again over their rows in the frame
      const int my0 = (lane == 0 ? bxy[0] : (lane == 1 ? bxy[1] : bxy[2])) >> 16;
      const bool clipped = fb && my0 + 16 > a.H;
      const unsigned m2 = __ballot_sync(0xffffffffu, clipped);
      if (m2) {
        int base2 = 0;
        if (lane == 0) base2 = atomicAdd(a.count2, __popc(m2));
        base2 = __shfl_sync(0xffffffffu, base2, 0);
        if (clipped) a.list2[base2 + __popc(m2 & ((1u << lane) - 1u))] = (int)(gb0 + lane);
      }
    }
  }
  const unsigned conf_mask = __ballot_sync(0xffffffffu, confident);
  if (conf_mask == 0) return;

  // ---- stage the confident blocks' windows and current blocks
  uint32_t* slots = smem + warp * kPer * kSlot;
  if (vec16) {
    // each window row as four 16-byte chunks from the 16-byte aligned column
    // at or left of its origin (lane = (row, chunk), three rounds of 8 rows);
    // the origin lies o = 0..3 words into chunk 0, so output chunk c takes
    // words o..3 of loaded chunk c and 0..o-1 of chunk c + 1 (the next lane)
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
      const int bc = __shfl_sync(0xffffffffu, cpk, k);
      if (!(conf_mask & (1u << k))) continue;
      const int x0 = bxy[k] & 0xFFFF, y0 = bxy[k] >> 16;
      const int cx = (int)(int16_t)(bc & 0xFFFF), cy = bc >> 16;
      const uint16_t* ref = a.ref + (long long)bp[k] * a.ref_bs;
      const int wx0 = x0 + cx - 4, wy0 = y0 + cy - 4;  // even; at least -4
      const int xa = (wx0 >> 3) << 3, o = (wx0 - xa) >> 1;
      const int ch = lane & 3;
      uint4 v[kWin / 8];
#pragma unroll
      for (int i = 0; i < kWin / 8; ++i) {
        // a chunk lies wholly inside or outside the frame (W a multiple of 16)
        const int gy = wy0 + (lane >> 2) + 8 * i, gx = xa + 8 * ch;
        v[i] = make_uint4(0, 0, 0, 0);
        if (gy >= 0 && gy < a.H && gx >= 0 && gx < a.W)
          v[i] = __ldg(reinterpret_cast<const uint4*>(ref + (long long)gy * a.pitch + gx));
      }
      uint32_t* wdst = slots + k * kSlot;
#pragma unroll
      for (int i = 0; i < kWin / 8; ++i) {
        const uint32_t n0 = __shfl_down_sync(0xffffffffu, v[i].x, 1), n1 = __shfl_down_sync(0xffffffffu, v[i].y, 1);
        const uint32_t n2 = __shfl_down_sync(0xffffffffu, v[i].z, 1);
        uint4 w;
        w.x = o == 0 ? v[i].x : (o == 1 ? v[i].y : (o == 2 ? v[i].z : v[i].w));
        w.y = o == 0 ? v[i].y : (o == 1 ? v[i].z : (o == 2 ? v[i].w : n0));
        w.z = o == 0 ? v[i].z : (o == 1 ? v[i].w : (o == 2 ? n0 : n1));
        w.w = o == 0 ? v[i].w : (o == 1 ? n0 : (o == 2 ? n1 : n2));
        if (ch < 3) *reinterpret_cast<uint4*>(wdst + ((lane >> 2) + 8 * i) * kWP + 4 * ch) = w;
      }
      reinterpret_cast<uint4*>(wdst + kCurOff)[lane] = rc16[k];  // row lane / 2, words 4 (lane % 2) ..
    }
  } else if (vec) {
    uint32_t raw[kPer][kPairsWin / 32];
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
      const int bc = __shfl_sync(0xffffffffu, cpk, k);
#pragma unroll
      for (int i = 0; i < kPairsWin / 32; ++i) raw[k][i] = 0;
      if (conf_mask & (1u << k)) {
        const int x0 = bxy[k] & 0xFFFF, y0 = bxy[k] >> 16;
        const int cx = (int)(int16_t)(bc & 0xFFFF), cy = bc >> 16;
        const uint16_t* ref = a.ref + (long long)bp[k] * a.ref_bs;
        const int wx0 = x0 + cx - 4, wy0 = y0 + cy - 4;
#pragma unroll
        for (int i = 0; i < kPairsWin / 32; ++i) {
          // the window may reach 4 samples past the frame; a pair is wholly in
          // or out (even origin, even W)
          const int e = lane + 32 * i;
          const int row = e / (kWin / 2), col = 2 * (e - row * (kWin / 2));
          const int gy = wy0 + row, gx = wx0 + col;
          if (gy >= 0 && gy < a.H && gx >= 0 && gx < a.W)
            raw[k][i] = __ldg(reinterpret_cast<const uint32_t*>(ref + (long long)gy * a.pitch + gx));
        }
      }
    }
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
      if (!(conf_mask & (1u << k))) continue;
#pragma unroll
      for (int i = 0; i < kPairsWin / 32; ++i) slots[k * kSlot + lane + 32 * i] = raw[k][i];  // pitch 12 = dense
#pragma unroll
      for (int i = 0; i < kPairsCur / 32; ++i) slots[k * kSlot + kCurOff + lane + 32 * i] = rc[k][i];
    }
  } else {
    // unaligned frames: one 16-bit load per sample
    for (int k = 0; k < kPer; ++k) {
      const int bc = __shfl_sync(0xffffffffu, cpk, k);
      if (!(conf_mask & (1u << k))) continue;
      const int x0 = bxy[k] & 0xFFFF, y0 = bxy[k] >> 16;
      const int cx = (int)(int16_t)(bc & 0xFFFF), cy = bc >> 16;
      const uint16_t* ref = a.ref + (long long)bp[k] * a.ref_bs;
      const uint16_t* cur = a.cur + (long long)bp[k] * a.cur_bs;
      for (int e = lane; e < kPairsWin; e += 32) {
        const int ry = e / kWP, wx = e - ry * kWP;
        const int gy = y0 + cy - 4 + ry, gx = x0 + cx - 4 + 2 * wx;
        uint32_t lo = 0, hi = 0;
        if (gy >= 0 && gy < a.H) {
          if (gx >= 0 && gx < a.W) lo = __ldg(ref + (long long)gy * a.pitch + gx);
          if (gx + 1 >= 0 && gx + 1 < a.W) hi = __ldg(ref + (long long)gy * a.pitch + gx + 1);
        }
        slots[k * kSlot + e] = lo | (hi << 16);
      }
      for (int e = lane; e < kPairsCur; e += 32) {
        const uint16_t* cp = cur + (long long)(y0 + (e >> 3)) * a.pitch + x0 + 2 * (e & 7);
        slots[k * kSlot + kCurOff + e] =
            (!CLIP || y0 + (e >> 3) < a.H) ? (uint32_t)__ldg(cp) | ((uint32_t)__ldg(cp + 1) << 16) : 0u;
      }
    }
  }
  __syncwarp();

  // ---- search: lane 10 j + 5 half + v
  const int j = lane / 10, r10 = lane - 10 * j, hh = r10 >= 5 ? 1 : 0, v = r10 - 5 * hh;
  const int jj = j < kPer ? j : 0;
  const int bc = __shfl_sync(0xffffffffu, cpk, jj);
  const int mxy = jj == 0 ? bxy[0] : (jj == 1 ? bxy[1] : bxy[2]);
  const bool live = j < kPer && (conf_mask & (1u << j));
  uint32_t acc[5] = {0, 0, 0, 0, 0};
  const int bhj = CLIP && (mxy >> 16) + 16 > a.H ? a.H - (mxy >> 16) : 16;  // the block's rows in the frame
  if (live) {
    // half hh: current words 4 hh .. 4 hh + 3, window words 4 hh .. 4 hh + 7 of rows 2 v + r
    const uint32_t* wb = slots + j * kSlot + 2 * v * kWP + 4 * hh;
    const uint32_t* cb = slots + j * kSlot + kCurOff + 4 * hh;
    uint32_t tw[8] = {0, 0, 0, 0, 0, 0, 0, 0};  // window column sums (lo + hi), 16 rows
    uint32_t pc[4] = {0, 0, 0, 0};              // current column sums, packed (each half <= 65520)
#pragma unroll 4
    for (int r = 0; r < 16; ++r) {
      uint32_t w[8], c[4];
#pragma unroll
      for (int k4 = 0; k4 < 2; ++k4) {
        const uint4 x = *reinterpret_cast<const uint4*>(wb + r * kWP + 4 * k4);
        w[4 * k4] = x.x;
        w[4 * k4 + 1] = x.y;
        w[4 * k4 + 2] = x.z;
        w[4 * k4 + 3] = x.w;
      }
      {
        const uint4 x = *reinterpret_cast<const uint4*>(cb + r * 8);
        c[0] = x.x;
        c[1] = x.y;
        c[2] = x.z;
        c[3] = x.w;
      }
#pragma unroll
      for (int u = 0; u < 5; ++u)
#pragma unroll
        for (int cc = 0; cc < 4; ++cc) acc[u] = dp2a_lo(min_u16x2(w[u + cc], c[cc]), 0x0202u, acc[u]);
      {
        const uint32_t wt = !CLIP || r < bhj ? 0x0101u : 0u;  // window rows past the block's own add nothing
#pragma unroll
        for (int t = 0; t < 8; ++t) tw[t] = dp2a_lo(w[t], wt, tw[t]);
      }
#pragma unroll
      for (int t = 0; t < 4; ++t) pc[t] += c[t];
    }
    // this half's SAD of candidate u: sum(cur) + sum(win of u) - 2 sum min
    uint32_t sc = 0;
#pragma unroll
    for (int t = 0; t < 4; ++t) sc = dp2a_lo(pc[t], 0x0101u, sc);
    uint32_t sw = tw[0] + tw[1] + tw[2] + tw[3];
#pragma unroll
    for (int u = 0; u < 5; ++u) {
      if (u > 0) sw += tw[u + 3] - tw[u - 1];
      acc[u] = sc + sw - acc[u];
    }
  }
  const int partner = lane < 30 ? (hh ? lane - 5 : lane + 5) : lane;
#pragma unroll
  for (int u = 0; u < 5; ++u) acc[u] += __shfl_sync(0xffffffffu, acc[u], partner);
  uint64_t key = kInvalidKey;
  if (live) {
    const int x0 = mxy & 0xFFFF, y0 = mxy >> 16;
    const int cx = (int)(int16_t)(bc & 0xFFFF), cy = bc >> 16;
    const int dy = cy + 2 * (v - 2);
#pragma unroll
    for (int u = 0; u < 5; ++u) {
      const int dx = cx + 2 * (u - 2);
      const bool ok = abs(dx) <= a.range && abs(dy) <= a.range && x0 + dx >= 0 && x0 + dx + 16 <= a.W &&
                      y0 + dy >= 0 && y0 + dy + bhj <= a.H;
      const uint64_t k = ok ? make_key(acc[u], dx, dy) : kInvalidKey;
      key = k < key ? k : key;
    }
  }
  // minimum over the block's five candidate rows (lanes 10j + v)
#pragma unroll
  for (int vv = 1; vv < 5; ++vv) {
    const uint64_t o = __shfl_sync(0xffffffffu, key, 10 * jj + vv);
    key = o < key ? o : key;
  }
  if (live && r10 == 0) a.out[gb0 + j] = key_to_mv(key);
}

}  // namespace

cudaError_t configure_seeded16() {
  cudaError_t e = cudaSuccess;
  for (int v = 0; v < 2 && e == cudaSuccess; ++v) {
    const void* fn = v ? (const void*)seeded16_kernel<true> : (const void*)seeded16_kernel<false>;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  }
  return e;
}

cudaError_t launch_seeded16(const Seeded16Args& in, cudaStream_t st) {
  Seeded16Args a = in;
  a.vec2 = (reinterpret_cast<uintptr_t>(a.ref) % 4) == 0 && (reinterpret_cast<uintptr_t>(a.cur) % 4) == 0 &&
           a.pitch % 2 == 0 && a.ref_bs % 2 == 0 && a.cur_bs % 2 == 0;
  a.vec16 = (reinterpret_cast<uintptr_t>(a.ref) % 16) == 0 && (reinterpret_cast<uintptr_t>(a.cur) % 16) == 0 &&
            a.pitch % 8 == 0 && a.ref_bs % 8 == 0 && a.cur_bs % 8 == 0 && a.W % 16 == 0;
  const long long nblk = (long long)a.batch * a.h * a.w;
  const long long per_cta = (long long)kSW * kPer;
  const dim3 grid((unsigned)((nblk + per_cta - 1) / per_cta));
  if (a.H % 16) return tc::launch_dependent(seeded16_kernel<true>, grid, dim3(kSW * 32), kSmem, st, a);
  return tc::launch_dependent(seeded16_kernel<false>, grid, dim3(kSW * 32), kSmem, st, a);
}

}  // namespace bme

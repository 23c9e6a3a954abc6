// One level of the paper's coarse-to-fine block matching (Sec. 3.2 "Parallel
// Coarse-to-fine Block Matching": large blocks first, each stage a (2R+1)^2
// grid of step s around the previous stage's best; "Matching Criterion":
// SAD, argmin = MV) on packed pixel pairs, for the EVEN phase (every step
// even) and whole blocks of 32 or 64 pixels.  Other levels take the generic
// kernel (me_generic.cu); both give the same MV field bit for bit.
//
// Mapping: one CTA (8 warps) per block.
//   * The union of the level's stage windows -- the block +- (sum of R*s)
//     around the level's start centre -- is staged once into shared memory as
//     packed pixel pairs (16-byte global loads, 32-bit stores; out-of-frame
//     samples 0) at an odd row pitch, so that 32 lanes reading one column of
//     32 different rows hit 32 different banks.
//   * Per stage: a table of B-row column sums of the stage window at each of
//     its 2R+1 row offsets (lo + hi of each pair word); then work items of
//     one candidate row and up to 9 consecutive candidate columns, round-robin
//     over the warps.  In an item lane r owns block row r (and r + 32 for
//     B = 64): it holds the current row in registers, reads each window word
//     of its row once and feeds it to every candidate of the item that uses
//     it (candidates are s/2 words apart), accumulating 2 min(cur, win) with
//     min.u16x2 + dp2a.  Then one warp reduction per candidate, and
//     SAD = sum(cur) + sum(win) - 2 sum min (the window sum from the table).
//   * A candidate whose displaced block leaves the frame is skipped; the
//     stage's minimum key (sad, |mv|_1, dy, dx) is the next stage's centre.
#include "common.cuh"
#include "kernels.cuh"

namespace bme {

namespace {

constexpr int kCW = 8;   // warps per CTA
constexpr int kUC = 9;   // candidate columns per work item (at most)

struct C2FLevel {
  int reach;    // sum over stages of R * s (pixels)
  int rows;     // union window rows = B + 2 reach
  int P;        // union window pitch (words, odd)
  int WWu;      // union window words per row
  int TP;       // table pitch (words)
  int tab_off;  // table offset in shared memory (words)
  int smem;     // bytes
};

// One work item: candidate row v of the stage (window row offset wr0 = first
// window row of block row 0 for this v), candidate columns u0 .. u0 + 8
// (first window word of candidate u: wb + u * H words).  Returns the lane's
// partial 2 sum min for each candidate in acc.  All nine columns are always
// computed -- straight-line code, no per-pair guards; columns past the
// stage's last (at most 8 H words past its window: inside the row pitch, or
// for the last row inside the column-sum table that follows) are discarded by
// the caller.
template <int B, int H>
__device__ __forceinline__ void c2f_item(const uint32_t* win, int P, int wr0, int wb,
                                         const uint32_t (&cr)[B / 32][B / 2], int lane, uint32_t* acc) {
  constexpr int BW = B / 2;                     // words per block row
  constexpr int NWW = (kUC - 1) * H + BW;       // window words an item touches
#pragma unroll
  for (int u = 0; u < kUC; ++u) acc[u] = 0;
#pragma unroll
  for (int half = 0; half < B / 32; ++half) {
    const int r = lane + 32 * half;
    const uint32_t* c = cr[half];
    const uint32_t* wrow = win + (wr0 + r) * P + wb;
#pragma unroll
    for (int w = 0; w < NWW; ++w) {
      const uint32_t x = wrow[w];
#pragma unroll
      for (int u = 0; u < kUC; ++u) {
        const int j = w - u * H;
        if (j >= 0 && j < BW) acc[u] = dp2a_lo(min_u16x2(x, c[j]), 0x0202u, acc[u]);
      }
    }
  }
}

template <int B>
__global__ void __launch_bounds__(kCW * 32) me_c2f_kernel(const GenericArgs a, const C2FLevel L) {
  extern __shared__ __align__(16) uint32_t smem[];
  uint32_t* win = smem;                 // rows x P
  uint32_t* tab = smem + L.tab_off;     // (2R+1) x TP per stage
  __shared__ uint64_t wbest[kCW];
  __shared__ uint32_t s_sc;
  constexpr int BW = B / 2;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int bx = blockIdx.x, by = blockIdx.y, pair = blockIdx.z;
  const uint16_t* ref = a.ref + (long long)pair * a.ref_bs;
  const uint16_t* curb = a.cur + (long long)pair * a.cur_bs + (long long)(by * B) * a.pitch + bx * B;
  const int x0 = bx * B, y0 = by * B;
  const long long bidx = ((long long)pair * a.h + by) * a.w + bx;

  // ---- level start centre
  int cx0 = 0, cy0 = 0;
  if (a.center_mode == 1) {
    const bayer_mv_t p = a.parent[((long long)pair * a.parent_h + y0 / a.parent_B) * a.parent_w + x0 / a.parent_B];
    cx0 = p.dx;
    cy0 = p.dy;
  }

  // ---- stage the union window: origin (ox, oy); 8-pixel chunks from the
  // 16-byte aligned column xa <= ox, word w of the window = pixel pair ox + 2w
  const int ox = x0 + cx0 - L.reach, oy = y0 + cy0 - L.reach;
  const int xa = ox - (((ox % 8) + 8) % 8);
  const int offw = (ox - xa) >> 1;  // 0..3
  {
    constexpr int kBatch = 9;  // loads of a thread in flight at once
    const int nch = (L.WWu + offw + 3) / 4;  // chunks per row
    const int total = L.rows * nch;
    for (int e0 = threadIdx.x; e0 < total; e0 += kBatch * kCW * 32) {
      uint4 v[kBatch];
#pragma unroll
      for (int i = 0; i < kBatch; ++i) {
        const int e = e0 + i * kCW * 32;
        v[i] = make_uint4(0, 0, 0, 0);
        if (e < total) {
          const int ry = e / nch, ch = e - ry * nch;
          const int gy = oy + ry, gx = xa + 8 * ch;
          if (gy >= 0 && gy < a.H && gx >= 0 && gx < a.W)
            v[i] = __ldg(reinterpret_cast<const uint4*>(ref + (long long)gy * a.pitch + gx));
        }
      }
#pragma unroll
      for (int i = 0; i < kBatch; ++i) {
        const int e = e0 + i * kCW * 32;
        if (e < total) {
          const int ry = e / nch, ch = e - ry * nch;
          const uint32_t t[4] = {v[i].x, v[i].y, v[i].z, v[i].w};
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const int wcol = 4 * ch + k - offw;
            if (wcol >= 0 && wcol < L.WWu) win[ry * L.P + wcol] = t[k];
          }
        }
      }
    }
  }
  // ---- the lane's current-block rows (lane, lane + 32), in registers for all stages
  uint32_t cr[B / 32][BW];
#pragma unroll
  for (int half = 0; half < B / 32; ++half) {
    const uint4* cp = reinterpret_cast<const uint4*>(curb + (long long)(lane + 32 * half) * a.pitch);
#pragma unroll
    for (int q = 0; q < BW / 4; ++q) {
      const uint4 t = __ldg(cp + q);
      cr[half][4 * q + 0] = t.x;
      cr[half][4 * q + 1] = t.y;
      cr[half][4 * q + 2] = t.z;
      cr[half][4 * q + 3] = t.w;
    }
  }
  // ---- sum of the current block
  {
    uint32_t sc = 0;
    for (int e = threadIdx.x; e < B * BW / 4; e += kCW * 32) {
      const int r = e / (BW / 4), q = e - r * (BW / 4);
      const uint4 t = __ldg(reinterpret_cast<const uint4*>(curb + (long long)r * a.pitch) + q);
      sc = dp2a_lo(t.x, 0x0101u, dp2a_lo(t.y, 0x0101u, dp2a_lo(t.z, 0x0101u, dp2a_lo(t.w, 0x0101u, sc))));
    }
    sc = __reduce_add_sync(0xffffffffu, sc);
    if (threadIdx.x == 0) s_sc = 0;
    __syncthreads();
    if (lane == 0) atomicAdd(&s_sc, sc);
  }
  __syncthreads();
  const uint32_t sc = s_sc;

  int cx = cx0, cy = cy0;
  uint64_t stage_best = kInvalidKey;
  for (int k = 0; k < a.nst; ++k) {
    const int R = a.R[k], s = a.S[k], n = 2 * R + 1;
    // stage window inside the union window: first row and first word
    const int r0 = L.reach - R * s + (cy - cy0);
    const int w0 = (L.reach - R * s + (cx - cx0)) >> 1;
    const int WT = BW + R * s;  // stage window words per row
    // ---- column-sum table: tab[v * TP + t] = sum of rows r0 + v s .. + B - 1 at word w0 + t
    for (int t = threadIdx.x; t < WT; t += kCW * 32) {
      const uint32_t* col = win + w0 + t;
      uint32_t acc = 0;
#pragma unroll 16
      for (int r = 0; r < B; ++r) acc = dp2a_lo(col[(r0 + r) * L.P], 0x0101u, acc);
      tab[t] = acc;
      for (int v = 1; v < n; ++v) {
        const int ra = r0 + (v - 1) * s;
#pragma unroll 8
        for (int q = 0; q < s; ++q) {
          acc = dp2a_lo(col[(ra + B + q) * L.P], 0x0101u, acc);
          acc -= dp2a_lo(col[(ra + q) * L.P], 0x0101u, 0u);
        }
        tab[v * L.TP + t] = acc;
      }
    }
    __syncthreads();
    // ---- work items: (candidate row v, columns u0 .. u0 + 8)
    const int nchunk = (n + kUC - 1) / kUC;
    uint64_t best = kInvalidKey;
    for (int it = warp; it < n * nchunk; it += kCW) {
      const int v = it / nchunk, u0 = (it - v * nchunk) * kUC;
      const int ucn = min(kUC, n - u0);
      uint32_t acc[kUC];
      const int wb = w0 + u0 * (s >> 1);
      if (s == 8) c2f_item<B, 4>(win, L.P, r0 + v * s, wb, cr, lane, acc);
      else if (s == 4) c2f_item<B, 2>(win, L.P, r0 + v * s, wb, cr, lane, acc);
      else c2f_item<B, 1>(win, L.P, r0 + v * s, wb, cr, lane, acc);
      // lane u < ucn finishes candidate u0 + u
      uint32_t mine = 0;
#pragma unroll
      for (int u = 0; u < kUC; ++u) {
        const uint32_t tot = __reduce_add_sync(0xffffffffu, acc[u]);
        if (lane == u) mine = tot;
      }
      uint64_t key = kInvalidKey;
      if (lane < ucn) {
        const int u = u0 + lane;
        const int dx = cx + (u - R) * s, dy = cy + (v - R) * s;
        if (abs(dx) <= a.lim && abs(dy) <= a.lim && x0 + dx >= 0 && x0 + dx + B <= a.W && y0 + dy >= 0 &&
            y0 + dy + B <= a.H) {
          const uint32_t* trow = tab + v * L.TP + u * (s >> 1);
          uint32_t sw = 0;
          for (int j = 0; j < BW; ++j) sw += trow[j];
          key = make_key(sc + sw - mine, dx, dy);
        }
      }
      key = warp_min_u64(key);
      best = key < best ? key : best;
    }
    if (lane == 0) wbest[warp] = best;
    __syncthreads();
    uint64_t b = wbest[0];
#pragma unroll
    for (int i = 1; i < kCW; ++i) b = wbest[i] < b ? wbest[i] : b;
    if (b != kInvalidKey) {
      const bayer_mv_t m = key_to_mv(b);
      cx = m.dx;
      cy = m.dy;
    }
    stage_best = b;
    __syncthreads();  // wbest and the table are reused by the next stage
  }
  if (threadIdx.x == 0) {
    bayer_mv_t m;
    if (stage_best == kInvalidKey) {
      m.dx = 0;
      m.dy = 0;
      m.sad = 0xFFFFFFFFu;
    } else {
      m = key_to_mv(stage_best);
    }
    a.out[bidx] = m;
  }
}

template <int B>
cudaError_t c2f_launch(const GenericArgs& a, int batch, const C2FLevel& L, cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute(me_c2f_kernel<B>, cudaFuncAttributeMaxDynamicSharedMemorySize, L.smem);
  if (e != cudaSuccess) return e;
  me_c2f_kernel<B><<<dim3(a.w, a.h, batch), kCW * 32, L.smem, st>>>(a, L);
  return cudaGetLastError();
}

}  // namespace

// The packed C2F level kernel serves EVEN-phase levels of whole 32- or
// 64-pixel blocks with steps 2, 4 or 8, 16-byte aligned frames, and a union
// window that fits shared memory; returns cudaErrorNotSupported otherwise
// (the caller then runs the generic kernel).
cudaError_t launch_c2f_level(const GenericArgs& a, int batch, cudaStream_t st) {
  if (a.B != 32 && a.B != 64) return cudaErrorNotSupported;
  if (a.center_mode == 2 || a.W % a.B || a.H % a.B) return cudaErrorNotSupported;
  if ((reinterpret_cast<uintptr_t>(a.ref) % 16) || (reinterpret_cast<uintptr_t>(a.cur) % 16) || a.pitch % 8 ||
      a.ref_bs % 8 || a.cur_bs % 8)
    return cudaErrorNotSupported;
  C2FLevel L{};
  int vmax = 0, wtmax = 0;
  for (int k = 0; k < a.nst; ++k) {
    if (a.S[k] != 2 && a.S[k] != 4 && a.S[k] != 8) return cudaErrorNotSupported;
    L.reach += a.R[k] * a.S[k];
    vmax = 2 * a.R[k] + 1 > vmax ? 2 * a.R[k] + 1 : vmax;
    wtmax = a.B / 2 + a.R[k] * a.S[k] > wtmax ? a.B / 2 + a.R[k] * a.S[k] : wtmax;
  }
  L.rows = a.B + 2 * L.reach;
  L.WWu = (a.B + 2 * L.reach) / 2;
  L.P = L.WWu | 1;  // odd pitch
  L.TP = wtmax;
  L.tab_off = (L.rows * L.P + 3) / 4 * 4;
  // + 64 words: an item's unused columns read up to 32 words past the window
  const long long bytes = ((long long)L.tab_off + (long long)vmax * L.TP + 64) * 4;
  if (bytes > 200 * 1024) return cudaErrorNotSupported;
  L.smem = (int)bytes;
  return a.B == 32 ? c2f_launch<32>(a, batch, L, st) : c2f_launch<64>(a, batch, L, st);
}

}  // namespace bme

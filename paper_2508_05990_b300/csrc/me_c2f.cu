// One level of the paper's coarse-to-fine block matching (Sec. 3.2 "Parallel
// Coarse-to-fine Block Matching": large blocks first, each stage a (2R+1)^2
// grid of step s around the previous stage's best; "Matching Criterion":
// SAD, argmin = MV) on packed pixel pairs, for the EVEN phase (every step
// even) and whole blocks of 32 or 64 pixels.  Other levels take the generic
// kernel (me_generic.cu); both give the same MV field bit for bit.
//
// Mapping: one CTA per tile of T x T blocks that start from the same centre
// (every block of level 0; at a finer level the blocks of one parent block).
//   * The union of the tile's stage windows -- the tile +- (sum of R*s)
//     around the common start centre -- is staged once into shared memory as
//     packed pixel pairs (16-byte global loads, 32-bit stores; out-of-frame
//     samples 0) at an odd row pitch, so that 32 lanes reading one column of
//     32 different rows hit 32 different banks.  Sharing it between T x T
//     blocks cuts the staged pixels per block (228^2 / 4 instead of 196^2 for
//     the 32-pixel level of the standard pyramid).
//   * Per stage and block: a table of B-row column sums of the block's stage
//     window at each of its 2R+1 row offsets (lo + hi of each pair word); then
//     work items of one block, one candidate row and up to 9 consecutive
//     candidate columns, round-robin over the warps.  In an item lane r owns
//     block row r (and r + 32 for B = 64): it holds the current rows in
//     registers, reads each window word of its row once and feeds it to every
//     candidate of the item that uses it (candidates are s/2 words apart),
//     accumulating 2 min(cur, win) with min.u16x2 + dp2a.  Then one warp
//     reduction per candidate, and SAD = sum(cur) + sum(win) - 2 sum min (the
//     window sum from the table).
//   * A candidate whose displaced block leaves the frame is skipped; each
//     block's minimum key (sad, |mv|_1, dy, dx) is its next stage's centre.
#include "common.cuh"
#include "kernels.cuh"

namespace bme {

namespace {

constexpr int kUC = 9;  // candidate columns per work item

struct C2FLevel {
  int reach;    // sum over stages of R * s (pixels)
  int rows;     // union window rows = T B + 2 reach
  int P;        // union window pitch (words, odd)
  int WWu;      // union window words per row
  int TP;       // table pitch (words)
  int tab_off;  // first table (words)
  int tab_sz;   // words per block's table
  int ms_off;   // per-candidate 2 sum min (words)
  int smem;     // bytes
};

// One work item: candidate row v of a stage (wr0: window row of block row 0),
// candidate columns u0 .. u0 + 8 (wb: first window word of column u0; column
// u starts H words further per step).  Returns the lane's partial 2 sum min
// per column in acc.  All nine columns are always computed -- straight-line
// code, no per-pair guards; columns past the stage's last (at most 8 H = 32
// words past its window: inside the row pitch, or past the last row inside
// the padding that follows the window) are discarded by the caller.
template <int B, int H>
__device__ __forceinline__ void c2f_item(const uint32_t* win, int P, int wr0, int wb,
                                         const uint32_t (&cr)[B / 32][B / 2], int lane, uint32_t* acc) {
  constexpr int BW = B / 2;                // words per block row
  constexpr int NWW = (kUC - 1) * H + BW;  // window words an item touches
#pragma unroll
  for (int u = 0; u < kUC; ++u) acc[u] = 0;
#pragma unroll
  for (int half = 0; half < B / 32; ++half) {
    const uint32_t* c = cr[half];
    const uint32_t* wrow = win + (wr0 + lane + 32 * half) * P + wb;
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

template <int B, int T, int NW>
__global__ void __launch_bounds__(NW * 32) me_c2f_kernel(const GenericArgs a, const C2FLevel L) {
  constexpr int NB = T * T;  // blocks per tile
  constexpr int BW = B / 2;
  constexpr int NT = NW * 32;
  extern __shared__ __align__(16) uint32_t smem[];
  uint32_t* win = smem;  // rows x P
  __shared__ unsigned long long sbest[NB];
  __shared__ int scx[NB], scy[NB];
  __shared__ uint32_t ssc[NB];

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int pair = blockIdx.z;
  const int tx0 = blockIdx.x * T * B, ty0 = blockIdx.y * T * B;  // tile origin (pixels)
  const uint16_t* ref = a.ref + (long long)pair * a.ref_bs;
  const uint16_t* cur = a.cur + (long long)pair * a.cur_bs;

  // ---- common start centre
  int cx0 = 0, cy0 = 0;
  if (a.center_mode == 1) {
    const bayer_mv_t p = a.parent[((long long)pair * a.parent_h + ty0 / a.parent_B) * a.parent_w + tx0 / a.parent_B];
    cx0 = p.dx;
    cy0 = p.dy;
  }

  // ---- stage the union window: origin (ox, oy); 8-pixel chunks from the
  // 16-byte aligned column xa <= ox, word w of the window = pixel pair ox + 2w
  const int ox = tx0 + cx0 - L.reach, oy = ty0 + cy0 - L.reach;
  const int xa = ox - (((ox % 8) + 8) % 8);
  const int offw = (ox - xa) >> 1;  // 0..3
  {
    // every thread takes chunks e = tid, tid + NT, ...; (row, chunk) of
    // consecutive ones advance by the constant divmod(NT, nch), so only the
    // first needs a division; all loads of a batch are in flight before the
    // stores
    constexpr int kBatch = 9;
    const int nch = (L.WWu + offw + 3) / 4;  // chunks per row
    const int dry = NT / nch, dch = NT - dry * nch;
    int ry = threadIdx.x / nch, ch = threadIdx.x - ry * nch;
    while (ry < L.rows) {
      uint4 v[kBatch];
      int rys[kBatch], chs[kBatch];
#pragma unroll
      for (int i = 0; i < kBatch; ++i) {
        rys[i] = ry;
        chs[i] = ch;
        const int gy = oy + ry, gx = xa + 8 * ch;
        v[i] = make_uint4(0, 0, 0, 0);
        if (ry < L.rows && gy >= 0 && gy < a.H && gx >= 0 && gx < a.W)
          v[i] = __ldg(reinterpret_cast<const uint4*>(ref + (long long)gy * a.pitch + gx));
        ry += dry;
        ch += dch;
        if (ch >= nch) {
          ch -= nch;
          ++ry;
        }
      }
#pragma unroll
      for (int i = 0; i < kBatch; ++i) {
        if (rys[i] < L.rows) {
          const uint32_t t[4] = {v[i].x, v[i].y, v[i].z, v[i].w};
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const int wcol = 4 * chs[i] + k - offw;
            if (wcol >= 0 && wcol < L.WWu) win[rys[i] * L.P + wcol] = t[k];
          }
        }
      }
    }
  }
  // ---- the tile's blocks: validity, the lane's current rows in registers, block sums
  bool valid[NB];
  uint32_t cr[NB][B / 32][BW];
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    const int bx = blockIdx.x * T + (b % T), by = blockIdx.y * T + (b / T);
    valid[b] = bx < a.w && by < a.h;
    const uint16_t* curb = cur + (long long)(by * B) * a.pitch + bx * B;
    uint32_t part = 0;
#pragma unroll
    for (int half = 0; half < B / 32; ++half) {
#pragma unroll
      for (int q = 0; q < BW / 4; ++q) {
        uint4 t = make_uint4(0, 0, 0, 0);
        if (valid[b]) t = __ldg(reinterpret_cast<const uint4*>(curb + (long long)(lane + 32 * half) * a.pitch) + q);
        cr[b][half][4 * q + 0] = t.x;
        cr[b][half][4 * q + 1] = t.y;
        cr[b][half][4 * q + 2] = t.z;
        cr[b][half][4 * q + 3] = t.w;
        part = dp2a_lo(t.x, 0x0101u, dp2a_lo(t.y, 0x0101u, dp2a_lo(t.z, 0x0101u, dp2a_lo(t.w, 0x0101u, part))));
      }
    }
    part = __reduce_add_sync(0xffffffffu, part);  // every warp holds the same rows
    if (threadIdx.x == 0) {
      ssc[b] = part;
      scx[b] = cx0;
      scy[b] = cy0;
    }
  }
  __syncthreads();

  for (int k = 0; k < a.nst; ++k) {
    const int R = a.R[k], s = a.S[k], n = 2 * R + 1, hs = s >> 1;
    const int WT = BW + R * s;  // stage window words per row
    // ---- (1) column-sum tables: tab_b[v * TP + t] = sum of the B rows from
    // the block's stage-window row v s, at the block's stage-window word t;
    // each column in up to three runs of row offsets, so that every thread
    // has some.  No barrier follows: the work items do not read the tables.
    constexpr int kParts = 3;
    const int vp = (n + kParts - 1) / kParts;
    for (int e = threadIdx.x; e < NB * kParts * WT; e += NT) {
      const int b = e / (kParts * WT), rem = e - b * kParts * WT;
      const int part = rem / WT, t = rem - part * WT;
      const int va = part * vp, vb = min(n, va + vp);
      if (va >= vb) continue;
      const int r0 = L.reach - R * s + (scy[b] - cy0) + (b / T) * B;
      const int w0 = ((L.reach - R * s + (scx[b] - cx0)) >> 1) + (b % T) * BW;
      uint32_t* tab = smem + L.tab_off + b * L.tab_sz;
      const uint32_t* col = win + w0 + t;
      uint32_t acc = 0;
#pragma unroll 16
      for (int r = 0; r < B; ++r) acc = dp2a_lo(col[(r0 + va * s + r) * L.P], 0x0101u, acc);
      tab[va * L.TP + t] = acc;
      for (int v = va + 1; v < vb; ++v) {
        const int ra = r0 + (v - 1) * s;
#pragma unroll 8
        for (int q = 0; q < s; ++q) {
          acc = dp2a_lo(col[(ra + B + q) * L.P], 0x0101u, acc);
          acc -= dp2a_lo(col[(ra + q) * L.P], 0x0101u, 0u);
        }
        tab[v * L.TP + t] = acc;
      }
    }
    if (threadIdx.x < NB) sbest[threadIdx.x] = kInvalidKey;
    // ---- (2) work items: (block b, candidate row v, columns u0 .. u0 + 8) ->
    // 2 sum min of each candidate into msum
    uint32_t* msum = smem + L.ms_off;
    const int nchunk = (n + kUC - 1) / kUC;
    for (int it = warp; it < NB * n * nchunk; it += NW) {
      const int b = it / (n * nchunk), rem = it - b * n * nchunk;
      if (!valid[b]) continue;  // warp-uniform
      const int v = rem / nchunk, u0 = (rem - v * nchunk) * kUC;
      const int r0 = L.reach - R * s + (scy[b] - cy0) + (b / T) * B;
      const int w0 = ((L.reach - R * s + (scx[b] - cx0)) >> 1) + (b % T) * BW;
      uint32_t acc[kUC];
      // b is warp-uniform; the register arrays are indexed statically
#pragma unroll
      for (int bb = 0; bb < NB; ++bb) {
        if (bb == b) {
          if (hs == 4) c2f_item<B, 4>(win, L.P, r0 + v * s, w0 + u0 * hs, cr[bb], lane, acc);
          else if (hs == 2) c2f_item<B, 2>(win, L.P, r0 + v * s, w0 + u0 * hs, cr[bb], lane, acc);
          else c2f_item<B, 1>(win, L.P, r0 + v * s, w0 + u0 * hs, cr[bb], lane, acc);
        }
      }
      const int ucn = min(kUC, n - u0);
      uint32_t mine = 0;
#pragma unroll
      for (int u = 0; u < kUC; ++u) {
        const uint32_t tot = __reduce_add_sync(0xffffffffu, acc[u]);
        if (lane == u) mine = tot;
      }
      if (lane < ucn) msum[(b * n + v) * n + u0 + lane] = mine;
    }
    __syncthreads();
    // ---- (3) keys, one thread per candidate; each block's minimum by warp
    // reductions and one shared atomicMin per warp and block
    for (int e0 = 0; e0 < NB * n * n; e0 += NT) {
      const int e = e0 + threadIdx.x;
      uint64_t key = kInvalidKey;
      int b = NB;
      if (e < NB * n * n) {
        b = e / (n * n);
        const int c = e - b * n * n, v = c / n, u = c - v * n;
        const int x0 = tx0 + (b % T) * B, y0 = ty0 + (b / T) * B;
        const int dx = scx[b] + (u - R) * s, dy = scy[b] + (v - R) * s;
        const int bx = blockIdx.x * T + (b % T), by = blockIdx.y * T + (b / T);
        if (bx < a.w && by < a.h && abs(dx) <= a.lim && abs(dy) <= a.lim && x0 + dx >= 0 && x0 + dx + B <= a.W &&
            y0 + dy >= 0 && y0 + dy + B <= a.H) {
          const uint32_t* trow = smem + L.tab_off + b * L.tab_sz + v * L.TP + u * hs;
          uint32_t sw = 0;
#pragma unroll 8
          for (int j = 0; j < BW; ++j) sw += trow[j];
          key = make_key(ssc[b] + sw - msum[(b * n + v) * n + u], dx, dy);
        }
      }
#pragma unroll
      for (int bb = 0; bb < NB; ++bb) {
        const uint64_t m = warp_min_u64(b == bb ? key : kInvalidKey);
        if (lane == 0 && m != kInvalidKey) atomicMin(&sbest[bb], (unsigned long long)m);
      }
    }
    __syncthreads();
    if (threadIdx.x < NB && sbest[threadIdx.x] != kInvalidKey) {
      const bayer_mv_t m = key_to_mv(sbest[threadIdx.x]);
      scx[threadIdx.x] = m.dx;
      scy[threadIdx.x] = m.dy;
    }
    __syncthreads();  // centres, tables and bests are reused by the next stage
  }
  if (threadIdx.x < NB) {
    const int b = threadIdx.x;
    const int bx = blockIdx.x * T + (b % T), by = blockIdx.y * T + (b / T);
    if (bx < a.w && by < a.h) {
      bayer_mv_t m;
      if (sbest[b] == kInvalidKey) {
        m.dx = 0;
        m.dy = 0;
        m.sad = 0xFFFFFFFFu;
      } else {
        m = key_to_mv(sbest[b]);
      }
      a.out[((long long)pair * a.h + by) * a.w + bx] = m;
    }
  }
}

template <int B, int T, int NW>
cudaError_t c2f_launch(const GenericArgs& a, int batch, const C2FLevel& L, cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute(me_c2f_kernel<B, T, NW>, cudaFuncAttributeMaxDynamicSharedMemorySize, L.smem);
  if (e != cudaSuccess) return e;
  me_c2f_kernel<B, T, NW><<<dim3((a.w + T - 1) / T, (a.h + T - 1) / T, batch), NW * 32, L.smem, st>>>(a, L);
  return cudaGetLastError();
}

bool plan(const GenericArgs& a, int T, C2FLevel* L) {
  *L = C2FLevel{};
  int vmax = 0, wtmax = 0;
  for (int k = 0; k < a.nst; ++k) {
    L->reach += a.R[k] * a.S[k];
    vmax = 2 * a.R[k] + 1 > vmax ? 2 * a.R[k] + 1 : vmax;
    wtmax = a.B / 2 + a.R[k] * a.S[k] > wtmax ? a.B / 2 + a.R[k] * a.S[k] : wtmax;
  }
  L->rows = T * a.B + 2 * L->reach;
  L->WWu = (T * a.B + 2 * L->reach) / 2;
  L->P = L->WWu | 1;  // odd pitch
  L->TP = wtmax;
  L->tab_sz = vmax * wtmax;
  // the window, 64 words of padding (an item's unused columns read up to 32
  // words past the window), then the tables
  L->tab_off = (L->rows * L->P + 64 + 3) / 4 * 4;
  L->ms_off = L->tab_off + T * T * L->tab_sz;
  const long long bytes = ((long long)L->ms_off + (long long)T * T * vmax * vmax) * 4;
  if (bytes > 220 * 1024) return false;
  L->smem = (int)bytes;
  return true;
}

}  // namespace

// The packed C2F level kernel serves EVEN-phase levels of whole 32- or
// 64-pixel blocks with steps 2, 4 or 8, 16-byte aligned frames, and a union
// window that fits shared memory; returns cudaErrorNotSupported otherwise
// (the caller then runs the generic kernel).  32-pixel levels with large
// windows take 2 x 2 tiles where the tile's blocks share a start centre
// (level 0, or a parent block that is a multiple of twice their size).
cudaError_t launch_c2f_level(const GenericArgs& a, int batch, cudaStream_t st) {
  if (a.B != 32 && a.B != 64) return cudaErrorNotSupported;
  if (a.center_mode == 2 || a.W % a.B || a.H % a.B) return cudaErrorNotSupported;
  if ((reinterpret_cast<uintptr_t>(a.ref) % 16) || (reinterpret_cast<uintptr_t>(a.cur) % 16) || a.pitch % 8 ||
      a.ref_bs % 8 || a.cur_bs % 8)
    return cudaErrorNotSupported;
  for (int k = 0; k < a.nst; ++k)
    if (a.S[k] != 2 && a.S[k] != 4 && a.S[k] != 8) return cudaErrorNotSupported;
  C2FLevel L{};
  if (a.B == 64) {
    if (!plan(a, 1, &L)) return cudaErrorNotSupported;
    return c2f_launch<64, 1, 8>(a, batch, L, st);
  }
  // a 2 x 2 tile when one block's window alone would leave at most two CTAs
  // per SM (its window is then mostly shared); else one block per CTA
  const bool shared_centre = a.center_mode == 0 || (a.parent_B % (2 * a.B) == 0);
  const bool one = plan(a, 1, &L);
  if (one && L.smem <= 76 * 1024) return c2f_launch<32, 1, 8>(a, batch, L, st);
  C2FLevel L2{};
  if (shared_centre && plan(a, 2, &L2)) return c2f_launch<32, 2, 16>(a, batch, L2, st);
  if (!one) return cudaErrorNotSupported;
  return c2f_launch<32, 1, 8>(a, batch, L, st);
}

}  // namespace bme

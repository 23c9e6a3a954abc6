// One level of the paper's coarse-to-fine block matching (Sec. 3.2 "Parallel
// Coarse-to-fine Block Matching": large blocks first, each stage a (2R+1)^2
// grid of step s around the previous stage's best; "Matching Criterion":
// SAD, argmin = MV) on packed pixel pairs, for the EVEN phase (every step
// even) and whole blocks of 8, 16, 32 or 64 pixels.  Other levels take the
// generic kernel (me_generic.cu); both give the same MV field bit for bit.
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
//   * Blocks of 8 or 16 pixels (2 x 2 tiles, the four children of one parent
//     block): a work item is one pair of candidate rows and up to 9 columns
//     of all four blocks; lane (b, vv, r) = 8 b + 4 vv + r holds rows r,
//     r + 4, ... of block b and reads them at candidate row 2 p + vv, so
//     every lane works.  Per pixel cur + win - 2 min(cur, win) = |cur - win|,
//     so a lane's partial Sum cur + Sum win - 2 Sum min is its pixels' exact
//     partial SAD: the window sums come from a running prefix sum along the
//     lane's row (two operations per column), two shuffles give each SAD,
//     and the lanes keep running minimum keys.  No tables, no key phase.
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

// Small-block work item: the partial SADs of the lane's B / 4 block rows
// (window row row0 + 4 k for block row r + 4 k) at candidate columns
// u0 .. u0 + 8 (wb as in c2f_item), csum = the lane's sum of current samples.
// Column u covers words [u H, u H + BW) of the row: its window sum is the
// difference of the row's running sum S at those two words.
template <int B, int H>
__device__ __forceinline__ void c2f_item_small(const uint32_t* win, int P, int row0, int wb,
                                               const uint32_t (&cr)[B / 4][B / 2], uint32_t csum, uint32_t* sad) {
  constexpr int BW = B / 2;
  constexpr int NWW = (kUC - 1) * H + BW;
  uint32_t m2[kUC];  // 2 sum min per column
#pragma unroll
  for (int u = 0; u < kUC; ++u) {
    sad[u] = csum;
    m2[u] = 0;
  }
#pragma unroll
  for (int k = 0; k < B / 4; ++k) {
    const uint32_t* c = cr[k];
    const uint32_t* wrow = win + (row0 + 4 * k) * P + wb;
    uint32_t S = 0;
#pragma unroll
    for (int w = 0; w < NWW; ++w) {
#pragma unroll
      for (int u = 0; u < kUC; ++u) {
        if (w == u * H) sad[u] -= S;
        if (w == u * H + BW) sad[u] += S;
      }
      const uint32_t x = wrow[w];
      S = dp2a_lo(x, 0x0101u, S);
#pragma unroll
      for (int u = 0; u < kUC; ++u) {
        const int j = w - u * H;
        if (j >= 0 && j < BW) m2[u] = dp2a_lo(min_u16x2(x, c[j]), 0x0202u, m2[u]);
      }
    }
    sad[kUC - 1] += S;  // the last column ends at the row's last word
  }
#pragma unroll
  for (int u = 0; u < kUC; ++u) sad[u] -= m2[u];  // modulo 2^32 throughout; the result is exact
}

template <int B, int T, int NW>
__global__ void __launch_bounds__(NW * 32) me_c2f_kernel(const GenericArgs a, const C2FLevel L) {
  constexpr int NB = T * T;  // blocks per tile
  constexpr int BW = B / 2;
  constexpr int NT = NW * 32;
  constexpr bool SMALL = B < 32;
  static_assert(!SMALL || T == 2, "8- and 16-pixel blocks: 2 x 2 tiles, 8 lanes per block");
  constexpr int KR = SMALL ? B / 4 : B / 32;  // block rows per lane
  constexpr int CRB = SMALL ? 1 : NB;         // blocks whose rows a lane holds
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
#pragma unroll
  for (int b = 0; b < NB; ++b) valid[b] = blockIdx.x * T + (b % T) < a.w && blockIdx.y * T + (b / T) < a.h;
  uint32_t cr[CRB][KR][BW];
  const int sb = lane >> 3, svv = (lane >> 2) & 1, sr = lane & 3;  // small blocks: the lane's (b, vv, r)
  uint32_t csum = 0;                                                 // small blocks: the lane's sum of cur
  if (threadIdx.x < NB) sbest[threadIdx.x] = kInvalidKey;
  if constexpr (SMALL) {
    const int bx = blockIdx.x * T + (sb % T), by = blockIdx.y * T + (sb / T);
    const uint16_t* curb = cur + (long long)(by * B) * a.pitch + bx * B;
#pragma unroll
    for (int k = 0; k < KR; ++k) {
#pragma unroll
      for (int q = 0; q < BW / 4; ++q) {
        uint4 t = make_uint4(0, 0, 0, 0);
        if (valid[sb]) t = __ldg(reinterpret_cast<const uint4*>(curb + (long long)(sr + 4 * k) * a.pitch) + q);
        cr[0][k][4 * q + 0] = t.x;
        cr[0][k][4 * q + 1] = t.y;
        cr[0][k][4 * q + 2] = t.z;
        cr[0][k][4 * q + 3] = t.w;
        csum = dp2a_lo(t.x, 0x0101u, dp2a_lo(t.y, 0x0101u, dp2a_lo(t.z, 0x0101u, dp2a_lo(t.w, 0x0101u, csum))));
      }
    }
    if (warp == 0 && (lane & 7) == 0) {
      scx[sb] = cx0;
      scy[sb] = cy0;
    }
  } else {
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      const int bx = blockIdx.x * T + (b % T), by = blockIdx.y * T + (b / T);
      const uint16_t* curb = cur + (long long)(by * B) * a.pitch + bx * B;
      uint32_t part = 0;
#pragma unroll
      for (int half = 0; half < KR; ++half) {
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
    for (int e = threadIdx.x; e < (SMALL ? 0 : NB * kParts * WT); e += NT) {
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
    if (!SMALL && threadIdx.x < NB) sbest[threadIdx.x] = kInvalidKey;
    // ---- (2) work items: (block b, candidate row v, columns u0 .. u0 + 8) ->
    // 2 sum min of each candidate into msum
    uint32_t* msum = smem + L.ms_off;
    const int nchunk = (n + kUC - 1) / kUC;
    if constexpr (SMALL) {
      // items (candidate-row pair p, columns u0 .. u0 + 8) of all four blocks: SADs and the
      // lanes' running minimum keys; a lane past the last candidate row recomputes the last
      // one and keeps nothing
      const int r0 = L.reach - R * s + (scy[sb] - cy0) + (sb / T) * B;
      const int w0 = ((L.reach - R * s + (scx[sb] - cx0)) >> 1) + (sb % T) * BW;
      const int x0 = tx0 + (sb % T) * B, y0 = ty0 + (sb / T) * B;
      const int npair = (n + 1) >> 1;
      uint64_t best = kInvalidKey;
      for (int it = warp; it < npair * nchunk; it += NW) {
        const int vp = it / nchunk, u0 = (it - vp * nchunk) * kUC;
        const int v = 2 * vp + svv, ve = min(v, n - 1);
        uint32_t sad[kUC];
        if (hs == 4) c2f_item_small<B, 4>(win, L.P, r0 + ve * s + sr, w0 + u0 * hs, cr[0], csum, sad);
        else if (hs == 2) c2f_item_small<B, 2>(win, L.P, r0 + ve * s + sr, w0 + u0 * hs, cr[0], csum, sad);
        else c2f_item_small<B, 1>(win, L.P, r0 + ve * s + sr, w0 + u0 * hs, cr[0], csum, sad);
#pragma unroll
        for (int u = 0; u < kUC; ++u) {
          sad[u] += __shfl_xor_sync(0xffffffffu, sad[u], 2);
          sad[u] += __shfl_xor_sync(0xffffffffu, sad[u], 1);
        }
        const int dy = scy[sb] + (v - R) * s;
        const bool row_ok = v < n && valid[sb] && abs(dy) <= a.lim && y0 + dy >= 0 && y0 + dy + B <= a.H;
#pragma unroll
        for (int u = 0; u < kUC; ++u) {
          const int dx = scx[sb] + (u0 + u - R) * s;
          if ((u & 3) == sr && row_ok && u0 + u < n && abs(dx) <= a.lim && x0 + dx >= 0 && x0 + dx + B <= a.W) {
            const uint64_t key = make_key(sad[u], dx, dy);
            best = key < best ? key : best;
          }
        }
      }
      // the block's eight lanes, then one shared atomic per warp and block
#pragma unroll
      for (int o = 4; o >= 1; o >>= 1) {
        const uint64_t other = __shfl_xor_sync(0xffffffffu, best, o);
        best = other < best ? other : best;
      }
      if ((lane & 7) == 0 && best != kInvalidKey) atomicMin(&sbest[sb], (unsigned long long)best);
    } else {
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
    }
    __syncthreads();
    // ---- (3) keys, one thread per candidate; each block's minimum by warp
    // reductions and one shared atomicMin per warp and block
    for (int e0 = 0; e0 < (SMALL ? 0 : NB * n * n); e0 += NT) {
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
      // small blocks take their atomics in the items phase: reset for the next stage here
      // (behind this stage's barriers); the last stage's minimum stays for the output
      if (SMALL && k + 1 < a.nst) sbest[threadIdx.x] = kInvalidKey;
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

bool plan(const GenericArgs& a, int T, C2FLevel* L, bool tables = true) {
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
  L->ms_off = L->tab_off + (tables ? T * T * L->tab_sz : 0);
  const long long bytes = ((long long)L->ms_off + (tables ? (long long)T * T * vmax * vmax : 0)) * 4;
  if (bytes > 220 * 1024) return false;
  L->smem = (int)bytes;
  return true;
}

}  // namespace

// The packed C2F level kernel serves EVEN-phase levels of whole 8-, 16-, 32-
// or 64-pixel blocks with steps 2, 4 or 8, 16-byte aligned frames, and a union
// window that fits shared memory; returns cudaErrorNotSupported otherwise
// (the caller then runs the generic kernel).  8- and 16-pixel levels, and
// 32-pixel levels with large windows, take 2 x 2 tiles where the tile's blocks
// share a start centre (level 0, or a parent block that is a multiple of
// twice their size); 8- and 16-pixel levels without one take the generic kernel.
cudaError_t launch_c2f_level(const GenericArgs& a, int batch, cudaStream_t st) {
  if (a.B != 8 && a.B != 16 && a.B != 32 && a.B != 64) return cudaErrorNotSupported;
  if (a.center_mode == 2 || a.W % a.B || a.H % a.B) return cudaErrorNotSupported;
  if ((reinterpret_cast<uintptr_t>(a.ref) % 16) || (reinterpret_cast<uintptr_t>(a.cur) % 16) || a.pitch % 8 ||
      a.ref_bs % 8 || a.cur_bs % 8)
    return cudaErrorNotSupported;
  for (int k = 0; k < a.nst; ++k)
    if (a.S[k] != 2 && a.S[k] != 4 && a.S[k] != 8) return cudaErrorNotSupported;
  C2FLevel L{};
  if (a.B <= 16) {
    if (!(a.center_mode == 0 || a.parent_B % (2 * a.B) == 0) || !plan(a, 2, &L, false)) return cudaErrorNotSupported;
    return a.B == 16 ? c2f_launch<16, 2, 8>(a, batch, L, st) : c2f_launch<8, 2, 8>(a, batch, L, st);
  }
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

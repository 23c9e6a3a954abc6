// One level of the paper's coarse-to-fine block matching (Sec. 3.2 "Parallel
// Coarse-to-fine Block Matching": large blocks first, each stage a (2R+1)^2
// grid of step s around the previous stage's best; "Matching Criterion":
// SAD, argmin = MV) on packed pixel pairs, for whole blocks of 8, 16, 32 or 64
// pixels: the EVEN phase (every step even) and the RAW phase's pyramids, whose
// steps are even but the last (step 1) and whose start centres may be odd.
// The frame width must be a multiple of the block size; a height that is not
// clips the last block row, whose SAD covers the rows inside the frame.
// Other levels take the generic kernel (me_generic.cu); both give the same MV
// field bit for bit.
//
// Mapping: one CTA per tile of T x T blocks that start from the same centre
// (every block of level 0; at a finer level the blocks of one parent block).
//   * The union of the tile's stage windows -- the tile +- (sum of R*s)
//     around the common start centre -- is staged once into shared memory as
//     packed pixel pairs (16-byte global loads, 32-bit stores; out-of-frame
//     samples 0) at an odd row pitch, so that lanes reading one column of
//     different rows hit different banks.  Sharing it between T x T blocks
//     cuts the staged pixels per block.  The pairs start at the centre's
//     column parity (an odd start joins the halves of adjacent aligned words
//     with a funnel shift), so every candidate of an even-step stage begins
//     on a word.
//   * A step-1 last stage (RAW): its candidates of each column parity form a
//     step-2 grid; each block stages one small window per parity in the
//     union window's space, and the same work items run on those.
//   * Work items: one candidate row (or pair of rows) and up to 9 consecutive
//     candidate columns.  A lane holds block rows of the current frame in
//     registers, reads each window word of its row once and feeds it to every
//     candidate of the item that uses it (candidates are s/2 words apart),
//     accumulating 2 min(cur, win) with min.u16x2 + dp2a, and the running sum
//     of its row's window words.  Per pixel cur + win - 2 min(cur, win) =
//     |cur - win|, so Sum cur + Sum win - 2 Sum min over the lane's pixels is
//     its exact partial SAD, a candidate column's window sum being the
//     difference of the running sum at the column's two ends.
//       - 32-pixel blocks: each warp serves one block of the tile; lane r
//         holds block row r; one warp reduction per candidate column gives
//         its SAD.
//       - 64-pixel blocks: lane r holds rows r and r + 32.  Where every stage
//         has at most 9 candidate rows (at most 9 items), warps pair up on an
//         item instead, one per 32-row half; the second warp hands its column
//         sums to the first through shared memory, behind a named barrier of
//         the pair, so the short stages split into more, shorter items.
//         Otherwise a stage whose last round holds only a few whole items
//         runs those as 3-column slices, all in that one round.
//       - 8- and 16-pixel blocks (2 x 2 tiles): an item covers a pair of
//         candidate rows of all four blocks; lane (b, vv, r) = 8 b + 4 vv + r
//         holds rows r, r + 4, ... of block b at candidate row 2 p + vv, and
//         two shuffles give each SAD.
//   * A candidate whose displaced block leaves the frame is skipped.  Lanes
//     keep running minimum keys (sad, |mv|_1, dy, dx); one shared atomic per
//     warp and block per stage gives the block's best, its next centre.
//     Two CTA barriers per stage.
#include "common.cuh"
#include "kernels.cuh"

namespace bme {

namespace {

constexpr int kUC = 9;  // candidate columns per work item

struct C2FLevel {
  int reach;  // sum over the even-step stages of R * s (pixels)
  int rows;   // union window rows = T B + 2 reach
  int P;      // union window pitch (words, odd)
  int WWu;    // union window words per row
  // an odd-step (s = 1) last stage: per block and column parity a half window
  int SR;     // its rows (B + 2R)
  int SWW;    // its words per row (B/2 + R)
  int SP;     // its pitch (words, odd)
  int SSZ;    // words per half window, padding included
  int smem;   // bytes
};

// Stage rows x WW words of packed pixel pairs into dst (row pitch P words):
// word w of row r holds the pixels gx0 + 2w and gx0 + 2w + 1 of frame row
// gy0 + r, samples outside the frame 0.  16-byte loads of 8-pixel chunks from
// the aligned column at or left of gx0; for an odd gx0 each word joins the
// high half of one aligned word and the low half of the next (one funnel
// shift), a chunk's last word taking the next chunk's first (one 4-byte
// load).  Every thread takes chunks tid, tid + NT, ...; (row, chunk) of
// consecutive ones advance by the constant divmod(NT, chunks per row), so
// only the first needs a division; the BATCH loads of a batch are in flight
// before its stores.  Every thread of the CTA calls it; no barrier.
template <int NT, int BATCH, bool ODD>
__device__ __forceinline__ void stage_window(uint32_t* dst, int P, int WW, int rows, int gx0, int gy0,
                                             const uint16_t* ref, int W, int H, int pitch) {
  const int par = ODD ? gx0 & 1 : 0;  // without ODD, gx0 is even
  const int e0 = gx0 - par;                   // even pixel of word 0's aligned pair
  const int xa = e0 - (((e0 % 8) + 8) % 8);   // its 16-byte aligned chunk
  const int offw = (e0 - xa) >> 1;            // 0..3
  constexpr int kBatch = BATCH;
  const int nch = (WW + offw + 3) / 4;  // chunks per row
  const int dry = NT / nch, dch = NT - dry * nch;
  int ry = threadIdx.x / nch, ch = threadIdx.x - ry * nch;
  while (ry < rows) {
    uint4 v[kBatch];
    uint32_t nx[kBatch];
    int rys[kBatch], chs[kBatch];
#pragma unroll
    for (int i = 0; i < kBatch; ++i) {
      rys[i] = ry;
      chs[i] = ch;
      const int gy = gy0 + ry, gx = xa + 8 * ch;
      v[i] = make_uint4(0, 0, 0, 0);
      nx[i] = 0;
      if (ry < rows && gy >= 0 && gy < H) {
        const uint16_t* rowp = ref + (long long)gy * pitch;
        if (gx >= 0 && gx < W) v[i] = __ldg(reinterpret_cast<const uint4*>(rowp + gx));
        if (par && gx + 8 >= 0 && gx + 8 < W) nx[i] = __ldg(reinterpret_cast<const uint32_t*>(rowp + gx + 8));
      }
      ry += dry;
      ch += dch;
      if (ch >= nch) {
        ch -= nch;
        ++ry;
      }
    }
#pragma unroll
    for (int i = 0; i < kBatch; ++i) {
      if (rys[i] < rows) {
        uint32_t t[4] = {v[i].x, v[i].y, v[i].z, v[i].w};
        if (par) {
          t[0] = __funnelshift_r(v[i].x, v[i].y, 16);
          t[1] = __funnelshift_r(v[i].y, v[i].z, 16);
          t[2] = __funnelshift_r(v[i].z, v[i].w, 16);
          t[3] = __funnelshift_r(v[i].w, nx[i], 16);
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int wcol = 4 * chs[i] + k - offw;
          if (wcol >= 0 && wcol < WW) dst[rys[i] * P + wcol] = t[k];
        }
      }
    }
  }
}

// One work item's partial SADs over the lane's KR block rows (window row
// row0 + RS k for the lane's k-th row, current words cr[k]) at candidate
// columns u0 .. u0 + NC - 1: wb is the first window word of column u0, column
// u starts H words further per step; csum = the lane's sum of current samples.
// ws[k] weighs row k's window samples in the running sums: 0x0101 (lo + hi),
// or 0 for a row below the frame in a block the frame clips, whose current
// words are 0 too, so that the row adds nothing to the SAD.
// All NC columns are always computed -- straight-line code, no per-pair
// guards; columns past the stage's last (at most 8 H = 32 words past its
// window: inside the row pitch, or past the last row inside the padding that
// follows the window) are discarded by the caller.
template <int KR, int RS, int BW, int H, int NC>
__device__ __forceinline__ void c2f_item(const uint32_t* win, int P, int row0, int wb, const uint32_t (&cr)[KR][BW],
                                         const uint32_t (&ws)[KR], uint32_t csum, uint32_t* sad) {
  constexpr int NWW = (NC - 1) * H + BW;  // window words of a row the item touches
  uint32_t m2[NC];                        // 2 sum min per column
#pragma unroll
  for (int u = 0; u < NC; ++u) {
    sad[u] = csum;
    m2[u] = 0;
  }
#pragma unroll
  for (int k = 0; k < KR; ++k) {
    const uint32_t* c = cr[k];
    const uint32_t* wrow = win + (row0 + RS * k) * P + wb;
    uint32_t S = 0;  // running sum of the row's window samples
#pragma unroll
    for (int w = 0; w < NWW; ++w) {
#pragma unroll
      for (int u = 0; u < NC; ++u) {
        if (w == u * H) sad[u] -= S;
        if (w == u * H + BW) sad[u] += S;
      }
      const uint32_t x = wrow[w];
      S = dp2a_lo(x, ws[k], S);
#pragma unroll
      for (int u = 0; u < NC; ++u) {
        const int j = w - u * H;
        if (j >= 0 && j < BW) m2[u] = dp2a_lo(min_u16x2(x, c[j]), 0x0202u, m2[u]);
      }
    }
    sad[NC - 1] += S;  // the last column ends at the row's last word
  }
#pragma unroll
  for (int u = 0; u < NC; ++u) sad[u] -= m2[u];  // modulo 2^32 throughout; the result is exact
}

template <int KR, int RS, int BW, int NC = kUC>
__device__ __forceinline__ void c2f_item_hs(int hs, const uint32_t* win, int P, int row0, int wb,
                                            const uint32_t (&cr)[KR][BW], const uint32_t (&ws)[KR], uint32_t csum,
                                            uint32_t* sad) {
  if (hs == 4) c2f_item<KR, RS, BW, 4, NC>(win, P, row0, wb, cr, ws, csum, sad);
  else if (hs == 2) c2f_item<KR, RS, BW, 2, NC>(win, P, row0, wb, cr, ws, csum, sad);
  else c2f_item<KR, RS, BW, 1, NC>(win, P, row0, wb, cr, ws, csum, sad);
}

// ODD: the level's last stage may step by 1 and its start centres may be odd
// (the RAW phase); without it every step and centre is even.  CLIP: the frame
// height is not a multiple of B, so the last block row is clipped (frames
// whose height is a multiple of B take the kernel without that logic).  The
// clipping logic pushes the 8-warp 64-pixel level past 128 registers, which
// would leave one CTA per SM (the shared memory allows two); its bound keeps
// two (a few bytes spilled).  Every other form has no minimum (0).
template <int B, int T, int NW, bool PAIRED = false, bool ODD = false, bool CLIP = false>
__global__ void __launch_bounds__(NW * 32, (CLIP && B == 64 && !PAIRED) ? 2 : 0)
    me_c2f_kernel(const GenericArgs a, const C2FLevel L) {
  constexpr int NB = T * T;  // blocks per tile
  constexpr int BW = B / 2;
  constexpr int NT = NW * 32;
  constexpr bool SMALL = B < 32;
  static_assert(!SMALL || T == 2, "8- and 16-pixel blocks: 2 x 2 tiles, 8 lanes per block");
  static_assert(SMALL || NW % NB == 0, "32- and 64-pixel blocks: the same number of warps per block");
  static_assert(!PAIRED || B == 64, "warp pairs: 64-pixel blocks");
  constexpr int KR = SMALL ? B / 4 : (PAIRED ? 1 : B / 32);  // block rows per lane
  constexpr int RS = SMALL ? 4 : 32;                         // row stride between a lane's rows
  constexpr int WPB = SMALL ? NW : NW / NB;                  // warps per block (large blocks)
  constexpr int NPAIR = PAIRED ? WPB / 2 : 1;
  static_assert(!PAIRED || (T == 1 && WPB % 2 == 0 && NPAIR <= 8), "64-pixel blocks: warp pairs");
  constexpr bool SLICE = B == 64 && !PAIRED;  // a stage's partial last round as 3-column slices
  extern __shared__ __align__(16) uint32_t smem[];
  uint32_t* win = smem;  // rows x P
  __shared__ unsigned long long sbest[NB];
  __shared__ int scx[NB], scy[NB];
  __shared__ uint32_t xsum[NPAIR][2][16];  // 64-pixel blocks: second half's column sums, by item parity

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

  // ---- stage the union window of the even-step stages: origin (ox, oy), of
  // the start centre's column parity
  stage_window<NT, 9, ODD>(win, L.P, L.WWu, L.rows, tx0 + cx0 - L.reach, ty0 + cy0 - L.reach, ref, a.W, a.H,
                           a.pitch);
  // ---- the lane's block (small blocks: lane group; large: the warp's) and its rows
  const int mb = SMALL ? lane >> 3 : warp / WPB;
  const int svv = (lane >> 2) & 1;                 // small blocks: candidate-row offset
  const int hb = PAIRED ? (warp - mb * WPB) / NPAIR : 0;  // 64-pixel blocks: the warp's 32-row half
  const int rl = SMALL ? (lane & 3) : lane + 32 * hb;     // the lane's first block row
  const int bx = blockIdx.x * T + (mb % T), by = blockIdx.y * T + (mb / T);
  const bool valid = bx < a.w && by < a.h;
  const int x0 = tx0 + (mb % T) * B, y0 = ty0 + (mb / T) * B;  // block origin (pixels)
  // a frame height that is not a multiple of B clips the last block row to bh
  // rows; the lane's rows below the frame keep zero current words and weigh
  // their window samples by 0, so they add nothing
  const int bh = CLIP ? min(B, a.H - y0) : B;
  uint32_t cr[KR][BW];
  uint32_t ws[KR];
  uint32_t csum = 0;  // the lane's sum of current samples
  {
    const uint16_t* curb = cur + (long long)y0 * a.pitch + x0;
#pragma unroll
    for (int k = 0; k < KR; ++k) {
      const bool in_frame = !CLIP || rl + RS * k < bh;
      ws[k] = in_frame ? 0x0101u : 0u;
#pragma unroll
      for (int q = 0; q < BW / 4; ++q) {
        uint4 t = make_uint4(0, 0, 0, 0);
        if (valid && in_frame) t = __ldg(reinterpret_cast<const uint4*>(curb + (long long)(rl + RS * k) * a.pitch) + q);
        cr[k][4 * q + 0] = t.x;
        cr[k][4 * q + 1] = t.y;
        cr[k][4 * q + 2] = t.z;
        cr[k][4 * q + 3] = t.w;
        csum = dp2a_lo(t.x, 0x0101u, dp2a_lo(t.y, 0x0101u, dp2a_lo(t.z, 0x0101u, dp2a_lo(t.w, 0x0101u, csum))));
      }
    }
  }
  if (threadIdx.x < NB) {
    sbest[threadIdx.x] = kInvalidKey;
    scx[threadIdx.x] = cx0;
    scy[threadIdx.x] = cy0;
  }
  __syncthreads();

  for (int k = 0; k < a.nst; ++k) {
    const int R = a.R[k], s = a.S[k], n = 2 * R + 1;
    // An odd step (s = 1, the last stage only): the candidates of each column
    // parity form a step-2 grid; each block stages one half window per parity
    // (set sg: columns u = 2j + sg, dx = centre + u - R) into the space of the
    // union window, which no later stage reads.
    const bool odd = ODD && (s & 1);
    if (odd) {
      // a short load batch: the lanes' current rows are live here
      for (int b = 0; b < NB; ++b)
        for (int sg = 0; sg < 2; ++sg)
          stage_window<NT, 2, true>(win + (b * 2 + sg) * L.SSZ, L.SP, L.SWW, L.SR,
                                    tx0 + (b % T) * B + scx[b] - R + sg, ty0 + (b / T) * B + scy[b] - R, ref, a.W,
                                    a.H, a.pitch);
      __syncthreads();
    }
    const int hs = odd ? 1 : s >> 1;          // words between an item's columns
    const int nset = odd ? 2 : 1;
    const int ncol = odd ? R + 1 : n;         // columns of set 0 (set 1: R)
    const int nchunk = (ncol + kUC - 1) / kUC;
    const bool narrow = ncol <= 3;            // 3-column items (e.g. the fine stage, R = 1 or 2)
    // the block's stage window: window row of block row 0 and word of candidate column 0
    const int r0 = L.reach - R * s + (scy[mb] - cy0) + (mb / T) * B;
    const int w0 = ((L.reach - R * s + (scx[mb] - cx0)) >> 1) + (mb % T) * BW;
    uint64_t best = kInvalidKey;
    if constexpr (SMALL) {
      // items (set sg, candidate-row pair p, columns u0 .. u0 + 8) of all four blocks; a lane
      // past the last candidate row recomputes the last one and keeps nothing
      const int npair = (n + 1) >> 1;
      for (int it = warp; it < nset * npair * nchunk; it += NW) {
        const int sg = ODD ? it / (npair * nchunk) : 0, rem = it - sg * npair * nchunk;
        const int vp = rem / nchunk, u0 = (rem - vp * nchunk) * kUC;
        const int v = 2 * vp + svv, ve = min(v, n - 1);
        const uint32_t* wsrc = odd ? win + (mb * 2 + sg) * L.SSZ : win;
        uint32_t sad[kUC];
        const int row = (odd ? 0 : r0) + ve * s + rl, wb = (odd ? 0 : w0) + u0 * hs;
        if (narrow) {
          c2f_item_hs<KR, RS, BW, 3>(hs, wsrc, odd ? L.SP : L.P, row, wb, cr, ws, csum, sad);
#pragma unroll
          for (int u = 0; u < 3; ++u) {
            sad[u] += __shfl_xor_sync(0xffffffffu, sad[u], 2);
            sad[u] += __shfl_xor_sync(0xffffffffu, sad[u], 1);
          }
        } else {
          c2f_item_hs<KR, RS, BW>(hs, wsrc, odd ? L.SP : L.P, row, wb, cr, ws, csum, sad);
#pragma unroll
          for (int u = 0; u < kUC; ++u) {
            sad[u] += __shfl_xor_sync(0xffffffffu, sad[u], 2);
            sad[u] += __shfl_xor_sync(0xffffffffu, sad[u], 1);
          }
        }
        const int dy = scy[mb] + (v - R) * s, cnt = odd ? ncol - sg : n;
        const bool row_ok = v < n && valid && abs(dy) <= a.lim && y0 + dy >= 0 && y0 + dy + bh <= a.H;
#pragma unroll
        for (int u = 0; u < kUC; ++u) {
          const int dx = scx[mb] + (odd ? 2 * (u0 + u) + sg - R : (u0 + u - R) * s);
          if ((u & 3) == rl && row_ok && u0 + u < cnt && (u < 3 || !narrow) && abs(dx) <= a.lim && x0 + dx >= 0 &&
              x0 + dx + B <= a.W) {
            const uint64_t key = make_key(sad[u], dx, dy);
            best = key < best ? key : best;
          }
        }
      }
      // the block's eight lanes
#pragma unroll
      for (int o = 4; o >= 1; o >>= 1) {
        const uint64_t other = __shfl_xor_sync(0xffffffffu, best, o);
        best = other < best ? other : best;
      }
      if ((lane & 7) == 0 && best != kInvalidKey) atomicMin(&sbest[mb], (unsigned long long)best);
    } else {
      // items (set sg, candidate row v, columns u0 .. u0 + 8) of the warp's block, over its WPB
      // warps.  64-pixel blocks: where an even-step stage's last round would hold only a few
      // whole items (3 x their number <= WPB), those items run as three 3-column slices each
      // instead, all in one round (a slice costs about 37 % of a whole item)
      if (valid) {
        const int wi = warp - mb * WPB, pi = PAIRED ? wi % NPAIR : wi;
        const int nitems = nset * n * nchunk;
        const int full = SLICE ? nitems / WPB * WPB : nitems;
        const bool sliced = SLICE && !odd && !narrow && nitems > full && 3 * (nitems - full) <= WPB;
        const int nwork = sliced ? full + 3 * (nitems - full) : nitems;
        int parity = 0;
        for (int it = pi; it < nwork; it += (PAIRED ? NPAIR : WPB), parity ^= 1) {
          const bool sl = sliced && it >= full;
          const int ti = sl ? full + (it - full) / 3 : it;  // the whole item
          const int sg = ODD ? ti / (n * nchunk) : 0, rem = ti - sg * n * nchunk;
          const int v = rem / nchunk, u0 = (rem - v * nchunk) * kUC + (sl ? 3 * ((it - full) % 3) : 0);
          const bool n3 = sl || narrow;  // a 3-column item
          const int nc = n3 ? 3 : kUC;
          const uint32_t* wsrc = odd ? win + (mb * 2 + sg) * L.SSZ : win;
          const int wp = odd ? L.SP : L.P;
          const int row = (odd ? 0 : r0) + v * s + rl, wb = (odd ? 0 : w0) + u0 * hs;
          uint32_t sad[kUC];
          uint32_t mine = 0;
          if (n3) {
            c2f_item_hs<KR, RS, BW, 3>(hs, wsrc, wp, row, wb, cr, ws, csum, sad);
#pragma unroll
            for (int u = 0; u < 3; ++u) {
              const uint32_t tot = __reduce_add_sync(0xffffffffu, sad[u]);
              if (lane == u) mine = tot;
            }
          } else {
            c2f_item_hs<KR, RS, BW>(hs, wsrc, wp, row, wb, cr, ws, csum, sad);
#pragma unroll
            for (int u = 0; u < kUC; ++u) {
              const uint32_t tot = __reduce_add_sync(0xffffffffu, sad[u]);
              if (lane == u) mine = tot;
            }
          }
          if constexpr (PAIRED) {
            // both warps of the pair run the same items; the parity buffers let the second
            // warp write the next item's sums while the first still reads these
            if (hb == 1 && lane < kUC) xsum[pi][parity][lane] = mine;
            asm volatile("bar.sync %0, 64;" ::"r"(1 + pi) : "memory");
            if (hb == 1) continue;
            mine += xsum[pi][parity][lane & 15];
          }
          // lane u: candidate column u0 + u of the set
          const int dx = scx[mb] + (odd ? 2 * (u0 + lane) + sg - R : (u0 + lane - R) * s);
          const int dy = scy[mb] + (v - R) * s, cnt = odd ? ncol - sg : n;
          if (lane < nc && u0 + lane < cnt && abs(dx) <= a.lim && abs(dy) <= a.lim && x0 + dx >= 0 &&
              x0 + dx + B <= a.W && y0 + dy >= 0 && y0 + dy + bh <= a.H) {
            const uint64_t key = make_key(mine, dx, dy);
            best = key < best ? key : best;
          }
        }
      }
      best = warp_min_u64(best);
      if (lane == 0 && best != kInvalidKey) atomicMin(&sbest[mb], (unsigned long long)best);
    }
    __syncthreads();
    if (threadIdx.x < NB && sbest[threadIdx.x] != kInvalidKey) {
      const bayer_mv_t m = key_to_mv(sbest[threadIdx.x]);
      scx[threadIdx.x] = m.dx;
      scy[threadIdx.x] = m.dy;
      if (k + 1 < a.nst) sbest[threadIdx.x] = kInvalidKey;  // the last stage's minimum stays for the output
    }
    __syncthreads();  // centres and bests are reused by the next stage
  }
  if (threadIdx.x < NB) {
    const int b = threadIdx.x;
    const int obx = blockIdx.x * T + (b % T), oby = blockIdx.y * T + (b / T);
    if (obx < a.w && oby < a.h) {
      bayer_mv_t m;
      if (sbest[b] == kInvalidKey) {
        m.dx = 0;
        m.dy = 0;
        m.sad = 0xFFFFFFFFu;
      } else {
        m = key_to_mv(sbest[b]);
      }
      a.out[((long long)pair * a.h + oby) * a.w + obx] = m;
    }
  }
}

template <int B, int T, int NW, bool PAIRED, bool ODD, bool CLIP>
cudaError_t c2f_launch_kc(const GenericArgs& a, int batch, const C2FLevel& L, cudaStream_t st) {
  auto kern = me_c2f_kernel<B, T, NW, PAIRED, ODD, CLIP>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, L.smem);
  if (e != cudaSuccess) return e;
  kern<<<dim3((a.w + T - 1) / T, (a.h + T - 1) / T, batch), NW * 32, L.smem, st>>>(a, L);
  return cudaGetLastError();
}

template <int B, int T, int NW, bool PAIRED, bool ODD>
cudaError_t c2f_launch_k(const GenericArgs& a, int batch, const C2FLevel& L, cudaStream_t st) {
  return (a.H % B) ? c2f_launch_kc<B, T, NW, PAIRED, ODD, true>(a, batch, L, st)
                   : c2f_launch_kc<B, T, NW, PAIRED, ODD, false>(a, batch, L, st);
}

// Every level runs the same stages, so only a step-1 last stage yields odd
// centres: such pyramids take the ODD kernels.
template <int B, int T, int NW, bool PAIRED = false>
cudaError_t c2f_launch(const GenericArgs& a, int batch, const C2FLevel& L, cudaStream_t st) {
  return (a.S[a.nst - 1] & 1) ? c2f_launch_k<B, T, NW, PAIRED, true>(a, batch, L, st)
                              : c2f_launch_k<B, T, NW, PAIRED, false>(a, batch, L, st);
}

bool plan(const GenericArgs& a, int T, C2FLevel* L) {
  *L = C2FLevel{};
  const int last = a.nst - 1;
  for (int k = 0; k < a.nst; ++k)
    if (!(a.S[k] & 1)) L->reach += a.R[k] * a.S[k];
  L->rows = T * a.B + 2 * L->reach;
  L->WWu = (T * a.B + 2 * L->reach) / 2;
  L->P = L->WWu | 1;  // odd pitch
  // the window, then 64 words of padding (an item's unused columns read up to
  // 32 words past the window)
  long long words = (long long)L->rows * L->P + 64;
  if (a.S[last] & 1) {
    // an odd-step last stage: two half windows per block, each padded like the window,
    // in the same space
    const int R = a.R[last];
    L->SR = a.B + 2 * R;
    L->SWW = a.B / 2 + R;
    L->SP = L->SWW | 1;
    L->SSZ = L->SR * L->SP + 64;
    const long long halves = (long long)T * T * 2 * L->SSZ;
    words = halves > words ? halves : words;
  }
  const long long bytes = words * 4;
  if (bytes > 220 * 1024) return false;
  L->smem = (int)bytes;
  return true;
}

}  // namespace

// The packed C2F level kernel serves levels of 8-, 16-, 32- or 64-pixel
// blocks on frames whose width is a multiple of the block (the last block row
// may be clipped by the frame height), with steps 2, 4 or 8 (and step 1 in the
// last stage: the RAW phase's fine stage), any start centre, 16-byte aligned
// frames, and a union window that fits shared memory; returns
// cudaErrorNotSupported otherwise
// (the caller then runs the generic kernel).  8-, 16- and 32-pixel levels
// take 2 x 2 tiles where the tile's blocks share a start centre (level 0, or
// a parent block that is a multiple of twice their size); without one, 32-pixel
// levels take one block per CTA and 8- and 16-pixel levels the generic kernel.
cudaError_t launch_c2f_level(const GenericArgs& a, int batch, cudaStream_t st) {
  if (a.B != 8 && a.B != 16 && a.B != 32 && a.B != 64) return cudaErrorNotSupported;
  if (a.center_mode == 2 || a.W % a.B) return cudaErrorNotSupported;
  if ((reinterpret_cast<uintptr_t>(a.ref) % 16) || (reinterpret_cast<uintptr_t>(a.cur) % 16) || a.pitch % 8 ||
      a.ref_bs % 8 || a.cur_bs % 8)
    return cudaErrorNotSupported;
  for (int k = 0; k < a.nst; ++k)
    if (a.S[k] != 2 && a.S[k] != 4 && a.S[k] != 8 && !(a.S[k] == 1 && k == a.nst - 1)) return cudaErrorNotSupported;
  const bool shared_centre = a.center_mode == 0 || (a.parent_B % (2 * a.B) == 0);
  C2FLevel L{};
  if (a.B <= 16) {
    if (!shared_centre || !plan(a, 2, &L)) return cudaErrorNotSupported;
    return a.B == 16 ? c2f_launch<16, 2, 8>(a, batch, L, st) : c2f_launch<8, 2, 8>(a, batch, L, st);
  }
  if (a.B == 64) {
    if (!plan(a, 1, &L)) return cudaErrorNotSupported;
    // a stage of n candidate rows is n (n <= 9) or more items of the block:
    // with n <= 9 everywhere, two warp pairs on half-block items split them
    // more evenly than eight warps on whole-block ones
    int nmax = 0;
    for (int k = 0; k < a.nst; ++k) nmax = 2 * a.R[k] + 1 > nmax ? 2 * a.R[k] + 1 : nmax;
    return nmax <= kUC ? c2f_launch<64, 1, 4, true>(a, batch, L, st) : c2f_launch<64, 1, 8>(a, batch, L, st);
  }
  // 32-pixel blocks: a 2 x 2 tile (two warps per block, one shared window)
  // where the blocks share a start centre, else one block per CTA
  if (shared_centre && plan(a, 2, &L)) return c2f_launch<32, 2, 8>(a, batch, L, st);
  if (!plan(a, 1, &L)) return cudaErrorNotSupported;
  return c2f_launch<32, 1, 8>(a, batch, L, st);
}

}  // namespace bme

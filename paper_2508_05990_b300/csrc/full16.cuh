// Exhaustive EVEN-phase search of 16x16 blocks: shared-memory plan, strip
// staging, window column sums and the per-warp block search, used by the
// strip kernel, the list-mode kernel (me_full16.cu) and the multi-stream
// search kernel (multistream.cu).  See me_full16.cu for the mapping.
//
// Packed pixel pairs.  Shared memory holds the frames' own layout: one 32-bit
// word = two horizontally adjacent 12-bit samples, the even column in the low
// half, so staging is a plain copy.  An EVEN offset moves a candidate by two
// pixels = one word, so word j of a current-block row always meets word k + j
// of the window row of candidate column k: whole pairs against whole pairs.
//
// SAD through the minimum (Sec. 3.2 "Matching Criterion" defines the SAD;
// this is an exact rewriting of it): |a - b| = a + b - 2 min(a, b), so
//   SAD(k) = sum(current block) + sum(window of k) - 2 * sum min(cur, win).
// min.u16x2 takes both halves' minima in one instruction, dp2a.lo with byte
// weights (2, 2) adds twice their sum to a 32-bit accumulator in another: one
// instruction per pixel-candidate at the issue rate, where sad.u32 needs one
// per pixel-candidate on the half-rate integer pipe.  The window sums come
// from a table of 16-row column sums at every even row offset, built once per
// window; a 16-row sum of 12-bit samples (<= 65520) stays inside its half.
#pragma once

#include "common.cuh"

namespace bme {

constexpr uint32_t kW11 = 0x0101u;  // dp2a byte weights (1, 1): lo + hi
constexpr uint32_t kW22 = 0x0202u;  // (2, 2): 2 * (lo + hi)

// Row pitch in words for rows of `words` words: a multiple of 4 whose quotient
// by 4 is odd, so rows 2v + r read by lanes v at one column hit distinct
// 16-byte bank groups (with the row rotation of half the lanes).
__host__ __device__ constexpr int pitch4odd(int words) {
  return ((words + 3) / 4) % 2 == 0 ? (words + 3) / 4 * 4 + 4 : (words + 3) / 4 * 4;
}

// Shared-memory plan of a strip of NW horizontally adjacent blocks (one warp
// each), in 32-bit words: the union of their search windows (WIN_H rows of WW
// words, pitch P), their current blocks (16 rows of 8 * NW words, pitch PC)
// and the window's column-sum table (NU rows of WW words, pitch P).
template <int R, int NW>
struct Full16Strip {
  static constexpr int NU = 2 * R + 1;         // candidates per row, and rows
  static constexpr int REACH = 2 * R;          // pixels each side
  static constexpr int WIN_W = 16 * NW + 2 * REACH;  // pixels
  static constexpr int WIN_H = 16 + 2 * REACH;
  static constexpr int WW = WIN_W / 2;         // words per window row
  static constexpr int P = pitch4odd(WW);
  static constexpr int PC = 8 * NW + 4;        // 4 * (2 NW + 1)
  static constexpr int SPANW = 8 + REACH;      // window words one block reads per row
  static constexpr int CUR_OFF = WIN_H * P;
  static constexpr int CS_OFF = CUR_OFF + 16 * PC;
  // TMA staging: the window as one box 2P pixels wide (its rows land at pitch
  // P), the current tile as one box 2PC pixels wide; both complete on one
  // mbarrier after the column-sum table
  static constexpr int BOX_W = 2 * P, CUR_BOX_W = 2 * PC;
  static constexpr uint32_t TX_BYTES = (uint32_t)(WIN_H * P + 16 * PC) * 4u;
  static constexpr int MBAR_OFF = (CS_OFF + NU * P + 1) / 2 * 2;  // 8-byte aligned
  static constexpr size_t SMEM = (size_t)MBAR_OFF * sizeof(uint32_t) + sizeof(uint64_t);
  static_assert(NU <= 33, "at most 33 candidate rows");
  static_assert(SPANW % 4 == 0, "R must be even (128-bit window loads)");
  static_assert((CUR_OFF * 4) % 128 == 0, "current tile 128-byte aligned (TMA destination)");
  static_assert(BOX_W <= 256 && CUR_BOX_W <= 256, "TMA box at most 256 elements wide");
};

// Accumulators of one lane: its candidate row (NU candidates), and for
// R = 16 the lane's candidate of the 33rd row and its share of the corner.
// During the row loop they hold 2 * sum min(cur, win); full16_finish turns
// them into SADs.
template <int R>
struct Full16Acc {
  static constexpr int NU = 2 * R + 1;
  uint32_t acc[NU];
  uint32_t accx, accc;
};

// cs[v * P + w] = sum of window rows 2v .. 2v + bh - 1 at word column w, both
// halves at once, for v = 0 .. 2R; bh (even, 2..16) is the block height: 16,
// or the rows left in a frame whose height is not a multiple of 16 (the last
// block row is clipped to the frame, and its SAD covers only those rows).
// Called by NT threads (index tid) after the window is staged; the caller
// synchronises before and after.  Two threads per column, each running a
// bh-row sum down half of the offsets (the 32-bit running sum is exact modulo
// 2^32, and its final halves each fit 16 bits).
template <int R, int P, int WW, int NT>
__device__ __forceinline__ void window_colsums(const uint32_t* win, uint32_t* cs, int tid, int bh = 16) {
  constexpr int NU = 2 * R + 1, HALF = (NU + 1) / 2;
  const int tail = (bh - 2) * P;  // the rows entering a sum that moves down by two
  for (int e = tid; e < 2 * WW; e += NT) {
    const int part = e >= WW, w = e - part * WW;
    const int v0 = part ? HALF : 0, v1 = part ? NU : HALF;
    const uint32_t* col = win + w;
    uint32_t s = 0;
#pragma unroll
    for (int r = 0; r < 16; ++r)
      if (r < bh) s += col[(2 * v0 + r) * P];
    cs[v0 * P + w] = s;
    for (int v = v0 + 1; v < v1; ++v) {
      s += col[2 * v * P + tail] + col[2 * v * P + tail + P];
      s -= col[(2 * v - 2) * P] + col[(2 * v - 1) * P];
      cs[v * P + w] = s;
    }
  }
}

// A lane's window sums gathered during the row loop (the variant without a
// column-sum table): per window word of its candidate row, the 16-row column
// sum -- the first half of the words packed (each half <= 65520, plain
// adds on the integer pipe), the rest as lo + hi (dp2a on the FMA pipe), so
// the extra work splits over both pipes -- and for R = 16 the window sum of
// its 33rd-row candidate and its share of the corner's.
template <int R>
struct Full16WinSums {
  static constexpr int SPANW = 8 + 2 * R;
  uint32_t cw[SPANW];
  uint32_t sx, scn;
};

// 2 * sum min(cur, win) of one 16x16 block against every candidate,
// accumulated by one warp from a staged window (wbase: the block's window
// origin, row pitch P words) and current block (cbase, row pitch PC words).
// Lane v owns candidate row v (lanes past the last row repeat it).  With
// SUMS the lane also gathers its window sums into S.  With CLIP the loop
// runs over the block's bh rows only (a last block row clipped by the frame),
// so that the window sums cover the rows the SAD covers.
template <int R, int P, int PC, bool SUMS = false, bool CLIP = false>
__device__ __forceinline__ void full16_accumulate(const uint32_t* wbase, const uint32_t* cbase, int lane,
                                                  Full16Acc<R>& A, Full16WinSums<R>& S, int bh = 16) {
  constexpr int NU = 2 * R + 1, SPANW = 8 + 2 * R;
  const int v = lane < NU ? lane : NU - 1;
  const int eps = (lane >> 2) & 1;  // row rotation for conflict-free loads

#pragma unroll
  for (int k = 0; k < NU; ++k) A.acc[k] = 0;
  A.accx = 0;
  A.accc = 0;
  if constexpr (SUMS) {
#pragma unroll
    for (int w = 0; w < SPANW; ++w) S.cw[w] = 0;
    S.sx = 0;
    S.scn = 0;
  }

  const int rows = CLIP ? bh : 16;
#pragma unroll 1
  for (int i = 0; i < rows; ++i) {
    int r;
    if constexpr (CLIP) {
      r = i + eps;
      r = r >= bh ? r - bh : r;
    } else {
      r = (i + eps) & 15;
    }
    uint32_t c[8];
    const uint4* cp = reinterpret_cast<const uint4*>(cbase + r * PC);
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const uint4 t = cp[q];
      c[4 * q + 0] = t.x;
      c[4 * q + 1] = t.y;
      c[4 * q + 2] = t.z;
      c[4 * q + 3] = t.w;
    }
    const uint4* wp = reinterpret_cast<const uint4*>(wbase + (2 * v + r) * P);
#pragma unroll
    for (int q = 0; q < SPANW / 4; ++q) {
      const uint4 t = wp[q];
      const uint32_t rr[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        const int w = 4 * q + s;
#pragma unroll
        for (int k = 0; k < NU; ++k) {
          const int j = w - k;
          if (j >= 0 && j < 8) A.acc[k] = dp2a_lo(min_u16x2(rr[s], c[j]), kW22, A.acc[k]);
        }
        if constexpr (SUMS) {
          if (w < SPANW / 2) S.cw[w] += rr[s];
          else S.cw[w] = dp2a_lo(rr[s], kW11, S.cw[w]);
        }
      }
    }
    if constexpr (NU == 33) {
      // row v = 32: candidate u = lane, window words lane .. lane + 7
      const uint32_t* xp = wbase + (64 + r) * P + lane;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const uint32_t x = xp[j];
        A.accx = dp2a_lo(min_u16x2(x, c[j]), kW22, A.accx);
        if constexpr (SUMS) S.sx = dp2a_lo(x, kW11, S.sx);
      }
      // corner candidate (u, v) = (32, 32): lane l < 8 takes word column l
      if (lane < 8) {
        const uint32_t x = wbase[(64 + r) * P + 32 + lane];
        A.accc = dp2a_lo(min_u16x2(x, cbase[r * PC + lane]), kW22, A.accc);
        if constexpr (SUMS) S.scn = dp2a_lo(x, kW11, S.scn);
      }
    }
  }
}

// The current block's sum (all lanes get it): lane l adds words
// 4 (l & 1) .. + 3 of row l / 2.
template <int PC>
__device__ __forceinline__ uint32_t block_sum(const uint32_t* cbase, int lane) {
  const uint4 t = *reinterpret_cast<const uint4*>(cbase + (lane >> 1) * PC + 4 * (lane & 1));
  const uint32_t sc = dp2a_lo(t.x, kW11, dp2a_lo(t.y, kW11, dp2a_lo(t.z, kW11, dp2a_lo(t.w, kW11, 0u))));
  return __reduce_add_sync(0xffffffffu, sc);
}

// full16_finish from the lane's own window sums (no table).
template <int R, int PC>
__device__ __forceinline__ void full16_finish_sums(const Full16WinSums<R>& S, const uint32_t* cbase, int lane,
                                                   Full16Acc<R>& A) {
  constexpr int NU = 2 * R + 1, SPANW = 8 + 2 * R;
  const uint32_t sc = block_sum<PC>(cbase, lane);
  uint32_t T[SPANW];
#pragma unroll
  for (int w = 0; w < SPANW; ++w) T[w] = w < SPANW / 2 ? dp2a_lo(S.cw[w], kW11, 0u) : S.cw[w];
  uint32_t s = 0;
#pragma unroll
  for (int j = 0; j < 8; ++j) s += T[j];
#pragma unroll
  for (int k = 0; k < NU; ++k) {
    if (k > 0) s += T[k + 7] - T[k - 1];
    A.acc[k] = sc + s - A.acc[k];
  }
  if constexpr (NU == 33) {
    A.accx = sc + S.sx - A.accx;
    const uint32_t part = lane < 8 ? S.scn - A.accc : 0u;
    A.accc = lane == 0 ? part + sc : part;
  }
}

// SAD = sum(cur) + sum(win) - 2 sum min: turns the accumulators into SADs.
// csbase: the column-sum table at the block's window origin (pitch P words);
// cbase: the block's current words (pitch PC).  The corner's SAD is the warp
// sum of accc afterwards.
template <int R, int P, int PC>
__device__ __forceinline__ void full16_finish(const uint32_t* csbase, const uint32_t* cbase, int lane,
                                              Full16Acc<R>& A) {
  constexpr int NU = 2 * R + 1, SPANW = 8 + 2 * R;
  const int v = lane < NU ? lane : NU - 1;
  const uint32_t sc = block_sum<PC>(cbase, lane);
  // window sums of row v: a sliding sum of 8 words along the column sums
  uint32_t T[SPANW];
  const uint4* cr = reinterpret_cast<const uint4*>(csbase + v * P);
#pragma unroll
  for (int q = 0; q < SPANW / 4; ++q) {
    const uint4 u = cr[q];
    T[4 * q + 0] = dp2a_lo(u.x, kW11, 0u);
    T[4 * q + 1] = dp2a_lo(u.y, kW11, 0u);
    T[4 * q + 2] = dp2a_lo(u.z, kW11, 0u);
    T[4 * q + 3] = dp2a_lo(u.w, kW11, 0u);
  }
  uint32_t s = 0;
#pragma unroll
  for (int j = 0; j < 8; ++j) s += T[j];
#pragma unroll
  for (int k = 0; k < NU; ++k) {
    if (k > 0) s += T[k + 7] - T[k - 1];
    A.acc[k] = sc + s - A.acc[k];
  }
  if constexpr (NU == 33) {
    const uint32_t* c32 = csbase + 32 * P;
    uint32_t sx = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) sx = dp2a_lo(c32[lane + j], kW11, sx);
    A.accx = sc + sx - A.accx;
    uint32_t part = lane < 8 ? dp2a_lo(c32[32 + lane], kW11, 0u) - A.accc : 0u;
    A.accc = lane == 0 ? part + sc : part;
  }
}

// The lane's best key (sad, |mv|_1, dy, dx) from its SADs; the warp minimum
// of the returned keys is the block's MV.  (xb, yb): the block's top-left
// pixel, bh its height (clipped to the frame), for the validity of
// out-of-frame candidates.
template <int R>
__device__ __forceinline__ uint64_t full16_select(const Full16Acc<R>& A, int lane, int xb, int yb, int W, int H,
                                                  int bh = 16) {
  constexpr int NU = 2 * R + 1, REACH = 2 * R;
  const int v = lane < NU ? lane : NU - 1;
  const int dy = 2 * v - REACH;
  uint64_t best = kInvalidKey;
  const bool interior = xb >= REACH && xb + 16 + REACH <= W && yb >= REACH && yb + bh + REACH <= H;
  if (interior) {
    // Every candidate is valid.  Within a lane dy is fixed, so the tie-break
    // (|dx|+|dy|, dy, dx) orders the row by rank = 0 for dx = 0, then -2, +2,
    // -4, +4, ...; sad * 64 + rank is a 32-bit key (sad < 2^25, rank <= 32).
    uint32_t m = 0xFFFFFFFFu;
#pragma unroll
    for (int k = 0; k < NU; ++k) {
      const uint32_t rank = k == R ? 0u : (k < R ? (uint32_t)(2 * (R - k) - 1) : (uint32_t)(2 * (k - R)));
      const uint32_t key = A.acc[k] * 64u + rank;
      m = key < m ? key : m;
    }
    const uint32_t rank = m & 63u;
    const int k = rank == 0 ? R : ((rank & 1u) ? R - (int)((rank + 1) >> 1) : R + (int)(rank >> 1));
    if (lane < NU) best = make_key(m >> 6, 2 * k - REACH, dy);
  } else {
    const bool row_ok = lane < NU && yb + dy >= 0 && yb + dy + bh <= H;
#pragma unroll
    for (int k = 0; k < NU; ++k) {
      const int dx = 2 * k - REACH;
      const bool ok = row_ok && xb + dx >= 0 && xb + dx + 16 <= W;
      const uint64_t key = ok ? make_key(A.acc[k], dx, dy) : kInvalidKey;
      best = key < best ? key : best;
    }
  }
  if constexpr (NU == 33) {
    {
      const int dx = 2 * lane - REACH;
      const bool ok = yb + 32 + bh <= H && xb + dx >= 0 && xb + dx + 16 <= W;
      const uint64_t key = ok ? make_key(A.accx, dx, 32) : kInvalidKey;
      best = key < best ? key : best;
    }
    const uint32_t corner = __reduce_add_sync(0xffffffffu, A.accc);
    if (lane == 0 && xb + 48 <= W && yb + 32 + bh <= H) {
      const uint64_t key = make_key(corner, 32, 32);
      best = key < best ? key : best;
    }
  }
  return best;
}

// Every candidate of one 16x16 block, by one warp: wbase / csbase are the
// window and its column-sum table at the block's origin (pitch P words),
// cbase its current words (pitch PC); returns the lane's best key.  A block
// clipped to bh < 16 rows has zero current rows below bh (min(win, 0) = 0
// adds nothing) and a table of bh-row sums.
template <int R, int P, int PC>
__device__ __forceinline__ uint64_t full16_block(const uint32_t* wbase, const uint32_t* csbase, const uint32_t* cbase,
                                                 int lane, int xb, int yb, int W, int H, int bh = 16) {
  Full16Acc<R> A;
  Full16WinSums<R> unused;
  full16_accumulate<R, P, PC, false>(wbase, cbase, lane, A, unused);
  full16_finish<R, P, PC>(csbase, cbase, lane, A);
  return full16_select<R>(A, lane, xb, yb, W, H, bh);
}

// A word of two samples (gx, gx + 1) of row gy, out-of-frame samples 0.
__device__ __forceinline__ uint32_t pair_word(const uint16_t* __restrict__ f, int W, int H, int pitch, int gx, int gy) {
  if (gy < 0 || gy >= H) return 0u;
  const uint16_t* row = f + (long long)gy * pitch;
  const uint32_t lo = (gx >= 0 && gx < W) ? (uint32_t)__ldg(row + gx) : 0u;
  const uint32_t hi = (gx + 1 >= 0 && gx + 1 < W) ? (uint32_t)__ldg(row + gx + 1) : 0u;
  return lo | (hi << 16);
}

// Stage the window and current tile of the strip whose first block is at
// (x0, y0) as packed pairs: 8 pixels per 16-byte load when vec_ok (x0 a
// multiple of 8, W a multiple of 16, rows 16-byte aligned), all loads of a
// thread in flight before the first store; out-of-frame samples are 0 (also
// the current rows below the frame of a clipped last block row).
// Called by all NW*32 threads.
template <int R, int NW>
__device__ __forceinline__ void stage_strip(const uint16_t* __restrict__ ref, const uint16_t* __restrict__ cur, int W,
                                            int H, int pitch, int x0, int y0, bool vec_ok, uint32_t* win,
                                            uint32_t* curt) {
  using C = Full16Strip<R, NW>;
  constexpr int kNT = NW * 32;
  if (vec_ok) {
    // The window origin x0 - 2R and the tile origin x0 are multiples of 8 and
    // W is a multiple of 16, so every 8-pixel chunk lies wholly inside or
    // wholly outside the frame.
    constexpr int WCH = C::WIN_W / 8, NWCH = WCH * C::WIN_H;
    constexpr int TCH = 2 * NW, NTCH = TCH * 16;
    constexpr int PER = (NWCH + NTCH + kNT - 1) / kNT;
    uint4 raw[PER];
#pragma unroll
    for (int i = 0; i < PER; ++i) {
      const int e = threadIdx.x + i * kNT;
      raw[i] = make_uint4(0, 0, 0, 0);
      if (e < NWCH) {
        const int ry = e / WCH, cx = e - ry * WCH;
        const int gy = y0 - C::REACH + ry, gx = x0 - C::REACH + 8 * cx;
        if (gy >= 0 && gy < H && gx >= 0 && gx < W)
          raw[i] = __ldg(reinterpret_cast<const uint4*>(ref + (long long)gy * pitch + gx));
      } else if (e < NWCH + NTCH) {
        const int f = e - NWCH, ry = f / TCH, cx = f - ry * TCH;
        const int gx = x0 + 8 * cx;
        if (gx < W && y0 + ry < H)
          raw[i] = __ldg(reinterpret_cast<const uint4*>(cur + (long long)(y0 + ry) * pitch + gx));
      }
    }
#pragma unroll
    for (int i = 0; i < PER; ++i) {
      const int e = threadIdx.x + i * kNT;
      if (e < NWCH) {
        const int ry = e / WCH, cx = e - ry * WCH;
        *reinterpret_cast<uint4*>(win + ry * C::P + 4 * cx) = raw[i];
      } else if (e < NWCH + NTCH) {
        const int f = e - NWCH, ry = f / TCH, cx = f - ry * TCH;
        *reinterpret_cast<uint4*>(curt + ry * C::PC + 4 * cx) = raw[i];
      }
    }
  } else {
    for (int e = threadIdx.x; e < C::WIN_H * C::WW; e += kNT) {
      const int ry = e / C::WW, wx = e - ry * C::WW;
      win[ry * C::P + wx] = pair_word(ref, W, H, pitch, x0 - C::REACH + 2 * wx, y0 - C::REACH + ry);
    }
    for (int e = threadIdx.x; e < 16 * 8 * NW; e += kNT) {
      const int ry = e / (8 * NW), wx = e - ry * (8 * NW);
      curt[ry * C::PC + wx] = pair_word(cur, W, H, pitch, x0 + 2 * wx, y0 + ry);
    }
  }
}

}  // namespace bme

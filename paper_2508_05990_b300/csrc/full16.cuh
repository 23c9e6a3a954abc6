// Exhaustive EVEN-phase search of 16x16 blocks: shared-memory plan, strip
// staging and the per-warp block search, used by the strip kernel, the
// list-mode kernel (me_full16.cu) and the multi-stream persistent kernel
// (multistream.cu).  See me_full16.cu for the mapping.
#pragma once

#include "common.cuh"

namespace bme {

// Shared-memory plan of a strip of NW horizontally adjacent blocks (one warp
// each): the union of their search windows (WIN_W x WIN_H pixels, row pitch P
// words = 4 * odd) and their current blocks (16 rows, pitch PC words).
template <int R, int NW>
struct Full16Strip {
  static constexpr int NU = 2 * R + 1;         // candidates per row
  static constexpr int REACH = 2 * R;          // pixels each side
  static constexpr int WIN_W = 16 * NW + 2 * REACH;
  static constexpr int WIN_H = 16 + 2 * REACH;
  static constexpr int P0 = (WIN_W + 3) / 4 * 4;
  static constexpr int P = ((P0 / 4) % 2 == 0) ? P0 + 4 : P0;  // 4 * odd words
  static constexpr int PC = 16 * NW + 4;       // current-tile pitch (words)
  static constexpr int SPAN = 16 + 2 * REACH;  // window pixels one block reads per row
  static constexpr size_t SMEM = (size_t)(WIN_H * P + 16 * PC) * sizeof(uint32_t);
  static_assert(NU <= 33, "at most 33 candidate rows");
  static_assert(SPAN % 4 == 0, "span must be a multiple of 4 words");
};

// Accumulators of one lane: its candidate row (NU candidates), and for
// R = 16 the lane's candidate of the 33rd row and its share of the corner.
template <int R>
struct Full16Acc {
  static constexpr int NU = 2 * R + 1;
  uint32_t acc[NU];
  uint32_t accx, accc;
};

// SADs of block rows RB .. RB + NRW - 1 of one 16x16 block against every
// candidate, accumulated by one warp from a staged window (wbase: the block's
// window origin, row pitch P words) and current block (cbase, row pitch PC
// words).  Lane v owns candidate row v (lanes past the last row repeat it).
template <int R, int P, int PC, int RB, int NRW>
__device__ __forceinline__ void full16_accumulate(const uint32_t* wbase, const uint32_t* cbase, int lane,
                                                  Full16Acc<R>& A) {
  constexpr int NU = 2 * R + 1, REACH = 2 * R, SPAN = 16 + 2 * REACH;
  static_assert(NRW == 4 || NRW == 8 || NRW == 16, "row ranges of 4, 8 or 16");
  const int v = lane < NU ? lane : NU - 1;
  const int eps = (lane >> 2) & 1;  // row rotation for conflict-free loads

#pragma unroll
  for (int k = 0; k < NU; ++k) A.acc[k] = 0;
  A.accx = 0;
  A.accc = 0;

#pragma unroll 1
  for (int i = 0; i < NRW; ++i) {
    const int r = RB + ((i + eps) & (NRW - 1));
    uint32_t c[16];
    const uint4* cp = reinterpret_cast<const uint4*>(cbase + r * PC);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const uint4 t = cp[q];
      c[4 * q + 0] = t.x;
      c[4 * q + 1] = t.y;
      c[4 * q + 2] = t.z;
      c[4 * q + 3] = t.w;
    }
    const uint4* wp = reinterpret_cast<const uint4*>(wbase + (2 * v + r) * P);
#pragma unroll
    for (int q = 0; q < SPAN / 4; ++q) {
      const uint4 t = wp[q];
      const uint32_t rr[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        const int p = 4 * q + s;
#pragma unroll
        for (int k = 0; k < NU; ++k) {
          const int cc = p - 2 * k;
          if (cc >= 0 && cc < 16) A.acc[k] = sad_u32(rr[s], c[cc], A.acc[k]);
        }
      }
    }
    if constexpr (NU == 33) {
      // row v = 32: candidate u = lane at window pixel 2*lane
      const uint2* xp = reinterpret_cast<const uint2*>(wbase + (64 + r) * P + 2 * lane);
#pragma unroll
      for (int t2 = 0; t2 < 8; ++t2) {
        const uint2 e2 = xp[t2];
        A.accx = sad_u32(e2.x, c[2 * t2], A.accx);
        A.accx = sad_u32(e2.y, c[2 * t2 + 1], A.accx);
      }
      // corner candidate (u, v) = (32, 32): lane l < 16 takes column l
      if (lane < 16) A.accc = sad_u32(wbase[(64 + r) * P + 64 + lane], cbase[r * PC + lane], A.accc);
    }
  }
}

// The lane's best key (sad, |mv|_1, dy, dx) from its complete accumulators;
// the warp minimum of the returned keys is the block's MV.  (xb, yb): the
// block's top-left pixel, for the validity of out-of-frame candidates.
template <int R>
__device__ __forceinline__ uint64_t full16_select(const Full16Acc<R>& A, int lane, int xb, int yb, int W, int H) {
  constexpr int NU = 2 * R + 1, REACH = 2 * R;
  const int v = lane < NU ? lane : NU - 1;
  const int dy = 2 * v - REACH;
  uint64_t best = kInvalidKey;
  const bool interior = xb >= REACH && xb + 16 + REACH <= W && yb >= REACH && yb + 16 + REACH <= H;
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
    const bool row_ok = lane < NU && yb + dy >= 0 && yb + dy + 16 <= H;
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
      const bool ok = yb + 48 <= H && xb + dx >= 0 && xb + dx + 16 <= W;
      const uint64_t key = ok ? make_key(A.accx, dx, 32) : kInvalidKey;
      best = key < best ? key : best;
    }
    const uint32_t corner = __reduce_add_sync(0xffffffffu, A.accc);
    if (lane == 0 && xb + 48 <= W && yb + 48 <= H) {
      const uint64_t key = make_key(corner, 32, 32);
      best = key < best ? key : best;
    }
  }
  return best;
}

// SAD of every candidate of one 16x16 block, computed by one warp from a
// staged window (wbase: the block's window origin, row pitch P words) and
// current block (cbase, row pitch PC words); returns the lane's best key.
template <int R, int P, int PC>
__device__ __forceinline__ uint64_t full16_block(const uint32_t* wbase, const uint32_t* cbase, int lane, int xb, int yb,
                                                 int W, int H) {
  Full16Acc<R> A;
  full16_accumulate<R, P, PC, 0, 16>(wbase, cbase, lane, A);
  return full16_select<R>(A, lane, xb, yb, W, H);
}

// Stage the window and current tile of the strip whose first block is at
// (x0, y0): 8 pixels per 16-byte load when vec_ok (x0 a multiple of 8, W a
// multiple of 16, rows 16-byte aligned), all loads of a thread in flight
// before conversion; out-of-frame samples are 0.  Called by all NW*32 threads.
template <int R, int NW>
__device__ __forceinline__ void stage_strip(const uint16_t* __restrict__ ref, const uint16_t* __restrict__ cur, int W,
                                            int H, int pitch, int x0, int y0, bool vec_ok, uint32_t* win,
                                            uint32_t* curt) {
  using C = Full16Strip<R, NW>;
  constexpr int kNW = NW;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (vec_ok) {
    // 8 pixels (16 bytes) per load: the window origin x0 - 2R and the tile
    // origin x0 are multiples of 8 and W is a multiple of 16, so every 8-pixel
    // chunk lies wholly inside or wholly outside the frame.  All loads of a
    // thread are issued before any conversion.
    constexpr int WCH = C::WIN_W / 8, NWCH = WCH * C::WIN_H;
    constexpr int TCH = 2 * kNW, NTCH = TCH * 16;
    constexpr int PER = (NWCH + NTCH + kNW * 32 - 1) / (kNW * 32);
    uint4 raw[PER];
#pragma unroll
    for (int i = 0; i < PER; ++i) {
      const int e = threadIdx.x + i * kNW * 32;
      raw[i] = make_uint4(0, 0, 0, 0);
      if (e < NWCH) {
        const int ry = e / WCH, cx = e - ry * WCH;
        const int gy = y0 - C::REACH + ry, gx = x0 - C::REACH + 8 * cx;
        if (gy >= 0 && gy < H && gx >= 0 && gx < W)
          raw[i] = __ldg(reinterpret_cast<const uint4*>(ref + (long long)gy * pitch + gx));
      } else if (e < NWCH + NTCH) {
        const int f = e - NWCH, ry = f / TCH, cx = f - ry * TCH;
        const int gx = x0 + 8 * cx;
        if (gx < W) raw[i] = __ldg(reinterpret_cast<const uint4*>(cur + (long long)(y0 + ry) * pitch + gx));
      }
    }
#pragma unroll
    for (int i = 0; i < PER; ++i) {
      const int e = threadIdx.x + i * kNW * 32;
      uint32_t* dst;
      if (e < NWCH) {
        const int ry = e / WCH, cx = e - ry * WCH;
        dst = win + ry * C::P + 8 * cx;
      } else if (e < NWCH + NTCH) {
        const int f = e - NWCH, ry = f / TCH, cx = f - ry * TCH;
        dst = curt + ry * C::PC + 8 * cx;
      } else {
        continue;
      }
      reinterpret_cast<uint4*>(dst)[0] = make_uint4(pix_lo(raw[i].x), pix_hi(raw[i].x), pix_lo(raw[i].y), pix_hi(raw[i].y));
      reinterpret_cast<uint4*>(dst)[1] = make_uint4(pix_lo(raw[i].z), pix_hi(raw[i].z), pix_lo(raw[i].w), pix_hi(raw[i].w));
    }
  } else {
    for (int ry = warp; ry < C::WIN_H; ry += kNW) {
      const int gy = y0 - C::REACH + ry;
      const bool row_in = gy >= 0 && gy < H;
      for (int rx = lane; rx < C::WIN_W; rx += 32) {
        const int gx = x0 - C::REACH + rx;
        uint32_t v = 0;
        if (row_in && gx >= 0 && gx < W) v = __ldg(ref + (long long)gy * pitch + gx);
        win[ry * C::P + rx] = pix_word(v);
      }
    }
    for (int ry = warp; ry < 16; ry += kNW) {
      const int gy = y0 + ry;
      for (int rx = lane; rx < 16 * kNW; rx += 32) {
        const int gx = x0 + rx;
        uint32_t v = 0;
        if (gy < H && gx < W) v = __ldg(cur + (long long)gy * pitch + gx);
        curt[ry * C::PC + rx] = pix_word(v);
      }
    }
  }
}

}  // namespace bme

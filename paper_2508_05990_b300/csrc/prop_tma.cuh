// NCHW bilinear propagation of one tile through shared memory (Sec. 3.3),
// shared by the batched propagation kernel (propagate.cu) and the
// multi-stream propagation kernel (multistream.cu).
//
// A CTA of kTT + 32 threads owns a tile of kTQY x kTQX quads (16 x 64 cells)
// and up to kTC channels of one map, with two or more feature cells per block
// side (the quad's four cells share one MV).  Per channel a TMA tile load
// stages the tile's source region -- the tile grown by kHalo cells on every
// side plus one more row and column for the second bilinear tap (25 x 76
// floats) -- into a ring of kNS buffers, so kNS channels' loads are in flight
// at once.  At the map's borders the load reads zeros outside; a tap row or
// column outside the map reads the staged edge row or column instead (its
// index clamped to the staged rows and columns inside the map, once per
// quad), which is the clamped element of the map.  Every quad whose integer
// MV offsets lie within +-kHalo cells takes its nine taps from the buffer:
// the same clamped elements as warp_quad reads from global memory, blended in
// the same order, so the output is the same bit for bit; a quad with a larger
// offset reads its taps from global memory (warp_quad).  Each warp covers one
// quad row of the tile: a channel's stores are 256-byte rows.  A ninth warp's
// lane 0 is the producer: it issues the loads and refills a buffer once all
// 256 quads have read their taps from it (an "empty" mbarrier of 256 arrivals
// per buffer; a "full" one completes with the load's bytes).  Every mbarrier
// wait is bounded (on expiry: BAYER_ERR_TIMEOUT and the thread stops; a
// consumer that stops leaves its buffer unreleased, so the producer's wait
// for it expires too).
#pragma once

#include "common.cuh"
#include "kernels.cuh"
#include "prop_common.cuh"
#include "tc_common.cuh"
#include "tma.cuh"

namespace bme {
namespace prop {

constexpr int kTQY = 8, kTQX = 32;             // quads per tile (rows, columns)
constexpr int kHalo = 4;                       // cells: +-32 pixels at stride 8
constexpr int kRH = 2 * kTQY + 2 * kHalo + 1;  // 25 staged rows
constexpr int kRW = 2 * kTQX + 2 * kHalo + 1;  // 73 staged columns
constexpr int kBW = (kRW + 3) / 4 * 4;         // 76: the box width (16-byte rows)
constexpr int kTT = kTQY * kTQX;               // 256 consumer threads
constexpr int kTileThreads = kTT + 32;         // + the producer warp
constexpr int kTC = 16;                        // channels per tile
constexpr int kNS = 6;                         // staging buffers
constexpr int kTileH = 2 * kTQY, kTileW = 2 * kTQX;  // tile size in cells
constexpr uint32_t kBoxBytes = kRH * kBW * 4;
constexpr int kBufF = (kBoxBytes + 127) / 128 * 32;  // floats per buffer: 128-byte aligned buffers
constexpr uint32_t kPropWait = 1u << 22;

struct TileStage {
  float buf[kNS][kBufF];
  uint64_t full[kNS], empty[kNS];
};

// One tile's work.  `tm` maps the planes of a stack of Hf x Wf float32
// planes (box kBW x kRH x 1); `feat` and `out` point at plane 0 of the input
// and output stacks; the tile covers planes plane0 .. plane0 + nc - 1 and
// cells [y0, y0 + kTileH) x [x0, x0 + kTileW); `mv` is the MV field of the
// map (mv_w blocks per row, 2^lc cells per block side, stride 2^ls).
// `map_in_global`: the tensor map lies in global memory, written before the
// launch, so the producer orders its reads after those writes first.
struct TileJob {
  const CUtensorMap* tm;
  const float* feat;
  float* out;
  const bayer_mv_t* mv;
  int mv_w;
  int Hf, Wf, ls, lc;
  int plane0, nc;
  int y0, x0;
  int* status;
  bool map_in_global;
};

// Run by all kTileThreads threads of the CTA (it holds a __syncthreads after
// the barrier set-up); returns in every thread, also after a timeout.
__device__ __forceinline__ void tma_tile(TileStage& s, const TileJob& j) {
  const int tid = threadIdx.x;
  const long long cells = (long long)j.Hf * j.Wf;

  if (tid == 0) {
    for (int i = 0; i < kNS; ++i) {
      tc::mbar_init(&s.full[i], 1);
      tc::mbar_init(&s.empty[i], kTT);
    }
    tc::fence_mbar_init();
  }
  __syncthreads();

  if (tid >= kTT) {
    // producer warp: one lane refills each buffer once its kTT readers are done
    if (tid == kTT) {
      if (j.map_in_global) tma::fence_map_acquire(j.tm);
      for (int c = 0; c < j.nc; ++c) {
        const int sl = c % kNS;
        if (c >= kNS && !tc::mbar_wait(&s.empty[sl], (uint32_t)(((c - kNS) / kNS) & 1), kPropWait)) {
          if (j.status) atomicExch(j.status, (int)BAYER_ERR_TIMEOUT);
          break;
        }
        tma::mbar_arrive_expect_tx(&s.full[sl], kBoxBytes);
        tma::load_3d(s.buf[sl], j.tm, j.x0 - kHalo, j.y0 - kHalo, j.plane0 + c, &s.full[sl]);
      }
    }
    return;
  }

  // this thread's quad
  const int qy = tid / kTQX, qx = tid - qy * kTQX;
  const int fy = j.y0 + 2 * qy, fx = j.x0 + 2 * qx;
  const bool live = fy < j.Hf && fx < j.Wf;
  bayer_mv_t mv{};
  if (live) mv = j.mv[(long long)(fy >> j.lc) * j.mv_w + (fx >> j.lc)];
  const Taps tp = bilinear_taps(j.ls, j.Hf, j.Wf, fy, fx, mv);
  const int oy = (int)mv.dy >> j.ls, ox = (int)mv.dx >> j.ls;
  const bool near = oy >= -kHalo && oy <= kHalo && ox >= -kHalo && ox <= kHalo;
  const bool row2 = fy + 1 < j.Hf, col2 = fx + 1 < j.Wf;
  const bool pair_store = col2 && (j.Wf & 1) == 0;
  // the staged rows [top, bot) and columns [lft, rgt) lie inside the map; a tap
  // outside them reads the nearest one inside, which is the clamped element
  const int top = max(0, kHalo - j.y0), bot = min(kRH, j.Hf - (j.y0 - kHalo));
  const int lft = max(0, kHalo - j.x0), rgt = min(kRW, j.Wf - (j.x0 - kHalo));
  int tr[3], tcol[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    tr[i] = clampi(2 * qy + oy + kHalo + i, top, bot - 1) * kBW;
    tcol[i] = clampi(2 * qx + ox + kHalo + i, lft, rgt - 1);
  }

  for (int c = 0; c < j.nc; ++c) {
    const int sl = c % kNS;
    const float* bf = s.buf[sl];
    if (!tc::mbar_wait(&s.full[sl], (uint32_t)((c / kNS) & 1), kPropWait)) {
      if (j.status) atomicExch(j.status, (int)BAYER_ERR_TIMEOUT);
      return;
    }
    if (live) {
      float* o = j.out + (long long)(j.plane0 + c) * cells + (long long)fy * j.Wf + fx;
      if (near) {
        float v[9];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
          for (int k = 0; k < 3; ++k) v[3 * i + k] = bf[tr[i] + tcol[k]];
        tc::mbar_arrive(&s.empty[sl]);  // the taps are in registers: the buffer may refill
        const float r00 = blend(tp, v[0], v[1], v[3], v[4]), r01 = blend(tp, v[1], v[2], v[4], v[5]);
        const float r10 = blend(tp, v[3], v[4], v[6], v[7]), r11 = blend(tp, v[4], v[5], v[7], v[8]);
        if (pair_store) {
          __stcs(reinterpret_cast<float2*>(o), make_float2(r00, r01));
          if (row2) __stcs(reinterpret_cast<float2*>(o + j.Wf), make_float2(r10, r11));
        } else {
          __stcs(o, r00);
          if (col2) __stcs(o + 1, r01);
          if (row2) {
            __stcs(o + j.Wf, r10);
            if (col2) __stcs(o + j.Wf + 1, r11);
          }
        }
        continue;
      }
      tc::mbar_arrive(&s.empty[sl]);
      warp_quad<1>(j.feat + (long long)(j.plane0 + c) * cells, j.out + (long long)(j.plane0 + c) * cells, cells, j.Hf,
                   j.Wf, j.ls, fy, fx, mv, 1);
    } else {
      tc::mbar_arrive(&s.empty[sl]);
    }
  }
}

}  // namespace prop
}  // namespace bme

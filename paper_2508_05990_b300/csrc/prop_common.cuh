// Propagation arithmetic shared by the propagation kernels (propagate.cu)
// and the multi-stream kernel (multistream.cu): Warp(z_R, MV) sampling
// positions and the fixed-order bilinear blend (Sec. 3.3).
#pragma once

#include "common.cuh"
#include "kernels.cuh"

namespace bme {
namespace prop {

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

// The feature stride s divides the block size (8, 16, 32 or 64), so s and the
// cells per block side are powers of two: with ls = log2(s), floor(a / s) is
// a >> ls, its remainder a & (s - 1), and r / s = r * 2^-ls exactly (the same
// bits as the rounded quotient).

// round(a / s), halves away from zero
__device__ __forceinline__ int rounddiv_pow2(int a, int ls) {
  return a >= 0 ? (2 * a + (1 << ls)) >> (ls + 1) : -((-2 * a + (1 << ls)) >> (ls + 1));
}

struct Taps {
  int y0, y1, x0, x1;
  float wy, wx, owy, owx;
};

__device__ __forceinline__ Taps bilinear_taps(int ls, int Hf, int Wf, int fy, int fx, bayer_mv_t m) {
  Taps t;
  const int qy = (int)m.dy >> ls, qx = (int)m.dx >> ls;
  const float inv_s = __int_as_float((127 - ls) << 23);  // 2^-ls
  t.wy = __fmul_rn((float)((int)m.dy & ((1 << ls) - 1)), inv_s);
  t.wx = __fmul_rn((float)((int)m.dx & ((1 << ls) - 1)), inv_s);
  t.owy = __fsub_rn(1.0f, t.wy);
  t.owx = __fsub_rn(1.0f, t.wx);
  t.y0 = clampi(fy + qy, 0, Hf - 1);
  t.y1 = clampi(fy + qy + 1, 0, Hf - 1);
  t.x0 = clampi(fx + qx, 0, Wf - 1);
  t.x1 = clampi(fx + qx + 1, 0, Wf - 1);
  return t;
}

__device__ __forceinline__ float blend(const Taps& t, float va, float vb, float vc, float vd) {
  const float top = __fadd_rn(__fmul_rn(t.owx, va), __fmul_rn(t.wx, vb));
  const float bot = __fadd_rn(__fmul_rn(t.owx, vc), __fmul_rn(t.wx, vd));
  return __fadd_rn(__fmul_rn(t.owy, top), __fmul_rn(t.wy, bot));
}

// BILINEAR warp of the 2 x 2 quad of cells with top-left cell (fy, fx) --
// fy, fx even, the four cells inside one block and sharing its MV -- for
// nc <= NCMAX channels of an NCHW map: `in` and `out` point at the first
// channel's plane, planes `cells` floats apart.  The quad's 16 taps are the
// 3 x 3 grid of rows y0..y0+2 and columns x0..x0+2, each clamped as for a
// single cell, so every output is bit for bit bilinear_taps / blend of its
// cell: 9 loads per channel for 4 outputs.  Cells past the map edge are not
// stored; float2 stores where the quad is whole and Wf is even.
template <int NCMAX>
__device__ __forceinline__ void warp_quad(const float* __restrict__ in, float* __restrict__ out, long long cells,
                                          int Hf, int Wf, int ls, int fy, int fx, bayer_mv_t mv, int nc) {
  const Taps tp = bilinear_taps(ls, Hf, Wf, fy, fx, mv);
  const int oy = (int)mv.dy >> ls, ox = (int)mv.dx >> ls;
  int ry[3], rx[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    ry[i] = clampi(fy + oy + i, 0, Hf - 1) * Wf;
    rx[i] = clampi(fx + ox + i, 0, Wf - 1);
  }
  float* o0 = out + (long long)fy * Wf + fx;
  const bool row2 = fy + 1 < Hf, col2 = fx + 1 < Wf;
  const bool pair_store = col2 && (Wf & 1) == 0;
#pragma unroll
  for (int c = 0; c < NCMAX; ++c) {
    if (c >= nc) break;
    const float* pl = in + (long long)c * cells;
    float v[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) v[3 * i + j] = __ldg(pl + ry[i] + rx[j]);
    const float r00 = blend(tp, v[0], v[1], v[3], v[4]), r01 = blend(tp, v[1], v[2], v[4], v[5]);
    const float r10 = blend(tp, v[3], v[4], v[6], v[7]), r11 = blend(tp, v[4], v[5], v[7], v[8]);
    float* o = o0 + (long long)c * cells;
    if (pair_store) {
      __stcs(reinterpret_cast<float2*>(o), make_float2(r00, r01));
      if (row2) __stcs(reinterpret_cast<float2*>(o + Wf), make_float2(r10, r11));
    } else {
      __stcs(o, r00);
      if (col2) __stcs(o + 1, r01);
      if (row2) {
        __stcs(o + Wf, r10);
        if (col2) __stcs(o + Wf + 1, r11);
      }
    }
  }
}

}  // namespace prop
}  // namespace bme

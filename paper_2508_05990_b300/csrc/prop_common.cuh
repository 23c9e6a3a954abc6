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

}  // namespace prop
}  // namespace bme

// Propagation arithmetic shared by the propagation kernels (propagate.cu)
// and the multi-stream kernel (multistream.cu): Warp(z_R, MV) sampling
// positions and the fixed-order bilinear blend (Sec. 3.3).
#pragma once

#include "common.cuh"
#include "kernels.cuh"

namespace bme {
namespace prop {

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

__device__ __forceinline__ int floordiv(int a, int b) {
  int q = a / b;
  if ((a % b != 0) && (a < 0)) --q;
  return q;
}

__device__ __forceinline__ int rounddiv(int a, int b) {
  return a >= 0 ? (2 * a + b) / (2 * b) : -((2 * (-a) + b) / (2 * b));
}

struct Taps {
  int y0, y1, x0, x1;
  float wy, wx, owy, owx;
};

__device__ __forceinline__ Taps bilinear_taps(int s, int Hf, int Wf, int fy, int fx, bayer_mv_t m) {
  Taps t;
  const int qy = floordiv(m.dy, s), qx = floordiv(m.dx, s);
  t.wy = __fdiv_rn((float)(m.dy - qy * s), (float)s);
  t.wx = __fdiv_rn((float)(m.dx - qx * s), (float)s);
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

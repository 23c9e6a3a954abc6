// Motion-vector feature propagation z_pred = Warp(z_R, MV) (Sec. 3.3).
//
// Feature cell (fy, fx) takes the MV of the block holding raw pixel
// (fy*s, fx*s) and samples z_R at (fy + dy/s, fx + dx/s).  NEAREST rounds the
// offsets half away from zero (a pure copy, bit-exact); BILINEAR evaluates
//   (1-wy)*((1-wx)*a + wx*b) + wy*((1-wx)*c + wx*d)
// with every product and sum rounded separately (__fmul_rn/__fadd_rn), so the
// result is reproducible bit for bit by any IEEE float evaluation in the same
// order.  Indices are clamped to the map.
//
// HBM-bound: per map C*Hf*Wf*4 bytes read once and written once.
//   NCHW: bilinear with two or more cells per block side -- one thread per
//         2 x 2 quad of cells (they share the MV: 9 tap loads per channel for
//         4 outputs) and chunk of 4 channels; otherwise one thread per cell and
//         chunk of 8 channels.
//   NHWC: one thread per (cell, 4 channels) of a feature row moves float4
//         vectors (taps are contiguous C-vectors), fully coalesced.
// Stride and cells per block are powers of two: all index divisions by them
// are shifts.
#include "common.cuh"
#include "kernels.cuh"
#include "prop_common.cuh"
#include "prop_tma.cuh"
#include "tc_common.cuh"
#include "tma.cuh"

namespace bme {

namespace {

using namespace prop;

// NCHW: one thread per output cell (fy, fx) and chunk of kCK channels
// (grid.y = map x channel chunk).  The MV lookup and tap arithmetic are paid
// once per chunk; all kCK x 4 tap loads are issued before any arithmetic, and
// each plane's store is a coalesced warp row.
constexpr int kCK = 8;

template <int INTERP>
__global__ void __launch_bounds__(256) prop_nchw_kernel(const PropArgs a, int nchunks) {
  const int cells = a.Hf * a.Wf;
  const int cell = blockIdx.x * blockDim.x + threadIdx.x;
  if (cell >= cells) return;
  const int m = blockIdx.y / nchunks;
  const int c0 = (blockIdx.y - m * nchunks) * kCK;
  const int fy = cell / a.Wf, fx = cell - fy * a.Wf;
  const bayer_mv_t mv = a.mv[((long long)m * a.mv_h + (fy >> a.lc)) * a.mv_w + (fx >> a.lc)];
  const float* in = a.feat + ((long long)m * a.C + c0) * cells;
  float* out = a.out + ((long long)m * a.C + c0) * cells + cell;
  const int nc = min(kCK, a.C - c0);
  if (INTERP == BAYER_INTERP_NEAREST) {
    const int sy = clampi(fy + rounddiv_pow2(mv.dy, a.ls), 0, a.Hf - 1);
    const int sx = clampi(fx + rounddiv_pow2(mv.dx, a.ls), 0, a.Wf - 1);
    const float* src = in + sy * a.Wf + sx;
    if (nc == kCK) {
      float v[kCK];
#pragma unroll
      for (int c = 0; c < kCK; ++c) v[c] = __ldg(src + (long long)c * cells);
#pragma unroll
      for (int c = 0; c < kCK; ++c) __stcs(out + (long long)c * cells, v[c]);
    } else {
      for (int c = 0; c < nc; ++c) __stcs(out + (long long)c * cells, __ldg(src + (long long)c * cells));
    }
  } else {
    const Taps tp = bilinear_taps(a.ls, a.Hf, a.Wf, fy, fx, mv);
    const int oa = tp.y0 * a.Wf + tp.x0, ob = tp.y0 * a.Wf + tp.x1;
    const int oc = tp.y1 * a.Wf + tp.x0, od = tp.y1 * a.Wf + tp.x1;
    if (nc == kCK) {
      float va[kCK], vb[kCK], vc[kCK], vd[kCK];
#pragma unroll
      for (int c = 0; c < kCK; ++c) {
        const float* pl = in + (long long)c * cells;
        va[c] = __ldg(pl + oa);
        vb[c] = __ldg(pl + ob);
        vc[c] = __ldg(pl + oc);
        vd[c] = __ldg(pl + od);
      }
#pragma unroll
      for (int c = 0; c < kCK; ++c) __stcs(out + (long long)c * cells, blend(tp, va[c], vb[c], vc[c], vd[c]));
    } else {
      for (int c = 0; c < nc; ++c) {
        const float* pl = in + (long long)c * cells;
        __stcs(out + (long long)c * cells, blend(tp, __ldg(pl + oa), __ldg(pl + ob), __ldg(pl + oc), __ldg(pl + od)));
      }
    }
  }
}

// NCHW bilinear, two or more feature cells per block side: one thread per
// 2 x 2 quad of cells (fy, fx even) and chunk of kQK channels.  The quad's
// cells share one MV, so their 16 taps are the 3 x 3 grid rows y0..y0+2 x
// columns x0..x0+2 (each clamped exactly as for a single cell): 9 loads per
// channel instead of 16, and each output row pair is a float2 store where
// the quad is whole and Wf is even.  Warps run along quad rows.
constexpr int kQK = 4;
constexpr int kQT = 128;

__global__ void __launch_bounds__(kQT) prop_nchw_quad_kernel(const PropArgs a, int nchunks, int qw, int nquads) {
  const int q = blockIdx.x * kQT + threadIdx.x;
  if (q >= nquads) return;
  const long long cells = (long long)a.Hf * a.Wf;
  const int m = blockIdx.y / nchunks;
  const int c0 = (blockIdx.y - m * nchunks) * kQK;
  const int qy = q / qw, qx = q - qy * qw;
  const int fy = 2 * qy, fx = 2 * qx;
  const bayer_mv_t mv = a.mv[((long long)m * a.mv_h + (fy >> a.lc)) * a.mv_w + (fx >> a.lc)];
  const long long base = ((long long)m * a.C + c0) * cells;
  warp_quad<kQK>(a.feat + base, a.out + base, cells, a.Hf, a.Wf, a.ls, fy, fx, mv, min(kQK, a.C - c0));
}

// NCHW bilinear, two or more cells per block side, through shared memory:
// one CTA per tile of 16 x 64 cells and kTC channels of one map (grid.z =
// map x channel chunk), the tile staged by TMA loads (prop_tma.cuh).
__global__ void __launch_bounds__(kTileThreads) prop_nchw_tma_kernel(const __grid_constant__ CUtensorMap tm,
                                                                      const PropArgs a, int nchunks) {
  __shared__ __align__(128) TileStage stage;
  const int m = blockIdx.z / nchunks;
  const int c0 = (blockIdx.z - m * nchunks) * kTC;
  TileJob j;
  j.tm = &tm;
  j.feat = a.feat;
  j.out = a.out;
  j.mv = a.mv + (long long)m * a.mv_h * a.mv_w;
  j.mv_w = a.mv_w;
  j.Hf = a.Hf;
  j.Wf = a.Wf;
  j.ls = a.ls;
  j.lc = a.lc;
  j.plane0 = m * a.C + c0;
  j.nc = min(kTC, a.C - c0);
  j.y0 = blockIdx.y * kTileH;
  j.x0 = blockIdx.x * kTileW;
  j.status = a.status;
  j.map_in_global = false;
  tma_tile(stage, j);
}

// NHWC with C % 4 == 0: one thread per (cell, 4 channels) of one feature row
// (grid.x = row's float4 vectors / 256, grid.y = fy, grid.z = map); c4n =
// C / 4 float4 vectors per cell, lc4 = log2(c4n) when that is a power of two
// (else -1: divide).
template <int INTERP>
__global__ void __launch_bounds__(256) prop_nhwc4_kernel(const PropArgs a, int c4n, int lc4) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= a.Wf * c4n) return;
  const int fy = blockIdx.y, m = blockIdx.z;
  const int fx = lc4 >= 0 ? t >> lc4 : t / c4n;
  const int c4 = t - fx * c4n;
  const bayer_mv_t mv = a.mv[((long long)m * a.mv_h + (fy >> a.lc)) * a.mv_w + (fx >> a.lc)];
  const float4* in = reinterpret_cast<const float4*>(a.feat) + (long long)m * a.Hf * a.Wf * c4n + c4;
  float4* out = reinterpret_cast<float4*>(a.out) + ((long long)m * a.Hf + fy) * a.Wf * c4n + t;
  if (INTERP == BAYER_INTERP_NEAREST) {
    const int sy = clampi(fy + rounddiv_pow2(mv.dy, a.ls), 0, a.Hf - 1);
    const int sx = clampi(fx + rounddiv_pow2(mv.dx, a.ls), 0, a.Wf - 1);
    __stcs(out, __ldg(in + (long long)(sy * a.Wf + sx) * c4n));
  } else {
    const Taps tp = bilinear_taps(a.ls, a.Hf, a.Wf, fy, fx, mv);
    const float4 va = __ldg(in + (long long)(tp.y0 * a.Wf + tp.x0) * c4n);
    const float4 vb = __ldg(in + (long long)(tp.y0 * a.Wf + tp.x1) * c4n);
    const float4 vc = __ldg(in + (long long)(tp.y1 * a.Wf + tp.x0) * c4n);
    const float4 vd = __ldg(in + (long long)(tp.y1 * a.Wf + tp.x1) * c4n);
    float4 r;
    r.x = blend(tp, va.x, vb.x, vc.x, vd.x);
    r.y = blend(tp, va.y, vb.y, vc.y, vd.y);
    r.z = blend(tp, va.z, vb.z, vc.z, vd.z);
    r.w = blend(tp, va.w, vb.w, vc.w, vd.w);
    __stcs(out, r);
  }
}

// NHWC with C % 4 == 0, bilinear, two or more cells per block side: one
// thread per (2 x 2 quad of cells, 4 channels) of a quad row (grid.x = the
// row's quads x float4 vectors / 256, grid.y = quad row, grid.z = map).  The
// quad's cells share one MV, so their 16 taps are the 3 x 3 grid of rows
// y0 .. y0 + 2 and columns x0 .. x0 + 2, each clamped as for a single cell:
// 9 float4 loads for 4 outputs, every output bit for bit bilinear_taps /
// blend of its cell (as in warp_quad); a warp's loads and stores are
// contiguous runs of the cells' channel vectors.
__global__ void __launch_bounds__(256) prop_nhwc4_quad_kernel(const PropArgs a, int c4n, int lc4, int qw) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= qw * c4n) return;
  const int m = blockIdx.z;
  const int qx = lc4 >= 0 ? t >> lc4 : t / c4n;
  const int c4 = t - qx * c4n;
  const int fy = 2 * blockIdx.y, fx = 2 * qx;
  const bayer_mv_t mv = a.mv[((long long)m * a.mv_h + (fy >> a.lc)) * a.mv_w + (fx >> a.lc)];
  const Taps tp = bilinear_taps(a.ls, a.Hf, a.Wf, fy, fx, mv);
  const int oy = (int)mv.dy >> a.ls, ox = (int)mv.dx >> a.ls;
  const float4* in = reinterpret_cast<const float4*>(a.feat) + (long long)m * a.Hf * a.Wf * c4n + c4;
  float4 v[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const long long row = (long long)clampi(fy + oy + i, 0, a.Hf - 1) * a.Wf;
#pragma unroll
    for (int j = 0; j < 3; ++j) v[i][j] = __ldg(in + (row + clampi(fx + ox + j, 0, a.Wf - 1)) * c4n);
  }
  auto quad_blend = [&](int i, int j) {
    float4 r;
    r.x = blend(tp, v[i][j].x, v[i][j + 1].x, v[i + 1][j].x, v[i + 1][j + 1].x);
    r.y = blend(tp, v[i][j].y, v[i][j + 1].y, v[i + 1][j].y, v[i + 1][j + 1].y);
    r.z = blend(tp, v[i][j].z, v[i][j + 1].z, v[i + 1][j].z, v[i + 1][j + 1].z);
    r.w = blend(tp, v[i][j].w, v[i][j + 1].w, v[i + 1][j].w, v[i + 1][j + 1].w);
    return r;
  };
  float4* out = reinterpret_cast<float4*>(a.out) + (((long long)m * a.Hf + fy) * a.Wf + fx) * c4n + c4;
  const bool row2 = fy + 1 < a.Hf, col2 = fx + 1 < a.Wf;
  __stcs(out, quad_blend(0, 0));
  if (col2) __stcs(out + c4n, quad_blend(0, 1));
  if (row2) {
    __stcs(out + (long long)a.Wf * c4n, quad_blend(1, 0));
    if (col2) __stcs(out + ((long long)a.Wf + 1) * c4n, quad_blend(1, 1));
  }
}

// NHWC, any C: one thread per (map, cell, channel).
template <int INTERP>
__global__ void __launch_bounds__(256) prop_nhwc1_kernel(const PropArgs a) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long cells = (long long)a.Hf * a.Wf;
  if (t >= (long long)a.n * cells * a.C) return;
  const int c = (int)(t % a.C);
  const long long cell = t / a.C;
  const int m = (int)(cell / cells);
  const int rem = (int)(cell - (long long)m * cells);
  const int fy = rem / a.Wf, fx = rem - fy * a.Wf;
  const bayer_mv_t mv = a.mv[((long long)m * a.mv_h + (fy >> a.lc)) * a.mv_w + (fx >> a.lc)];
  const float* in = a.feat + (long long)m * cells * a.C;
  if (INTERP == BAYER_INTERP_NEAREST) {
    const int sy = clampi(fy + rounddiv_pow2(mv.dy, a.ls), 0, a.Hf - 1);
    const int sx = clampi(fx + rounddiv_pow2(mv.dx, a.ls), 0, a.Wf - 1);
    a.out[t] = __ldg(in + ((long long)sy * a.Wf + sx) * a.C + c);
  } else {
    const Taps tp = bilinear_taps(a.ls, a.Hf, a.Wf, fy, fx, mv);
    a.out[t] = blend(tp, __ldg(in + ((long long)tp.y0 * a.Wf + tp.x0) * a.C + c),
                     __ldg(in + ((long long)tp.y0 * a.Wf + tp.x1) * a.C + c),
                     __ldg(in + ((long long)tp.y1 * a.Wf + tp.x0) * a.C + c),
                     __ldg(in + ((long long)tp.y1 * a.Wf + tp.x1) * a.C + c));
  }
}

inline int log2_exact(int v) {  // log2 of a power of two, else -1
  if (v <= 0 || (v & (v - 1))) return -1;
  int l = 0;
  while ((1 << l) < v) ++l;
  return l;
}

inline unsigned blocks_for(long long threads, int per) { return (unsigned)((threads + per - 1) / per); }

}  // namespace

cudaError_t launch_propagate(const PropArgs& args, int layout, int interp, cudaStream_t st) {
  PropArgs a = args;
  a.ls = log2_exact(a.s);
  a.lc = log2_exact(a.cells);
  if (a.ls < 0 || a.lc < 0) return cudaErrorInvalidValue;  // stride and block are powers of two
  const long long cells = (long long)a.n * a.Hf * a.Wf;
  if (cells == 0 || a.C == 0) return cudaSuccess;
  CUtensorMap tm{};
  if (layout == BAYER_LAYOUT_NCHW && interp == BAYER_INTERP_BILINEAR && a.lc >= 1 &&
      (long long)a.n * ((a.C + kTC - 1) / kTC) <= 65535 && (long long)a.n * a.C <= (1ll << 31) &&
      (long long)a.Hf * a.Wf <= (1ll << 31) - 256 &&
      tma::encode_f32_planes(&tm, a.feat, a.Wf, a.Hf, (long long)a.n * a.C, kBW, kRH)) {
    const int nchunks = (a.C + kTC - 1) / kTC;
    dim3 g((a.Wf + kTileW - 1) / kTileW, (a.Hf + kTileH - 1) / kTileH, a.n * nchunks);
    prop_nchw_tma_kernel<<<g, kTileThreads, 0, st>>>(tm, a, nchunks);
  } else if (layout == BAYER_LAYOUT_NCHW && interp == BAYER_INTERP_BILINEAR && a.lc >= 1 &&
             (long long)a.n * ((a.C + kQK - 1) / kQK) <= 65535 && (long long)a.Hf * a.Wf <= (1ll << 31) - 256) {
    const int nchunks = (a.C + kQK - 1) / kQK;
    const int qw = (a.Wf + 1) / 2, nquads = ((a.Hf + 1) / 2) * qw;
    dim3 g(blocks_for(nquads, kQT), a.n * nchunks);
    prop_nchw_quad_kernel<<<g, kQT, 0, st>>>(a, nchunks, qw, nquads);
  } else if (layout == BAYER_LAYOUT_NCHW) {
    const int nchunks = (a.C + kCK - 1) / kCK;
    if ((long long)a.n * nchunks > 65535 || (long long)a.Hf * a.Wf > (1ll << 31) - 256) return cudaErrorInvalidValue;
    dim3 g(blocks_for((long long)a.Hf * a.Wf, 256), a.n * nchunks);
    if (interp == BAYER_INTERP_NEAREST)
      prop_nchw_kernel<BAYER_INTERP_NEAREST><<<g, 256, 0, st>>>(a, nchunks);
    else
      prop_nchw_kernel<BAYER_INTERP_BILINEAR><<<g, 256, 0, st>>>(a, nchunks);
  } else if ((a.C & 3) == 0 && (reinterpret_cast<uintptr_t>(a.feat) & 15) == 0 &&
             (reinterpret_cast<uintptr_t>(a.out) & 15) == 0 && a.n <= 65535 && a.Hf <= 65535 &&
             (long long)a.Hf * a.Wf * (a.C >> 2) < (1ll << 31) - 256) {
    const int c4n = a.C >> 2;
    if (interp == BAYER_INTERP_BILINEAR && a.lc >= 1) {
      // quads: the cells of a 2 x 2 quad share their block's MV
      const int qw = (a.Wf + 1) / 2;
      dim3 g(blocks_for((long long)qw * c4n, 256), (a.Hf + 1) / 2, a.n);
      prop_nhwc4_quad_kernel<<<g, 256, 0, st>>>(a, c4n, log2_exact(c4n), qw);
    } else {
      dim3 g(blocks_for((long long)a.Wf * c4n, 256), a.Hf, a.n);
      if (interp == BAYER_INTERP_NEAREST)
        prop_nhwc4_kernel<BAYER_INTERP_NEAREST><<<g, 256, 0, st>>>(a, c4n, log2_exact(c4n));
      else
        prop_nhwc4_kernel<BAYER_INTERP_BILINEAR><<<g, 256, 0, st>>>(a, c4n, log2_exact(c4n));
    }
  } else {
    const unsigned g = blocks_for(cells * a.C, 256);
    if (interp == BAYER_INTERP_NEAREST)
      prop_nhwc1_kernel<BAYER_INTERP_NEAREST><<<g, 256, 0, st>>>(a);
    else
      prop_nhwc1_kernel<BAYER_INTERP_BILINEAR><<<g, 256, 0, st>>>(a);
  }
  return cudaGetLastError();
}

}  // namespace bme

// Backward of the proposal network's 3x3 stride-2 convolutions (zero pad 1,
// 32 output channels) on the 5th-generation tensor cores: BF16 operands in
// shared memory, FP32 accumulators in tensor memory.  The pre-activation
// gradients dpre (NHWC bf16, [batch][H][W][32]) are the operands, as the
// network's training definition stores them; weights and activations are the
// forward's bf16 values.
//
// Input gradient (layers 2..4), conv_dx_tc_kernel:
//   dpre_in[b, iy, ix, ci] = [x_in > 0] * sum_{ky, kx, co} w[co, ci, ky, kx] * dpre_out[b, oy, ox, co],
//   iy = 2 oy + ky - 1, ix = 2 ox + kx - 1.
// Input pixels split into four parity classes (iy % 2, ix % 2).  An even row
// takes ky = 1 from output row iy/2; an odd row ky = 0 from row (iy+1)/2 and
// ky = 2 from row (iy-1)/2; columns likewise.  So the class (py, px) pixels
// (2a + py, 2c + px), c = c0 .. c0+127, of one tile are a sum of 1, 2, 2 and 4
// taps, each an MMA of the staged output-gradient rows a and a+1 (A: 128
// pixels x 32 co, K-major, shifted by one pixel for the "+1" taps) with the
// tap's transposed weights (B: 32 ci x 32 co).  Four accumulators of 32 TMEM
// columns hold the four classes; the epilogue masks with the staged input
// activations, rounds to bf16 and writes two input rows x 256 columns.
//
// Weight gradient (all four layers), conv_dw_tc_kernel:
//   dW[co, ci, tap] = sum_{b, oy, ox} dpre_out[b, oy, ox, co] * x_in[b, iy, ix, ci],
//   db[co] = sum dpre_out[b, oy, ox, co],
// a GEMM with the output pixels as the reduction: D[k, co] = sum_p A[k, p] B[co, p]
// with k = tap * CIN + ci (M, 3 tiles of 128 rows for CIN = 32, 2 for layer
// 1's 16 operand channels) and the pixels as K.  Per chunk of 64 output
// pixels (one row segment) the patches (im2col: one 16-byte cell per pixel,
// tap and 8 channels) and the output gradients are staged MN-major -- the
// natural order of NHWC memory -- and the MMAs read them with the transpose
// bits of the instruction descriptor.  Row k = 9 * CIN of A holds 1.0 for
// every pixel, so row 9 * CIN of D is the bias gradient.  The copies of the
// next chunks are in flight while the MMAs of the current one run.  Each CTA
// accumulates a contiguous range of chunks in TMEM and adds its partial
// gradients to the output once.
// Layer 1's patches are the Bayer frames, split exactly as in the forward:
// channel 2c + h of a tap is the hi (h = 0) or lo (h = 1) part of input plane
// c, so dW1[co, c, tap] = D[hi] + D[lo] / 128, where each thread loads the
// samples of its patches (any alignment).  With 16-byte aligned frame rows the
// six raw rows and the output gradients of a chunk are copied whole (cp.async,
// two chunks ahead) and converted in shared memory to K-major TF32 operands
// instead: v/2048 - 1 has at most 11 significant bits, so TF32 holds it
// exactly, and the bf16 gradients widen exactly (kind::tf32 MMAs, products
// exact as well), at a quarter of the split's conversion work per sample.
//
// Every mbarrier wait is bounded; on expiry the kernel records
// BAYER_ERR_TIMEOUT in the status word, frees its TMEM and finishes.
#include <cuda_bf16.h>

#include "common.cuh"
#include "kernels.cuh"
#include "tc_common.cuh"

namespace bme {

namespace {

constexpr int kC = 32;                 // channels of every hidden map
constexpr uint32_t kWaitLimit = 1u << 20;

// ---------------------------------------------------------------------------
// input gradient
// ---------------------------------------------------------------------------

constexpr int kDxM = 128;                    // class pixels per tile (MMA M)
constexpr int kDxNP = kDxM + 1;              // staged output-gradient columns
constexpr int kDxWBytes = 9 * 4 * 4 * 128;   // transposed weights of one layer
constexpr int kDxDBytes = 2 * 4 * kDxNP * 16;  // two output-gradient rows
constexpr int kDxXBytes = 2 * 4 * 2 * kDxM * 16;  // two input-activation rows, 256 pixels
constexpr int kDxSmem = kDxWBytes + kDxDBytes + kDxXBytes + 64;
constexpr int kDxTmemCols = 128;
static_assert(kDxWBytes % 128 == 0 && kDxDBytes % 16 == 0 && kDxXBytes % 16 == 0, "alignment");

// Transposed weight images of layers 2..4 (B operand of the input gradient,
// K-major): element (n = ci, k = tap * 32 + co) = w[co, ci, tap] at
// (n/8) * (36*128) + (k/8) * 128 + (n%8) * 16 + (k%8) * 2.  One thread per
// element of the three images; image l - 2 at img + (l - 2) * kDxWBytes.
struct PackDxArgs {
  const __nv_bfloat16* w;
  int w_off[3];
};

__global__ void pack_dx_weights_kernel(const PackDxArgs pa, __nv_bfloat16* __restrict__ img) {
  constexpr int kL = kC * 9 * kC;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 3 * kL) return;
  const int l = i / kL, r = i - l * kL;
  const int n = r / (9 * kC), k = r - n * (9 * kC);
  const int tap = k / kC, co = k - tap * kC;
  const int off = l == 0 ? pa.w_off[0] : (l == 1 ? pa.w_off[1] : pa.w_off[2]);
  img[(l * kDxWBytes + (n >> 3) * (36 * 128) + (k >> 3) * 128 + (n & 7) * 16) / 2 + (k & 7)] =
      pa.w[off + (co * kC + n) * 9 + tap];
}

__global__ void __launch_bounds__(kDxM) conv_dx_tc_kernel(const ConvBwdArgs a) {
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* sW = smem;
  uint8_t* sD = smem + kDxWBytes;
  uint8_t* sX = sD + kDxDBytes;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(sX + kDxXBytes);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mbar + 1);
  const int tid = threadIdx.x, warp = tid >> 5;

  if (tid == 0) {
    tc::mbar_init(&mbar[0], 1);
    tc::fence_mbar_init();
  }
  if (warp == 0) tc::tmem_alloc(tmem_slot, kDxTmemCols);
  for (int i = tid; i < kDxWBytes / 16; i += kDxM) reinterpret_cast<uint4*>(sW)[i] = __ldg(a.wimg_t + i);
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tmem_slot;
  const uint32_t sW_addr = tc::smem_addr(sW), sD_addr = tc::smem_addr(sD), sX_addr = tc::smem_addr(sX);
  constexpr uint32_t idesc = tc::idesc_bf16_f32(kDxM, kC);
  const int segs = (a.Wo + kDxM - 1) / kDxM;
  const long long ntiles = (long long)a.batch * a.Ho * segs;
  uint32_t phase = 0;
  bool ok = true;

  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int seg = (int)(tile % segs);
    const long long row = tile / segs;
    const int b = (int)(row / a.Ho), ra = (int)(row - (long long)b * a.Ho);
    const int c0 = seg * kDxM;

    // ---- stage output-gradient rows ra, ra + 1, columns c0 .. c0 + 128 (zero
    // outside the map): cell (r, kc, p) at ((r*4 + kc)*NP + p)*16
    for (int it = tid; it < 2 * kDxNP * 4; it += kDxM) {
      const int kc = it & 3, rp = it >> 2;
      const int r = rp / kDxNP, p = rp - r * kDxNP;
      const int oy = ra + r, ox = c0 + p;
      const bool in = oy < a.Ho && ox < a.Wo;
      const __nv_bfloat16* src = in ? a.dout + (((long long)b * a.Ho + oy) * a.Wo + ox) * kC + kc * 8 : a.dout;
      tc::cp_async16(sD_addr + ((r * 4 + kc) * kDxNP + p) * 16, src, in ? 16u : 0u);
    }
    // ---- stage input-activation rows 2ra, 2ra + 1, columns 2c0 .. 2c0 + 255:
    // cell (r, kc, j) at ((r*4 + kc)*256 + j)*16
    for (int it = tid; it < 2 * 2 * kDxM * 4; it += kDxM) {
      const int kc = it & 3, rj = it >> 2;
      const int r = rj / (2 * kDxM), j = rj - r * (2 * kDxM);
      const int iy = 2 * ra + r, ix = 2 * c0 + j;
      const bool in = iy < a.Hi && ix < a.Wi;
      const __nv_bfloat16* src = in ? a.xin + (((long long)b * a.Hi + iy) * a.Wi + ix) * kC + kc * 8 : a.xin;
      tc::cp_async16(sX_addr + ((r * 4 + kc) * (2 * kDxM) + j) * 16, src, in ? 16u : 0u);
    }
    tc::cp_async_wait_all();
    tc::fence_proxy_async();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after_sync();
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int py = q >> 1, px = q & 1;
        int nt = 0;
#pragma unroll
        for (int ty = 0; ty <= py; ++ty) {
          // even rows: ky = 1 from row ra; odd rows: ky = 0 from ra + 1, ky = 2 from ra
          const int ky = py ? 2 * ty : 1, dr = (py && ty == 0) ? 1 : 0;
#pragma unroll
          for (int tx = 0; tx <= px; ++tx) {
            const int kx = px ? 2 * tx : 1, dc = (px && tx == 0) ? 1 : 0;
            const int tap = ky * 3 + kx;
#pragma unroll
            for (int s2 = 0; s2 < 2; ++s2) {
              const uint64_t ad = tc::smem_desc(sD_addr + ((dr * 4 + 2 * s2) * kDxNP + dc) * 16, kDxNP * 16, 128);
              const uint64_t bd = tc::smem_desc(sW_addr + (tap * 4 + 2 * s2) * 128, 128, 36 * 128);
              tc::mma_bf16(tmem + 32 * q, ad, bd, idesc, nt > 0 ? 1u : 0u);
              ++nt;
            }
          }
        }
      }
      tc::commit(&mbar[0]);
    }
    ok &= tc::mbar_wait(&mbar[0], phase & 1, kWaitLimit);
    ++phase;
    tc::fence_after_sync();

    // ---- epilogue: thread = class column c0 + tid, both column parities of
    // one input row per pass (128 contiguous output bytes)
    const uint32_t lane = (uint32_t)(warp * 32) << 16;
#pragma unroll 1
    for (int py = 0; py < 2; ++py) {
      float v[2][32];
      tc::tmem_ld32(tmem + lane + 32 * (2 * py), v[0]);
      tc::tmem_ld32(tmem + lane + 32 * (2 * py + 1), v[1]);
      const int iy = 2 * ra + py;
      if (iy < a.Hi) {
#pragma unroll
        for (int px = 0; px < 2; ++px) {
          const int j = 2 * tid + px, ix = 2 * c0 + j;
          if (ix < a.Wi) {
            uint4* dst = reinterpret_cast<uint4*>(a.din + (((long long)b * a.Hi + iy) * a.Wi + ix) * kC);
#pragma unroll
            for (int kc = 0; kc < 4; ++kc) {
              const uint4 xv = *reinterpret_cast<const uint4*>(sX + ((py * 4 + kc) * (2 * kDxM) + j) * 16);
              const uint32_t xw[4] = {xv.x, xv.y, xv.z, xv.w};
              uint32_t o[4];
#pragma unroll
              for (int e = 0; e < 4; ++e) {
                // bf16 > 0: sign bit clear and not +0
                const bool lo_on = (xw[e] & 0x8000u) == 0 && (xw[e] & 0x7FFFu) != 0;
                const bool hi_on = (xw[e] & 0x80000000u) == 0 && (xw[e] & 0x7FFF0000u) != 0;
                o[e] = tc::bf2(lo_on ? v[px][8 * kc + 2 * e] : 0.f, hi_on ? v[px][8 * kc + 2 * e + 1] : 0.f);
              }
              dst[kc] = make_uint4(o[0], o[1], o[2], o[3]);
            }
          }
        }
      }
    }
    tc::fence_before_sync();
    // TMEM read and staged rows consumed before the next tile; a timed-out
    // wait anywhere in the CTA ends the loop for all threads
    if (__syncthreads_or(!ok)) break;
  }
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, kDxTmemCols);
  if (!ok && tid == 0 && a.status) atomicExch(a.status, (int)BAYER_ERR_TIMEOUT);
}

// ---------------------------------------------------------------------------
// weight gradient
// ---------------------------------------------------------------------------

constexpr int kDwThreads = 256;
constexpr int kDwP = 64;         // output pixels per chunk: one row segment (4 MMA K-steps of 16)
constexpr int kRawPieces = 33;   // 16-byte pieces of a staged raw row: samples 4*ox0 - 8 .. 4*ox0 + 255

// MODE 0: hidden maps (patches gathered by cp.async in 16-byte channel chunks);
// MODE 1: Bayer frames, any alignment (per-thread sample loads, the exact
// bf16 hi/lo split).  Layer 1 with 16-byte aligned frame rows has a kernel of
// its own (conv_dw1_ring_tc_kernel, TF32 operands).
template <int MODE>
struct DwLayout {
  static constexpr bool FRAMES = MODE != 0;
  static constexpr int KOP = FRAMES ? 16 : kC;  // operand channels per tap
  static constexpr int KCH = 9 * KOP / 8;       // 16-byte patch chunks per pixel (18 or 36)
  static constexpr int MT = FRAMES ? 2 : 3;     // M tiles of 128 rows (patch rows + ones row + padding)
  static constexpr int NCH = MT * 16;           // 8-row chunks of A
  // A: cell (chunk j, pixel p) at (j * P + p) * 16: 8 consecutive patch rows
  // of one pixel, the 8 pixels of a core matrix 16 bytes apart.
  static constexpr int A_BYTES = NCH * kDwP * 16;
  // B: cell (co chunk, pixel p) at (chunk * P + p) * 16.
  static constexpr int B_BYTES = 4 * kDwP * 16;
  static constexpr int B_OFF = 2 * A_BYTES;
  static constexpr int MBAR_OFF = B_OFF + 2 * B_BYTES;
  static constexpr int SMEM = MBAR_OFF + 64;
  static constexpr int GS = KCH * 8 + 1;  // epilogue row stride: the patch rows and the ones row
  static constexpr int TMEM_COLS = MT == 2 ? 64 : 128;
  static_assert(kC * GS * 4 <= 2 * A_BYTES, "epilogue scratch fits in the A buffers");
  static_assert(KCH < NCH, "room for the ones row");
  static_assert(B_OFF % 16 == 0 && MBAR_OFF % 8 == 0, "alignment");
  static_assert(SMEM <= 113 * 1024, "two CTAs per SM");
};

// Chunk c of the (b, oy, segment) order: output pixels ox0 .. ox0 + 63 of row
// oy of image b (those at ox >= Wo are padding: zero output gradient).
struct Seg {
  int b, oy, ox0;
};
__device__ __forceinline__ Seg seg_of(int c, int Ho, int segs) {
  Seg s;
  const int row = c / segs;
  s.ox0 = (c - row * segs) * kDwP;
  s.b = row / Ho;
  s.oy = row - s.b * Ho;
  return s;
}

// Output gradients of a chunk into a B buffer: 4 lanes per pixel (64
// contiguous bytes), 8 pixels per warp.
__device__ __forceinline__ void dw_stage_dout(const ConvBwdArgs& a, const Seg& s, uint32_t sB, int tid) {
  const int kc = tid & 3, p = tid >> 2;  // kDwThreads == 4 * kDwP
  const int ox = s.ox0 + p;
  const bool in = ox < a.Wo;
  const __nv_bfloat16* src = in ? a.dout + (((long long)s.b * a.Ho + s.oy) * a.Wo + ox) * kC + kc * 8 : a.dout;
  tc::cp_async16(sB + (kc * kDwP + p) * 16, src, in ? 16u : 0u);
}

// MODE 0 patches: lanes = 8 pixels x 4 channel chunks of one tap (64
// contiguous bytes per pixel); items (tap, pixel octet) across warps.
__device__ __forceinline__ void dw_stage_hidden(const ConvBwdArgs& a, const Seg& s, uint32_t sA, int tid) {
  const int p_lo = tid & 7, kc = (tid >> 3) & 3;
  const long long img = (long long)s.b * a.Hi;
#pragma unroll 3
  for (int rest = tid >> 5; rest < 9 * (kDwP / 8); rest += kDwThreads / 32) {
    const int tap = rest % 9, p = (rest / 9) * 8 + p_lo;
    const int ox = s.ox0 + p;
    const int iy = 2 * s.oy + tap / 3 - 1, ix = 2 * ox + tap % 3 - 1;
    const bool in = ox < a.Wo && iy >= 0 && iy < a.Hi && ix >= 0 && ix < a.Wi;
    const __nv_bfloat16* src = in ? a.xin + ((img + iy) * a.Wi + ix) * kC + kc * 8 : a.xin;
    tc::cp_async16(sA + ((tap * 4 + kc) * kDwP + p) * 16, src, in ? 16u : 0u);
  }
}

// The A cell of Bayer patch (pixel, tap, frame): the RGGB quad's samples
// (row 0: w0, row 1: w1; two samples each, left one low) split into hi/lo
// pairs, or zeros outside the half-resolution map.
__device__ __forceinline__ uint4 bayer_cell(bool in, uint32_t w0, uint32_t w1) {
  if (!in) return make_uint4(0, 0, 0, 0);
  return make_uint4(tc::split12(w0 & 0xFFFFu), tc::split12(w0 >> 16), tc::split12(w1 & 0xFFFFu),
                    tc::split12(w1 >> 16));
}

// MODE 1 patches: item (pixel, tap, frame), loads first, then conversion.
__device__ __forceinline__ void dw_stage_bayer_direct(const ConvBwdArgs& a, const Seg& s, uint8_t* sA, int tid) {
  constexpr int NIT = kDwP * 9 * 2;
  constexpr int PER = (NIT + kDwThreads - 1) / kDwThreads;
  const int Hh = a.fr.H / 2, Wh = a.fr.W / 2;
  uint32_t r0[PER], r1[PER];
  bool in[PER];
#pragma unroll
  for (int u = 0; u < PER; ++u) {
    const int it = tid + u * kDwThreads;
    const int p = it & (kDwP - 1), tf = it / kDwP;
    const int tap = tf >> 1, f = tf & 1;
    const int ox = s.ox0 + p;
    const int hy = 2 * s.oy + tap / 3 - 1, hx = 2 * ox + tap % 3 - 1;
    in[u] = it < NIT && ox < a.Wo && hy >= 0 && hy < Hh && hx >= 0 && hx < Wh;
    r0[u] = r1[u] = 0;
    if (in[u]) {
      const uint16_t* fp = f ? a.fr.cur + (long long)s.b * a.fr.cur_bs : a.fr.ref + (long long)s.b * a.fr.ref_bs;
      const uint16_t* s0 = fp + (long long)(2 * hy) * a.fr.pitch + 2 * hx;
      const uint16_t* s1 = s0 + a.fr.pitch;
      if (a.vec) {
        r0[u] = __ldg(reinterpret_cast<const uint32_t*>(s0));
        r1[u] = __ldg(reinterpret_cast<const uint32_t*>(s1));
      } else {
        r0[u] = (uint32_t)__ldg(s0) | ((uint32_t)__ldg(s0 + 1) << 16);
        r1[u] = (uint32_t)__ldg(s1) | ((uint32_t)__ldg(s1 + 1) << 16);
      }
    }
  }
#pragma unroll
  for (int u = 0; u < PER; ++u) {
    const int it = tid + u * kDwThreads;
    if (it < NIT) *reinterpret_cast<uint4*>(sA + ((it / kDwP) * kDwP + (it & (kDwP - 1))) * 16) =
        bayer_cell(in[u], r0[u], r1[u]);
  }
}

// Layer 1 (aligned frames): raw rows 4oy - 2 .. 4oy + 3 of both frames, samples 4ox0 - 8 ..
// 4ox0 + 255 (zero-filled outside the frame) into a raw buffer.
__device__ __forceinline__ void dw_stage_raw(const ConvBwdArgs& a, const Seg& s, uint32_t sR, int tid) {
  const uint16_t* ref = a.fr.ref + (long long)s.b * a.fr.ref_bs;
  const uint16_t* cur = a.fr.cur + (long long)s.b * a.fr.cur_bs;
  for (int it = tid; it < 2 * 6 * kRawPieces; it += kDwThreads) {
    const int q = it % kRawPieces, fr = it / kRawPieces;
    const int f = fr / 6, r = fr - 6 * f;
    const int y = 4 * s.oy - 2 + r, x = 4 * s.ox0 - 8 + 8 * q;
    const bool in = y >= 0 && y < a.fr.H && x >= 0 && x < a.fr.W;  // W % 8 == 0: whole pieces
    const uint16_t* src = in ? (f ? cur : ref) + (long long)y * a.fr.pitch + x : a.fr.ref;
    tc::cp_async16(sR + it * 16, src, in ? 16u : 0u);
  }
}

// The ones row (row KCH*8 of A: element 0 of chunk KCH) and the zero padding
// rows of both A buffers; the patch staging never touches them.
template <int MODE>
__device__ __forceinline__ void dw_init_pad(uint8_t* smem, int tid) {
  using L = DwLayout<MODE>;
  constexpr int PAD = (L::NCH - L::KCH) * kDwP;
  for (int i = tid; i < 2 * PAD; i += kDwThreads) {
    const int s = i / PAD, r = i - s * PAD;
    const int j = L::KCH + r / kDwP, p = r % kDwP;
    *reinterpret_cast<uint4*>(smem + s * L::A_BYTES + (j * kDwP + p) * 16) =
        make_uint4(j == L::KCH ? 0x3F80u : 0u, 0u, 0u, 0u);
  }
}

// MMAs of one chunk (thread 0): K step = 16 pixels; core matrices are 8
// pixels (K, 128 bytes apart) x 8 rows (M or N, kDwP * 16 bytes apart).
template <int MT>
__device__ __forceinline__ void dw_mma(uint32_t tmem, uint32_t sa, uint32_t sb, bool first) {
  constexpr uint32_t idesc = tc::idesc_bf16_f32(128, kC) | (1u << 15) | (1u << 16);  // A, B MN-major
#pragma unroll
  for (int s = 0; s < kDwP / 16; ++s) {
    const uint64_t bd = tc::smem_desc(sb + s * 256, 128, kDwP * 16);
#pragma unroll
    for (int mt = 0; mt < MT; ++mt) {
      const uint64_t ad = tc::smem_desc(sa + mt * 16 * kDwP * 16 + s * 256, 128, kDwP * 16);
      tc::mma_bf16(tmem + 32 * mt, ad, bd, idesc, (!first || s > 0) ? 1u : 0u);
    }
  }
}

// TMEM partial sums -> shared scratch G[co][k] (over the A buffers) -> the
// gradient, once per CTA.  ok is CTA-uniform; every MMA has completed.
template <int MODE>
__device__ __forceinline__ void dw_epilogue(const ConvBwdArgs& a, uint8_t* smem, uint32_t tmem, bool live, int tid) {
  using L = DwLayout<MODE>;
  const int warp = tid >> 5;
  float* G = reinterpret_cast<float*>(smem);
  if (live) {
    const int quarter = warp & 3;
    for (int mt = warp >> 2; mt < L::MT; mt += 2) {
      float v[32];
      tc::tmem_ld32(tmem + ((uint32_t)(quarter * 32) << 16) + 32 * mt, v);
      const int k = mt * 128 + quarter * 32 + (tid & 31);
      if (k < L::GS) {
#pragma unroll
        for (int co = 0; co < kC; ++co) G[co * L::GS + k] = v[co];
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (live) {
    // dW in the flat order [co][ci][tap], 4 consecutive entries per thread
    constexpr int CIN = L::FRAMES ? 8 : kC, PER_CO = CIN * 9;
    for (int i = tid; i < kC * PER_CO / 4; i += kDwThreads) {
      const int co = (4 * i) / PER_CO, j0 = 4 * i - co * PER_CO;
      float g[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int j = j0 + e, ci = j / 9, tap = j - 9 * ci;
        const float* gr = G + co * L::GS;
        g[e] = L::FRAMES ? gr[tap * 16 + 2 * ci] + gr[tap * 16 + 2 * ci + 1] * (1.0f / 128.0f) : gr[tap * kC + ci];
      }
      float* dst = a.gw + co * PER_CO + j0;
      if (a.vec_atomics) {
        atomicAdd(reinterpret_cast<float4*>(dst), make_float4(g[0], g[1], g[2], g[3]));
      } else {
#pragma unroll
        for (int e = 0; e < 4; ++e) atomicAdd(dst + e, g[e]);
      }
    }
    if (tid < kC) atomicAdd(a.gb + tid, G[tid * L::GS + L::KCH * 8]);
  }
}

// MODE 0 and 1: two stages, the copies of chunk i + 1 in flight while the MMAs
// of chunk i run.
template <int MODE>
__global__ void __launch_bounds__(kDwThreads, 2) conv_dw_tc_kernel(const ConvBwdArgs a, int chunks_per_cta) {
  using L = DwLayout<MODE>;
  extern __shared__ __align__(1024) uint8_t smem[];
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + L::MBAR_OFF);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mbar + 2);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int segs = (a.Wo + kDwP - 1) / kDwP;
  const int nchunks = a.batch * a.Ho * segs;
  const int c_begin = blockIdx.x * chunks_per_cta;
  const int c_end = min(c_begin + chunks_per_cta, nchunks);
  const int n = c_begin < c_end ? c_end - c_begin : 0;

  if (tid == 0) {
    tc::mbar_init(&mbar[0], 1);
    tc::mbar_init(&mbar[1], 1);
    tc::fence_mbar_init();
  }
  if (warp == 0) tc::tmem_alloc(tmem_slot, L::TMEM_COLS);
  dw_init_pad<MODE>(smem, tid);
  const uint32_t s0 = tc::smem_addr(smem);
  bool ok = true;

  auto stage = [&](int i, int buf) {
    const Seg s = seg_of(c_begin + i, a.Ho, segs);
    dw_stage_dout(a, s, s0 + L::B_OFF + buf * L::B_BYTES, tid);
    if (MODE == 0)
      dw_stage_hidden(a, s, s0 + buf * L::A_BYTES, tid);
    else
      dw_stage_bayer_direct(a, s, smem + buf * L::A_BYTES, tid);
  };
  if (n > 0) stage(0, 0);
  tc::cp_async_commit();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tmem_slot;

  for (int i = 0; i < n; ++i) {
    const int buf = i & 1;
    if (i + 1 < n) {
      // the other stage was read by the MMAs of chunk i - 1
      if (i >= 1) ok &= tc::mbar_wait(&mbar[buf ^ 1], ((i - 1) >> 1) & 1, kWaitLimit);
      stage(i + 1, buf ^ 1);
      tc::cp_async_commit();
      tc::cp_async_wait<1>();
    } else {
      tc::cp_async_wait<0>();
    }
    tc::fence_proxy_async();
    if (__syncthreads_or(!ok)) {  // a timed-out wait anywhere in the CTA: stop issuing
      tc::cp_async_wait_all();
      break;
    }
    if (tid == 0) {
      tc::fence_after_sync();
      dw_mma<L::MT>(tmem, s0 + buf * L::A_BYTES, s0 + L::B_OFF + buf * L::B_BYTES, i == 0);
      tc::commit(&mbar[buf]);
    }
  }
  if (n > 0 && ok) ok &= tc::mbar_wait(&mbar[(n - 1) & 1], ((n - 1) >> 1) & 1, kWaitLimit);
  ok = __syncthreads_and(ok);  // every buffer consumed: the A buffers become the epilogue scratch
  tc::fence_after_sync();
  dw_epilogue<MODE>(a, smem, tmem, n > 0 && ok, tid);
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, L::TMEM_COLS);
  if (!ok && tid == 0 && a.status) atomicExch(a.status, (int)BAYER_ERR_TIMEOUT);
}

// Layer 1 with 16-byte aligned frame rows (launch MODE 2): TF32 operands,
// K-major.  The raw rows and the output gradients of a chunk are copied two
// chunks ahead (rings of 3); per chunk the threads convert them into the A and
// B buffers the MMAs of chunk i - 2 have released:
//   A (M = 128 rows: patch row m = tap * 8 + frame * 4 + plane, 72 of them,
//     row 72 = 1.0 for the bias, K = the chunk's 64 pixels): element (m, p) at
//     (m/8) * kT1SBO + (p/4) * kT1LBO + (m%8) * 16 + (p%4) * 4, the float32
//     value v/2048 - 1 (exact in TF32) of the patch's sample;
//   B (N = 32 channels): element (co, p) at the same offsets, the bf16
//     gradient widened exactly.
// kT1LBO = 144 bytes (9 words) spreads the 4-pixel groups over distinct banks,
// so a warp's 32 pixel stores of one row are conflict-free.  Only the first 10
// of A's 16 row groups hold data (the MMA reads the others from whatever lies
// after them: rows 80..127 of D are not used).
constexpr int kT1LBO = 144, kT1SBO = (kDwP / 4) * kT1LBO;  // 2304
constexpr int kT1ABytes = 10 * kT1SBO;                       // written part of A
constexpr int kT1BBytes = 4 * kT1SBO;
constexpr int kT1R = 2 * 6 * kRawPieces * 16;                // raw rows of a chunk (both frames)
constexpr int kT1D = kDwP * kC * 2;                          // raw gradients of a chunk
constexpr int kT1B_OFF = 2 * kT1ABytes;
constexpr int kT1R_OFF = kT1B_OFF + 2 * kT1BBytes;
constexpr int kT1D_OFF = kT1R_OFF + 3 * kT1R;
constexpr int kT1MBAR_OFF = kT1D_OFF + 3 * kT1D;
constexpr int kT1Smem = kT1MBAR_OFF + 64;
constexpr int kT1GS = 73;  // epilogue row stride: 72 patch rows and the ones row
static_assert(kT1MBAR_OFF - kT1ABytes >= 16 * kT1SBO, "the second A buffer's unused row groups stay in bounds");
static_assert(kT1R_OFF % 16 == 0 && kT1D_OFF % 16 == 0 && kT1MBAR_OFF % 8 == 0, "alignment");
static_assert(kT1Smem <= 113 * 1024, "two CTAs per SM");
static_assert(kC * kT1GS * 4 <= 2 * kT1ABytes, "epilogue scratch fits in the A buffers");

// The chunk's converted operands from its raw buffers.  Items (pixel p, tap,
// frame) -> 4 plane values of patch rows tap*8 + frame*4 + plane; items (p,
// channel group g of 8) -> 8 widened gradients.
__device__ __forceinline__ void dw1_convert_tf32(const ConvBwdArgs& a, const Seg& s, const uint8_t* R,
                                                 const uint8_t* Dr, uint8_t* A, uint8_t* B, int tid) {
  const int Hh = a.fr.H / 2, Wh = a.fr.W / 2;
  const int p = tid & (kDwP - 1), q = tid / kDwP;  // q = 0..3
  const int ox = s.ox0 + p;
  const int pix = (p >> 2) * kT1LBO + (p & 3) * 4;
#pragma unroll
  for (int u = 0; u < 5; ++u) {
    const int tf = q + 4 * u;
    if (tf < 18) {
      const int tap = tf >> 1, f = tf & 1, ky = tap / 3, kx = tap - 3 * ky;
      const int hy = 2 * s.oy + ky - 1, hx = 2 * ox + kx - 1;
      const bool in = ox < a.Wo && hy >= 0 && hy < Hh && hx >= 0 && hx < Wh;
      uint32_t w0 = 0, w1 = 0;
      if (in) {
        const uint8_t* row = R + (f * 6 + 2 * ky) * (kRawPieces * 16) + 2 * (4 * p + 2 * kx + 6);
        w0 = *reinterpret_cast<const uint32_t*>(row);
        w1 = *reinterpret_cast<const uint32_t*>(row + kRawPieces * 16);
      }
      uint8_t* dst = A + tap * kT1SBO + f * 4 * 16 + pix;
      *reinterpret_cast<uint32_t*>(dst) = in ? tc::tf32_sample12(w0 & 0xFFFFu) : 0u;
      *reinterpret_cast<uint32_t*>(dst + 16) = in ? tc::tf32_sample12(w0 >> 16) : 0u;
      *reinterpret_cast<uint32_t*>(dst + 32) = in ? tc::tf32_sample12(w1 & 0xFFFFu) : 0u;
      *reinterpret_cast<uint32_t*>(dst + 48) = in ? tc::tf32_sample12(w1 >> 16) : 0u;
    }
  }
  // B: pixel p, channels 8q .. 8q + 7 (n-group q, rows n % 8)
  const uint4 v = *reinterpret_cast<const uint4*>(Dr + p * 64 + q * 16);
  const uint32_t w[4] = {v.x, v.y, v.z, v.w};
  uint8_t* dst = B + q * kT1SBO + pix;
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    *reinterpret_cast<uint32_t*>(dst + (2 * e) * 16) = w[e] << 16;
    *reinterpret_cast<uint32_t*>(dst + (2 * e + 1) * 16) = w[e] & 0xFFFF0000u;
  }
}

__global__ void __launch_bounds__(kDwThreads, 2) conv_dw1_ring_tc_kernel(const ConvBwdArgs a, int chunks_per_cta) {
  extern __shared__ __align__(1024) uint8_t smem[];
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + kT1MBAR_OFF);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mbar + 2);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int segs = (a.Wo + kDwP - 1) / kDwP;
  const int nchunks = a.batch * a.Ho * segs;
  const int c_begin = blockIdx.x * chunks_per_cta;
  const int c_end = min(c_begin + chunks_per_cta, nchunks);
  const int n = c_begin < c_end ? c_end - c_begin : 0;

  if (tid == 0) {
    tc::mbar_init(&mbar[0], 1);
    tc::mbar_init(&mbar[1], 1);
    tc::fence_mbar_init();
  }
  if (warp == 0) tc::tmem_alloc(tmem_slot, 32);
  // row group 9 of both A buffers: row 72 = 1.0, rows 73..79 = 0 (never rewritten)
  for (int i = tid; i < 2 * 8 * kDwP; i += kDwThreads) {
    const int sb = i / (8 * kDwP), r = i - sb * (8 * kDwP);
    const int row = r / kDwP, p = r - row * kDwP;
    *reinterpret_cast<uint32_t*>(smem + sb * kT1ABytes + 9 * kT1SBO + (p >> 2) * kT1LBO + row * 16 + (p & 3) * 4) =
        row == 0 ? 0x3F800000u : 0u;
  }
  const uint32_t s0 = tc::smem_addr(smem);
  bool ok = true;

  auto issue = [&](int i) {  // copies of chunk i, one cp.async group (empty past the end)
    if (i < n) {
      const Seg s = seg_of(c_begin + i, a.Ho, segs);
      dw_stage_raw(a, s, s0 + kT1R_OFF + (i % 3) * kT1R, tid);
      const int kc = tid & 3, p = tid >> 2;  // raw gradients: pixel p at p * 64
      const int ox = s.ox0 + p;
      const bool in = ox < a.Wo;
      const __nv_bfloat16* src =
          in ? a.dout + (((long long)s.b * a.Ho + s.oy) * a.Wo + ox) * kC + kc * 8 : a.dout;
      tc::cp_async16(s0 + kT1D_OFF + (i % 3) * kT1D + (p * 4 + kc) * 16, src, in ? 16u : 0u);
    }
    tc::cp_async_commit();
  };
  issue(0);
  issue(1);
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tmem_slot;
  constexpr uint32_t idesc = tc::idesc_tf32_f32(128, kC);  // K-major A and B

  for (int i = 0; i < n; ++i) {
    const int buf = i & 1;
    // A[buf] and B[buf] were read by the MMAs of chunk i - 2
    if (i >= 2) ok &= tc::mbar_wait(&mbar[buf], ((i - 2) >> 1) & 1, kWaitLimit);
    issue(i + 2);
    tc::cp_async_wait<2>();  // chunk i's copies (this thread's) have landed
    if (__syncthreads_or(!ok)) {
      tc::cp_async_wait_all();
      break;
    }
    dw1_convert_tf32(a, seg_of(c_begin + i, a.Ho, segs), smem + kT1R_OFF + (i % 3) * kT1R,
                     smem + kT1D_OFF + (i % 3) * kT1D, smem + buf * kT1ABytes, smem + kT1B_OFF + buf * kT1BBytes,
                     tid);
    tc::fence_proxy_async();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after_sync();
      const uint32_t sa = s0 + buf * kT1ABytes, sb = s0 + kT1B_OFF + buf * kT1BBytes;
#pragma unroll
      for (int k = 0; k < kDwP / 8; ++k) {  // K step = 8 pixels = 2 groups of 4
        const uint64_t ad = tc::smem_desc(sa + k * 2 * kT1LBO, kT1LBO, kT1SBO);
        const uint64_t bd = tc::smem_desc(sb + k * 2 * kT1LBO, kT1LBO, kT1SBO);
        tc::mma_tf32(tmem, ad, bd, idesc, (i > 0 || k > 0) ? 1u : 0u);
      }
      tc::commit(&mbar[buf]);
    }
  }
  if (n > 0 && ok) ok &= tc::mbar_wait(&mbar[(n - 1) & 1], ((n - 1) >> 1) & 1, kWaitLimit);
  tc::cp_async_wait_all();
  ok = __syncthreads_and(ok);
  tc::fence_after_sync();
  // TMEM -> G[co][m] (over the A buffers) -> dW1[co][ci][tap] = G[co][tap*8 + ci], db = G[co][72]
  float* G = reinterpret_cast<float*>(smem);
  const bool live = n > 0 && ok;
  if (live && warp < 4) {
    float v[32];
    tc::tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16), v);
    const int m = warp * 32 + (tid & 31);
    if (m < kT1GS) {
#pragma unroll
      for (int co = 0; co < kC; ++co) G[co * kT1GS + m] = v[co];
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (live) {
    for (int i = tid; i < kC * 72 / 4; i += kDwThreads) {
      const int co = (4 * i) / 72, j0 = 4 * i - co * 72;
      float g[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int j = j0 + e, ci = j / 9, tap = j - 9 * ci;
        g[e] = G[co * kT1GS + tap * 8 + ci];
      }
      float* dst = a.gw + co * 72 + j0;
      if (a.vec_atomics) {
        atomicAdd(reinterpret_cast<float4*>(dst), make_float4(g[0], g[1], g[2], g[3]));
      } else {
#pragma unroll
        for (int e = 0; e < 4; ++e) atomicAdd(dst + e, g[e]);
      }
    }
    if (tid < kC) atomicAdd(a.gb + tid, G[tid * kT1GS + 72]);
  }
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, 32);
  if (!ok && tid == 0 && a.status) atomicExch(a.status, (int)BAYER_ERR_TIMEOUT);
}

int sm_count() {
  int dev = 0, nsm = 148;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  return nsm;
}

template <typename K>
cudaError_t launch_dw(K kern, const ConvBwdArgs& a, int smem, int tmem_cols, cudaStream_t st) {
  const long long nchunks = (long long)a.batch * a.Ho * ((a.Wo + kDwP - 1) / kDwP);
  if (nchunks < 1) return cudaSuccess;
  if (nchunks > 0x7FFFFFFFll) return cudaErrorInvalidValue;
  const int per_sm = tc::ctas_per_sm(kern, kDwThreads, smem, tmem_cols);
  const long long slots = (long long)sm_count() * per_sm;
  // at least 4 chunks per CTA: the partial sums are added once per CTA
  long long per = (nchunks + slots - 1) / slots;
  if (per < 4) per = 4;
  const long long grid = (nchunks + per - 1) / per;
  kern<<<(unsigned)grid, kDwThreads, smem, st>>>(a, (int)per);
  return cudaGetLastError();
}

template <typename K>
cudaError_t configure_dw(K kern, int smem) {
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  return e;
}

}  // namespace

size_t conv_dx_weight_bytes() { return (size_t)3 * kDxWBytes; }

cudaError_t pack_conv_dx_weights(const uint16_t* w, const int* w_off, uint16_t* img, cudaStream_t st) {
  PackDxArgs pa;
  pa.w = reinterpret_cast<const __nv_bfloat16*>(w);
  for (int l = 0; l < 3; ++l) pa.w_off[l] = w_off[l];
  const int n = 3 * kC * 9 * kC;
  pack_dx_weights_kernel<<<(n + 255) / 256, 256, 0, st>>>(pa, reinterpret_cast<__nv_bfloat16*>(img));
  return cudaGetLastError();
}

cudaError_t configure_conv_bwd_tc() {
  cudaError_t e = cudaFuncSetAttribute(conv_dx_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kDxSmem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(conv_dx_tc_kernel, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  if (e == cudaSuccess) e = configure_dw(conv_dw_tc_kernel<0>, DwLayout<0>::SMEM);
  if (e == cudaSuccess) e = configure_dw(conv_dw_tc_kernel<1>, DwLayout<1>::SMEM);
  if (e == cudaSuccess) e = configure_dw(conv_dw1_ring_tc_kernel, kT1Smem);
  return e;
}

cudaError_t launch_conv_dx_tc(const ConvBwdArgs& a, cudaStream_t st) {
  const int per_sm = tc::ctas_per_sm(conv_dx_tc_kernel, kDxM, kDxSmem, kDxTmemCols);
  const long long ntiles = (long long)a.batch * a.Ho * ((a.Wo + kDxM - 1) / kDxM);
  if (ntiles < 1) return cudaSuccess;
  long long grid = (long long)sm_count() * per_sm;
  if (grid > ntiles) grid = ntiles;
  conv_dx_tc_kernel<<<(unsigned)grid, kDxM, kDxSmem, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_conv_dw_tc(const ConvBwdArgs& a, bool frames, cudaStream_t st) {
  if (!frames) return launch_dw(conv_dw_tc_kernel<0>, a, DwLayout<0>::SMEM, DwLayout<0>::TMEM_COLS, st);
  // the raw-row ring copies 16-byte pieces: 16-byte aligned frames, pitch and
  // batch strides multiples of 8 samples (W is a multiple of 32)
  const bool ring = (reinterpret_cast<uintptr_t>(a.fr.ref) & 15) == 0 &&
                    (reinterpret_cast<uintptr_t>(a.fr.cur) & 15) == 0 && a.fr.pitch % 8 == 0 &&
                    a.fr.ref_bs % 8 == 0 && a.fr.cur_bs % 8 == 0 && a.fr.W % 8 == 0;
  if (ring) return launch_dw(conv_dw1_ring_tc_kernel, a, kT1Smem, 32, st);
  return launch_dw(conv_dw_tc_kernel<1>, a, DwLayout<1>::SMEM, DwLayout<1>::TMEM_COLS, st);
}

}  // namespace bme

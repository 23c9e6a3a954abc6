// 3x3 stride-2 convolution (zero pad 1), 32 output channels, as an implicit
// GEMM on the 5th-generation tensor cores: BF16 operands in shared memory,
// FP32 accumulators in tensor memory (TMEM) -- layers 3 and 4 of the learned
// proposal network (few output rows; layers 1 and 2 stream rows through
// conv_s2_tc.cu), and the weight packing of all four layers.
//
//   D[m, n] = sum_k A[m, k] * B[k, n],  m = output pixel, n = output channel,
//   k = tap * CIN + ci,  A[m, k] = input at (2*oy + ky - 1, 2*ox + kx - 1, ci).
//
// Tile = 128 consecutive output pixels of one output row (MMA M = 128, N = 32);
// CTA = 128 threads, persistent over tiles.
//   Prologue: the layer's weights, packed once per forward into the kernels'
//   shared-memory image (one launch of pack_conv_tc_weights for all four
//   layers), are copied in with 16-byte loads and stay resident.
//   Staging: per tile the three NHWC bf16 input rows, once (no im2col copy),
//   through asynchronous 16-byte copies (cp.async, zero-filled outside the
//   map), so every load of the tile is in flight at once.
//   MMA: after one barrier thread 0 issues 9 * CIN/16 MMAs whose A operands
//   are shifted views of the staged rows and commits them to an mbarrier.
//   Epilogue: TMEM -> registers -> bias, ReLU -> bf16 NHWC, or, for layer 4
//   with the head fused, the 1x1 head, tanh and sigmoid straight to the
//   per-block proposals.
// Several CTAs per SM overlap one tile's staging with another's MMAs and
// epilogue.  Every mbarrier wait is bounded; on expiry the kernel records
// BAYER_ERR_TIMEOUT in the status word, frees its TMEM and finishes.
//
// Layer 1 (conv_s2_tc.cu) takes its operands as TF32: each 12-bit sample v as
// v/2048 - 1 (exact in TF32), the bf16 weights widened exactly; the packing
// below builds that layer's TF32 weight image too.
#include <cuda_bf16.h>

#include "common.cuh"
#include "kernels.cuh"
#include "tc_common.cuh"

namespace bme {

namespace {

constexpr int kM = 128;    // output pixels per tile (MMA M)
constexpr int kN = 32;     // output channels (MMA N)
constexpr int kS = 2;      // stride
constexpr int kHeadW = 12 * kN + 12;  // head weights + biases
constexpr uint32_t kWaitLimit = 1u << 20;

// Shared-memory plan of one CTA.  The three input rows a tile needs are staged
// once, split into 2 column-parity planes and into 16-byte channel chunks:
// element (row rho, plane q, chunk kc, pixel p) at
// (((rho*2 + q)*KC + kc)*NP + p)*16.  Output pixel m of tap (ky, kx) then reads
// plane q = kx % 2 at pixel m + kx / 2, so every tap's A operand is the staged
// tensor itself at a shifted start address: core matrices of 8 consecutive
// pixels (SBO = 128 bytes), the next K chunk one plane further (LBO = NP*16).
template <int CIN, int EPI>
struct RowConvLayout {
  static constexpr int KC = CIN / 8;
  static constexpr int NJ = kS * (kM - 1) + 3;      // staged input columns
  static constexpr int NP = (NJ + kS - 1) / kS;     // pixels per parity plane
  static constexpr int STAGE_BYTES = 3 * kS * KC * NP * 16;
  static constexpr int B_BYTES = 9 * CIN * kN * 2;  // packed weights
  static constexpr int HEAD_BYTES = EPI == 1 ? kHeadW * 4 : 0;
  static constexpr int TMEM_COLS = 32;
  static constexpr int SMEM = B_BYTES + STAGE_BYTES + HEAD_BYTES + 64;
  static_assert(CIN % 16 == 0, "shape");
  static_assert(B_BYTES % 128 == 0 && STAGE_BYTES % 16 == 0, "alignment");
  static_assert(SMEM <= 227 * 1024, "shared memory");
};

using tc::bf2;

using tc::cp_async16;
using tc::cp_async_wait_all;

// Weight images of the four layers (K-major B operand, all 32 output
// channels): for layers 2..4 (32 input channels), element (n, k), k =
// tap*32 + ci, bf16 at (n/8)*(9*4)*128 + (k/8)*128 + (n%8)*16 + (k%8)*2.
// Layer 1 (8 input planes, TF32 operands): element (n, k), k = tap*8 + ci, the
// float32 value of the bf16 weight at (n/8)*(9*2)*128 + (k/4)*128 + (n%8)*16 +
// (k%4)*4 (core matrices of 8 rows x 4 TF32 values); the same 9216 bytes.
// One thread per element of all four images; image l starts at byte
// img_off[l] of img and is built from w + w_off[l].
struct PackArgs {
  const __nv_bfloat16* w;
  int w_off[4];
  unsigned img_off[4];
  int* zero_words;  // optional: two ints set to 0 (counters that kernels after the network fill)
};

// Launched as a dependent of whatever precedes it on the stream (its launch
// overlaps that kernel's last CTAs); it reads the weights only after the wait,
// since the kernel before may have written them (an optimizer step).
__global__ void pack_conv_tc_weights_kernel(const PackArgs pa, __nv_bfloat16* __restrict__ img) {
  constexpr int kL1 = kN * 9 * 8, kL = kN * 9 * 32;
  tc::grid_dep_wait();
  tc::grid_dep_launch();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0 && pa.zero_words) pa.zero_words[0] = pa.zero_words[1] = 0;
  if (i < kL1) {
    const int n = i / 72, k = i - n * 72;
    const int tap = k / 8, ci = k - tap * 8;
    const float wv = __bfloat162float(pa.w[pa.w_off[0] + (n * 8 + ci) * 9 + tap]);
    reinterpret_cast<float*>(reinterpret_cast<uint8_t*>(img) + pa.img_off[0] + (n >> 3) * (18 * 128) +
                             (k >> 2) * 128 + (n & 7) * 16)[k & 3] = wv;
    return;
  }
  i -= kL1;
  const int l = 1 + i / kL;
  i -= (l - 1) * kL;
  if (l > 3) return;
  constexpr int cin_op = 32, K = 9 * cin_op;
  const int n = i / K, k = i - n * K;
  const int tap = k / cin_op, ci = k - tap * cin_op;
  const __nv_bfloat16* w = pa.w + (l == 1 ? pa.w_off[1] : (l == 2 ? pa.w_off[2] : pa.w_off[3]));
  const float wv = __bfloat162float(w[(n * cin_op + ci) * 9 + tap]);
  const unsigned off = l == 1 ? pa.img_off[1] : (l == 2 ? pa.img_off[2] : pa.img_off[3]);
  constexpr int kc = cin_op / 8;
  img[(off + (n >> 3) * (9 * kc) * 128 + (k >> 3) * 128 + (n & 7) * 16) / 2 + (k & 7)] = __float2bfloat16_rn(wv);
}

// EPI: 0 bias + ReLU -> bf16 NHWC output; 1 bias + ReLU -> bf16 rounding ->
// 1x1 head (12 outputs) -> (range*tanh, range*tanh, sigmoid) of the 4 blocks
// of the pixel.
template <int CIN, int EPI>
__global__ void __launch_bounds__(kM) conv3x3_tc_kernel(const ConvTcArgs a) {
  using L = RowConvLayout<CIN, EPI>;
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* sB = smem;
  uint8_t* sX = smem + L::B_BYTES;
  float* sHead = reinterpret_cast<float*>(smem + L::B_BYTES + L::STAGE_BYTES);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + L::B_BYTES + L::STAGE_BYTES + L::HEAD_BYTES);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mbar + 1);
  const int tid = threadIdx.x, warp = tid >> 5;

  if (tid == 0) {
    tc::mbar_init(&mbar[0], 1);
    tc::fence_mbar_init();
  }
  if (warp == 0) tc::tmem_alloc(tmem_slot, L::TMEM_COLS);
  for (int i = tid; i < L::B_BYTES / 16; i += kM) reinterpret_cast<uint4*>(sB)[i] = __ldg(a.wimg + i);
  if (EPI == 1)
    for (int i = tid; i < kHeadW; i += kM) sHead[i] = __bfloat162float(a.whead[i]);
  // launched as a dependent of the previous layer (whose own wait covered the
  // weight packing): its output is read only after this wait
  tc::grid_dep_wait();
  tc::grid_dep_launch();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tmem_slot;
  const uint32_t sX_addr = tc::smem_addr(sX), sB_addr = tc::smem_addr(sB);
  constexpr uint32_t idesc = tc::idesc_bf16_f32(kM, kN);
  const int segs = (a.Wo + kM - 1) / kM;
  const long long ntiles = (long long)a.batch * a.Ho * segs;
  uint32_t phase = 0;
  bool ok = true;

  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int seg = (int)(tile % segs);
    const long long row = tile / segs;
    const int b = (int)(row / a.Ho), oy = (int)(row - (long long)b * a.Ho);
    const int ox0 = seg * kM;
    const int c0 = kS * ox0 - 1;  // input column of staged column 0

    // ---- stage rows 2*oy - 1 .. 2*oy + 1, columns c0 .. c0 + NJ - 1
    {
      // item = (row rho, column j, chunk kc), kc fastest: a warp copies whole pixels
      constexpr int NITEM = 3 * L::NJ * L::KC;
      for (int it = tid; it < NITEM; it += kM) {
        const int rho = it / (L::NJ * L::KC), r = it - rho * (L::NJ * L::KC);
        const int j = r / L::KC, kc = r - j * L::KC;
        const int iy = kS * oy - 1 + rho, ix = c0 + j;
        const bool in_ok = iy >= 0 && iy < a.Hi && ix >= 0 && ix < a.Wi;
        const __nv_bfloat16* src = in_ok ? a.in + (((long long)b * a.Hi + iy) * a.Wi + ix) * CIN + kc * 8 : a.in;
        const int q = j & 1, pp = j >> 1;
        cp_async16(sX_addr + (((rho * kS + q) * L::KC + kc) * L::NP + pp) * 16, src, in_ok ? 16u : 0u);
      }
      cp_async_wait_all();
    }
    tc::fence_proxy_async();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after_sync();
#pragma unroll
      for (int tap = 0; tap < 9; ++tap) {
        const int ky = tap / 3, kx = tap % 3;
        const int q = kx % kS, dp = kx / kS;
#pragma unroll
        for (int s2 = 0; s2 < CIN / 16; ++s2) {
          const uint32_t a_addr = sX_addr + (((ky * kS + q) * L::KC + 2 * s2) * L::NP + dp) * 16;
          const uint64_t ad = tc::smem_desc(a_addr, L::NP * 16, 128);
          const uint64_t bd = tc::smem_desc(sB_addr + (tap * L::KC + 2 * s2) * 128, 128, 9 * L::KC * 128);
          tc::mma_bf16(tmem, ad, bd, idesc, (tap > 0 || s2 > 0) ? 1u : 0u);
        }
      }
      tc::commit(&mbar[0]);
    }
    ok &= tc::mbar_wait(&mbar[0], phase & 1, kWaitLimit);
    ++phase;
    tc::fence_after_sync();
    const int ox = ox0 + tid;
    const bool valid = ox < a.Wo;
    float v[32];
    tc::tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16), v);
    if (valid) {
#pragma unroll
      for (int j = 0; j < 32; ++j) v[j] = fmaxf(v[j] + __bfloat162float(a.bias[j]), 0.f);
      if (EPI == 0) {
        const long long opix = ((long long)b * a.Ho + oy) * a.Wo + ox;
        uint4* dst = reinterpret_cast<uint4*>(a.out + opix * kN);
#pragma unroll
        for (int q4 = 0; q4 < 4; ++q4)
          dst[q4] = make_uint4(bf2(v[8 * q4], v[8 * q4 + 1]), bf2(v[8 * q4 + 2], v[8 * q4 + 3]),
                               bf2(v[8 * q4 + 4], v[8 * q4 + 5]), bf2(v[8 * q4 + 6], v[8 * q4 + 7]));
      } else {
        // the head sees the bf16 activation, as it would read it back from memory
#pragma unroll
        for (int j = 0; j < 32; ++j) v[j] = __bfloat162float(__float2bfloat16_rn(v[j]));
        // the block grid: ceil(H / 16) rows (the network's 2 Ho rows cropped), 2 Wo columns
        const int hb = (a.fr.H + 15) / 16, wb = 2 * a.Wo;
#pragma unroll
        for (int s = 0; s < 4; ++s) {
          if (2 * oy + (s >> 1) >= hb) continue;
          float z[3];
#pragma unroll
          for (int q = 0; q < 3; ++q) {
            const int j = 3 * s + q;
            float acc = sHead[12 * kN + j];
#pragma unroll
            for (int c = 0; c < kN; ++c) acc = fmaf(sHead[j * kN + c], v[c], acc);
            z[q] = acc;
          }
          const long long blk = ((long long)b * hb + 2 * oy + (s >> 1)) * wb + 2 * ox + (s & 1);
          a.prop[2 * blk] = (float)a.range * tanhf(z[0]);
          a.prop[2 * blk + 1] = (float)a.range * tanhf(z[1]);
          a.conf[blk] = 1.0f / (1.0f + expf(-z[2]));
        }
      }
    }
    tc::fence_before_sync();
    __syncthreads();  // TMEM read and staged rows consumed before the next tile
  }
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, L::TMEM_COLS);
  if (!ok && tid == 0 && a.status) atomicExch(a.status, (int)BAYER_ERR_TIMEOUT);
}

// ---------------------------------------------------------------------------
// Layers 3 and 4 and the head in one kernel (inference; layer-3 rows of at most
// 128 pixels).  CTA = (image, pair of layer-4 rows u0, u0 + 1): the 11 layer-2
// rows 4u0 - 3 .. 4u0 + 7 they depend on are staged at once (slot r = row 4u0
// - 3 + r, the tile kernel's layout, zero outside the map); layer-3 row t (=
// 2u0 - 1 + t, t = 0..4) reads slots 2t .. 2t + 2, so once its MMAs are done
// (and those of row t - 1) slot 2t is free and its epilogue writes the row
// there, bias + ReLU + bf16, in the same layout as layer 4's input; layer-4 row
// u0 + v then reads slots 2(2v + ky) and its epilogue evaluates the head.
// Layer-3 rows alternate between two TMEM accumulators, so the MMAs of row t + 1
// run while row t drains.  The layer-3 map never goes to memory.
// ---------------------------------------------------------------------------

constexpr int k34Rows = 11;                       // staged layer-2 rows
constexpr int k34Slot = 2 * 4 * 129 * 16;         // one staged row (NP = 129 pixels per parity)
constexpr int k34B = 9 * 32 * kN * 2;             // one layer's weight image
constexpr int k34Smem = 2 * k34B + kHeadW * 4 + k34Rows * k34Slot + 64 + 2 * kN * 4;
static_assert(k34Smem <= 227 * 1024, "shared memory");

struct Conv34Args {
  ConvTcArgs l3;              // layer 3: in = layer-2 map, wimg, bias, Ho/Wo = layer-3 dims; head fields
  const uint4* wimg4;         // layer 4 weights
  const __nv_bfloat16* bias4;
  int H4, W4;
};

constexpr int k34Threads = 256;  // two warps per TMEM lane quarter: channel halves, or the two layer-4 rows

__global__ void __launch_bounds__(k34Threads) conv34_head_tc_kernel(const Conv34Args c) {
  const ConvTcArgs& a = c.l3;
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* sB3 = smem;
  uint8_t* sB4 = smem + k34B;
  float* sHead = reinterpret_cast<float*>(smem + 2 * k34B);
  uint8_t* sX = smem + 2 * k34B + kHeadW * 4;  // kHeadW * 4 = 1584, a multiple of 16
  uint64_t* mbar = reinterpret_cast<uint64_t*>(sX + k34Rows * k34Slot);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mbar + 3);
  float* sBias = reinterpret_cast<float*>(sX + k34Rows * k34Slot + 64);  // layer 3, then layer 4
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int bands = (c.H4 + 1) / 2;
  const int b = blockIdx.x / bands, u0 = 2 * (blockIdx.x - b * bands);
  const int H3 = a.Ho, W3 = a.Wo, H2 = a.Hi, W2 = a.Wi;

  if (tid == 0) {
    for (int i = 0; i < 3; ++i) tc::mbar_init(&mbar[i], 1);
    tc::fence_mbar_init();
  }
  if (warp == 0) tc::tmem_alloc(tmem_slot, 128);  // acc 0, 1: layer 3; 2, 3: layer 4
  for (int i = tid; i < k34B / 16; i += k34Threads) {
    reinterpret_cast<uint4*>(sB3)[i] = __ldg(a.wimg + i);
    reinterpret_cast<uint4*>(sB4)[i] = __ldg(c.wimg4 + i);
  }
  for (int i = tid; i < kHeadW; i += k34Threads) sHead[i] = __bfloat162float(a.whead[i]);
  if (tid < 2 * kN) sBias[tid] = __bfloat162float(tid < kN ? a.bias[tid] : c.bias4[tid - kN]);
  // launched as a dependent of layer 2: read its output only after this wait
  tc::grid_dep_wait();
  tc::grid_dep_launch();
  const uint32_t sX_addr = tc::smem_addr(sX);
  // ---- stage layer-2 rows 4u0 - 3 .. 4u0 + 7, columns -1 .. 255, as five
  // cp.async groups: rows 0-2 (what layer-3 row 0 reads), then 2 rows each
  // (what row t adds), so that row t's MMAs wait only for groups 0..t
  {
    constexpr int NJ = 2 * kM + 1;
#pragma unroll 1
    for (int g = 0; g < 5; ++g) {
      const int r0 = g == 0 ? 0 : 2 * g + 1, nr = g == 0 ? 3 : 2;
      for (int it = tid; it < nr * NJ * 4; it += k34Threads) {
        const int rr = it / (NJ * 4), rem = it - rr * (NJ * 4);
        const int r = r0 + rr, j = rem >> 2, kc = rem & 3;
        const int iy = 4 * u0 - 3 + r, ix = j - 1;
        const bool in = iy >= 0 && iy < H2 && ix >= 0 && ix < W2;
        const __nv_bfloat16* src = in ? a.in + (((long long)b * H2 + iy) * W2 + ix) * 32 + kc * 8 : a.in;
        tc::cp_async16(sX_addr + r * k34Slot + (((j & 1) * 4 + kc) * 129 + (j >> 1)) * 16, src, in ? 16u : 0u);
      }
      tc::cp_async_commit();
    }
  }
  // groups 0..t landed for every thread, visible to the tensor cores
  auto rows_ready = [&](int t) {
    switch (t) {
      case 0: tc::cp_async_wait<4>(); break;
      case 1: tc::cp_async_wait<3>(); break;
      case 2: tc::cp_async_wait<2>(); break;
      case 3: tc::cp_async_wait<1>(); break;
      default: tc::cp_async_wait<0>(); break;
    }
    tc::fence_proxy_async();
  };
  rows_ready(0);
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tmem_slot;
  const uint32_t sB3_addr = tc::smem_addr(sB3), sB4_addr = tc::smem_addr(sB4);
  constexpr uint32_t idesc = tc::idesc_bf16_f32(kM, kN);
  const uint64_t a_base = tc::smem_desc(sX_addr, 129 * 16, 128);
  // a 3x3 conv row: 9 taps x 2 K steps, tap row ky from slot slot_of(ky)
  auto conv_row = [&](uint32_t bimg, int slot0, int slot_step, uint32_t d) {
    const uint64_t b_base = tc::smem_desc(bimg, 128, 9 * 4 * 128);
#pragma unroll
    for (int tap = 0; tap < 9; ++tap) {
      const int ky = tap / 3, kx = tap % 3;
      const uint64_t a_row = a_base + (uint64_t)((slot0 + slot_step * ky) * (k34Slot / 16));
#pragma unroll
      for (int s2 = 0; s2 < 2; ++s2) {
        const uint64_t ad = a_row + (uint64_t)(((kx & 1) * 4 + 2 * s2) * 129 + (kx >> 1));
        const uint64_t bd = b_base + (uint64_t)((tap * 4 + 2 * s2) * 8);
        tc::mma_bf16(d, ad, bd, idesc, (tap > 0 || s2 > 0) ? 1u : 0u);
      }
    }
  };
  bool ok = true;
  if (tid == 0) {
    tc::fence_after_sync();
    conv_row(sB3_addr, 0, 1, tmem);
    tc::commit(&mbar[0]);
  }
  rows_ready(1);
  __syncthreads();
  if (tid == 0) {
    tc::fence_after_sync();
    conv_row(sB3_addr, 2, 1, tmem + 32);
    tc::commit(&mbar[1]);
  }
  // warp w reads TMEM lanes 32 (w % 4) .. (pixel x); layer 3: channel half w / 4
  const int quarter = warp & 3, half = warp >> 2;
  const uint32_t lane_base = (uint32_t)(quarter * 32) << 16;
  const int x = quarter * 32 + lane;
  for (int t = 0; t < 5; ++t) {
    ok &= tc::mbar_wait(&mbar[t & 1], (uint32_t)((t >> 1) & 1), kWaitLimit);
    tc::fence_after_sync();
    float v[16];
    tc::tmem_ld16(tmem + lane_base + (uint32_t)(32 * (t & 1) + 16 * half), v);
    // layer-3 row y3 -> slot 2t as layer 4's input: pixel x at staged column x + 1
    const int y3 = 2 * u0 - 1 + t;
    const bool valid = y3 >= 0 && y3 < H3 && x < W3;
    uint8_t* dst = sX + 2 * t * k34Slot;
    const int j = x + 1;
#pragma unroll
    for (int k2 = 0; k2 < 2; ++k2) {
      const int kc = 2 * half + k2;
      uint4 o = make_uint4(0, 0, 0, 0);
      if (valid) {
        float u[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) u[e] = v[8 * k2 + e] + sBias[8 * kc + e];
        o = make_uint4(tc::bf2_relu(u[0], u[1]), tc::bf2_relu(u[2], u[3]), tc::bf2_relu(u[4], u[5]),
                       tc::bf2_relu(u[6], u[7]));
      }
      *reinterpret_cast<uint4*>(dst + (((j & 1) * 4 + kc) * 129 + (j >> 1)) * 16) = o;
      if (x == 0) *reinterpret_cast<uint4*>(dst + (kc * 129) * 16) = make_uint4(0, 0, 0, 0);  // column -1
    }
    tc::fence_before_sync();
    if (t + 2 <= 4) rows_ready(t + 2);
    tc::fence_proxy_async();  // the row is layer 4's operand (async proxy)
    __syncthreads();          // accumulator t & 1 drained, slot 2t written, row t + 2's inputs landed
    if (tid == 0 && t + 2 <= 4) {
      tc::fence_after_sync();
      conv_row(sB3_addr, 2 * (t + 2), 1, tmem + (uint32_t)(32 * (t & 1)));
      tc::commit(&mbar[t & 1]);
    }
  }
  // ---- layer 4: rows u0 + v, v = 0, 1, tap row ky from layer-3 row 2v + ky in slot 2(2v + ky)
  if (tid == 0) {
    tc::fence_after_sync();
    conv_row(sB4_addr, 0, 2, tmem + 64);
    conv_row(sB4_addr, 4, 2, tmem + 96);
    tc::commit(&mbar[2]);
  }
  ok &= tc::mbar_wait(&mbar[2], 0, kWaitLimit);
  tc::fence_after_sync();
  const int hb = (a.fr.H + 15) / 16, wb = 2 * c.W4;  // the block grid (2 H4 rows cropped to ceil(H / 16))
  {
    // warps 0-3: layer-4 row u0, warps 4-7: row u0 + 1
    const int v2 = half;
    float v[32];
    tc::tmem_ld32(tmem + lane_base + (uint32_t)(64 + 32 * v2), v);
    const int y4 = u0 + v2;
    if (y4 < c.H4 && x < c.W4) {
      // the head sees the bf16 activation, as it would read it back from memory
#pragma unroll
      for (int jj = 0; jj < 32; ++jj)
        v[jj] = __bfloat162float(__float2bfloat16_rn(fmaxf(v[jj] + sBias[kN + jj], 0.f)));
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        if (2 * y4 + (s >> 1) >= hb) continue;
        float z[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          const int jh = 3 * s + q;
          float acc = sHead[12 * kN + jh];
#pragma unroll
          for (int cc = 0; cc < kN; ++cc) acc = fmaf(sHead[jh * kN + cc], v[cc], acc);
          z[q] = acc;
        }
        const long long blk = ((long long)b * hb + 2 * y4 + (s >> 1)) * wb + 2 * x + (s & 1);
        a.prop[2 * blk] = (float)a.range * tanhf(z[0]);
        a.prop[2 * blk + 1] = (float)a.range * tanhf(z[1]);
        a.conf[blk] = 1.0f / (1.0f + expf(-z[2]));
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, 128);
  if (!ok && tid == 0 && a.status) atomicExch(a.status, (int)BAYER_ERR_TIMEOUT);
}

template <int CIN, int EPI>
cudaError_t launch_t(const ConvTcArgs& a, cudaStream_t st) {
  using L = RowConvLayout<CIN, EPI>;
  auto kern = conv3x3_tc_kernel<CIN, EPI>;
  int dev = 0, nsm = 148;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int per_sm = tc::ctas_per_sm(kern, kM, L::SMEM, L::TMEM_COLS);
  const long long ntiles = (long long)a.batch * a.Ho * ((a.Wo + kM - 1) / kM);
  if (ntiles < 1) return cudaSuccess;
  long long grid = (long long)nsm * per_sm;
  if (grid > ntiles) grid = ntiles;
  return tc::launch_dependent(kern, dim3((unsigned)grid), dim3(kM), L::SMEM, st, a);
}

template <int CIN, int EPI>
cudaError_t configure_t() {
  using L = RowConvLayout<CIN, EPI>;
  auto kern = conv3x3_tc_kernel<CIN, EPI>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, L::SMEM);
  // prefer the largest shared-memory carveout so several CTAs fit per SM
  if (e == cudaSuccess) e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  return e;
}

}  // namespace

size_t conv_tc_weight_bytes(int cin_op) { return (size_t)9 * cin_op * kN * 2; }

cudaError_t pack_conv_tc_weights(const uint16_t* w, const int* w_off, const size_t* img_off, uint16_t* img,
                                 int* zero_words, cudaStream_t st) {
  PackArgs pa;
  pa.zero_words = zero_words;
  pa.w = reinterpret_cast<const __nv_bfloat16*>(w);
  for (int l = 0; l < 4; ++l) {
    pa.w_off[l] = w_off[l];
    pa.img_off[l] = (unsigned)img_off[l];
  }
  const int n = kN * 9 * 8 + 3 * kN * 9 * 32;
  return tc::launch_dependent(pack_conv_tc_weights_kernel, dim3((n + 255) / 256), dim3(256), 0, st, pa,
                              reinterpret_cast<__nv_bfloat16*>(img));
}

cudaError_t configure_conv_tc() {
  cudaError_t e;
  if ((e = configure_t<32, 0>()) != cudaSuccess) return e;
  if ((e = configure_t<32, 1>()) != cudaSuccess) return e;
  return cudaFuncSetAttribute(conv34_head_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, k34Smem);
}

bool conv34_head_supported(int W3) { return W3 >= 1 && W3 <= kM; }

cudaError_t launch_conv34_head_tc(const ConvTcArgs& l3, const uint4* wimg4, const __nv_bfloat16* bias4, int H4, int W4,
                                  cudaStream_t st) {
  if (!conv34_head_supported(l3.Wo)) return cudaErrorInvalidValue;
  Conv34Args c;
  c.l3 = l3;
  c.wimg4 = wimg4;
  c.bias4 = bias4;
  c.H4 = H4;
  c.W4 = W4;
  const long long grid = (long long)l3.batch * ((H4 + 1) / 2);
  if (grid < 1) return cudaSuccess;
  return tc::launch_dependent(conv34_head_tc_kernel, dim3((unsigned)grid), dim3(k34Threads), k34Smem, st, c);
}

cudaError_t launch_conv_tc(const ConvTcArgs& a, int layer, bool head, cudaStream_t st) {
  if (layer > 1 && !head) return launch_t<32, 0>(a, st);
  if (layer > 1 && head) return launch_t<32, 1>(a, st);
  return cudaErrorInvalidValue;
}

}  // namespace bme

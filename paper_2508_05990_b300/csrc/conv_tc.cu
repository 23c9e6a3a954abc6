// 3x3 convolution (zero pad 1, stride 1 or 2) as an implicit GEMM on the 5th-
// generation tensor cores: BF16 operands in shared memory, FP32 accumulators
// in tensor memory (TMEM), bias + optional ReLU epilogue, BF16 NHWC output.
//
//   D[m, n] = sum_k A[m, k] * B[k, n],  m = output pixel, n = output channel,
//   k = tap * CIN + ci,  A[m, k] = input at (S*oy + ky - 1, S*ox + kx - 1, ci).
//
// Tile = 128 consecutive output pixels of one output row (MMA M = 128,
// N = COUT); CTA = 128 threads, persistent over tiles, all nine taps' weights
// resident in shared memory.  Per tile the CTA stages the three input rows
// once (coalesced 16-byte loads; no im2col copy), after one barrier thread 0
// issues 9 * CIN/16 MMAs whose A operands are shifted views of the staged rows
// and commits them to an mbarrier that gates the epilogue (TMEM -> registers
// -> bias, ReLU, bf16 -> global).  Several CTAs per SM overlap one tile's
// staging with another's MMAs and epilogue.  Every mbarrier wait is bounded;
// on expiry the kernel records BAYER_ERR_TIMEOUT in the status word, frees its
// TMEM and finishes.
//
// SRC 1 (layer 1 of the proposal network) gathers straight from the Bayer
// frames: the 8 half-resolution planes x = v/2048 - 1 are split exactly into
// two bf16 channels, hi = (v >> 4)/128 - 1 and lo = (v & 15)/16, with weights w
// and w/128, so that hi*w + lo*(w/128) = x*w exactly.
#include <cuda_bf16.h>

#include "common.cuh"
#include "kernels.cuh"
#include "tc_common.cuh"

namespace bme {

namespace {

constexpr int kM = 128;  // output pixels per tile (MMA M)
constexpr uint32_t kWaitLimit = 1u << 20;

// Shared-memory plan of one CTA.  The three input rows a tile needs are staged
// once, split into S column-parity planes (S = stride) and into 16-byte
// channel chunks: element (row rho, plane q, chunk kc, pixel p) at
// (((rho*S + q)*KC + kc)*NP + p)*16.  Output pixel m of tap (ky, kx) then reads
// plane q = kx % S at pixel m + kx / S, so every tap's A operand is the staged
// tensor itself at a shifted start address: core matrices of 8 consecutive
// pixels (SBO = 128 bytes), the next K chunk one plane further (LBO = NP*16).
template <int CIN, int NB, int S>
struct RowConvLayout {
  static constexpr int KC = CIN / 8;
  static constexpr int NJ = S * (kM - 1) + 3;       // staged input columns
  static constexpr int NP = (NJ + S - 1) / S;       // pixels per parity plane
  static constexpr int STAGE_BYTES = 3 * S * KC * NP * 16;
  static constexpr int B_BYTES = 9 * CIN * NB * 2;  // this CTA's NB output channels
  static constexpr int TMEM_COLS = NB < 32 ? 32 : NB;
  static constexpr int SMEM = B_BYTES + STAGE_BYTES + 64;
  static_assert(CIN % 16 == 0 && NB % 32 == 0 && NB <= 256, "shape");
  static_assert(B_BYTES % 128 == 0 && STAGE_BYTES % 16 == 0, "alignment");
  static_assert(SMEM <= 227 * 1024, "shared memory");
};

__device__ __forceinline__ uint32_t bf2(float a, float b) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t*>(&v);
}

// hi/lo bf16 pair of a 12-bit sample (SRC 1): hi = (v >> 4)/128 - 1, lo = (v & 15)/16.
__device__ __forceinline__ uint32_t split12(uint32_t v) {
  return bf2((float)(v >> 4) * (1.0f / 128.0f) - 1.0f, (float)(v & 15u) * (1.0f / 16.0f));
}

// SRC: 0 bf16 NHWC input, 1 Bayer frames (hi/lo split), 2 float32 NHWC input
// rounded to bf16 while staging.  OUTF: 0 bf16 NHWC output, 1 float32 NHWC.
// Output channels are split over CTAs, NB per CTA (a.cout = total).
template <int CIN, int NB, int S, int SRC, int OUTF, bool RELU>
__global__ void __launch_bounds__(kM) conv3x3_tc_kernel(const ConvTcArgs a) {
  using L = RowConvLayout<CIN, NB, S>;
  constexpr int COUT = NB;
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* sB = smem;
  uint8_t* sX = smem + L::B_BYTES;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + L::B_BYTES + L::STAGE_BYTES);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mbar + 1);
  const int tid = threadIdx.x, warp = tid >> 5;

  if (tid == 0) {
    tc::mbar_init(&mbar[0], 1);
    tc::fence_mbar_init();
  }
  if (warp == 0) tc::tmem_alloc(tmem_slot, L::TMEM_COLS);
  const int nsplit = a.cout / NB;
  const int split = blockIdx.x % nsplit;
  const int n0 = split * NB;
  // weights of channels n0..n0+NB-1 -> B (K-major, k = tap*CIN + ci): element
  // (n, k) at (n/8)*(9*KC)*128 + (k/8)*128 + (n%8)*16 + (k%8)*2
  for (int i = tid; i < COUT * 9 * CIN; i += kM) {
    const int n = i / (9 * CIN), k = i - n * 9 * CIN;
    const int tap = k / CIN, ci = k - tap * CIN;
    float wv;
    if (SRC != 1) {
      wv = __bfloat162float(a.w[((n0 + n) * CIN + ci) * 9 + tap]);
    } else {
      wv = __bfloat162float(a.w[(n * 8 + (ci >> 1)) * 9 + tap]);
      if (ci & 1) wv *= (1.0f / 128.0f);
    }
    __nv_bfloat16* dst =
        reinterpret_cast<__nv_bfloat16*>(sB + (n >> 3) * (9 * L::KC) * 128 + (k >> 3) * 128 + (n & 7) * 16) + (k & 7);
    *dst = __float2bfloat16_rn(wv);
  }
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tmem_slot;
  const uint32_t sX_addr = tc::smem_addr(sX), sB_addr = tc::smem_addr(sB);
  constexpr uint32_t idesc = tc::idesc_bf16_f32(kM, COUT);
  const int segs = (a.Wo + kM - 1) / kM;
  const long long ntiles = (long long)a.batch * a.Ho * segs;
  uint32_t phase = 0;
  bool ok = true;

  const int cta_stride = gridDim.x / nsplit;
  for (long long tile = blockIdx.x / nsplit; tile < ntiles; tile += cta_stride) {
    const int seg = (int)(tile % segs);
    const long long row = tile / segs;
    const int b = (int)(row / a.Ho), oy = (int)(row - (long long)b * a.Ho);
    const int ox0 = seg * kM;
    const int c0 = S * ox0 - 1;  // input column of staged column 0

    // ---- stage rows S*oy - 1 .. S*oy + 1, columns c0 .. c0 + NJ - 1
    constexpr int NITEM = 3 * L::NJ;
    for (int it0 = 0; it0 < NITEM; it0 += 2 * kM) {
      if (SRC == 2) {
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const int it = it0 + u * kM + tid;
          if (it >= NITEM) continue;
          const int rho = it / L::NJ, j = it - rho * L::NJ;
          const int iy = S * oy - 1 + rho, ix = c0 + j;
          const bool in_ok = iy >= 0 && iy < a.Hi && ix >= 0 && ix < a.Wi;
          const float4* src = reinterpret_cast<const float4*>(a.in_f32 + (((long long)b * a.Hi + iy) * a.Wi + ix) * CIN);
          const int q = j % S, pp = j / S;
#pragma unroll 4
          for (int kc = 0; kc < L::KC; ++kc) {
            const float4 f0 = in_ok ? __ldg(src + 2 * kc) : make_float4(0.f, 0.f, 0.f, 0.f);
            const float4 f1 = in_ok ? __ldg(src + 2 * kc + 1) : make_float4(0.f, 0.f, 0.f, 0.f);
            *reinterpret_cast<uint4*>(sX + (((rho * S + q) * L::KC + kc) * L::NP + pp) * 16) =
                make_uint4(bf2(f0.x, f0.y), bf2(f0.z, f0.w), bf2(f1.x, f1.y), bf2(f1.z, f1.w));
          }
        }
      } else if (SRC == 0) {
        uint4 v[2][L::KC];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const int it = it0 + u * kM + tid;
          const int rho = it / L::NJ, j = it - rho * L::NJ;
          const int iy = S * oy - 1 + rho, ix = c0 + j;
          const bool in_ok = it < NITEM && iy >= 0 && iy < a.Hi && ix >= 0 && ix < a.Wi;
          const uint4* src = reinterpret_cast<const uint4*>(a.in + (((long long)b * a.Hi + iy) * a.Wi + ix) * CIN);
#pragma unroll
          for (int kc = 0; kc < L::KC; ++kc) v[u][kc] = in_ok ? __ldg(src + kc) : make_uint4(0, 0, 0, 0);
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const int it = it0 + u * kM + tid;
          if (it >= NITEM) continue;
          const int rho = it / L::NJ, j = it - rho * L::NJ;
          const int q = j % S, pp = j / S;
#pragma unroll
          for (int kc = 0; kc < L::KC; ++kc)
            *reinterpret_cast<uint4*>(sX + (((rho * S + q) * L::KC + kc) * L::NP + pp) * 16) = v[u][kc];
        }
      } else {
        uint32_t raw[2][8];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const int it = it0 + u * kM + tid;
          const int rho = it / L::NJ, j = it - rho * L::NJ;
          const int iy = S * oy - 1 + rho, ix = c0 + j;
          const bool in_ok = it < NITEM && iy >= 0 && iy < a.Hi && ix >= 0 && ix < a.Wi;
#pragma unroll
          for (int c = 0; c < 8; ++c) {
            const uint16_t* f = (c < 4 ? a.fr.ref + (long long)b * a.fr.ref_bs : a.fr.cur + (long long)b * a.fr.cur_bs);
            const int pl = c & 3;
            raw[u][c] = in_ok ? (uint32_t)__ldg(f + (long long)(2 * iy + (pl >> 1)) * a.fr.pitch + 2 * ix + (pl & 1))
                              : 0xFFFFFFFFu;
          }
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const int it = it0 + u * kM + tid;
          if (it >= NITEM) continue;
          const int rho = it / L::NJ, j = it - rho * L::NJ;
          const int q = j % S, pp = j / S;
          uint32_t wd[8];
#pragma unroll
          for (int c = 0; c < 8; ++c) wd[c] = raw[u][c] == 0xFFFFFFFFu ? 0u : split12(raw[u][c]);
          *reinterpret_cast<uint4*>(sX + (((rho * S + q) * L::KC + 0) * L::NP + pp) * 16) =
              make_uint4(wd[0], wd[1], wd[2], wd[3]);
          *reinterpret_cast<uint4*>(sX + (((rho * S + q) * L::KC + 1) * L::NP + pp) * 16) =
              make_uint4(wd[4], wd[5], wd[6], wd[7]);
        }
      }
    }
    tc::fence_proxy_async();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after_sync();
#pragma unroll
      for (int tap = 0; tap < 9; ++tap) {
        const int ky = tap / 3, kx = tap % 3;
        const int q = kx % S, dp = kx / S;
#pragma unroll
        for (int s2 = 0; s2 < CIN / 16; ++s2) {
          const uint32_t a_addr = sX_addr + (((ky * S + q) * L::KC + 2 * s2) * L::NP + dp) * 16;
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
    const long long opix = ((long long)b * a.Ho + oy) * a.Wo + ox;
#pragma unroll
    for (int cc = 0; cc < COUT; cc += 32) {
      float v[32];
      tc::tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)cc, v);
      if (valid) {
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          v[j] += __bfloat162float(a.bias[n0 + cc + j]);
          if (RELU) v[j] = fmaxf(v[j], 0.f);
        }
        if (OUTF == 0) {
          uint4* dst = reinterpret_cast<uint4*>(a.out + opix * a.cout + n0 + cc);
#pragma unroll
          for (int q4 = 0; q4 < 4; ++q4)
            dst[q4] = make_uint4(bf2(v[8 * q4], v[8 * q4 + 1]), bf2(v[8 * q4 + 2], v[8 * q4 + 3]),
                                 bf2(v[8 * q4 + 4], v[8 * q4 + 5]), bf2(v[8 * q4 + 6], v[8 * q4 + 7]));
        } else {
          float4* dst = reinterpret_cast<float4*>(a.out_f32 + opix * a.cout + n0 + cc);
#pragma unroll
          for (int q4 = 0; q4 < 8; ++q4) dst[q4] = make_float4(v[4 * q4], v[4 * q4 + 1], v[4 * q4 + 2], v[4 * q4 + 3]);
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

template <int CIN, int NB, int S, int SRC, int OUTF, bool RELU>
cudaError_t launch_t(const ConvTcArgs& a, cudaStream_t st) {
  using L = RowConvLayout<CIN, NB, S>;
  auto kern = conv3x3_tc_kernel<CIN, NB, S, SRC, OUTF, RELU>;
  if (a.cout % NB != 0) return cudaErrorInvalidValue;
  const int nsplit = a.cout / NB;
  int dev = 0, nsm = 148;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int per_sm = tc::ctas_per_sm(kern, kM, L::SMEM, L::TMEM_COLS);
  const long long ntiles = (long long)a.batch * a.Ho * ((a.Wo + kM - 1) / kM);
  long long per_split = (long long)nsm * per_sm / nsplit;
  if (per_split > ntiles) per_split = ntiles;
  if (per_split < 1) per_split = 1;
  if (ntiles < 1) return cudaSuccess;
  kern<<<(unsigned)(per_split * nsplit), kM, L::SMEM, st>>>(a);
  return cudaGetLastError();
}

template <int CIN, int NB, int S, int SRC, int OUTF, bool RELU>
cudaError_t configure_t() {
  using L = RowConvLayout<CIN, NB, S>;
  auto kern = conv3x3_tc_kernel<CIN, NB, S, SRC, OUTF, RELU>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, L::SMEM);
  // prefer the largest shared-memory carveout so several CTAs fit per SM
  if (e == cudaSuccess) e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  return e;
}

}  // namespace

cudaError_t configure_conv_tc() {
  cudaError_t e;
  if ((e = configure_t<16, 32, 2, 1, 0, true>()) != cudaSuccess) return e;
  return configure_t<32, 32, 2, 0, 0, true>();
}

cudaError_t launch_conv_tc(const ConvTcArgs& a, int cin, int stride, int src, int outf, bool relu, cudaStream_t st) {
  if (cin == 16 && stride == 2 && src == 1 && outf == 0 && relu && a.cout == 32)
    return launch_t<16, 32, 2, 1, 0, true>(a, st);
  if (cin == 32 && stride == 2 && src == 0 && outf == 0 && relu && a.cout == 32)
    return launch_t<32, 32, 2, 0, 0, true>(a, st);
  return cudaErrorInvalidValue;
}

}  // namespace bme

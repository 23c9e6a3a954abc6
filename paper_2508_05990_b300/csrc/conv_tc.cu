// 3x3 convolution (zero pad 1, stride 1 or 2) as an implicit GEMM on the 5th-
// generation tensor cores: BF16 operands in shared memory, FP32 accumulators
// in tensor memory (TMEM), bias + optional ReLU epilogue, BF16 NHWC output.
//
//   D[m, n] = sum_k A[m, k] * B[k, n],  m = output pixel, n = output channel,
//   k = tap * CIN + ci,  A[m, k] = input at (S*oy + ky - 1, S*ox + kx - 1, ci).
//
// CTA = 128 threads = 128 output pixels (MMA M = 128, N = COUT); persistent
// over pixel tiles.  All nine taps' weights stay in shared memory.  Per tile
// each thread gathers its pixel's 9 x CIN input values into the A tile
// (canonical no-swizzle K-major layout: 8-row x 16-byte core matrices), three
// taps' loads in flight at a time; after one barrier thread 0 issues the
// 9*CIN/16 MMAs (K = 16 each) and commits them to an mbarrier that gates the
// epilogue (TMEM -> registers -> bias, ReLU, bf16 -> global).  Several CTAs
// per SM overlap one tile's gather with another's MMAs and epilogue.  Every
// mbarrier wait is bounded; on expiry the kernel records BAYER_ERR_TIMEOUT in
// the status word, frees its TMEM and finishes.
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

constexpr int kM = 128;
constexpr uint32_t kWaitLimit = 1u << 20;

template <int CIN, int COUT>
struct ConvTcLayout {
  static constexpr int KC = CIN / 8;            // 16-byte K chunks per tap
  static constexpr int A_BYTES = kM * 9 * CIN * 2;  // all nine taps of one tile
  static constexpr int B_BYTES = 9 * CIN * COUT * 2;
  static constexpr int TMEM_COLS = COUT < 32 ? 32 : COUT;
  static constexpr int SMEM = B_BYTES + A_BYTES + 64;
  static_assert(CIN % 16 == 0 && COUT % 32 == 0 && COUT <= 256, "shape");
};

__device__ __forceinline__ uint32_t bf2(float a, float b) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t*>(&v);
}

template <int CIN, int COUT, int STRIDE, int SRC, bool RELU>
__global__ void __launch_bounds__(kM) conv3x3_tc_kernel(const ConvTcArgs a) {
  using L = ConvTcLayout<CIN, COUT>;
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* sB = smem;
  uint8_t* sA = smem + L::B_BYTES;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + L::B_BYTES + L::A_BYTES);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mbar + 2);
  const int tid = threadIdx.x, warp = tid >> 5;

  if (tid == 0) {
    tc::mbar_init(&mbar[0], 1);
    tc::fence_mbar_init();
  }
  if (warp == 0) tc::tmem_alloc(tmem_slot, L::TMEM_COLS);
  // weights -> B (K-major, k = tap*CIN + ci): element (n, k) at
  // (n/8)*(9*KC)*128 + (k/8)*128 + (n%8)*16 + (k%8)*2
  for (int i = tid; i < COUT * 9 * CIN; i += kM) {
    const int n = i / (9 * CIN), k = i - n * 9 * CIN;
    const int tap = k / CIN, ci = k - tap * CIN;
    float wv;
    if (SRC == 0) {
      wv = __bfloat162float(a.w[(n * CIN + ci) * 9 + tap]);
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
  const uint32_t sA_addr = tc::smem_addr(sA), sB_addr = tc::smem_addr(sB);
  constexpr uint32_t idesc = tc::idesc_bf16_f32(kM, COUT);
  constexpr int KCA = 9 * L::KC;  // K chunks of the full A tile
  const long long npix = (long long)a.batch * a.Ho * a.Wo;
  const long long ntiles = (npix + kM - 1) / kM;
  uint32_t phase = 0;
  bool ok = true;
  // A tile (K-major, k = tap*CIN + ci): row m, chunk kc at (m/8)*KCA*128 + kc*128 + (m%8)*16
  uint8_t* arow = sA + (tid >> 3) * (KCA * 128) + (tid & 7) * 16;

  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const long long pix = tile * kM + tid;
    const bool valid = pix < npix;
    int b = 0, oy = 0, ox = 0;
    if (valid) {
      b = (int)(pix / ((long long)a.Ho * a.Wo));
      const int r = (int)(pix - (long long)b * a.Ho * a.Wo);
      oy = r / a.Wo;
      ox = r - oy * a.Wo;
    }
    // gather the nine taps, three at a time (all loads of a group in flight together)
#pragma unroll
    for (int g = 0; g < 3; ++g) {
      if (SRC == 0) {
        uint4 v[3][L::KC];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          const int tap = 3 * g + j, ky = tap / 3, kx = tap % 3;
          const int iy = STRIDE * oy + ky - 1, ix = STRIDE * ox + kx - 1;
          const bool in_ok = valid && iy >= 0 && iy < a.Hi && ix >= 0 && ix < a.Wi;
          const uint4* src = reinterpret_cast<const uint4*>(a.in + (((long long)b * a.Hi + iy) * a.Wi + ix) * CIN);
#pragma unroll
          for (int kc = 0; kc < L::KC; ++kc) v[j][kc] = in_ok ? __ldg(src + kc) : make_uint4(0, 0, 0, 0);
        }
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
          for (int kc = 0; kc < L::KC; ++kc)
            *reinterpret_cast<uint4*>(arow + ((3 * g + j) * L::KC + kc) * 128) = v[j][kc];
      } else {
        uint32_t raw[3][8];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          const int tap = 3 * g + j, ky = tap / 3, kx = tap % 3;
          const int iy = 2 * oy + ky - 1, ix = 2 * ox + kx - 1;
          const bool in_ok = valid && iy >= 0 && iy < a.Hi && ix >= 0 && ix < a.Wi;
#pragma unroll
          for (int c = 0; c < 8; ++c) {
            const uint16_t* f = (c < 4 ? a.fr.ref + (long long)b * a.fr.ref_bs : a.fr.cur + (long long)b * a.fr.cur_bs);
            const int p = c & 3;
            raw[j][c] = in_ok ? (uint32_t)__ldg(f + (long long)(2 * iy + (p >> 1)) * a.fr.pitch + 2 * ix + (p & 1))
                              : 0xFFFFFFFFu;  // marks zero padding
          }
        }
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          uint32_t wd[8];
#pragma unroll
          for (int c = 0; c < 8; ++c) {
            const uint32_t v = raw[j][c];
            const float hi = v == 0xFFFFFFFFu ? 0.f : (float)(v >> 4) * (1.0f / 128.0f) - 1.0f;
            const float lo = v == 0xFFFFFFFFu ? 0.f : (float)(v & 15u) * (1.0f / 16.0f);
            wd[c] = bf2(hi, lo);
          }
          const int tap = 3 * g + j;
          *reinterpret_cast<uint4*>(arow + (tap * 2) * 128) = make_uint4(wd[0], wd[1], wd[2], wd[3]);
          *reinterpret_cast<uint4*>(arow + (tap * 2 + 1) * 128) = make_uint4(wd[4], wd[5], wd[6], wd[7]);
        }
      }
    }
    tc::fence_proxy_async();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after_sync();
#pragma unroll
      for (int s = 0; s < 9 * CIN / 16; ++s) {
        const uint64_t ad = tc::smem_desc(sA_addr + 2 * s * 128, 128, KCA * 128);
        const uint64_t bd = tc::smem_desc(sB_addr + 2 * s * 128, 128, KCA * 128);
        tc::mma_bf16(tmem, ad, bd, idesc, s > 0 ? 1u : 0u);
      }
      tc::commit(&mbar[0]);
    }
    ok &= tc::mbar_wait(&mbar[0], phase & 1, kWaitLimit);
    ++phase;
    tc::fence_after_sync();
#pragma unroll
    for (int c0 = 0; c0 < COUT; c0 += 32) {
      float v[32];
      tc::tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
      if (valid) {
        uint32_t o[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          float x0 = v[2 * j] + __bfloat162float(a.bias[c0 + 2 * j]);
          float x1 = v[2 * j + 1] + __bfloat162float(a.bias[c0 + 2 * j + 1]);
          if (RELU) {
            x0 = fmaxf(x0, 0.f);
            x1 = fmaxf(x1, 0.f);
          }
          o[j] = bf2(x0, x1);
        }
        uint4* dst = reinterpret_cast<uint4*>(a.out + pix * COUT + c0);
#pragma unroll
        for (int q = 0; q < 4; ++q) dst[q] = make_uint4(o[4 * q], o[4 * q + 1], o[4 * q + 2], o[4 * q + 3]);
      }
    }
    tc::fence_before_sync();
    __syncthreads();  // TMEM read and A consumed before the next tile overwrites them
  }
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, L::TMEM_COLS);
  if (!ok && tid == 0 && a.status) atomicExch(a.status, (int)BAYER_ERR_TIMEOUT);
}

template <int CIN, int COUT, int STRIDE, int SRC, bool RELU>
cudaError_t launch_t(const ConvTcArgs& a, cudaStream_t st) {
  using L = ConvTcLayout<CIN, COUT>;
  auto kern = conv3x3_tc_kernel<CIN, COUT, STRIDE, SRC, RELU>;
  int dev = 0, nsm = 148, per_sm = 1;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kM, L::SMEM);
  if (e != cudaSuccess) return e;
  const int tmem_limit = 512 / L::TMEM_COLS;
  if (per_sm > tmem_limit) per_sm = tmem_limit;
  if (per_sm < 1) per_sm = 1;
  const long long ntiles = ((long long)a.batch * a.Ho * a.Wo + kM - 1) / kM;
  long long grid = (long long)nsm * per_sm;
  if (grid > ntiles) grid = ntiles;
  if (grid < 1) return cudaSuccess;
  kern<<<(unsigned)grid, kM, L::SMEM, st>>>(a);
  return cudaGetLastError();
}

template <int CIN, int COUT, int STRIDE, int SRC, bool RELU>
cudaError_t configure_t() {
  using L = ConvTcLayout<CIN, COUT>;
  return cudaFuncSetAttribute(conv3x3_tc_kernel<CIN, COUT, STRIDE, SRC, RELU>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, L::SMEM);
}

}  // namespace

cudaError_t configure_conv_tc() {
  cudaError_t e;
  if ((e = configure_t<16, 32, 2, 1, true>()) != cudaSuccess) return e;
  return configure_t<32, 32, 2, 0, true>();
}

cudaError_t launch_conv_tc(const ConvTcArgs& a, int cin, int cout, int stride, int src, bool relu, cudaStream_t st) {
  if (cin == 16 && cout == 32 && stride == 2 && src == 1 && relu) return launch_t<16, 32, 2, 1, true>(a, st);
  if (cin == 32 && cout == 32 && stride == 2 && src == 0 && relu) return launch_t<32, 32, 2, 0, true>(a, st);
  return cudaErrorInvalidValue;
}

}  // namespace bme

// 3x3 stride-1 convolution in float32 on the SIMT cores (the FP32 run of the
// refine convolution, beside the BF16 tensor-core run).
//
// CTA = 128 threads = an 8 x 16 tile of output pixels for one group of 32
// output channels; input channels are consumed in chunks of 16: the CTA
// stages the 10 x 18 input halo tile of the chunk and the chunk's
// 9 x 16 x 32 weights in shared memory, and each thread accumulates its
// pixel's 32 outputs in registers (weights read as broadcast 128-bit loads).
#include "common.cuh"
#include "kernels.cuh"

namespace bme {

namespace {

constexpr int kTY = 8, kTX = 16, kCI = 16, kCO = 32;

__global__ void __launch_bounds__(kTY * kTX) conv3x3_f32_kernel(const float* __restrict__ in, int H, int W, int cin,
                                                                 const float* __restrict__ w,
                                                                 const float* __restrict__ bias, int cout, int relu,
                                                                 float* __restrict__ out) {
  __shared__ float xs[(kTY + 2) * (kTX + 2) * kCI];
  __shared__ __align__(16) float ws[9 * kCI * kCO];  // [tap][ci][co]
  const int ngroups = cout / kCO;
  const int b = blockIdx.z / ngroups, co0 = (blockIdx.z % ngroups) * kCO;
  const int ty = threadIdx.x / kTX, tx = threadIdx.x % kTX;
  const int oy = blockIdx.y * kTY + ty, ox = blockIdx.x * kTX + tx;
  const float* inb = in + (long long)b * H * W * cin;
  float acc[kCO];
#pragma unroll
  for (int c = 0; c < kCO; ++c) acc[c] = bias[co0 + c];
  for (int ci0 = 0; ci0 < cin; ci0 += kCI) {
    __syncthreads();
    for (int i = threadIdx.x; i < (kTY + 2) * (kTX + 2) * kCI; i += blockDim.x) {
      const int c = i % kCI, p = i / kCI;
      const int yy = blockIdx.y * kTY - 1 + p / (kTX + 2), xx = blockIdx.x * kTX - 1 + p % (kTX + 2);
      xs[i] = (yy >= 0 && yy < H && xx >= 0 && xx < W) ? __ldg(inb + ((long long)yy * W + xx) * cin + ci0 + c) : 0.f;
    }
    for (int i = threadIdx.x; i < 9 * kCI * kCO; i += blockDim.x) {
      const int co = i % kCO, r = i / kCO, ci = r % kCI, tap = r / kCI;
      ws[i] = __ldg(w + ((long long)(co0 + co) * cin + ci0 + ci) * 9 + tap);
    }
    __syncthreads();
#pragma unroll 1
    for (int tap = 0; tap < 9; ++tap) {
      const int ky = tap / 3, kx = tap % 3;
      const float* xp = xs + ((ty + ky) * (kTX + 2) + tx + kx) * kCI;
#pragma unroll 4
      for (int ci = 0; ci < kCI; ++ci) {
        const float x = xp[ci];
        const float4* wr = reinterpret_cast<const float4*>(ws + (tap * kCI + ci) * kCO);
#pragma unroll
        for (int q = 0; q < kCO / 4; ++q) {
          const float4 wv = wr[q];
          acc[4 * q + 0] = fmaf(x, wv.x, acc[4 * q + 0]);
          acc[4 * q + 1] = fmaf(x, wv.y, acc[4 * q + 1]);
          acc[4 * q + 2] = fmaf(x, wv.z, acc[4 * q + 2]);
          acc[4 * q + 3] = fmaf(x, wv.w, acc[4 * q + 3]);
        }
      }
    }
  }
  if (oy < H && ox < W) {
    float4* dst = reinterpret_cast<float4*>(out + (((long long)b * H + oy) * W + ox) * cout + co0);
#pragma unroll
    for (int q = 0; q < kCO / 4; ++q) {
      float4 v = make_float4(acc[4 * q], acc[4 * q + 1], acc[4 * q + 2], acc[4 * q + 3]);
      if (relu) {
        v.x = fmaxf(v.x, 0.f);
        v.y = fmaxf(v.y, 0.f);
        v.z = fmaxf(v.z, 0.f);
        v.w = fmaxf(v.w, 0.f);
      }
      dst[q] = v;
    }
  }
}

}  // namespace

cudaError_t launch_conv3x3_f32(const float* in, int batch, int H, int W, int cin, const float* w, const float* bias,
                               int cout, bool relu, float* out, cudaStream_t st) {
  if (cin % kCI != 0 || cout % kCO != 0) return cudaErrorInvalidValue;
  dim3 grid((W + kTX - 1) / kTX, (H + kTY - 1) / kTY, batch * (cout / kCO));
  conv3x3_f32_kernel<<<grid, kTY * kTX, 0, st>>>(in, H, W, cin, w, bias, cout, relu ? 1 : 0, out);
  return cudaGetLastError();
}

}  // namespace bme

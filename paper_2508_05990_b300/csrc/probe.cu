// Roofline probe: throughput of the exact SAD primitive on the running device.
//
// A register-only loop (no memory traffic) of independent accumulator chains,
// NCH per thread, on every SM.  Variants:
//   0  sad.u32 on 32-bit pixel words (integer pipe)
//   1  float subtract + absolute-value add (two float ops per pixel-candidate)
//   2  both interleaved (the two pipes side by side)
//   3  packed pixel pairs: min.u16x2 then dp2a.lo into a 32-bit accumulator
//      (two pixel-candidates per instruction pair; the exhaustive search's
//      primitive)
// The SM clock during the run is measured from %clock64 against %globaltimer
// in one thread, so the peak can be stated per clock and at the clock seen.
#include "common.cuh"
#include "kernels.cuh"

namespace bme {

namespace {

constexpr int kNCH = 8;
constexpr int kIters = 2048;
constexpr int kUnroll = 4;

template <int VARIANT>
__global__ void __launch_bounds__(256) probe_kernel(const uint32_t* __restrict__ seed, uint32_t* __restrict__ sink,
                                                    unsigned long long* __restrict__ clk) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t xi[kNCH], ai[kNCH];
  float xf[kNCH], af[kNCH];
#pragma unroll
  for (int k = 0; k < kNCH; ++k) {
    xi[k] = pix_word(seed[(t + k) & 255] & 4095u);
    xf[k] = __uint_as_float(xi[k]);
    ai[k] = 0;
    af[k] = 0.f;
  }
  uint32_t yi = pix_word(seed[(t + 77) & 255] & 4095u);
  float yf = __uint_as_float(yi);
  uint32_t xp[kNCH];
#pragma unroll
  for (int k = 0; k < kNCH; ++k) xp[k] = (seed[(t + k) & 255] & 0x0FFF0FFFu);
  uint32_t yp = seed[(t + 77) & 255] & 0x0FFF0FFFu;
  unsigned long long c0, g0, c1, g1;
  asm volatile("mov.u64 %0, %%clock64;" : "=l"(c0));
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(g0));
  for (int i = 0; i < kIters; ++i) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
      for (int k = 0; k < kNCH; ++k) {
        if (VARIANT == 0 || VARIANT == 2) ai[k] = sad_u32(xi[k], yi, ai[k]);
        if (VARIANT == 1 || VARIANT == 2) af[k] += fabsf(xf[k] - yf);
        if (VARIANT == 3) ai[k] = dp2a_lo(min_u16x2(xp[k], yp), 0x0202u, ai[k]);
      }
      yi += 1u;
      yf = __uint_as_float(yi);
      yp += 0x00010001u;
    }
  }
  asm volatile("mov.u64 %0, %%clock64;" : "=l"(c1));
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(g1));
  uint32_t s = 0;
#pragma unroll
  for (int k = 0; k < kNCH; ++k) s ^= ai[k] ^ __float_as_uint(af[k]);
  sink[t] = s;
  if (t == 0) {
    clk[0] = c1 - c0;
    clk[1] = g1 - g0;
  }
}

template <int V>
cudaError_t run_variant(int grid, const uint32_t* seed, uint32_t* sink, unsigned long long* clk, float* ms) {
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  for (int w = 0; w < 2; ++w) probe_kernel<V><<<grid, 256>>>(seed, sink, clk);
  cudaEventRecord(e0);
  probe_kernel<V><<<grid, 256>>>(seed, sink, clk);
  cudaEventRecord(e1);
  cudaError_t e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e == cudaSuccess) e = cudaGetLastError();
  return e;
}

}  // namespace

cudaError_t run_probe_alu(int variant, double* pc_per_clk_per_sm, double* sm_mhz, int* sm_count) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  int nsm = 0;
  e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int grid = nsm * 8;
  uint32_t *seed = nullptr, *sink = nullptr;
  unsigned long long* clk = nullptr;
  if ((e = cudaMalloc(&seed, 256 * sizeof(uint32_t))) != cudaSuccess) return e;
  if ((e = cudaMalloc(&sink, (size_t)grid * 256 * sizeof(uint32_t))) != cudaSuccess) {
    cudaFree(seed);
    return e;
  }
  if ((e = cudaMalloc(&clk, 2 * sizeof(unsigned long long))) != cudaSuccess) {
    cudaFree(seed);
    cudaFree(sink);
    return e;
  }
  uint32_t h[256];
  for (int i = 0; i < 256; ++i) h[i] = (uint32_t)i * 2654435761u;
  e = cudaMemcpy(seed, h, sizeof(h), cudaMemcpyHostToDevice);
  float ms = 0.f;
  if (e == cudaSuccess) {
    if (variant == 0) e = run_variant<0>(grid, seed, sink, clk, &ms);
    else if (variant == 1) e = run_variant<1>(grid, seed, sink, clk, &ms);
    else if (variant == 2) e = run_variant<2>(grid, seed, sink, clk, &ms);
    else e = run_variant<3>(grid, seed, sink, clk, &ms);
  }
  unsigned long long hc[2] = {0, 1};
  if (e == cudaSuccess) e = cudaMemcpy(hc, clk, sizeof(hc), cudaMemcpyDeviceToHost);
  cudaFree(seed);
  cudaFree(sink);
  cudaFree(clk);
  if (e != cudaSuccess) return e;
  const double mhz = (double)hc[0] / (double)(hc[1] ? hc[1] : 1) * 1000.0;
  const double pcs = (double)grid * 256 * kIters * kUnroll * kNCH * (variant >= 2 ? 2 : 1);
  const double cycles = (double)ms * 1e-3 * mhz * 1e6;
  *pc_per_clk_per_sm = pcs / (cycles * nsm);
  *sm_mhz = mhz;
  *sm_count = nsm;
  return cudaSuccess;
}

}  // namespace bme

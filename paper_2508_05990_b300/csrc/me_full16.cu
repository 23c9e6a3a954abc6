// Exhaustive EVEN-phase block matching for 16 x 16 blocks (Sec. 2.2 "Block
// Matching-based ME"; Sec. 3.2 "Matching Criterion": SAD, argmin = MV).
//
// Mapping (B300: 148 SMs, INT32 sad.u32 at 64 lanes/clk/SM):
//   * one CTA = NW (8) warps = NW horizontally adjacent blocks of one block
//     row of one frame pair; the CTA stages the union of their search windows
//     ((16*NW + 4R) x (16 + 4R) pixels) and their current blocks into shared
//     memory as 32-bit pixel words, 8 pixels per 16-byte load with every load
//     of a thread in flight before the first conversion;
//   * one warp = one block; lane v owns candidate row v (dy = 2v - 2R) and all
//     2R+1 candidates of that row (dx = 2u - 2R).  Adjacent candidates of a
//     row are one 32-bit word apart (EVEN offsets), so every reference word a
//     lane loads feeds up to 8 accumulators (register-blocked sliding SAD);
//   * for R = 16 the 33rd row (dy = +32) is spread one candidate per lane and
//     the corner candidate (+32, +32) is split over 16 lanes and summed with a
//     warp reduction, so the 1089 candidates divide evenly over 32 lanes;
//   * half the lanes walk the block rows rotated by one, which together with a
//     window pitch of 4*(odd) words makes every 128-bit shared load
//     conflict-free;
//   * argmin: each lane folds its candidates into a uint64 key
//     (sad, |dx|+|dy|, dy, dx) -- on interior blocks through a 32-bit
//     sad*64 + rank key, rank being the tie-break order within the lane's row
//     -- then a 5-step shuffle minimum.
#include "common.cuh"
#include "full16.cuh"
#include "kernels.cuh"
#include "tc_common.cuh"

namespace bme {

namespace {

constexpr int kNW = 8;  // warps (blocks) per CTA

template <int R>
__global__ void __launch_bounds__(kNW * 32) me_full16_even_kernel(const uint16_t* __restrict__ ref_base,
                                                                   const uint16_t* __restrict__ cur_base, int W,
                                                                   int H, int pitch, long long ref_bs,
                                                                   long long cur_bs, int h, int w,
                                                                   bayer_mv_t* __restrict__ out, bool vec_ok) {
  using C = Full16Strip<R, kNW>;
  extern __shared__ __align__(16) uint32_t smem[];
  uint32_t* win = smem;                 // WIN_H x P
  uint32_t* curt = smem + C::WIN_H * C::P;  // 16 x PC

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int pair = blockIdx.z;
  const uint16_t* ref = ref_base + (long long)pair * ref_bs;
  const uint16_t* cur = cur_base + (long long)pair * cur_bs;
  const int x0 = blockIdx.x * kNW * 16, y0 = blockIdx.y * 16;

  stage_strip<R, kNW>(ref, cur, W, H, pitch, x0, y0, vec_ok, win, curt);
  __syncthreads();

  const int bx = blockIdx.x * kNW + warp;
  if (bx >= w) return;

  const uint64_t best = warp_min_u64(
      full16_block<R, C::P, C::PC>(win + 16 * warp, curt + 16 * warp, lane, bx * 16, y0, W, H));
  if (lane == 0) out[((long long)pair * h + blockIdx.y) * w + bx] = key_to_mv(best);
}

template <int R>
cudaError_t launch_r(const uint16_t* ref, const uint16_t* cur, int W, int H, int pitch, long long ref_bs,
                     long long cur_bs, int batch, bayer_mv_t* out, cudaStream_t st) {
  using C = Full16Strip<R, kNW>;
  const int h = H / 16, w = W / 16;
  dim3 grid((w + kNW - 1) / kNW, h, batch);
  // 16-byte loads need 16-byte aligned rows in every frame of the batch
  const bool vec_ok = (reinterpret_cast<uintptr_t>(ref) % 16) == 0 && (reinterpret_cast<uintptr_t>(cur) % 16) == 0 &&
                      pitch % 8 == 0 && ref_bs % 8 == 0 && cur_bs % 8 == 0;
  me_full16_even_kernel<R><<<grid, kNW * 32, C::SMEM, st>>>(ref, cur, W, H, pitch, ref_bs, cur_bs, h, w, out, vec_ok);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// List mode: the exhaustive search of the blocks named in a device list (the
// low-confidence blocks of the learned-seeded search).  Each warp stages its
// own block's window, so the blocks need not be adjacent; warps loop over the
// list (grid-stride) up to the count found in device memory.
constexpr int kLW = 4;  // warps per CTA in list mode

template <int R>
struct Full16List {
  static constexpr int REACH = 2 * R;
  static constexpr int WIN_W = 16 + 2 * REACH;
  static constexpr int WIN_H = 16 + 2 * REACH;
  static constexpr int P0 = (WIN_W + 3) / 4 * 4;
  static constexpr int P = ((P0 / 4) % 2 == 0) ? P0 + 4 : P0;  // 4 * odd words
  static constexpr int PC = 20;                                // 4 * odd words
  static constexpr int WARP_WORDS = WIN_H * P + 16 * PC;
  static constexpr size_t SMEM = (size_t)kLW * WARP_WORDS * sizeof(uint32_t);
};

template <int R>
__global__ void __launch_bounds__(kLW * 32) me_full16_list_kernel(const uint16_t* __restrict__ ref_base,
                                                                   const uint16_t* __restrict__ cur_base, int W,
                                                                   int H, int pitch, long long ref_bs,
                                                                   long long cur_bs, int h, int w,
                                                                   const int* __restrict__ list,
                                                                   const int* __restrict__ count,
                                                                   bayer_mv_t* __restrict__ out, bool vec_ok) {
  using C = Full16List<R>;
  extern __shared__ __align__(16) uint32_t smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint32_t* win = smem + warp * C::WARP_WORDS;
  uint32_t* curt = win + C::WIN_H * C::P;
  const int n = *count;
  for (int gi = blockIdx.x * kLW + warp; gi < n; gi += gridDim.x * kLW) {
    const int gb = list[gi];
    const int pair = gb / (h * w), rem = gb - pair * h * w;
    const int by = rem / w, bx = rem - by * w;
    const uint16_t* ref = ref_base + (long long)pair * ref_bs;
    const uint16_t* cur = cur_base + (long long)pair * cur_bs;
    const int x0 = bx * 16, y0 = by * 16;
    __syncwarp();  // the previous block's reads are done
    if (vec_ok) {
      constexpr int WCH = C::WIN_W / 8, NW = WCH * C::WIN_H, NT = NW + 32, BATCH = 8;
      for (int e0 = 0; e0 < NT; e0 += 32 * BATCH) {
        uint4 raw[BATCH];
#pragma unroll
        for (int j = 0; j < BATCH; ++j) {
          const int e = e0 + lane + 32 * j;
          raw[j] = make_uint4(0, 0, 0, 0);
          if (e < NW) {
            const int ry = e / WCH, cx = e - ry * WCH;
            const int gy = y0 - C::REACH + ry, gx = x0 - C::REACH + 8 * cx;
            if (gy >= 0 && gy < H && gx >= 0 && gx < W)
              raw[j] = __ldg(reinterpret_cast<const uint4*>(ref + (long long)gy * pitch + gx));
          } else if (e < NT) {
            const int f = e - NW, ry = f >> 1, cx = f & 1;
            raw[j] = __ldg(reinterpret_cast<const uint4*>(cur + (long long)(y0 + ry) * pitch + x0 + 8 * cx));
          }
        }
#pragma unroll
        for (int j = 0; j < BATCH; ++j) {
          const int e = e0 + lane + 32 * j;
          if (e >= NT) continue;
          uint32_t* dst;
          if (e < NW) {
            const int ry = e / WCH, cx = e - ry * WCH;
            dst = win + ry * C::P + 8 * cx;
          } else {
            const int f = e - NW;
            dst = curt + (f >> 1) * C::PC + 8 * (f & 1);
          }
          reinterpret_cast<uint4*>(dst)[0] = make_uint4(pix_lo(raw[j].x), pix_hi(raw[j].x), pix_lo(raw[j].y), pix_hi(raw[j].y));
          reinterpret_cast<uint4*>(dst)[1] = make_uint4(pix_lo(raw[j].z), pix_hi(raw[j].z), pix_lo(raw[j].w), pix_hi(raw[j].w));
        }
      }
    } else {
      for (int e = lane; e < C::WIN_H * C::WIN_W; e += 32) {
        const int ry = e / C::WIN_W, rx = e - ry * C::WIN_W;
        const int gy = y0 - C::REACH + ry, gx = x0 - C::REACH + rx;
        uint32_t v = 0;
        if (gy >= 0 && gy < H && gx >= 0 && gx < W) v = __ldg(ref + (long long)gy * pitch + gx);
        win[ry * C::P + rx] = pix_word(v);
      }
      for (int e = lane; e < 256; e += 32)
        curt[(e >> 4) * C::PC + (e & 15)] = pix_word(__ldg(cur + (long long)(y0 + (e >> 4)) * pitch + x0 + (e & 15)));
    }
    __syncwarp();
    const uint64_t best = warp_min_u64(full16_block<R, C::P, C::PC>(win, curt, lane, x0, y0, W, H));
    if (lane == 0) out[gb] = key_to_mv(best);
  }
}

template <int R>
cudaError_t launch_list_r(const uint16_t* ref, const uint16_t* cur, int W, int H, int pitch, long long ref_bs,
                          long long cur_bs, int h, int w, const int* list, const int* count, int max_count,
                          bayer_mv_t* out, cudaStream_t st) {
  using C = Full16List<R>;
  int dev = 0, nsm = 148;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int per_sm = tc::ctas_per_sm(me_full16_list_kernel<R>, kLW * 32, (int)C::SMEM, 0);
  int grid = (max_count + kLW - 1) / kLW;
  if (grid > per_sm * nsm) grid = per_sm * nsm;
  if (grid < 1) grid = 1;
  const bool vec_ok = (reinterpret_cast<uintptr_t>(ref) % 16) == 0 && (reinterpret_cast<uintptr_t>(cur) % 16) == 0 &&
                      pitch % 8 == 0 && ref_bs % 8 == 0 && cur_bs % 8 == 0;
  me_full16_list_kernel<R><<<grid, kLW * 32, C::SMEM, st>>>(ref, cur, W, H, pitch, ref_bs, cur_bs, h, w, list, count,
                                                             out, vec_ok);
  return cudaGetLastError();
}

template <int R>
cudaError_t configure_list_r() {
  cudaError_t e = cudaFuncSetAttribute(me_full16_list_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)Full16List<R>::SMEM);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(me_full16_list_kernel<R>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  return e;
}

template <int R>
cudaError_t configure_r() {
  cudaError_t e = cudaFuncSetAttribute(me_full16_even_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)Full16Strip<R, kNW>::SMEM);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(me_full16_even_kernel<R>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  return e;
}

}  // namespace

cudaError_t configure_full16() {
  cudaError_t e;
  if ((e = configure_r<4>()) != cudaSuccess) return e;
  if ((e = configure_r<8>()) != cudaSuccess) return e;
  if ((e = configure_r<12>()) != cudaSuccess) return e;
  return configure_r<16>();
}

cudaError_t configure_full16_list() {
  cudaError_t e;
  if ((e = configure_list_r<4>()) != cudaSuccess) return e;
  if ((e = configure_list_r<8>()) != cudaSuccess) return e;
  if ((e = configure_list_r<12>()) != cudaSuccess) return e;
  return configure_list_r<16>();
}

cudaError_t launch_full16_list(const uint16_t* ref, const uint16_t* cur, int W, int H, int pitch, long long ref_bs,
                               long long cur_bs, int h, int w, int range, const int* list, const int* count,
                               int max_count, bayer_mv_t* out, cudaStream_t st) {
  switch (range) {
    case 8: return launch_list_r<4>(ref, cur, W, H, pitch, ref_bs, cur_bs, h, w, list, count, max_count, out, st);
    case 16: return launch_list_r<8>(ref, cur, W, H, pitch, ref_bs, cur_bs, h, w, list, count, max_count, out, st);
    case 24: return launch_list_r<12>(ref, cur, W, H, pitch, ref_bs, cur_bs, h, w, list, count, max_count, out, st);
    case 32: return launch_list_r<16>(ref, cur, W, H, pitch, ref_bs, cur_bs, h, w, list, count, max_count, out, st);
    default: return cudaErrorInvalidValue;
  }
}

bool full16_even_supported(int range) { return range == 8 || range == 16 || range == 24 || range == 32; }

cudaError_t launch_full16_even(const uint16_t* ref, const uint16_t* cur, int W, int H, int pitch, long long ref_bs,
                               long long cur_bs, int batch, int range, bayer_mv_t* out, cudaStream_t st) {
  switch (range) {
    case 8: return launch_r<4>(ref, cur, W, H, pitch, ref_bs, cur_bs, batch, out, st);
    case 16: return launch_r<8>(ref, cur, W, H, pitch, ref_bs, cur_bs, batch, out, st);
    case 24: return launch_r<12>(ref, cur, W, H, pitch, ref_bs, cur_bs, batch, out, st);
    case 32: return launch_r<16>(ref, cur, W, H, pitch, ref_bs, cur_bs, batch, out, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace bme

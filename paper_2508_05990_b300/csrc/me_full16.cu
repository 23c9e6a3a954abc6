// Exhaustive EVEN-phase block matching for 16 x 16 blocks (Sec. 2.2 "Block
// Matching-based ME"; Sec. 3.2 "Matching Criterion": SAD, argmin = MV).
//
// Mapping (B300: 148 SMs; packed 16-bit min + dp2a at the issue rate):
//   * one CTA = NW (4) warps = NW horizontally adjacent blocks of one block
//     row of one frame pair; the CTA stages the union of their search windows
//     ((16*NW + 4R) x (16 + 4R) pixels) and their current blocks into shared
//     memory as packed pixel pairs -- two TMA tensor tiles whose rows land at
//     the pitches below (16-byte register-staged loads for unaligned frames)
//     -- then a table of 16-row column sums of the window at every even row
//     offset;
//   * one warp = one block; lane v owns candidate row v (dy = 2v - 2R) and all
//     2R+1 candidates of that row (dx = 2u - 2R).  Adjacent candidates of a
//     row are one packed word apart (EVEN offsets), so every window word a
//     lane loads feeds up to 8 accumulators (register-blocked sliding sum of
//     2 min(cur, win) over pixel pairs); SAD = sum(cur) + sum(win) - that sum;
//   * for R = 16 the 33rd row (dy = +32) is spread one candidate per lane and
//     the corner candidate (+32, +32) is split over 8 lanes and summed with a
//     warp reduction, so the 1089 candidates divide evenly over 32 lanes;
//   * half the lanes walk the block rows rotated by one, which together with a
//     window pitch of 4*(odd) words makes every 128-bit shared load
//     conflict-free;
//   * a frame height that is not a multiple of 16 clips the last block row
//     to bh rows: its current rows below the frame are staged as zeros (their
//     min(cur, win) adds nothing) and its column-sum table sums bh rows, so
//     its SAD covers exactly the rows inside the frame, as the definition of
//     a clipped edge block asks;
//   * argmin: each lane folds its candidates into a uint64 key
//     (sad, |dx|+|dy|, dy, dx) -- on interior blocks through a 32-bit
//     sad*64 + rank key, rank being the tie-break order within the lane's row
//     -- then a 5-step shuffle minimum.
#include "common.cuh"
#include "full16.cuh"
#include "kernels.cuh"
#include "tc_common.cuh"
#include "tma.cuh"

namespace bme {

namespace {

// Warps (blocks) per CTA.  4-block strips at 6 CTAs (24 warps) per SM issue
// faster than 8-block strips at 4 (0.531 vs 0.559 ms for the 1080p clip),
// although each block stages a third more window.
constexpr int kNW = 4;
constexpr uint32_t kStripWaitLimit = 1u << 22;

// TMA: the window and the current tile arrive as two tensor tiles (16-byte
// aligned frames); the rows land at the pitches the sliding loads want, and
// samples outside the frame read 0 -- the current rows below the frame of a
// clipped last block row too.  Without TMA, 16-byte register-staged loads.
template <int R, bool TMA>
__global__ void __launch_bounds__(kNW * 32, 6) me_full16_even_kernel(const __grid_constant__ CUtensorMap tm_ref,
                                                                   const __grid_constant__ CUtensorMap tm_cur,
                                                                   const uint16_t* __restrict__ ref_base,
                                                                   const uint16_t* __restrict__ cur_base, int W,
                                                                   int H, int pitch, long long ref_bs,
                                                                   long long cur_bs, int h, int w,
                                                                   bayer_mv_t* __restrict__ out, bool vec_ok,
                                                                   int* __restrict__ status) {
  using C = Full16Strip<R, kNW>;
  extern __shared__ __align__(128) uint32_t smem[];
  uint32_t* win = smem;                // WIN_H x P
  uint32_t* curt = smem + C::CUR_OFF;  // 16 x PC
  uint32_t* cs = smem + C::CS_OFF;     // NU x P

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int pair = blockIdx.z;
  const int x0 = blockIdx.x * kNW * 16, y0 = blockIdx.y * 16;

  // the last block row of a frame whose height is not a multiple of 16 is
  // clipped to bh rows (its SAD covers the rows inside the frame)
  const int bh = min(16, H - y0);
  if constexpr (TMA) {
    uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + C::MBAR_OFF);
    if (threadIdx.x == 0) {
      tc::mbar_init(mbar, 1);
      tc::fence_mbar_init();
      tma::mbar_arrive_expect_tx(mbar, C::TX_BYTES);
      tma::load_3d(win, &tm_ref, x0 - C::REACH, y0 - C::REACH, pair, mbar);
      tma::load_3d(curt, &tm_cur, x0, y0, pair, mbar);
    }
    __syncthreads();  // the barrier is initialised before anyone waits on it
    const bool ok = tc::mbar_wait(mbar, 0, kStripWaitLimit);
    if (!__syncthreads_and(ok)) {
      // record the expiry, give the copies a last bounded wait, and stop
      if (threadIdx.x == 0) {
        if (status) atomicExch(status, (int)BAYER_ERR_TIMEOUT);
        tc::mbar_wait(mbar, 0, kStripWaitLimit);
      }
      __syncthreads();
      return;
    }
  } else {
    stage_strip<R, kNW>(ref_base + (long long)pair * ref_bs, cur_base + (long long)pair * cur_bs, W, H, pitch, x0,
                        y0, vec_ok, win, curt);
    __syncthreads();
  }
  window_colsums<R, C::P, C::WW, kNW * 32>(win, cs, threadIdx.x, bh);
  __syncthreads();

  const int bx = blockIdx.x * kNW + warp;
  if (bx >= w) return;

  const uint64_t best = warp_min_u64(
      full16_block<R, C::P, C::PC>(win + 8 * warp, cs + 8 * warp, curt + 8 * warp, lane, bx * 16, y0, W, H, bh));
  if (lane == 0) out[((long long)pair * h + blockIdx.y) * w + bx] = key_to_mv(best);
}

template <int R>
cudaError_t launch_r(const uint16_t* ref, const uint16_t* cur, int W, int H, int pitch, long long ref_bs,
                     long long cur_bs, int batch, bayer_mv_t* out, int* status, cudaStream_t st) {
  using C = Full16Strip<R, kNW>;
  const int h = (H + 15) / 16, w = W / 16;
  dim3 grid((w + kNW - 1) / kNW, h, batch);
  // 16-byte loads and TMA tiles need 16-byte aligned rows in every frame of the batch
  const bool vec_ok = (reinterpret_cast<uintptr_t>(ref) % 16) == 0 && (reinterpret_cast<uintptr_t>(cur) % 16) == 0 &&
                      pitch % 8 == 0 && ref_bs % 8 == 0 && cur_bs % 8 == 0;
  CUtensorMap tref{}, tcur{};
  const bool use_tma = vec_ok && tma::encode_u16_frames(&tref, ref, W, H, batch, pitch, ref_bs, C::BOX_W, C::WIN_H) &&
                       tma::encode_u16_frames(&tcur, cur, W, H, batch, pitch, cur_bs, C::CUR_BOX_W, 16);
  if (use_tma)
    me_full16_even_kernel<R, true><<<grid, kNW * 32, C::SMEM, st>>>(tref, tcur, ref, cur, W, H, pitch, ref_bs, cur_bs,
                                                                     h, w, out, vec_ok, status);
  else
    me_full16_even_kernel<R, false><<<grid, kNW * 32, C::SMEM, st>>>(tref, tcur, ref, cur, W, H, pitch, ref_bs,
                                                                      cur_bs, h, w, out, vec_ok, status);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// List mode: the exhaustive search of the blocks named in a device list (the
// low-confidence blocks of the learned-seeded search).  Each warp searches
// its own block from its own window, so the blocks need not be adjacent;
// warps loop over the list (grid-stride) up to the count found in device
// memory.  One CTA of 15 warps per SM (the 15 windows fill shared memory).
//
// Window sums: each lane gathers its own during the row loop
// (full16_accumulate with SUMS), so no column-sum table or table pass is
// needed and a warp's shared memory is just its window and current block.
//
// Staging: with 16-byte aligned frames, two TMA tile loads per block (the
// window as a box 2P pixels wide, which lands at the 4*odd-word pitch the
// sliding loads want, and the 16 x 16 current block), completing on one
// mbarrier per warp.  The next block's window is requested as soon as the
// row loop is done with the current one and its current block after the SAD
// finish, so the copies overlap the finish and the argmin.  Every wait is
// bounded: on expiry the kernel records BAYER_ERR_TIMEOUT and the warp stops.
// Other layouts stage with plain loads.
constexpr int kLW = 15;  // warps per CTA in list mode
constexpr uint32_t kWaitLimit = 1u << 22;

template <int R>
struct Full16List {
  static constexpr int REACH = 2 * R;
  static constexpr int WIN_W = 16 + 2 * REACH;  // pixels
  static constexpr int WIN_H = 16 + 2 * REACH;
  static constexpr int WW = WIN_W / 2;          // words
  static constexpr int P = pitch4odd(WW);
  static constexpr int BOX_W = 2 * P;           // TMA window box width (pixels)
  static constexpr int PC = 8;                  // current block: dense rows (read as broadcasts)
  static constexpr int CUR_OFF = WIN_H * P;
  static constexpr int WARP_WORDS = (CUR_OFF + 16 * PC + 31) / 32 * 32;  // 128-byte aligned windows
  static constexpr uint32_t TX_BYTES = (uint32_t)(WIN_H * P + 16 * PC) * 4u;
  static constexpr int MBAR_OFF = kLW * WARP_WORDS;  // one mbarrier per warp after the windows
  static constexpr size_t SMEM = (size_t)MBAR_OFF * sizeof(uint32_t) + kLW * sizeof(uint64_t);
  static_assert((CUR_OFF * 4) % 128 == 0, "current block 128-byte aligned");
};

// Plain-load staging of one block's window and current block (any layout).
template <int R>
__device__ __forceinline__ void list_stage(const uint16_t* __restrict__ ref, const uint16_t* __restrict__ cur, int W,
                                           int H, int pitch, int x0, int y0, bool vec_ok, int lane, uint32_t* win,
                                           uint32_t* curt) {
  using C = Full16List<R>;
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
          if (y0 + ry < H)  // a clipped last block row keeps zero rows below the frame
            raw[j] = __ldg(reinterpret_cast<const uint4*>(cur + (long long)(y0 + ry) * pitch + x0 + 8 * cx));
        }
      }
#pragma unroll
      for (int j = 0; j < BATCH; ++j) {
        const int e = e0 + lane + 32 * j;
        if (e < NW) {
          const int ry = e / WCH, cx = e - ry * WCH;
          *reinterpret_cast<uint4*>(win + ry * C::P + 4 * cx) = raw[j];
        } else if (e < NT) {
          const int f = e - NW;
          *reinterpret_cast<uint4*>(curt + (f >> 1) * C::PC + 4 * (f & 1)) = raw[j];
        }
      }
    }
  } else {
    for (int e = lane; e < C::WIN_H * C::WW; e += 32) {
      const int ry = e / C::WW, wx = e - ry * C::WW;
      win[ry * C::P + wx] = pair_word(ref, W, H, pitch, x0 - C::REACH + 2 * wx, y0 - C::REACH + ry);
    }
    for (int e = lane; e < 128; e += 32)
      curt[(e >> 3) * C::PC + (e & 7)] = pair_word(cur, W, H, pitch, x0 + 2 * (e & 7), y0 + (e >> 3));
  }
}

// Block gb of the list: its pair and tile origin (x0, y0).
__device__ __forceinline__ void list_where(int gb, int h, int w, int& pair, int& x0, int& y0) {
  pair = gb / (h * w);
  const int rem = gb - pair * h * w;
  const int by = rem / w;
  y0 = by * 16;
  x0 = (rem - by * w) * 16;
}

// CLIP: a block of a last block row clipped by the frame (H % 16 != 0) runs
// over its bh = H - y0 rows (the current rows below the frame are staged as
// zeros: TMA fills them, the plain loads skip them).  This form makes every
// block slower (list search of the 1080p clip's fallback blocks: 127.6 ->
// ~150 us), so it only runs a second list of the clipped row's blocks.
template <int R, bool TMA, bool CLIP>
__global__ void __launch_bounds__(kLW * 32) me_full16_list_kernel(const __grid_constant__ CUtensorMap tm_ref,
                                                                   const __grid_constant__ CUtensorMap tm_cur,
                                                                   const uint16_t* __restrict__ ref_base,
                                                                   const uint16_t* __restrict__ cur_base, int W,
                                                                   int H, int pitch, long long ref_bs,
                                                                   long long cur_bs, int h, int w,
                                                                   const int* __restrict__ list,
                                                                   const int* __restrict__ count,
                                                                   bayer_mv_t* __restrict__ out, bool vec_ok,
                                                                   int* __restrict__ status) {
  using C = Full16List<R>;
  extern __shared__ __align__(128) uint32_t smem[];
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + C::MBAR_OFF);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint32_t* win = smem + warp * C::WARP_WORDS;
  uint32_t* curt = win + C::CUR_OFF;
  // launched as a dependent of the kernel that built the list: read it (and
  // write the fallback blocks' fields) only after this wait
  tc::grid_dep_wait();
  tc::grid_dep_launch();
  const int n = *count;
  // warp-major: consecutive entries go to different CTAs, so that a partial
  // last round (or a short list) spreads over every SM
  const int step = gridDim.x * kLW;
  int gi = warp * gridDim.x + blockIdx.x;

  if constexpr (TMA) {
    if (lane == 0) {
      tc::mbar_init(&mbar[warp], 1);
      tc::fence_mbar_init();
    }
    __syncwarp();
    if (lane == 0 && gi < n) {
      int pr, x0, y0;
      list_where(list[gi], h, w, pr, x0, y0);
      tma::mbar_arrive_expect_tx(&mbar[warp], C::TX_BYTES);
      tma::load_3d(win, &tm_ref, x0 - C::REACH, y0 - C::REACH, pr, &mbar[warp]);
      tma::load_3d(curt, &tm_cur, x0, y0, pr, &mbar[warp]);
    }
  }
  uint32_t phase = 0;
  for (; gi < n; gi += step) {
    const int gb = list[gi];
    int pair, x0, y0;
    list_where(gb, h, w, pair, x0, y0);
    if constexpr (TMA) {
      const bool ok = __all_sync(0xffffffffu, tc::mbar_wait(&mbar[warp], phase, kWaitLimit));
      phase ^= 1u;
      if (!ok) {
        if (lane == 0 && status) atomicExch(status, (int)BAYER_ERR_TIMEOUT);
        return;
      }
    } else {
      __syncwarp();  // the previous block's reads are done
      list_stage<R>(ref_base + (long long)pair * ref_bs, cur_base + (long long)pair * cur_bs, W, H, pitch, x0, y0,
                    vec_ok, lane, win, curt);
      __syncwarp();
    }
    Full16Acc<R> A;
    Full16WinSums<R> S;
    const int bh = CLIP && y0 + 16 > H ? H - y0 : 16;
    full16_accumulate<R, C::P, C::PC, true, CLIP>(win, curt, lane, A, S, bh);
    const int gn = gi + step;
    int pn = 0, xn = 0, yn = 0;
    if constexpr (TMA) {
      __syncwarp();  // every lane is done reading the window
      if (lane == 0 && gn < n) {
        list_where(list[gn], h, w, pn, xn, yn);
        tc::fence_proxy_async();
        tma::mbar_arrive_expect_tx(&mbar[warp], C::TX_BYTES);
        tma::load_3d(win, &tm_ref, xn - C::REACH, yn - C::REACH, pn, &mbar[warp]);
      }
    }
    full16_finish_sums<R, C::PC>(S, curt, lane, A);
    if constexpr (TMA) {
      __syncwarp();  // every lane is done reading the current block
      if (lane == 0 && gn < n) {
        tc::fence_proxy_async();
        tma::load_3d(curt, &tm_cur, xn, yn, pn, &mbar[warp]);
      }
    }
    const uint64_t best = warp_min_u64(full16_select<R>(A, lane, x0, y0, W, H, bh));
    if (lane == 0) out[gb] = key_to_mv(best);
  }
}

template <int R>
cudaError_t launch_list_r(const uint16_t* ref, const uint16_t* cur, int W, int H, int pitch, long long ref_bs,
                          long long cur_bs, int batch, int h, int w, const int* list, const int* count, int max_count,
                          bool clip, bayer_mv_t* out, int* status, cudaStream_t st) {
  using C = Full16List<R>;
  int dev = 0, nsm = 148;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const bool vec_ok = (reinterpret_cast<uintptr_t>(ref) % 16) == 0 && (reinterpret_cast<uintptr_t>(cur) % 16) == 0 &&
                      pitch % 8 == 0 && ref_bs % 8 == 0 && cur_bs % 8 == 0;
  CUtensorMap tref{}, tcur{};
  const bool use_tma = vec_ok &&
                       tma::encode_u16_frames(&tref, ref, W, H, batch, pitch, ref_bs, C::BOX_W, C::WIN_H) &&
                       tma::encode_u16_frames(&tcur, cur, W, H, batch, pitch, cur_bs, 16, 16);
  auto kern = use_tma ? (clip ? me_full16_list_kernel<R, true, true> : me_full16_list_kernel<R, true, false>)
                      : (clip ? me_full16_list_kernel<R, false, true> : me_full16_list_kernel<R, false, false>);
  const int per_sm = tc::ctas_per_sm(kern, kLW * 32, (int)C::SMEM, 0);
  int grid = max_count;
  if (grid > per_sm * nsm) grid = per_sm * nsm;
  if (grid < 1) grid = 1;
  return tc::launch_dependent(kern, dim3(grid), dim3(kLW * 32), C::SMEM, st, tref, tcur, ref, cur, W, H, pitch,
                              ref_bs, cur_bs, h, w, list, count, out, vec_ok, status);
}

template <int R>
cudaError_t configure_list_r() {
  cudaError_t e = cudaSuccess;
  const void* fns[4] = {(const void*)me_full16_list_kernel<R, true, false>,
                        (const void*)me_full16_list_kernel<R, false, false>,
                        (const void*)me_full16_list_kernel<R, true, true>,
                        (const void*)me_full16_list_kernel<R, false, true>};
  for (int v = 0; v < 4 && e == cudaSuccess; ++v) {
    const void* fn = fns[v];
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Full16List<R>::SMEM);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  }
  return e;
}

template <int R>
cudaError_t configure_r() {
  cudaError_t e = cudaSuccess;
  for (int v = 0; v < 2 && e == cudaSuccess; ++v) {
    const void* fn = v ? (const void*)me_full16_even_kernel<R, true> : (const void*)me_full16_even_kernel<R, false>;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Full16Strip<R, kNW>::SMEM);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  }
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
                               long long cur_bs, int batch, int h, int w, int range, const int* list, const int* count,
                               int max_count, bool clip, bayer_mv_t* out, int* status, cudaStream_t st) {
  switch (range) {
    case 8:
      return launch_list_r<4>(ref, cur, W, H, pitch, ref_bs, cur_bs, batch, h, w, list, count, max_count, clip,
                              out, status, st);
    case 16:
      return launch_list_r<8>(ref, cur, W, H, pitch, ref_bs, cur_bs, batch, h, w, list, count, max_count, clip,
                              out, status, st);
    case 24:
      return launch_list_r<12>(ref, cur, W, H, pitch, ref_bs, cur_bs, batch, h, w, list, count, max_count, clip,
                               out, status, st);
    case 32:
      return launch_list_r<16>(ref, cur, W, H, pitch, ref_bs, cur_bs, batch, h, w, list, count, max_count, clip,
                               out, status, st);
    default: return cudaErrorInvalidValue;
  }
}

bool full16_even_supported(int range) { return range == 8 || range == 16 || range == 24 || range == 32; }

cudaError_t launch_full16_even(const uint16_t* ref, const uint16_t* cur, int W, int H, int pitch, long long ref_bs,
                               long long cur_bs, int batch, int range, bayer_mv_t* out, int* status, cudaStream_t st) {
  switch (range) {
    case 8: return launch_r<4>(ref, cur, W, H, pitch, ref_bs, cur_bs, batch, out, status, st);
    case 16: return launch_r<8>(ref, cur, W, H, pitch, ref_bs, cur_bs, batch, out, status, st);
    case 24: return launch_r<12>(ref, cur, W, H, pitch, ref_bs, cur_bs, batch, out, status, st);
    case 32: return launch_r<16>(ref, cur, W, H, pitch, ref_bs, cur_bs, batch, out, status, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace bme

// 3x3 stride-1 convolution (zero pad 1) on the 5th-generation tensor cores,
// streamed row by row: the refine convolutions of propagated features.
//
//   out[y, x, n] = bias[n] + sum_{ky, kx, ci} in[y + ky - 1, x + kx - 1, ci] * w[n, ci, ky, kx]
//
// Work: the output is cut into segments of 128 pixels of one row (the MMA M);
// each CTA (one per SM, persistent) owns a contiguous range of rows of one or
// more column strips and walks down each strip.  Every input row of a strip
// is staged in shared memory exactly once and feeds three output rows: input
// row r adds tap row ky = 0 to output row r + 1, ky = 1 to row r and ky = 2 to
// row r - 1, each output row accumulating in its own TMEM accumulator (four
// rotate, so the epilogue of one row overlaps the MMAs of the next ones).
//
// Warp roles (416 threads):
//   warps 0-3   epilogue: TMEM -> registers -> bias, ReLU -> bf16 / float32 NHWC
//               (warp w reads TMEM lanes 32w..32w+31 = pixels of the segment),
//               each 32-channel chunk turned around in a per-warp shared-memory
//               tile so that a store instruction writes 64 / 128 contiguous bytes
//               per pixel instead of 16 bytes at a stride of one pixel;
//   warp 4      one thread issues the MMAs (9 * CIN/16 per input row and
//               output row it touches) and commits them to mbarriers;
//   warps 5-12  producers: global loads of the next input row (float32 input
//               is rounded to bf16 here), stored as K-major core matrices.
// Ring of NR staged rows with full / empty mbarriers; weights (all nine taps,
// all output channels) stay resident in shared memory for the whole launch.
// Every wait is bounded: on expiry the CTA raises an abort flag, records
// BAYER_ERR_TIMEOUT, waits (bounded) for its own MMAs and frees its TMEM.
#include <cuda_bf16.h>

#include "common.cuh"
#include "kernels.cuh"
#include "tc_common.cuh"

namespace bme {

namespace {

constexpr int kM = 128;     // output pixels per row segment (MMA M)
constexpr int kNJ = 130;    // staged input pixels per row segment (128 + 2 halo)
constexpr int kNP = 137;    // pitch of a staged chunk plane: 137 * 16 B = 16 mod 128 (conflict-free stores)
constexpr int kAcc = 4;     // TMEM accumulators (output rows in flight)
constexpr int kEpiWarps = 4, kMmaWarp = 4, kProdWarp0 = 5, kProdWarps = 8;
constexpr int kProdThreads = kProdWarps * 32;
constexpr int kThreads = (kProdWarp0 + kProdWarps) * 32;
constexpr uint32_t kWaitLimit = 1u << 22;

// Shared-memory plan.  Staged row: element (chunk kc of 8 channels, pixel p)
// at (kc * kNP + p) * 16, so the A operand of tap column kx and K step s2 is
// the staged row at start (2 * s2 * kNP + kx) * 16: core matrices of 8
// consecutive pixels (SBO 128 B), next K chunk one plane further (LBO kNP * 16).
// Weights: element (n, k), k = tap * CIN + ci, at
// (n / 8) * (9 * KC) * 128 + (k / 8) * 128 + (n % 8) * 16 + (k % 8) * 2.
//
// COUT = 64 layers stack the three tap rows along N: B row n = ky * 64 + co,
// K index k = kx * CIN + ci, element (n, k) at
// (n / 8) * (3 * KC) * 128 + (k / 8) * 128 + (n % 8) * 16 + (k % 8) * 2.  One
// MMA with N = 192 then applies an input row's three tap rows at once, to the
// accumulators of output rows r + 1, r and r - 1, which sit in adjacent
// 64-column TMEM slots: slot(o) = NS - 1 - o % NS for the CTA's o-th output
// row.  Where those slots wrap around or a row lies outside the run, the MMA
// is split into N = 64 / 128 pieces.  Every MMA accumulates: the epilogue
// zeroes a slot after draining it (and all slots at the start).  A staged row
// is read by 24 MMAs instead of 72, which cuts the tensor cores' shared-memory
// operand traffic by 44 %.
template <int CIN, int COUT, int SRC, int OUTF>
struct RowStreamLayout {
  static constexpr bool STACK = COUT == 64;
  static constexpr int NS = STACK ? 8 : kAcc;  // accumulator slots
  static constexpr int KC = CIN / 8;
  static constexpr int SLOT_BYTES = KC * kNP * 16;
  // ring slots: float32 input leaves room for 2; float32 output gives one up to the store transpose
  static constexpr int NR = SRC == 2 ? 2 : (OUTF == 1 ? 3 : 4);
  static constexpr int NG = SRC == 2 ? 1 : 2;  // producer groups taking alternate rows
  static constexpr int GT = kProdThreads / NG;
  static constexpr int B_BYTES = 9 * CIN * COUT * 2;
  static constexpr int BAR_OFF = B_BYTES + NR * SLOT_BYTES;
  static constexpr int NBAR = 2 * NR + 2 * NS + 1;
  static constexpr int BIAS_OFF = (BAR_OFF + NBAR * 8 + 16 + 15) / 16 * 16;  // float32 bias, read as broadcasts
  // store transpose: per epilogue warp a tile of 32 pixels x 32 channels (float32: 4 KB,
  // bf16: 2 KB) that turns the pixel-per-lane TMEM rows into contiguous runs of 128 / 64
  // bytes per pixel for the global stores
  static constexpr int XB_OFF = (BIAS_OFF + COUT * 4 + 127) / 128 * 128;
  static constexpr int XB_BYTES = kEpiWarps * 32 * (OUTF == 1 ? 128 : 64);
  static constexpr int SMEM = XB_OFF + XB_BYTES;
  static constexpr int TMEM_COLS = NS * COUT;
  static_assert(CIN % 16 == 0 && (COUT == 64 || COUT == 128), "shape");
  static_assert(B_BYTES % 16 == 0 && SLOT_BYTES % 16 == 0, "alignment");
  static_assert(SMEM <= 227 * 1024, "shared memory");
  static_assert(TMEM_COLS <= 512, "tensor memory");
};

using tc::bf2;

// The CTA's output rows [t0, t1) of the (b, segment, y)-ordered list, cut into
// runs that stay inside one column strip.
struct Runs {
  long long t, t1;
  int Ho, segs;
  int b, seg, ya, yb;
  __device__ bool next() {
    if (t >= t1) return false;
    const long long bs = t / Ho;
    ya = (int)(t - bs * Ho);
    const long long left = t1 - t;
    yb = left < (long long)(Ho - ya) ? ya + (int)left : Ho;
    b = (int)(bs / segs);
    seg = (int)(bs - (long long)b * segs);
    t += yb - ya;
    return true;
  }
};

__device__ __forceinline__ void raise_abort(volatile int* abort_flag, int* status) {
  *abort_flag = 1;
  if (status) atomicExch(status, (int)BAYER_ERR_TIMEOUT);
}

template <int CIN, int COUT, int SRC, int OUTF, bool RELU>
__global__ void __launch_bounds__(kThreads, 1) conv3x3_rows_tc_kernel(const ConvRowsArgs a) {
  using L = RowStreamLayout<CIN, COUT, SRC, OUTF>;
  constexpr int KC = L::KC;
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* sB = smem;
  uint8_t* sX = smem + L::B_BYTES;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + L::BAR_OFF);
  uint64_t* empty = full + L::NR;
  uint64_t* acc_full = empty + L::NR;
  uint64_t* acc_empty = acc_full + L::NS;
  uint64_t* mma_done = acc_empty + L::NS;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mma_done + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (tid == 0) {
    for (int s = 0; s < L::NR; ++s) {
      tc::mbar_init(&full[s], L::GT);
      tc::mbar_init(&empty[s], 1);
    }
    for (int i = 0; i < L::NS; ++i) {
      tc::mbar_init(&acc_full[i], 1);
      tc::mbar_init(&acc_empty[i], kEpiWarps);
    }
    tc::mbar_init(mma_done, 1);
    *abort_flag = 0;
    tc::fence_mbar_init();
  }
  if (warp == 0) tc::tmem_alloc(tmem_slot, L::TMEM_COLS);
  // weights: the packed image is the shared-memory layout, copied as is
  for (int i = tid; i < L::B_BYTES / 16; i += kThreads) reinterpret_cast<uint4*>(sB)[i] = __ldg(a.wimg + i);
  float* sBias = reinterpret_cast<float*>(smem + L::BIAS_OFF);
  for (int i = tid; i < COUT; i += kThreads) sBias[i] = __ldg(a.bias + i);
  tc::fence_proxy_async();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tmem_slot;

  const int segs = (a.W + kM - 1) / kM;
  const long long T = (long long)a.batch * segs * a.H;
  Runs runs{T * blockIdx.x / gridDim.x, T * (blockIdx.x + 1) / gridDim.x, a.H, segs, 0, 0, 0, 0};

  if (warp >= kProdWarp0) {
    // ---- producers: input rows ya-1 .. yb of each run, group g takes rows j % NG == g
    const int ptid = tid - kProdWarp0 * 32;
    const int group = ptid / L::GT, gtid = ptid - group * L::GT;
    constexpr int NITEM = kNJ * KC;
    constexpr int PER = (NITEM + L::GT - 1) / L::GT;
    long long j = 0;
    bool stop = false;
    while (!stop && runs.next()) {
      const int c0 = runs.seg * kM - 1;
      for (int r = runs.ya - 1; r <= runs.yb; ++r, ++j) {
        if ((int)(j % L::NG) != group) continue;
        if (*abort_flag) {
          stop = true;
          break;
        }
        const int slot = (int)(j % L::NR);
        const long long f = j / L::NR;
        const bool row_ok = r >= 0 && r < a.H;
        const long long rowbase = ((long long)runs.b * a.H + r) * a.W;
        uint8_t* dst = sX + slot * L::SLOT_BYTES;
        if (SRC == 2) {
          float4 v[PER][2];
#pragma unroll
          for (int u = 0; u < PER; ++u) {
            const int it = gtid + u * L::GT;
            const int p = it / KC, kc = it - p * KC, ix = c0 + p;
            const bool ok = row_ok && it < NITEM && ix >= 0 && ix < a.W;
            const float4* src = reinterpret_cast<const float4*>(a.in_f32 + (rowbase + ix) * CIN + kc * 8);
            v[u][0] = ok ? __ldg(src) : make_float4(0.f, 0.f, 0.f, 0.f);
            v[u][1] = ok ? __ldg(src + 1) : make_float4(0.f, 0.f, 0.f, 0.f);
          }
          if (f > 0 && !tc::mbar_wait(&empty[slot], (uint32_t)((f - 1) & 1), kWaitLimit)) {
            raise_abort(abort_flag, a.status);
            stop = true;
            break;
          }
#pragma unroll
          for (int u = 0; u < PER; ++u) {
            const int it = gtid + u * L::GT;
            if (it >= NITEM) continue;
            const int p = it / KC, kc = it - p * KC;
            *reinterpret_cast<uint4*>(dst + (kc * kNP + p) * 16) =
                make_uint4(bf2(v[u][0].x, v[u][0].y), bf2(v[u][0].z, v[u][0].w), bf2(v[u][1].x, v[u][1].y),
                           bf2(v[u][1].z, v[u][1].w));
          }
        } else {
          uint4 v[PER];
#pragma unroll
          for (int u = 0; u < PER; ++u) {
            const int it = gtid + u * L::GT;
            const int p = it / KC, kc = it - p * KC, ix = c0 + p;
            const bool ok = row_ok && it < NITEM && ix >= 0 && ix < a.W;
            v[u] = ok ? __ldg(reinterpret_cast<const uint4*>(a.in + (rowbase + ix) * CIN + kc * 8))
                      : make_uint4(0, 0, 0, 0);
          }
          if (f > 0 && !tc::mbar_wait(&empty[slot], (uint32_t)((f - 1) & 1), kWaitLimit)) {
            raise_abort(abort_flag, a.status);
            stop = true;
            break;
          }
#pragma unroll
          for (int u = 0; u < PER; ++u) {
            const int it = gtid + u * L::GT;
            if (it >= NITEM) continue;
            const int p = it / KC, kc = it - p * KC;
            *reinterpret_cast<uint4*>(dst + (kc * kNP + p) * 16) = v[u];
          }
        }
        tc::fence_proxy_async();  // generic-proxy stores -> tensor-core (async proxy) reads
        tc::mbar_arrive(&full[slot]);
      }
    }
  } else if (warp == kMmaWarp) {
    // ---- MMA issue: one thread
    if (lane == 0) {
      const uint32_t sX_addr = tc::smem_addr(sX), sB_addr = tc::smem_addr(sB);
      long long j = 0, o = 0;
      bool stop = false;
      while (!stop && runs.next()) {
        for (int r = runs.ya - 1; r <= runs.yb; ++r, ++j) {
          const int slot = (int)(j % L::NR);
          if (*abort_flag || !tc::mbar_wait(&full[slot], (uint32_t)((j / L::NR) & 1), kWaitLimit)) {
            raise_abort(abort_flag, a.status);
            stop = true;
            break;
          }
          tc::fence_after_sync();
          const uint32_t xs = sX_addr + slot * L::SLOT_BYTES;
          if constexpr (L::STACK) {
            // tap row ky of input row r goes to output row r + 1 - ky, held in slot s_ky
            const int y0 = r + 1;
            const bool v0 = y0 >= runs.ya && y0 < runs.yb, v1 = y0 - 1 >= runs.ya && y0 - 1 < runs.yb,
                       v2 = y0 - 2 >= runs.ya && y0 - 2 < runs.yb;
            const int s0 = L::NS - 1 - (int)((o + (y0 - runs.ya)) % L::NS);
            const int s1 = s0 == L::NS - 1 ? 0 : s0 + 1, s2 = s1 == L::NS - 1 ? 0 : s1 + 1;
            if (v0) {  // first contribution to row r + 1: its slot must be drained and zeroed
              const long long use = (o + (y0 - runs.ya)) / L::NS;
              if (!tc::mbar_wait(&acc_empty[s0], (uint32_t)(use & 1), kWaitLimit)) {
                raise_abort(abort_flag, a.status);
                stop = true;
                break;
              }
              tc::fence_after_sync();
            }
            // one MMA of N = 64 * cnt for tap rows kys .. kys + cnt - 1 (adjacent slots from sidx)
            auto issue = [&](int kys, int cnt, int sidx) {
              const uint32_t d = tmem + (uint32_t)(sidx * COUT);
              const uint32_t idesc = tc::idesc_bf16_f32(kM, 64 * cnt);
              const uint32_t bstack = sB_addr + (uint32_t)(kys * 8 * (3 * KC * 128));
#pragma unroll 1
              for (int kx = 0; kx < 3; ++kx) {
#pragma unroll
                for (int t2 = 0; t2 < CIN / 16; ++t2) {
                  const uint64_t ad = tc::smem_desc(xs + (uint32_t)((2 * t2 * kNP + kx) * 16), kNP * 16, 128);
                  const uint64_t bd = tc::smem_desc(bstack + (uint32_t)((kx * KC + 2 * t2) * 128), 128, 3 * KC * 128);
                  tc::mma_bf16(d, ad, bd, idesc, 1u);
                }
              }
            };
            const bool a01 = s1 == s0 + 1, a12 = s2 == s1 + 1;  // no wrap-around between the slots
            if (v0 && v1 && v2 && a01 && a12) {
              issue(0, 3, s0);
            } else {
              if (v0 && v1 && a01) {
                issue(0, 2, s0);
                if (v2) issue(2, 1, s2);
              } else if (v1 && v2 && a12) {
                if (v0) issue(0, 1, s0);
                issue(1, 2, s1);
              } else {
                if (v0) issue(0, 1, s0);
                if (v1) issue(1, 1, s1);
                if (v2) issue(2, 1, s2);
              }
            }
            if (v2) tc::commit(&acc_full[s2]);  // output row r - 1 complete
          } else {
            constexpr uint32_t idesc = tc::idesc_bf16_f32(kM, COUT);
#pragma unroll
            for (int ky = 0; ky < 3; ++ky) {
              const int y = r + 1 - ky;
              if (y < runs.ya || y >= runs.yb) continue;
              const long long oo = o + (y - runs.ya);
              const int acc = (int)(oo % kAcc);
              const long long use = oo / kAcc;
              if (ky == 0 && use > 0) {  // first contribution: the accumulator's previous row must be drained
                if (!tc::mbar_wait(&acc_empty[acc], (uint32_t)((use - 1) & 1), kWaitLimit)) {
                  raise_abort(abort_flag, a.status);
                  stop = true;
                  break;
                }
                tc::fence_after_sync();
              }
              const uint32_t d = tmem + (uint32_t)(acc * COUT);
#pragma unroll
              for (int kx = 0; kx < 3; ++kx) {
#pragma unroll
                for (int s2 = 0; s2 < CIN / 16; ++s2) {
                  const uint64_t ad = tc::smem_desc(xs + (uint32_t)((2 * s2 * kNP + kx) * 16), kNP * 16, 128);
                  const uint64_t bd =
                      tc::smem_desc(sB_addr + (uint32_t)(((ky * 3 + kx) * KC + 2 * s2) * 128), 128, 9 * KC * 128);
                  tc::mma_bf16(d, ad, bd, idesc, (ky == 0 && kx == 0 && s2 == 0) ? 0u : 1u);
                }
              }
              if (ky == 2) tc::commit(&acc_full[acc]);  // last contribution to output row y
            }
          }
          if (stop) break;
          tc::commit(&empty[slot]);  // staged row consumed once these MMAs finish
        }
        o += runs.yb - runs.ya;
      }
      // all MMAs of this CTA complete before teardown
      tc::commit(mma_done);
      if (!tc::mbar_wait(mma_done, 0, kWaitLimit)) raise_abort(abort_flag, a.status);
    }
    __syncwarp();
  } else {
    // ---- epilogue: thread = pixel of the segment = TMEM lane
    if constexpr (L::STACK) {
      // every slot starts zeroed (first phase of its acc_empty barrier)
      for (int sidx = 0; sidx < L::NS; ++sidx) {
#pragma unroll
        for (int cc = 0; cc < COUT; cc += 32)
          tc::tmem_zero32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(sidx * COUT + cc));
        tc::fence_before_sync();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&acc_empty[sidx]);
      }
    }
    long long o = 0;
    bool stop = false;
    while (!stop && runs.next()) {
      for (int y = runs.ya; y < runs.yb; ++y, ++o) {
        const int acc = L::STACK ? L::NS - 1 - (int)(o % L::NS) : (int)(o % kAcc);
        const bool got = !*abort_flag && tc::mbar_wait(&acc_full[acc], (uint32_t)((o / L::NS) & 1), kWaitLimit);
        if (!__all_sync(0xffffffffu, got)) {
          raise_abort(abort_flag, a.status);
          stop = true;
          break;
        }
        tc::fence_after_sync();
#pragma unroll
        for (int cc = 0; cc < COUT; cc += 32) {
          float v[32];
          tc::tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(acc * COUT + cc), v);
          if (L::STACK) tc::tmem_zero32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(acc * COUT + cc));
          if (cc + 32 == COUT) {  // accumulator drained (and zeroed): hand it back to the MMA thread
            tc::fence_before_sync();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&acc_empty[acc]);
          }
#pragma unroll
          for (int q4 = 0; q4 < 8; ++q4) {
            const float4 b4 = *reinterpret_cast<const float4*>(sBias + cc + 4 * q4);
            v[4 * q4] += b4.x;
            v[4 * q4 + 1] += b4.y;
            v[4 * q4 + 2] += b4.z;
            v[4 * q4 + 3] += b4.w;
          }
          if (RELU) {
#pragma unroll
            for (int q = 0; q < 32; ++q) v[q] = fmaxf(v[q], 0.f);
          }
          const int ox0 = runs.seg * kM + warp * 32;  // pixel of the warp's lane 0
          const long long opix0 = ((long long)runs.b * a.H + y) * a.W + ox0;
          if (OUTF == 0) {
            // lane = pixel row of 64 bytes (four 16-byte slots), slot q stored at q ^ ((row >> 1) & 3):
            // conflict-free both when a lane writes its row and when 4 lanes read one row
            uint4* xb = reinterpret_cast<uint4*>(smem + L::XB_OFF) + warp * 128;
#pragma unroll
            for (int q = 0; q < 4; ++q)
              xb[lane * 4 + (q ^ ((lane >> 1) & 3))] =
                  make_uint4(bf2(v[8 * q], v[8 * q + 1]), bf2(v[8 * q + 2], v[8 * q + 3]),
                             bf2(v[8 * q + 4], v[8 * q + 5]), bf2(v[8 * q + 6], v[8 * q + 7]));
            __syncwarp();
            // each store instruction: 8 pixels x 64 contiguous bytes (lanes 4i..4i+3 one pixel)
            const int q = lane & 3;
            __nv_bfloat16* obase = a.out + opix0 * COUT + cc + 8 * q;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
              const int p = 8 * i + (lane >> 2);
              const uint4 t = xb[p * 4 + (q ^ ((p >> 1) & 3))];
              if (ox0 + p < a.W) *reinterpret_cast<uint4*>(obase + (long long)p * COUT) = t;
            }
            __syncwarp();
          } else {
            // lane = pixel row of the warp's tile, 16-byte slot q stored at q ^ (row & 7):
            // conflict-free both when a lane writes its row and when 8 lanes read one row
            float4* xb = reinterpret_cast<float4*>(smem + L::XB_OFF) + warp * 256;
#pragma unroll
            for (int q = 0; q < 8; ++q)
              xb[lane * 8 + (q ^ (lane & 7))] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
            __syncwarp();
            // each store instruction: 4 pixels x 128 contiguous bytes (lanes 8i..8i+7 one pixel)
            const int q = lane & 7;
            float* obase = a.out_f32 + opix0 * COUT + cc + 4 * q;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
              const int p = 4 * i + (lane >> 3);
              const float4 t = xb[p * 8 + (q ^ (p & 7))];
              if (ox0 + p < a.W) *reinterpret_cast<float4*>(obase + (long long)p * COUT) = t;
            }
            __syncwarp();
          }
        }
      }
    }
  }
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, L::TMEM_COLS);
  }
}

// float32 [cout][cin][3][3] -> bf16 image of the shared-memory weight layout:
// tap-major K (k = tap * cin + ci) for cout != 64, tap rows stacked along N
// (n = ky * 64 + co, k = kx * cin + ci) for cout == 64.
__global__ void pack_rows_weights_kernel(const float* __restrict__ w, int cout, int cin, uint16_t* __restrict__ img) {
  const int n_el = cout * 9 * cin;
  const int kc = cin / 8;
  const bool stack = cout == 64;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_el; i += gridDim.x * blockDim.x) {
    int n, k, co, ci, ky, kx;
    if (stack) {
      n = i / (3 * cin);
      k = i - n * 3 * cin;
      ky = n / cout;
      co = n - ky * cout;
      kx = k / cin;
      ci = k - kx * cin;
    } else {
      n = i / (9 * cin);
      k = i - n * 9 * cin;
      const int tap = k / cin;
      ci = k - tap * cin;
      co = n;
      ky = tap / 3;
      kx = tap - 3 * ky;
    }
    const __nv_bfloat16 v = __float2bfloat16_rn(w[(((long long)co * cin + ci) * 3 + ky) * 3 + kx]);
    const int kchunks = stack ? 3 * kc : 9 * kc;
    img[(n >> 3) * kchunks * 64 + (k >> 3) * 64 + (n & 7) * 8 + (k & 7)] = *reinterpret_cast<const uint16_t*>(&v);
  }
}

template <int CIN, int COUT, int SRC, int OUTF, bool RELU>
cudaError_t launch_rows(const ConvRowsArgs& a, cudaStream_t st) {
  using L = RowStreamLayout<CIN, COUT, SRC, OUTF>;
  const long long T = (long long)a.batch * ((a.W + kM - 1) / kM) * a.H;
  if (T < 1) return cudaSuccess;
  int dev = 0, nsm = 148;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int grid = T < nsm ? (int)T : nsm;  // one CTA per SM (shared memory and TMEM admit one)
  conv3x3_rows_tc_kernel<CIN, COUT, SRC, OUTF, RELU><<<grid, kThreads, L::SMEM, st>>>(a);
  return cudaGetLastError();
}

template <int CIN, int COUT, int SRC, int OUTF, bool RELU>
cudaError_t configure_rows() {
  using L = RowStreamLayout<CIN, COUT, SRC, OUTF>;
  return cudaFuncSetAttribute(conv3x3_rows_tc_kernel<CIN, COUT, SRC, OUTF, RELU>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, L::SMEM);
}

}  // namespace

cudaError_t configure_conv_rows_tc() {
  cudaError_t e;
  if ((e = configure_rows<128, 64, 2, 0, true>()) != cudaSuccess) return e;
  if ((e = configure_rows<64, 64, 0, 0, true>()) != cudaSuccess) return e;
  return configure_rows<64, 128, 0, 1, false>();
}

size_t conv_rows_weight_bytes(int cin, int cout) { return (size_t)9 * cin * cout * 2; }

cudaError_t pack_conv_rows_weights(const float* w, int cout, int cin, uint16_t* img, cudaStream_t st) {
  if (cin % 16 || cout % 8) return cudaErrorInvalidValue;
  const int n = cout * 9 * cin;
  pack_rows_weights_kernel<<<(n + 255) / 256, 256, 0, st>>>(w, cout, cin, img);
  return cudaGetLastError();
}

cudaError_t launch_conv_rows_tc(const ConvRowsArgs& a, int cin, int cout, int src, int outf, bool relu,
                                cudaStream_t st) {
  if (cin == 128 && cout == 64 && src == 2 && outf == 0 && relu) return launch_rows<128, 64, 2, 0, true>(a, st);
  if (cin == 64 && cout == 64 && src == 0 && outf == 0 && relu) return launch_rows<64, 64, 0, 0, true>(a, st);
  if (cin == 64 && cout == 128 && src == 0 && outf == 1 && !relu) return launch_rows<64, 128, 0, 1, false>(a, st);
  return cudaErrorInvalidValue;
}

}  // namespace bme

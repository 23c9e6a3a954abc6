// 3x3 stride-2 convolution (zero pad 1), 32 output channels, streamed row by
// row on the 5th-generation tensor cores: layers 1 and 2 of the learned
// proposal network, the layers with enough output rows to keep a pipeline
// full (layers 3 and 4 use the per-tile kernel of conv_tc.cu).
//
//   out[y, x, n] = relu(bias[n] + sum_{ky, kx, ci} in[2y + ky - 1, 2x + kx - 1, ci] * w[n, ci, ky, kx])
//
// Work: the output is cut into segments of 128 pixels of one row (the MMA M);
// each CTA owns a contiguous range of output rows of the (image, segment, row)
// order and walks down each column strip.  Input row r is staged in shared
// memory exactly once, split into two column-parity planes, and feeds the
// output rows it touches: an odd row r adds tap row ky = 2 to output row
// (r - 1) / 2 and ky = 0 to row (r + 1) / 2, an even row adds ky = 1 to row
// r / 2.  Output row pixel x of tap column kx reads plane kx % 2 at pixel
// x + kx / 2, so every tap's A operand is a shifted view of the staged row.
// Each output row accumulates in one of four rotating TMEM accumulators, so
// the epilogue of one row overlaps the MMAs of the next ones.
//
// Warp roles (416 threads):
//   warps 0-3   epilogue: TMEM -> registers -> bias, ReLU -> bf16 NHWC
//               (warp w reads TMEM lanes 32w..32w+31 = pixels of the segment);
//   warp 4      one thread issues the MMAs and commits them to mbarriers;
//   warps 5-12  producers in groups taking input rows round-robin: global
//               loads of the row (16-byte NHWC chunks, or for layer 1 the
//               Bayer frames with 16-byte loads, each 12-bit sample split into
//               two exact bf16 operand channels), stored as K-major core
//               matrices.
// Ring of staged rows with full / empty mbarriers; weights (packed once per
// forward by pack_conv_tc_weights) and bias resident in shared memory.  Every
// wait is bounded: on expiry the CTA raises an abort flag, records
// BAYER_ERR_TIMEOUT, waits (bounded) for its own MMAs and frees its TMEM.
#include <cuda_bf16.h>

#include "common.cuh"
#include "kernels.cuh"
#include "tc_common.cuh"

namespace bme {

namespace {

constexpr int kM = 128;     // output pixels per row segment (MMA M)
constexpr int kN = 32;      // output channels (MMA N)
constexpr int kNJ = 2 * kM + 1;  // staged input columns per row segment (257)
constexpr int kNP = 129;    // pixels per parity plane; 129 * 16 B = 16 mod 128 (conflict-free stores)
constexpr int kAcc = 4;     // TMEM accumulators (output rows in flight)
constexpr int kEpiWarps = 4, kMmaWarp = 4, kProdWarp0 = 5, kProdWarps = 8;
constexpr int kProdThreads = kProdWarps * 32;
constexpr int kThreads = (kProdWarp0 + kProdWarps) * 32;
constexpr int kTmemCols = kAcc * kN;
constexpr uint32_t kWaitLimit = 1u << 22;

// Shared-memory plan.  Staged row: element (parity q, chunk kc of 8 channels,
// pixel p) at ((q * KC + kc) * kNP + p) * 16: the A operand of tap column kx
// and K step s2 starts at ((kx % 2) * KC + 2 * s2) * kNP + kx / 2 (units of
// 16 bytes), core matrices of 8 consecutive pixels (SBO 128 B), the next K
// chunk one plane further (LBO kNP * 16).  Weights as packed by
// pack_conv_tc_weights: element (n, k), k = tap * CIN + ci, at
// (n / 8) * (9 * KC) * 128 + (k / 8) * 128 + (n % 8) * 16 + (k % 8) * 2.
// Ring: NR slots filled by G producer groups taking rows j % G (slot j % NR
// always belongs to group j % G).  Layer 1 (Bayer frames) has small rows and
// little work per loaded byte, so it keeps more rows in flight: 8 slots, 8
// one-warp groups; layer 2: 4 slots, 2 groups.
template <int CIN, int SRC>
struct S2Layout {
  static constexpr int KC = CIN / 8;
  static constexpr int NR = SRC == 1 ? 8 : 4;
  static constexpr int G = SRC == 1 ? 8 : 2;
  static constexpr int GT = kProdThreads / G;
  static constexpr int SLOT_BYTES = 2 * KC * kNP * 16;
  static constexpr int B_BYTES = 9 * CIN * kN * 2;
  static constexpr int BAR_OFF = B_BYTES + NR * SLOT_BYTES;
  static constexpr int NBAR = 2 * NR + 2 * kAcc + 1;
  static constexpr int BIAS_OFF = (BAR_OFF + NBAR * 8 + 16 + 15) / 16 * 16;
  static constexpr int SMEM = BIAS_OFF + kN * 4;
  static_assert(CIN % 16 == 0, "shape");
  static_assert(B_BYTES % 16 == 0 && SLOT_BYTES % 16 == 0, "alignment");
  static_assert(SMEM <= 113 * 1024, "two CTAs per SM");
  static_assert(NR % G == 0, "a slot belongs to one group");
};

using tc::bf2;
using tc::split12;

// The CTA's output rows [t, t1) of the (image, segment, y)-ordered list, cut
// into runs that stay inside one column strip.
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

// SRC 0: bf16 NHWC input [batch][Hi][Wi][CIN]; SRC 1: the Bayer frames (CIN =
// 16 operand channels from 8 half-resolution planes).
template <int CIN, int SRC>
__global__ void __launch_bounds__(kThreads, 2) conv3x3s2_rows_tc_kernel(const ConvTcArgs a) {
  using L = S2Layout<CIN, SRC>;
  constexpr int KC = L::KC, kNR = L::NR, kGroups = L::G, kGT = L::GT;
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* sB = smem;
  uint8_t* sX = smem + L::B_BYTES;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + L::BAR_OFF);
  uint64_t* empty = full + kNR;
  uint64_t* acc_full = empty + kNR;
  uint64_t* acc_empty = acc_full + kAcc;
  uint64_t* mma_done = acc_empty + kAcc;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mma_done + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  float* sBias = reinterpret_cast<float*>(smem + L::BIAS_OFF);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (tid == 0) {
    for (int s = 0; s < kNR; ++s) {
      tc::mbar_init(&full[s], kGT);
      tc::mbar_init(&empty[s], 1);
    }
    for (int i = 0; i < kAcc; ++i) {
      tc::mbar_init(&acc_full[i], 1);
      tc::mbar_init(&acc_empty[i], kEpiWarps);
    }
    tc::mbar_init(mma_done, 1);
    *abort_flag = 0;
    tc::fence_mbar_init();
  }
  if (warp == 0) tc::tmem_alloc(tmem_slot, kTmemCols);
  for (int i = tid; i < L::B_BYTES / 16; i += kThreads) reinterpret_cast<uint4*>(sB)[i] = __ldg(a.wimg + i);
  for (int i = tid; i < kN; i += kThreads) sBias[i] = __bfloat162float(a.bias[i]);
  tc::fence_proxy_async();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tmem_slot;

  const int segs = (a.Wo + kM - 1) / kM;
  const long long T = (long long)a.batch * segs * a.Ho;
  Runs runs{T * blockIdx.x / gridDim.x, T * (blockIdx.x + 1) / gridDim.x, a.Ho, segs, 0, 0, 0, 0};

  if (warp >= kProdWarp0) {
    // ---- producers: input rows 2ya-1 .. 2yb-1 of each run; group g takes rows j % G == g
    const int ptid = tid - kProdWarp0 * 32;
    const int group = ptid / kGT, gtid = ptid - group * kGT;
    long long j = 0;
    bool stop = false;
    while (!stop && runs.next()) {
      const int c0 = 2 * runs.seg * kM - 1;  // input column of staged column 0
      for (int r = 2 * runs.ya - 1; r <= 2 * runs.yb - 1; ++r, ++j) {
        if ((int)(j % kGroups) != group) continue;
        if (*abort_flag) {
          stop = true;
          break;
        }
        const int slot = (int)(j % kNR);
        const long long f = j / kNR;
        const bool row_ok = r >= 0 && r < a.Hi;
        uint8_t* dst = sX + slot * L::SLOT_BYTES;
        if (SRC == 0) {
          constexpr int NITEM = kNJ * KC;
          constexpr int PER = (NITEM + kGT - 1) / kGT;
          const long long rowbase = ((long long)runs.b * a.Hi + r) * a.Wi;
          uint4 v[PER];
#pragma unroll
          for (int u = 0; u < PER; ++u) {
            const int it = gtid + u * kGT;
            const int p = it / KC, kc = it - p * KC, ix = c0 + p;
            const bool ok = row_ok && it < NITEM && ix >= 0 && ix < a.Wi;
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
            const int it = gtid + u * kGT;
            if (it >= NITEM) continue;
            const int p = it / KC, kc = it - p * KC;
            *reinterpret_cast<uint4*>(dst + (((p & 1) * KC + kc) * kNP + (p >> 1)) * 16) = v[u];
          }
        } else if (a.vec) {
          // item = (frame, group of 4 half-resolution columns hx .. hx + 3,
          // hx = c0 - 3 + 4g a multiple of 4): two 16-byte loads (raw rows
          // 2r, 2r + 1) hold the 4 planes of 4 pixels; Wi % 4 == 0, so a
          // group is wholly inside or outside the map
          constexpr int NGRP = (kNJ - 1) / 4 + 1;
          constexpr int NITEM = 2 * NGRP;
          constexpr int PER = (NITEM + kGT - 1) / kGT;
          uint4 r0[PER], r1[PER];
#pragma unroll
          for (int u = 0; u < PER; ++u) {
            const int it = gtid + u * kGT;
            const int fr = it / NGRP, g = it - fr * NGRP;
            const int hx = c0 - 3 + 4 * g;
            r0[u] = r1[u] = make_uint4(0, 0, 0, 0);
            if (row_ok && it < NITEM && hx >= 0 && hx < a.Wi) {
              const uint16_t* fb = fr == 0 ? a.fr.ref + (long long)runs.b * a.fr.ref_bs
                                           : a.fr.cur + (long long)runs.b * a.fr.cur_bs;
              const uint16_t* p = fb + (long long)(2 * r) * a.fr.pitch + 2 * hx;
              r0[u] = __ldg(reinterpret_cast<const uint4*>(p));
              r1[u] = __ldg(reinterpret_cast<const uint4*>(p + a.fr.pitch));
            }
          }
          if (f > 0 && !tc::mbar_wait(&empty[slot], (uint32_t)((f - 1) & 1), kWaitLimit)) {
            raise_abort(abort_flag, a.status);
            stop = true;
            break;
          }
#pragma unroll
          for (int u = 0; u < PER; ++u) {
            const int it = gtid + u * kGT;
            if (it >= NITEM) continue;
            const int fr = it / NGRP, g = it - fr * NGRP;
            const int hx = c0 - 3 + 4 * g;
            const bool in_ok = row_ok && hx >= 0 && hx < a.Wi;
            const uint32_t w0[4] = {r0[u].x, r0[u].y, r0[u].z, r0[u].w};
            const uint32_t w1[4] = {r1[u].x, r1[u].y, r1[u].z, r1[u].w};
#pragma unroll
            for (int t = 0; t < 4; ++t) {
              const int jj = 4 * g - 3 + t;
              if (jj < 0 || jj >= kNJ) continue;
              uint4 val = make_uint4(0, 0, 0, 0);
              if (in_ok)
                val = make_uint4(split12(w0[t] & 0xFFFFu), split12(w0[t] >> 16), split12(w1[t] & 0xFFFFu),
                                 split12(w1[t] >> 16));
              *reinterpret_cast<uint4*>(dst + (((jj & 1) * KC + fr) * kNP + (jj >> 1)) * 16) = val;
            }
          }
        } else {
          // unaligned frames: one 2-byte load per plane sample, item by item
          // once the slot is free (the rare path)
          if (f > 0 && !tc::mbar_wait(&empty[slot], (uint32_t)((f - 1) & 1), kWaitLimit)) {
            raise_abort(abort_flag, a.status);
            stop = true;
            break;
          }
          for (int jj = gtid; jj < kNJ; jj += kGT) {
            const int ix = c0 + jj;
            const bool ok = row_ok && ix >= 0 && ix < a.Wi;
            uint32_t wd[8];
#pragma unroll
            for (int c = 0; c < 8; ++c) {
              const uint16_t* fb = c < 4 ? a.fr.ref + (long long)runs.b * a.fr.ref_bs
                                         : a.fr.cur + (long long)runs.b * a.fr.cur_bs;
              const int pl = c & 3;
              wd[c] = ok ? split12(__ldg(fb + (long long)(2 * r + (pl >> 1)) * a.fr.pitch + 2 * ix + (pl & 1))) : 0u;
            }
            *reinterpret_cast<uint4*>(dst + (((jj & 1) * KC + 0) * kNP + (jj >> 1)) * 16) =
                make_uint4(wd[0], wd[1], wd[2], wd[3]);
            *reinterpret_cast<uint4*>(dst + (((jj & 1) * KC + 1) * kNP + (jj >> 1)) * 16) =
                make_uint4(wd[4], wd[5], wd[6], wd[7]);
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
      constexpr uint32_t idesc = tc::idesc_bf16_f32(kM, kN);
      long long j = 0, o = 0;
      bool stop = false;
      while (!stop && runs.next()) {
        for (int r = 2 * runs.ya - 1; r <= 2 * runs.yb - 1; ++r, ++j) {
          const int slot = (int)(j % kNR);
          if (*abort_flag || !tc::mbar_wait(&full[slot], (uint32_t)((j / kNR) & 1), kWaitLimit)) {
            raise_abort(abort_flag, a.status);
            stop = true;
            break;
          }
          tc::fence_after_sync();
          const uint32_t xs = sX_addr + slot * L::SLOT_BYTES;
          // odd rows: ky = 2 (finishes output row (r-1)/2), then ky = 0 (starts row (r+1)/2);
          // even rows: ky = 1 of row r/2
#pragma unroll
          for (int pass = 0; pass < 2; ++pass) {
            int ky, y;
            if (r & 1) {
              ky = pass == 0 ? 2 : 0;
              y = pass == 0 ? (r - 1) >> 1 : (r + 1) >> 1;
            } else {
              if (pass == 1) break;
              ky = 1;
              y = r >> 1;
            }
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
            const uint32_t d = tmem + (uint32_t)(acc * kN);
#pragma unroll
            for (int kx = 0; kx < 3; ++kx) {
#pragma unroll
              for (int s2 = 0; s2 < CIN / 16; ++s2) {
                const uint64_t ad =
                    tc::smem_desc(xs + (uint32_t)((((kx & 1) * KC + 2 * s2) * kNP + (kx >> 1)) * 16), kNP * 16, 128);
                const uint64_t bd =
                    tc::smem_desc(sB_addr + (uint32_t)(((ky * 3 + kx) * KC + 2 * s2) * 128), 128, 9 * KC * 128);
                tc::mma_bf16(d, ad, bd, idesc, (ky == 0 && kx == 0 && s2 == 0) ? 0u : 1u);
              }
            }
            if (ky == 2) tc::commit(&acc_full[acc]);  // last contribution to output row y
          }
          if (stop) break;
          tc::commit(&empty[slot]);  // staged row consumed once these MMAs finish
        }
        o += runs.yb - runs.ya;
      }
      tc::commit(mma_done);
      if (!tc::mbar_wait(mma_done, 0, kWaitLimit)) raise_abort(abort_flag, a.status);
    }
    __syncwarp();
  } else {
    // ---- epilogue: thread = pixel of the segment = TMEM lane
    long long o = 0;
    bool stop = false;
    while (!stop && runs.next()) {
      for (int y = runs.ya; y < runs.yb; ++y, ++o) {
        const int acc = (int)(o % kAcc);
        const bool got = !*abort_flag && tc::mbar_wait(&acc_full[acc], (uint32_t)((o / kAcc) & 1), kWaitLimit);
        if (!__all_sync(0xffffffffu, got)) {
          raise_abort(abort_flag, a.status);
          stop = true;
          break;
        }
        tc::fence_after_sync();
        float v[32];
        tc::tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(acc * kN), v);
        tc::fence_before_sync();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&acc_empty[acc]);  // accumulator drained
        const int ox = runs.seg * kM + tid;
        if (ox < a.Wo) {
#pragma unroll
          for (int q4 = 0; q4 < 8; ++q4) {
            const float4 b4 = *reinterpret_cast<const float4*>(sBias + 4 * q4);
            v[4 * q4] = fmaxf(v[4 * q4] + b4.x, 0.f);
            v[4 * q4 + 1] = fmaxf(v[4 * q4 + 1] + b4.y, 0.f);
            v[4 * q4 + 2] = fmaxf(v[4 * q4 + 2] + b4.z, 0.f);
            v[4 * q4 + 3] = fmaxf(v[4 * q4 + 3] + b4.w, 0.f);
          }
          const long long opix = ((long long)runs.b * a.Ho + y) * a.Wo + ox;
          uint4* o4 = reinterpret_cast<uint4*>(a.out + opix * kN);
#pragma unroll
          for (int q4 = 0; q4 < 4; ++q4)
            o4[q4] = make_uint4(bf2(v[8 * q4], v[8 * q4 + 1]), bf2(v[8 * q4 + 2], v[8 * q4 + 3]),
                                bf2(v[8 * q4 + 4], v[8 * q4 + 5]), bf2(v[8 * q4 + 6], v[8 * q4 + 7]));
        }
      }
    }
  }
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, kTmemCols);
  }
}

template <int CIN, int SRC>
cudaError_t launch_s2(const ConvTcArgs& a, cudaStream_t st) {
  using L = S2Layout<CIN, SRC>;
  auto kern = conv3x3s2_rows_tc_kernel<CIN, SRC>;
  const long long T = (long long)a.batch * ((a.Wo + kM - 1) / kM) * a.Ho;
  if (T < 1) return cudaSuccess;
  int dev = 0, nsm = 148;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int per_sm = tc::ctas_per_sm(kern, kThreads, L::SMEM, kTmemCols);
  long long grid = (long long)nsm * per_sm;
  // at least ~4 output rows per CTA keep the ring and the accumulators busy
  if (grid > (T + 3) / 4) grid = (T + 3) / 4;
  if (grid < 1) grid = 1;
  kern<<<(unsigned)grid, kThreads, L::SMEM, st>>>(a);
  return cudaGetLastError();
}

template <int CIN, int SRC>
cudaError_t configure_s2() {
  using L = S2Layout<CIN, SRC>;
  auto kern = conv3x3s2_rows_tc_kernel<CIN, SRC>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, L::SMEM);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  return e;
}

}  // namespace

cudaError_t configure_conv_s2_rows_tc() {
  cudaError_t e;
  if ((e = configure_s2<16, 1>()) != cudaSuccess) return e;
  return configure_s2<32, 0>();
}

cudaError_t launch_conv_s2_rows_tc(const ConvTcArgs& a, int layer, cudaStream_t st) {
  if (layer == 1) return launch_s2<16, 1>(a, st);
  if (layer == 2) return launch_s2<32, 0>(a, st);
  return cudaErrorInvalidValue;
}

}  // namespace bme

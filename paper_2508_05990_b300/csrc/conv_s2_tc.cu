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
// Warp roles (416 threads; 320 for layer 1 with TMA):
//   warps 0-3   epilogue: TMEM -> registers -> bias, ReLU -> bf16 NHWC
//               (warp w reads TMEM lanes 32w..32w+31 = pixels of the segment);
//   warp 4      one thread issues the MMAs and commits them to mbarriers;
//   warps 5-12  producers in groups taking input rows round-robin (layer 1
//               with TMA: warps 5-8, two groups of two warps): layer 2
//               loads the row's 16-byte NHWC chunks and stores them as K-major
//               core matrices; layer 1 turns each 12-bit Bayer sample v into
//               the TF32 operand v/2048 - 1 (exact), its MMAs running in
//               kind::tf32 on the bf16 weights widened exactly to float32;
//   warp 9      (layer 1 with 16-byte aligned frame rows) one thread copies
//               the two raw rows of each staged half-resolution row of both
//               frames by TMA (one box per frame) into a ring that the
//               producers convert from, four columns per 16-byte word of
//               each raw row, so that they do no global address arithmetic
//               or loads.
//               Otherwise the producers load the frames themselves.
// Ring of staged rows: full mbarriers, and a slot is free again once the
// commit that completes an output row covers its last MMA; weights (packed once per
// forward by pack_conv_tc_weights) and bias resident in shared memory.  Every
// wait is bounded: on expiry the CTA raises an abort flag, records
// BAYER_ERR_TIMEOUT, waits (bounded) for its own MMAs and frees its TMEM.
#include <cuda_bf16.h>

#include "common.cuh"
#include "kernels.cuh"
#include "tc_common.cuh"
#include "tma.cuh"

namespace bme {

namespace {

constexpr int kM = 128;     // output pixels per row segment (MMA M)
constexpr int kN = 32;      // output channels (MMA N)
constexpr int kNJ = 2 * kM + 1;  // staged input columns per row segment (257)
constexpr int kNP = 129;    // pixels per parity plane; 129 * 16 B = 16 mod 128 (conflict-free stores)
constexpr int kAcc = 4;     // TMEM accumulators (output rows in flight)
// Epilogue transpose buffer: one row of 16 bf16x2 words per pixel, pitch 20
// words (16-byte stores of a pixel row and 16-byte loads across pixels both
// take few wavefronts).
constexpr int kTP = 20;
// Warp roles: 4 epilogue warps, the MMA warp, 8 producer warps and, for SRC
// 2, one TMA warp.
template <int SRC>
struct Roles {
  static constexpr int EPI = 4;
  static constexpr int MMA = EPI;
  static constexpr int PROD0 = MMA + 1;
  static constexpr int PROD = SRC == 2 ? 4 : 8;
  static constexpr int TMA = PROD0 + PROD;  // SRC 2 only
  static constexpr int THREADS = (PROD0 + PROD + (SRC == 2 ? 1 : 0)) * 32;
};
template <int SRC>
__host__ __device__ constexpr int threads_of() {
  return Roles<SRC>::THREADS;
}
// SRC 2 raw ring: per staged row, for each frame, one TMA box of 66 16-byte
// chunks x 2 raw rows (samples 512 * seg - 8 .. + 527 of raw rows 2r, 2r + 1,
// 1056 bytes per row), the frames 2176 bytes (128-byte aligned) apart.
constexpr int kRawChunks = 66, kRawRowBytes = kRawChunks * 16, kRawBoxBytes = 2 * kRawRowBytes, kRawBoxStep = 2176;
constexpr int kRawSlot = 2 * kRawBoxStep;
constexpr int kTmemCols = kAcc * kN;
constexpr uint32_t kWaitLimit = 1u << 22;

// Shared-memory plan.  Staged row: 16-byte chunk (parity q, chunk kc, pixel p)
// at ((q * KC + kc) * kNP + p) * 16, a chunk holding 8 bf16 channels (layer 2)
// or, for layer 1, the 4 planes of one frame as TF32 (CIN = 16 counts the
// bytes of two such chunks as 16 bf16 would): the A operand of tap column kx
// and K step s2 starts at ((kx % 2) * KC + 2 * s2) * kNP + kx / 2 (units of
// 16 bytes), core matrices of 8 consecutive pixels (SBO 128 B), the next K
// chunk one plane further (LBO kNP * 16).  Weights as packed by
// pack_conv_tc_weights, in the same chunk arithmetic: element (n, k), k = tap
// * CIN + ci, at (n / 8) * (9 * KC) * 128 + (k / 8) * 128 + (n % 8) * 16 +
// (k % 8) * 2 for bf16 (layer 1: 4 TF32 values per 16-byte chunk).
// Ring: NR slots filled by G producer groups taking rows j % G (slot j % NR
// always belongs to group j % G).  Layer 1 (Bayer frames) has small rows and
// little work per loaded byte, so it keeps more rows in flight: 8 slots, 8
// one-warp groups; converting TMA-staged rows, 4 slots, 2 two-warp groups and
// 4 raw slots, so that three CTAs fit an SM (70 KB, 320 threads); layer 2: 4
// slots, 2 groups of 4 warps.
template <int CIN, int SRC>
struct S2Layout {
  static constexpr int KC = CIN / 8;
  static constexpr int NR = SRC == 2 ? 4 : (SRC != 0 ? 8 : 4);
  static constexpr int G = SRC == 0 ? 2 : (SRC == 1 ? 8 : 2);
  static constexpr int GT = Roles<SRC>::PROD * 32 / G;
  static constexpr int RR = SRC == 2 ? 4 : 0;  // raw ring slots
  static constexpr int SLOT_BYTES = 2 * KC * kNP * 16;
  static constexpr int B_BYTES = 9 * CIN * kN * 2;
  static constexpr int RAW_OFF = B_BYTES + NR * SLOT_BYTES;
  static constexpr int BAR_OFF = RAW_OFF + RR * kRawSlot;
  static constexpr int NBAR = 2 * NR + 2 * kAcc + 1 + 2 * RR;
  static constexpr int BIAS_OFF = (BAR_OFF + NBAR * 8 + 16 + 15) / 16 * 16;
  static constexpr int TR_OFF = BIAS_OFF + kN * 4;  // epilogue transpose buffers (16-byte aligned)
  static constexpr int SMEM = TR_OFF + Roles<SRC>::EPI * 32 * kTP * 4;
  static_assert(CIN % 16 == 0, "shape");
  static_assert(B_BYTES % 16 == 0 && SLOT_BYTES % 16 == 0, "alignment");
  static_assert(SMEM <= 113 * 1024, "two CTAs per SM (three for layer 1 with TMA)");
  static_assert(NR % G == 0, "a slot belongs to one group");
  static_assert(RAW_OFF % 128 == 0, "TMA destinations 128-byte aligned");
};

using tc::bf2;
using tc::tf32_sample12;

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
// 16: the bytes of 8 TF32 half-resolution planes), loaded by the producers;
// SRC 2: the same, raw rows staged by TMA (tm_ref, tm_cur: boxes of
// 66 chunks of 8 samples x 2 rows over [batch][H][W/8][8]).
template <int CIN, int SRC>
__global__ void __launch_bounds__(threads_of<SRC>(), SRC == 2 ? 3 : 2)
    conv3x3s2_rows_tc_kernel(const ConvTcArgs a, const __grid_constant__ CUtensorMap tm_ref,
                             const __grid_constant__ CUtensorMap tm_cur) {
  using L = S2Layout<CIN, SRC>;
  constexpr int KC = L::KC, kNR = L::NR, kGroups = L::G, kGT = L::GT, kRR = L::RR;
  constexpr int kRRm = kRR > 0 ? kRR : 1;  // divisor for the SRC 2 ring arithmetic
  constexpr int kThreads = threads_of<SRC>();
  using R = Roles<SRC>;
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* sB = smem;
  uint8_t* sX = smem + L::B_BYTES;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + L::BAR_OFF);
  uint64_t* acc_full = full + 2 * kNR;
  uint64_t* acc_empty = acc_full + kAcc;
  uint64_t* mma_done = acc_empty + kAcc;
  uint64_t* raw_full = mma_done + 1;  // SRC 2
  uint64_t* raw_empty = raw_full + kRR;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(raw_empty + kRR);
  uint8_t* sRaw = smem + L::RAW_OFF;
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  float* sBias = reinterpret_cast<float*>(smem + L::BIAS_OFF);
  uint32_t* sTr = reinterpret_cast<uint32_t*>(smem + L::TR_OFF);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (tid == 0) {
    for (int s = 0; s < kNR; ++s) {
      tc::mbar_init(&full[s], kGT);
    }
    for (int i = 0; i < kAcc; ++i) {
      tc::mbar_init(&acc_full[i], 1);
      tc::mbar_init(&acc_empty[i], R::EPI);
    }
    tc::mbar_init(mma_done, 1);
    for (int s = 0; s < kRR; ++s) {
      tc::mbar_init(&raw_full[s], 1);
      tc::mbar_init(&raw_empty[s], kGT);
    }
    *abort_flag = 0;
    tc::fence_mbar_init();
  }
  if (warp == 0) tc::tmem_alloc(tmem_slot, kTmemCols);
  // Launched as a dependent of the previous kernel: layer 2's weights (packed
  // before layer 1 ran, which waited for them before triggering) load while
  // layer 1 finishes; layer 1 waits for the packing kernel first.  Trigger the
  // next layer only after this wait, so that it may rely on the same.
  if (SRC == 0) {
    for (int i = tid; i < L::B_BYTES / 16; i += kThreads) reinterpret_cast<uint4*>(sB)[i] = __ldg(a.wimg + i);
    for (int i = tid; i < kN; i += kThreads) sBias[i] = __bfloat162float(a.bias[i]);
  }
  tc::grid_dep_wait();
  tc::grid_dep_launch();
  if (SRC != 0) {
    for (int i = tid; i < L::B_BYTES / 16; i += kThreads) reinterpret_cast<uint4*>(sB)[i] = __ldg(a.wimg + i);
    for (int i = tid; i < kN; i += kThreads) sBias[i] = __bfloat162float(a.bias[i]);
  }
  tc::fence_proxy_async();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tmem_slot;

  const int segs = (a.Wo + kM - 1) / kM;
  const long long T = (long long)a.batch * segs * a.Ho;
  Runs runs{T * blockIdx.x / gridDim.x, T * (blockIdx.x + 1) / gridDim.x, a.Ho, segs, 0, 0, 0, 0};

  if (SRC == 2 && warp == R::TMA) {
    // ---- raw rows by TMA, every staged row in order (rows outside the map:
    // an arrival without copies; the producers write zeros)
    if (lane == 0) {
      long long j = 0;
      bool stop = false;
      while (!stop && runs.next()) {
        for (int r = 2 * runs.ya - 1; r <= 2 * runs.yb - 1; ++r, ++j) {
          const int s = (int)(j % kRRm);
          const long long u = j / kRRm;
          if (*abort_flag ||
              (u > 0 && !tc::mbar_wait(&raw_empty[s], (uint32_t)((u - 1) & 1), kWaitLimit))) {
            raise_abort(abort_flag, a.status);
            stop = true;
            break;
          }
          if (r >= 0 && r < a.Hi) {
            tma::mbar_arrive_expect_tx(&raw_full[s], 2 * kRawBoxBytes);
            tma::load_4d(sRaw + s * kRawSlot, &tm_ref, 0, (4 * runs.seg * kM - 8) / 8, 2 * r, runs.b, &raw_full[s]);
            tma::load_4d(sRaw + s * kRawSlot + kRawBoxStep, &tm_cur, 0, (4 * runs.seg * kM - 8) / 8, 2 * r, runs.b,
                         &raw_full[s]);
          } else {
            tc::mbar_arrive(&raw_full[s]);
          }
        }
      }
      // the copies still in flight land before the CTA may exit
      for (long long k = j - 1; k >= 0 && k >= j - kRR; --k)
        tc::mbar_wait(&raw_full[k % kRRm], (uint32_t)((k / kRRm) & 1), kWaitLimit);
    }
    __syncwarp();
  } else if (warp >= R::PROD0) {
    // ---- producers: input rows 2ya-1 .. 2yb-1 of each run; group g takes rows j % G == g
    const int ptid = tid - R::PROD0 * 32;
    const int group = ptid / kGT, gtid = ptid - group * kGT;
    // SRC 2: staged columns 1 .. 256 form 64 groups of four, jj = 4g + 1 ..
    // 4g + 4, whose raw samples 8g + 8 .. 8g + 15 are one 16-byte word per
    // raw row; column 0 (samples 6, 7) is converted on its own.  Task tau =
    // gtid + kGT k (k = 0, 1) is (frame fr, group g): per 8-lane phase the
    // eight raw loads read eight consecutive 16-byte words (distinct bank
    // groups) and the 16-byte stores of one column of the four land on
    // plane chunks 2g + c + fr * kNP (kNP = 1 mod 8), eight distinct groups
    static_assert(SRC != 2 || (kGT == 64 && kNJ == 257), "two tasks per thread cover the 128 (frame, group) tasks");
    int cv_fr[2], cv_g[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const int tau = gtid + kGT * k, l = tau & 31, k8 = l >> 3, r = l & 7;
      cv_g[k] = 16 * (tau >> 5) + 8 * (k8 >> 1) + r;
      cv_fr[k] = (r >> 2) ^ (k8 & 1);
    }
    // A staged row is released by the commit of output row o_base + max(0,
    // (t - 1) / 2) (t: its index in the run; the MMA issues an odd row's ky = 0
    // pass before the ky = 2 pass that completes the previous output row);
    // the group remembers, per slot it owns, the release of the occupant.
    constexpr int kOwn = kNR / kGroups;
    int rel[kOwn];
#pragma unroll
    for (int q = 0; q < kOwn; ++q) rel[q] = -1;
    long long j = 0;
    int o_base = 0;
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
        const int own = (int)((j / kGroups) % kOwn);
        int prev = rel[0];
#pragma unroll
        for (int q = 1; q < kOwn; ++q)
          if (own == q) prev = rel[q];
        const int t = r - (2 * runs.ya - 1);
        const int cn = o_base + (t >= 1 ? (t - 1) / 2 : 0);
#pragma unroll
        for (int q = 0; q < kOwn; ++q)
          if (own == q) rel[q] = cn;
        // the slot's previous row has been consumed (its output row's commit)
        auto slot_free = [&]() -> bool {
          return prev < 0 || tc::mbar_wait(&acc_full[prev % kAcc], (uint32_t)((prev / kAcc) & 1), kWaitLimit);
        };
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
            // the map's last read: evict-first
            v[u] = ok ? __ldcs(reinterpret_cast<const uint4*>(a.in + (rowbase + ix) * CIN + kc * 8))
                      : make_uint4(0, 0, 0, 0);
          }
          if (!slot_free()) {
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
        } else if (SRC == 2) {
          // convert the TMA-staged raw rows: staged column jj (half-resolution
          // column c0 + jj) of frame fr reads raw samples 2jj + 6, 2jj + 7 of
          // the frame's two rows in the slot
          const int s = (int)(j % kRRm);
          if (!tc::mbar_wait(&raw_full[s], (uint32_t)((j / kRRm) & 1), kWaitLimit) ||
              !slot_free()) {
            raise_abort(abort_flag, a.status);
            stop = true;
            break;
          }
          const uint8_t* raw = sRaw + s * kRawSlot;
          const int jlo = -c0, jhi = a.Wi - c0;  // staged columns inside the map: [jlo, jhi)
#pragma unroll
          for (int k = 0; k < 2; ++k) {
            const int fr = cv_fr[k], g = cv_g[k];
            const uint8_t* p0 = raw + fr * kRawBoxStep + 16 * g + 16;
            uint4 ra = make_uint4(0, 0, 0, 0), rb = make_uint4(0, 0, 0, 0);
            if (row_ok) {
              ra = *reinterpret_cast<const uint4*>(p0);
              rb = *reinterpret_cast<const uint4*>(p0 + kRawRowBytes);
            }
            const uint32_t wa[4] = {ra.x, ra.y, ra.z, ra.w}, wb[4] = {rb.x, rb.y, rb.z, rb.w};
#pragma unroll
            for (int t = 0; t < 4; ++t) {
              const int jj = 4 * g + 1 + t;
              uint4 val = make_uint4(0, 0, 0, 0);
              if (row_ok && jj >= jlo && jj < jhi)  // outside the map: zero operands (not v = 0)
                val = make_uint4(tf32_sample12(wa[t] & 0xFFFFu), tf32_sample12(wa[t] >> 16),
                                 tf32_sample12(wb[t] & 0xFFFFu), tf32_sample12(wb[t] >> 16));
              *reinterpret_cast<uint4*>(dst + (((jj & 1) * KC + fr) * kNP + (jj >> 1)) * 16) = val;
            }
          }
          if (gtid < 2) {  // column 0 of frame gtid: raw samples 6, 7
            const int fr = gtid;
            uint4 val = make_uint4(0, 0, 0, 0);
            if (row_ok && 0 >= jlo && 0 < jhi) {
              const uint8_t* p0 = raw + fr * kRawBoxStep + 12;
              const uint32_t w0 = *reinterpret_cast<const uint32_t*>(p0);
              const uint32_t w1 = *reinterpret_cast<const uint32_t*>(p0 + kRawRowBytes);
              val = make_uint4(tf32_sample12(w0 & 0xFFFFu), tf32_sample12(w0 >> 16), tf32_sample12(w1 & 0xFFFFu),
                               tf32_sample12(w1 >> 16));
            }
            *reinterpret_cast<uint4*>(dst + (fr * kNP) * 16) = val;
          }
          tc::fence_proxy_async();
          tc::mbar_arrive(&full[slot]);
          tc::mbar_arrive(&raw_empty[s]);
          continue;
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
          if (!slot_free()) {
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
                val = make_uint4(tf32_sample12(w0[t] & 0xFFFFu), tf32_sample12(w0[t] >> 16),
                                 tf32_sample12(w1[t] & 0xFFFFu), tf32_sample12(w1[t] >> 16));
              *reinterpret_cast<uint4*>(dst + (((jj & 1) * KC + fr) * kNP + (jj >> 1)) * 16) = val;
            }
          }
        } else {
          // unaligned frames: one 2-byte load per plane sample, item by item
          // once the slot is free (the rare path)
          if (!slot_free()) {
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
              wd[c] = ok ? tf32_sample12(__ldg(fb + (long long)(2 * r + (pl >> 1)) * a.fr.pitch + 2 * ix + (pl & 1)))
                         : 0u;
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
      o_base += runs.yb - runs.ya;
    }
  } else if (warp == R::MMA) {
    // ---- MMA issue: one thread
    if (lane == 0) {
      // Descriptors: the start-address field (bits 0-13, address / 16) is the
      // only part that varies, so each MMA adds a 16-byte offset to a base
      // descriptor (shared addresses < 256 KB: no carry out of the field).
      const uint64_t a_base = tc::smem_desc(tc::smem_addr(sX), kNP * 16, 128);
      const uint64_t b_base = tc::smem_desc(tc::smem_addr(sB), 128, 9 * KC * 128);
      // layer 1: TF32 operands, K = 8 = the 4 planes of both frames per tap
      constexpr uint32_t idesc = SRC != 0 ? tc::idesc_tf32_f32(kM, kN) : tc::idesc_bf16_f32(kM, kN);
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
          const uint64_t a_row = a_base + (uint64_t)(slot * (L::SLOT_BYTES / 16));
          // odd rows: ky = 0 (starts output row (r+1)/2), then ky = 2 (finishes
          // row (r-1)/2); even rows: ky = 1 of row r/2
#pragma unroll
          for (int pass = 0; pass < 2; ++pass) {
            int ky, y;
            if (r & 1) {
              // ky = 0 (starts row (r+1)/2) first, so that the commit after the
              // ky = 2 pass (finishing row (r-1)/2) covers the whole staged row
              ky = pass == 0 ? 0 : 2;
              y = pass == 0 ? (r + 1) >> 1 : (r - 1) >> 1;
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
            const uint64_t b_ky = b_base + (uint64_t)(ky * 3 * KC * 8);
#pragma unroll
            for (int kx = 0; kx < 3; ++kx) {
#pragma unroll
              for (int s2 = 0; s2 < CIN / 16; ++s2) {
                const uint64_t ad = a_row + (uint64_t)(((kx & 1) * KC + 2 * s2) * kNP + (kx >> 1));
                const uint64_t bd = b_ky + (uint64_t)((kx * KC + 2 * s2) * 8);
                if (SRC != 0)
                  tc::mma_tf32(d, ad, bd, idesc, (ky == 0 && kx == 0 && s2 == 0) ? 0u : 1u);
                else
                  tc::mma_bf16(d, ad, bd, idesc, (ky == 0 && kx == 0 && s2 == 0) ? 0u : 1u);
              }
            }
            // last contribution to output row y: its accumulator is complete and
            // every staged row up to this one consumed (the producers' release)
            if (ky == 2) tc::commit(&acc_full[acc]);
          }
          if (stop) break;
        }
        o += runs.yb - runs.ya;
      }
      tc::commit(mma_done);
      if (!tc::mbar_wait(mma_done, 0, kWaitLimit)) raise_abort(abort_flag, a.status);
    }
    __syncwarp();
  } else {
    // ---- epilogue: thread = pixel of the segment = TMEM lane (warp w reads
    // lanes 32w .. 32w + 31)
    const int quarter = warp;
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
        tc::tmem_ld32(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(acc * kN), v);
        tc::fence_before_sync();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&acc_empty[acc]);  // accumulator drained
#pragma unroll
        for (int q4 = 0; q4 < 8; ++q4) {
          const float4 b4 = *reinterpret_cast<const float4*>(sBias + 4 * q4);
          v[4 * q4] += b4.x;
          v[4 * q4 + 1] += b4.y;
          v[4 * q4 + 2] += b4.z;
          v[4 * q4 + 3] += b4.w;
        }
        // the warp's 32 pixels x 64 bytes are one contiguous NHWC run: each
        // lane puts its pixel's 64 bytes into the transpose buffer, then the
        // warp stores the run as four 512-byte rows of 16 bytes per lane
        uint32_t* tb = sTr + quarter * (32 * kTP);
#pragma unroll
        for (int q4 = 0; q4 < 4; ++q4)
          *reinterpret_cast<uint4*>(tb + lane * kTP + 4 * q4) =
              make_uint4(tc::bf2_relu(v[8 * q4], v[8 * q4 + 1]), tc::bf2_relu(v[8 * q4 + 2], v[8 * q4 + 3]),
                         tc::bf2_relu(v[8 * q4 + 4], v[8 * q4 + 5]), tc::bf2_relu(v[8 * q4 + 6], v[8 * q4 + 7]));
        __syncwarp();
        const int px0 = runs.seg * kM + quarter * 32;  // the warp's first pixel
        const long long obase = ((long long)runs.b * a.Ho + y) * a.Wo + px0;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int p = 8 * q + (lane >> 2), piece = lane & 3;
          const uint4 val = *reinterpret_cast<const uint4*>(tb + p * kTP + 4 * piece);
          // evict-first: the next layer reads the map once; the frames, which the
          // refine and fallback searches read after the network, stay in L2
          if (px0 + p < a.Wo) __stcs(reinterpret_cast<uint4*>(a.out + (obase + p) * kN) + piece, val);
        }
        __syncwarp();  // the buffer is rewritten by the next row
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
cudaError_t launch_s2(const ConvTcArgs& a, const CUtensorMap& tm_ref, const CUtensorMap& tm_cur, cudaStream_t st) {
  using L = S2Layout<CIN, SRC>;
  auto kern = conv3x3s2_rows_tc_kernel<CIN, SRC>;
  constexpr int kThreads = threads_of<SRC>();
  const long long T = (long long)a.batch * ((a.Wo + kM - 1) / kM) * a.Ho;
  if (T < 1) return cudaSuccess;
  int dev = 0, nsm = 148;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int per_sm = tc::ctas_per_sm(kern, kThreads, L::SMEM, kTmemCols);
  long long grid = (long long)nsm * per_sm;
  // at least ~4 output rows per CTA keep the ring and the accumulators busy
  if (grid > (T + 3) / 4) grid = (T + 3) / 4;
  if (grid < 1) grid = 1;
  return tc::launch_dependent(kern, dim3((unsigned)grid), dim3(kThreads), L::SMEM, st, a, tm_ref, tm_cur);
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
  if ((e = configure_s2<16, 2>()) != cudaSuccess) return e;
  return configure_s2<32, 0>();
}

cudaError_t launch_conv_s2_rows_tc(const ConvTcArgs& a, int layer, cudaStream_t st) {
  CUtensorMap tm_ref{}, tm_cur{};
  if (layer == 1) {
    // TMA raw rows where the frames' layout allows it (16-byte aligned rows
    // and batch strides), else the producers' own loads
    if (a.vec &&
        tma::encode_u16_frame_chunks(&tm_ref, a.fr.ref, a.fr.W, a.fr.H, a.batch, a.fr.pitch, a.fr.ref_bs, kRawChunks,
                                     2) &&
        tma::encode_u16_frame_chunks(&tm_cur, a.fr.cur, a.fr.W, a.fr.H, a.batch, a.fr.pitch, a.fr.cur_bs, kRawChunks,
                                     2))
      return launch_s2<16, 2>(a, tm_ref, tm_cur, st);
    return launch_s2<16, 1>(a, tm_ref, tm_cur, st);
  }
  if (layer == 2) return launch_s2<32, 0>(a, tm_ref, tm_cur, st);
  return cudaErrorInvalidValue;
}

}  // namespace bme

// Launchers of the device kernels (called by the C ABI in api.cu).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/bayer_me.h"

namespace bme {

// Exhaustive EVEN search, block 16, radius R = range/2 steps of 2, zero
// centre, W and H multiples of 16.  Specialised for range 8, 16, 24, 32; the
// caller checks full16_even_supported and otherwise uses the generic kernel.
bool full16_even_supported(int range);
cudaError_t configure_full16();  // once per device: shared-memory opt-in
cudaError_t launch_full16_even(const uint16_t* ref, const uint16_t* cur, int W, int H, int pitch, long long ref_bs,
                               long long cur_bs, int batch, int range, bayer_mv_t* out, cudaStream_t st);

// Generic matching kernel: one CTA per block, up to BAYER_MAX_STAGES stages
// run in order, each centred on the previous stage's best.
struct GenericArgs {
  const uint16_t* ref;
  const uint16_t* cur;
  int W, H, pitch;
  long long ref_bs, cur_bs;  // batch strides (elements)
  int B, h, w;               // block size and field shape
  int nst;
  int R[BAYER_MAX_STAGES];
  int S[BAYER_MAX_STAGES];
  int lim;                   // |dx|, |dy| limit
  int center_mode;           // 0 zero, 1 parent field, 2 seeded proposal
  const bayer_mv_t* parent;  // center_mode 1: previous level's field
  int parent_B, parent_h, parent_w;
  const float* prop;         // center_mode 2: [batch][h][w][2]
  const float* conf;         // center_mode 2: [batch][h][w]
  float thresh;
  int range;                 // center_mode 2: full-search range and clamp
  uint8_t* fallback;         // center_mode 2: optional flags
  bayer_mv_t* out;
};
cudaError_t launch_generic(const GenericArgs& a, int batch, cudaStream_t st);

// Propagation z_pred = Warp(z_R, MV).
struct PropArgs {
  const float* feat;
  float* out;
  int n, C, Hf, Wf;
  const bayer_mv_t* mv;
  int mv_h, mv_w;
  int cells;  // feature cells per block side = block / stride
  int s;      // stride
};
cudaError_t launch_propagate(const PropArgs& a, int layout, int interp, cudaStream_t st);

// Roofline probe of the SAD primitive.
cudaError_t run_probe_alu(int variant, double* pc_per_clk_per_sm, double* sm_mhz, int* sm_count);

}  // namespace bme

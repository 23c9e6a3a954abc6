// Launchers of the device kernels (called by the C ABI in api.cu).
#pragma once

#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "../../include/bayer_me.h"

namespace bme {

// Exhaustive EVEN search, block 16, radius R = range/2 steps of 2, zero
// centre, W a multiple of 16 (any even H >= 16: a last block row that the
// frame clips is searched over its rows inside the frame).  Specialised for
// range 8, 16, 24, 32; the caller checks full16_even_supported and otherwise
// uses another kernel.
bool full16_even_supported(int range);
cudaError_t configure_full16();  // once per device: shared-memory opt-in
// status: device word that receives BAYER_ERR_TIMEOUT if the TMA staging's
// bounded wait expires.
cudaError_t launch_full16_even(const uint16_t* ref, const uint16_t* cur, int W, int H, int pitch, long long ref_bs,
                               long long cur_bs, int batch, int range, bayer_mv_t* out, int* status, cudaStream_t st);

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
// One C2F level on packed pixel pairs (me_c2f.cu): EVEN steps 2/4/8, whole
// 32- or 64-pixel blocks, 16-byte aligned frames; cudaErrorNotSupported when
// the level falls outside that (the caller runs launch_generic).
cudaError_t launch_c2f_level(const GenericArgs& a, int batch, cudaStream_t st);

// Propagation z_pred = Warp(z_R, MV).
struct PropArgs {
  const float* feat;
  float* out;
  int n, C, Hf, Wf;
  const bayer_mv_t* mv;
  int mv_h, mv_w;
  int cells;  // feature cells per block side = block / stride
  int s;      // stride (a power of two dividing the block size)
  int ls, lc;  // log2(s), log2(cells): filled in by launch_propagate
  int* status = nullptr;  // device status word: BAYER_ERR_TIMEOUT if a bounded wait expired
};
cudaError_t launch_propagate(const PropArgs& a, int layout, int interp, cudaStream_t st);

// Learned proposal network (cnn.cu).
struct CnnFrames {
  const uint16_t* ref;
  const uint16_t* cur;
  int W, H, pitch;
  long long ref_bs, cur_bs;
};
struct CnnShapes {
  int H[5], W[5];  // [0] half-resolution input, [1..4] layer outputs
};
CnnShapes cnn_shapes(int W, int H);
size_t cnn_act_bytes(int W, int H, int batch);   // bf16 activations of layers 1..4 + packed weights
size_t cnn_grad_bytes(int W, int H, int batch);  // bf16 pre-activation gradients of layers 1..4
// zero_words (optional): two ints the forward's first launch sets to 0 (the
// fallback lists' counters of a learned search, so that no separate memset
// sits between the previous kernel and the network).
cudaError_t cnn_forward(const CnnFrames& fr, int batch, const uint16_t* wbf16, int range, void* acts, float* prop,
                        float* conf, int* status, cudaStream_t st, int* zero_words = nullptr);
cudaError_t cnn_loss_grad(const CnnFrames& fr, int batch, const uint16_t* wbf16, const bayer_mv_t* labels, int range,
                          float neg_weight, void* acts, void* dpre, float* grad, float* loss, int* status,
                          cudaStream_t st);

// 3x3 stride-2 convolutions, 32 output channels, on the tensor cores: the
// proposal network's layers.  NHWC bf16 in (layer 1: the Bayer frames), bias +
// ReLU, NHWC bf16 out, or (head fused, layer 4) the 1x1 head straight to the
// per-block proposals and confidences.  Layers 1 and 2 stream rows
// (conv_s2_tc.cu: launch_conv_s2_rows_tc); layers 3 and 4 work in tiles
// (conv_tc.cu: launch_conv_tc, which also packs the weights of all four).
struct ConvTcArgs {
  const __nv_bfloat16* in;  // layers 2..4: [batch][Hi][Wi][32] bf16
  CnnFrames fr;             // layer 1: frames; Hi, Wi are the half-resolution dims
  bool vec;                 // layer 1: 16-byte frame loads allowed (aligned rows, Wi % 4 == 0)
  int Hi, Wi;
  const uint4* wimg;          // weights packed by pack_conv_tc_weights
  const __nv_bfloat16* bias;  // [32]
  __nv_bfloat16* out;         // [batch][Ho][Wo][32] bf16 (no head)
  const __nv_bfloat16* whead;  // head: [12][32] weights then [12] biases
  float* prop;                 // head: [batch][2Ho][2Wo][2]
  float* conf;                 // head: [batch][2Ho][2Wo]
  int range;                   // head: proposal scale
  int Ho, Wo, batch;
  int* status;  // device status word: BAYER_ERR_TIMEOUT if a bounded wait expired
};
cudaError_t configure_conv_tc();
// Packed weight image of one layer in bytes: cin_op = 32 for layers 2..4, 16
// for layer 1 (whose TF32 image of 8 planes has the same 9216 bytes).  pack_conv_tc_weights builds all four layers'
// images in one launch: layer l from the [32][cin][3][3] bf16 block at
// w + w_off[l], written at byte img_off[l] (256-byte aligned) of img;
// zero_word (optional) is set to 0 by the same launch.
size_t conv_tc_weight_bytes(int cin_op);
cudaError_t pack_conv_tc_weights(const uint16_t* w, const int* w_off, const size_t* img_off, uint16_t* img,
                                 int* zero_word, cudaStream_t st);
cudaError_t launch_conv_tc(const ConvTcArgs& a, int layer, bool head, cudaStream_t st);  // layers 3, 4
// Inference: layers 3 and 4 and the head in one kernel (the layer-3 map stays
// in shared memory); l3 describes layer 3 (and carries the head's fields),
// wimg4 / bias4 layer 4.  Layer-3 rows of at most 128 pixels.
bool conv34_head_supported(int W3);
cudaError_t launch_conv34_head_tc(const ConvTcArgs& l3, const uint4* wimg4, const __nv_bfloat16* bias4, int H4, int W4,
                                  cudaStream_t st);
cudaError_t configure_conv_s2_rows_tc();
cudaError_t launch_conv_s2_rows_tc(const ConvTcArgs& a, int layer, cudaStream_t st);

// Backward of those convolutions on the tensor cores (conv_bwd_tc.cu): the
// input gradient of layers 2..4 masked by the layer below's ReLU (bf16 out),
// and the weight and bias gradients of all four layers (added to gw, gb).
struct ConvBwdArgs {
  const __nv_bfloat16* dout;  // [batch][Ho][Wo][32] bf16 pre-activation gradient of this layer
  int Ho, Wo;
  const __nv_bfloat16* xin;   // layers 2..4: [batch][Hi][Wi][32] bf16 input activation
  CnnFrames fr;               // layer 1 (weight gradient): frames; Hi, Wi the half-resolution dims
  bool vec;                   // layer 1: 4-byte frame loads allowed (even pitch, 4-byte aligned rows)
  int Hi, Wi, batch;
  const uint4* wimg_t;        // input gradient: this layer's transposed weight image
  __nv_bfloat16* din;         // input gradient: [batch][Hi][Wi][32] bf16 out
  float* gw;                  // weight gradient: [32][cin][3][3], accumulated
  float* gb;                  // bias gradient: [32], accumulated
  bool vec_atomics;           // gw 16-byte aligned: float4 atomics
  int* status;                // device status word: BAYER_ERR_TIMEOUT if a bounded wait expired
};
cudaError_t configure_conv_bwd_tc();
// Transposed weight images of layers 2..4 (the [32][32][3][3] bf16 blocks at
// w + w_off[0..2]) for the input gradient, written to img (16-byte aligned).
size_t conv_dx_weight_bytes();
cudaError_t pack_conv_dx_weights(const uint16_t* w, const int* w_off, uint16_t* img, cudaStream_t st);
cudaError_t launch_conv_dx_tc(const ConvBwdArgs& a, cudaStream_t st);
cudaError_t launch_conv_dw_tc(const ConvBwdArgs& a, bool frames, cudaStream_t st);

// 3x3 stride-1 convolution streamed row by row on the tensor cores
// (conv_rows_tc.cu): NHWC input (bf16, or float32 rounded to bf16 when
// staged), weights pre-packed by pack_conv_rows_weights into the kernel's
// shared-memory image, float32 bias, bf16 or float32 NHWC output.
struct ConvRowsArgs {
  const __nv_bfloat16* in;  // src 0: [batch][H][W][cin] bf16
  const float* in_f32;      // src 2: [batch][H][W][cin] float32
  int H, W, batch;
  const uint4* wimg;  // packed bf16 weights, conv_rows_weight_bytes(cin, cout) bytes, 16-byte aligned
  const float* bias;  // [cout]
  __nv_bfloat16* out;  // outf 0: [batch][H][W][cout] bf16
  float* out_f32;      // outf 1: [batch][H][W][cout] float32
  int* status;         // device status word: BAYER_ERR_TIMEOUT if a bounded wait expired
};
cudaError_t configure_conv_rows_tc();
size_t conv_rows_weight_bytes(int cin, int cout);
cudaError_t pack_conv_rows_weights(const float* w, int cout, int cin, uint16_t* img, cudaStream_t st);
cudaError_t launch_conv_rows_tc(const ConvRowsArgs& a, int cin, int cout, int src, int outf, bool relu,
                                cudaStream_t st);

// 3x3 stride-1 convolution in float32 on the SIMT cores (refine_f32.cu):
// NHWC float32 in and out, bias, optional ReLU.
cudaError_t launch_conv3x3_f32(const float* in, int batch, int H, int W, int cin, const float* w, const float* bias,
                               int cout, bool relu, float* out, cudaStream_t st);
cudaError_t cnn_adamw(float* w, uint16_t* wbf16, const float* g, float* m, float* v, int n, int step, float lr,
                      float b1, float b2, float eps, float wd, cudaStream_t st);
cudaError_t cnn_to_bf16(const float* w, uint16_t* wbf16, int n, cudaStream_t st);

// Seeded +-4 refine of 16x16 blocks (warp per block) with a compacted list of
// the low-confidence blocks, and the exhaustive search of a block list.
struct Seeded16Args {
  const uint16_t* ref;
  const uint16_t* cur;
  int W, H, pitch;
  long long ref_bs, cur_bs;
  int h, w, batch;
  const float* prop;  // [batch][h][w][2]
  const float* conf;  // [batch][h][w]
  float thresh;
  int range;
  bayer_mv_t* out;
  uint8_t* fallback;  // optional
  int* list;          // [batch*h*w] global block indices needing the full search
  int* count;         // number of entries in list (zeroed by the caller)
  int* list2;         // H % 16 != 0: the entries of list in the clipped last block row, again
  int* count2;        // number of entries in list2 (zeroed by the caller)
  bool vec2;          // set by launch_seeded16: 32-bit sample-pair loads allowed
  bool vec16;         // set by launch_seeded16: 16-byte loads of frame rows allowed
};
cudaError_t configure_seeded16();  // once per device: shared-memory opt-in
cudaError_t launch_seeded16(const Seeded16Args& a, cudaStream_t st);
// clip: the list holds blocks of a last block row clipped by the frame
// (H % 16 != 0), searched over their rows in the frame; without it every
// block is searched as 16 rows (the rows below the frame read as zeros).
cudaError_t launch_full16_list(const uint16_t* ref, const uint16_t* cur, int W, int H, int pitch, long long ref_bs,
                               long long cur_bs, int batch, int h, int w, int range, const int* list, const int* count,
                               int max_count, bool clip, bayer_mv_t* out, int* status, cudaStream_t st);
cudaError_t configure_full16_list();

// Multi-stream search + propagation (multistream.cu); status: the handle's
// device status word, where a propagation wait that expires records
// BAYER_ERR_TIMEOUT.
struct MultiStream;
MultiStream* ms_create(int device, int* status);
void ms_destroy(MultiStream* m);
cudaError_t configure_multistream();
// force: a schedule code to run instead of the autotuned one (0: autotune).
bool ms_schedule_valid(int code);
cudaError_t ms_run(MultiStream* m, const bayer_pair_t* pairs, int n, int range, int interp, long long* end_ns,
                   int force, cudaStream_t st);
int ms_config_nw(MultiStream* m, const bayer_pair_t* pairs, int n, int range, int interp, int force);

// Self-test of the bounded mbarrier wait (tc_common.cuh) every tcgen05 kernel
// uses: BAYER_ERR_TIMEOUT lands in *status when nothing arrives.
cudaError_t launch_wait_selftest(int* status, bool arrive, unsigned limit, cudaStream_t st);

// Roofline probe of the SAD primitive.
cudaError_t run_probe_alu(int variant, double* pc_per_clk_per_sm, double* sm_mhz, int* sm_count);

}  // namespace bme

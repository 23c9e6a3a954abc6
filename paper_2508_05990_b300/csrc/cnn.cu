// Learned MV proposal network: forward, loss gradient and AdamW (BF16
// weights and activations, FP32 accumulation).  Not in the paper: it seeds the
// +-4 refine of the learned-seeded search.  Training follows the paper's
// recipe for its learned module (AdamW, cosine schedule; Sec. 4.1 "Training
// Details") and its BerHu loss (Sec. 3.3).
//
// Network (flat parameter order = BAYER_CNN_* offsets in bayer_me.h):
//   x0 = the four RGGB planes of ref and cur at half resolution, v/2048 - 1
//   x_l = ReLU(conv3x3(x_{l-1}, stride 2, pad 1) + b_l), 32 channels, l = 1..4
//   z = 1x1 conv (32 -> 12) + b_h; channel 3*(2*sy + sx) + q of L4 cell (i, k)
//       is quantity q of block (2i + sy, 2k + sx)
//   dx = range*tanh(z_0), dy = range*tanh(z_1), conf = sigmoid(z_2)
// Activations are NHWC bf16 [B][H][W][32].  The four convolutions run on the
// tensor cores (conv_s2_tc.cu, conv_tc.cu; layer 1 gathers the Bayer frames
// directly, the packing fused into its operand staging; in inference layers
// 3, 4 and the head run as one kernel, the layer-3 map kept in shared memory,
// where its rows fit one tile), and so do the convolutions' input and
// weight gradients (conv_bwd_tc.cu), on bf16 pre-activation gradients; the
// training head and loss are SIMT (one thread per layer-4 cell).
// Loss per block:
//   BerHu_4(dx - dx*) + BerHu_4(dy - dy*) - t log(conf) - w_neg (1 - t) log(1 - conf),
//   t = [round_even(dx) within +-4 of dx* and likewise for dy],
// averaged over all blocks of the batch.
#include <cuda_bf16.h>

#include "common.cuh"
#include "kernels.cuh"
#include "tc_common.cuh"

namespace bme {

namespace {

constexpr int kC = 32;

__device__ __forceinline__ float bf(const __nv_bfloat16 v) { return __bfloat162float(v); }

// 8 bf16 packed in a uint4 -> 8 floats
__device__ __forceinline__ void unpack8(const uint4 u, float* f) {
  const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    f[2 * i] = __uint_as_float(w[i] << 16);
    f[2 * i + 1] = __uint_as_float(w[i] & 0xFFFF0000u);
  }
}

// ---------------------------------------------------------------------------
// training: loss and gradients
// ---------------------------------------------------------------------------

__device__ __forceinline__ float round_even(float v) { return 2.0f * roundf(v * 0.5f); }
__device__ __forceinline__ float berhu(float e) {
  const float a = fabsf(e);
  return a <= 4.0f ? a : (e * e + 16.0f) * 0.125f;
}
__device__ __forceinline__ float berhu_grad(float e) {
  return fabsf(e) <= 4.0f ? (e > 0.f ? 1.f : (e < 0.f ? -1.f : 0.f)) : e * 0.25f;
}

// Head forward + loss + head backward.  One thread per L4 cell, 128 cells per
// CTA.  Writes dpre4 = dL/d(L4 pre-activation) (bf16 NHWC, rounded to nearest
// even); the CTA's cells stage their dL/dz and activations in shared memory,
// then thread t sums the head-weight gradients t, t + 128, t + 256 (and t <
// 12 a head-bias gradient) over the 128 cells and adds them to grad once, so
// that grad receives one atomic per parameter per CTA.  The loss sum goes to
// *loss.  Both already scaled by 1/n.
constexpr int kHeadCells = 128;

__global__ void __launch_bounds__(kHeadCells) head_loss_bwd_kernel(const __nv_bfloat16* __restrict__ x4, int H4,
                                                                   int W4, const __nv_bfloat16* __restrict__ w,
                                                                   int range, const bayer_mv_t* __restrict__ labels,
                                                                   float inv_n, float neg_w,
                                                                   __nv_bfloat16* __restrict__ dpre4,
                                                                   float* __restrict__ grad,
                                                                   float* __restrict__ loss) {
  __shared__ float wh[12 * kC + 12];
  __shared__ float sdz[kHeadCells][13];
  __shared__ float sx[kHeadCells][kC + 1];
  __shared__ float lsum[kHeadCells / 32];
  for (int i = threadIdx.x; i < 12 * kC + 12; i += blockDim.x) wh[i] = bf(w[BAYER_CNN_WH + i]);
  __syncthreads();
  const int cells = H4 * W4;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int b = blockIdx.y;
  float x[kC], dz[12];
  float l = 0.f;
#pragma unroll
  for (int c = 0; c < kC; ++c) x[c] = 0.f;
#pragma unroll
  for (int j = 0; j < 12; ++j) dz[j] = 0.f;
  if (t < cells) {
    const int i = t / W4, k = t - i * W4;
    const uint4* src = reinterpret_cast<const uint4*>(x4 + ((long long)b * cells + t) * kC);
#pragma unroll
    for (int q = 0; q < 4; ++q) unpack8(__ldg(src + q), x + 8 * q);
    const int h = 2 * H4, wb = 2 * W4;
#pragma unroll 1  // unrolled, the four blocks' live ranges spill
    for (int s = 0; s < 4; ++s) {
      float z[3];
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const int j = 3 * s + q;
        float a = wh[12 * kC + j];
#pragma unroll
        for (int c = 0; c < kC; ++c) a = fmaf(wh[j * kC + c], x[c], a);
        z[q] = a;
      }
      const long long blk = ((long long)b * h + 2 * i + (s >> 1)) * wb + 2 * k + (s & 1);
      const bayer_mv_t lab = labels[blk];
      const float tx = tanhf(z[0]), ty = tanhf(z[1]);
      const float dx = (float)range * tx, dy = (float)range * ty;
      const float cf = 1.0f / (1.0f + expf(-z[2]));
      const float ex = dx - (float)lab.dx, ey = dy - (float)lab.dy;
      const float tgt = (fabsf(round_even(dx) - (float)lab.dx) <= 4.f && fabsf(round_even(dy) - (float)lab.dy) <= 4.f)
                            ? 1.f : 0.f;
      l += berhu(ex) + berhu(ey) - (tgt * logf(cf + 1e-12f) + neg_w * (1.f - tgt) * logf(1.f - cf + 1e-12f));
      dz[3 * s + 0] = berhu_grad(ex) * (float)range * (1.f - tx * tx) * inv_n;
      dz[3 * s + 1] = berhu_grad(ey) * (float)range * (1.f - ty * ty) * inv_n;
      dz[3 * s + 2] = (cf * (tgt + neg_w * (1.f - tgt)) - tgt) * inv_n;
    }
    // d x4, masked by ReLU (x4 > 0 iff its pre-activation > 0)
    float d[kC];
#pragma unroll
    for (int c = 0; c < kC; ++c) {
      float a = 0.f;
#pragma unroll
      for (int j = 0; j < 12; ++j) a = fmaf(wh[j * kC + c], dz[j], a);
      d[c] = x[c] > 0.f ? a : 0.f;
    }
    uint4* dst = reinterpret_cast<uint4*>(dpre4 + ((long long)b * cells + t) * kC);
#pragma unroll
    for (int q = 0; q < 4; ++q)
      dst[q] = make_uint4(tc::bf2(d[8 * q], d[8 * q + 1]), tc::bf2(d[8 * q + 2], d[8 * q + 3]),
                          tc::bf2(d[8 * q + 4], d[8 * q + 5]), tc::bf2(d[8 * q + 6], d[8 * q + 7]));
  }
  const int tl = threadIdx.x;
#pragma unroll
  for (int j = 0; j < 12; ++j) sdz[tl][j] = dz[j];
#pragma unroll
  for (int c = 0; c < kC; ++c) sx[tl][c] = x[c];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
  if ((tl & 31) == 0) lsum[tl >> 5] = l;
  __syncthreads();
  // head weight gradients (j, c) = (g / 32, g % 32): a warp shares j (dL/dz
  // broadcast) and reads 32 consecutive activations
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    const int g = tl + r * kHeadCells, j = g >> 5, c = g & 31;
    float a = 0.f;
    for (int m = 0; m < kHeadCells; ++m) a = fmaf(sdz[m][j], sx[m][c], a);
    atomicAdd(&grad[BAYER_CNN_WH + g], a);
  }
  if (tl < 12) {
    float a = 0.f;
    for (int m = 0; m < kHeadCells; ++m) a += sdz[m][tl];
    atomicAdd(&grad[BAYER_CNN_BH + tl], a);
  }
  if (tl == 0) atomicAdd(loss, (lsum[0] + lsum[1] + lsum[2] + lsum[3]) * inv_n);
}

__global__ void adamw_kernel(float* __restrict__ w, __nv_bfloat16* __restrict__ wb, const float* __restrict__ g,
                             float* __restrict__ m, float* __restrict__ v, int n, float lr, float b1, float b2,
                             float eps, float wd, float bc1, float bc2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float mh = mi / bc1, vh = vi / bc2;
  const float wi = w[i] - lr * (mh / (sqrtf(vh) + eps) + wd * w[i]);
  w[i] = wi;
  wb[i] = __float2bfloat16_rn(wi);
}

__global__ void f32_to_bf16_kernel(const float* __restrict__ a, __nv_bfloat16* __restrict__ b, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = __float2bfloat16_rn(a[i]);
}

inline int conv_out(int n) { return (n - 1) / 2 + 1; }

}  // namespace

CnnShapes cnn_shapes(int W, int H) {
  CnnShapes s;
  s.H[0] = H / 2;
  s.W[0] = W / 2;
  for (int l = 1; l <= 4; ++l) {
    s.H[l] = conv_out(s.H[l - 1]);
    s.W[l] = conv_out(s.W[l - 1]);
  }
  return s;
}

namespace {

size_t act_elems(const CnnShapes& s, int batch) {
  size_t n = 0;
  for (int l = 1; l <= 4; ++l) n += (size_t)s.H[l] * s.W[l] * kC;
  return n * batch;
}

// Workspace: the bf16 activations of layers 1..4, then the packed weight
// images of the four convolutions and the transposed images of layers 2..4
// for the input gradient (256-byte aligned).
size_t wimg_offset(int W, int H, int batch) {
  return (act_elems(cnn_shapes(W, H), batch) * sizeof(__nv_bfloat16) + 255) / 256 * 256;
}

size_t wimg_bytes() {
  size_t n = 0;
  for (int l = 1; l <= 4; ++l) n += (conv_tc_weight_bytes(l == 1 ? 16 : 32) + 255) / 256 * 256;
  return n;
}

size_t wimg_t_offset() { return wimg_bytes(); }

size_t wimg_all_bytes() { return wimg_bytes() + (conv_dx_weight_bytes() + 255) / 256 * 256; }

// Forward through the four convolutions.  head: layer 4's epilogue evaluates
// the head (activations of layer 4 are then not stored); otherwise all four
// layers' activations are written.
cudaError_t cnn_forward_acts(const CnnFrames& fr, int batch, const uint16_t* wbf16, void* acts, int* status, bool head,
                             int range, float* prop, float* conf, cudaStream_t st, int* zero_words = nullptr) {
  const CnnShapes s = cnn_shapes(fr.W, fr.H);
  const __nv_bfloat16* w = reinterpret_cast<const __nv_bfloat16*>(wbf16);
  __nv_bfloat16* a[5];
  a[1] = static_cast<__nv_bfloat16*>(acts);
  for (int l = 2; l <= 4; ++l) a[l] = a[l - 1] + (size_t)batch * s.H[l - 1] * s.W[l - 1] * kC;
  const int woff[5] = {0, BAYER_CNN_W1, BAYER_CNN_W2, BAYER_CNN_W3, BAYER_CNN_W4};
  const int boff[5] = {0, BAYER_CNN_B1, BAYER_CNN_B2, BAYER_CNN_B3, BAYER_CNN_B4};
  char* img = static_cast<char*>(acts) + wimg_offset(fr.W, fr.H, batch);
  const uint4* wimg[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  size_t img_off[4];
  size_t off = 0;
  for (int l = 1; l <= 4; ++l) {
    img_off[l - 1] = off;
    wimg[l] = reinterpret_cast<const uint4*>(img + off);
    off += (conv_tc_weight_bytes(l == 1 ? 16 : 32) + 255) / 256 * 256;
  }
  cudaError_t e0 = pack_conv_tc_weights(wbf16, woff + 1, img_off, reinterpret_cast<uint16_t*>(img), zero_words, st);
  if (e0 != cudaSuccess) return e0;
  const bool vec = (reinterpret_cast<uintptr_t>(fr.ref) % 16) == 0 && (reinterpret_cast<uintptr_t>(fr.cur) % 16) == 0 &&
                   fr.pitch % 8 == 0 && fr.ref_bs % 8 == 0 && fr.cur_bs % 8 == 0 && s.W[0] % 4 == 0;
  for (int l = 1; l <= 4; ++l) {
    ConvTcArgs c{};
    c.in = l == 1 ? nullptr : a[l - 1];
    c.fr = fr;
    c.vec = vec;
    c.Hi = s.H[l - 1];
    c.Wi = s.W[l - 1];
    c.wimg = wimg[l];
    c.bias = w + boff[l];
    c.out = a[l];
    c.Ho = s.H[l];
    c.Wo = s.W[l];
    c.batch = batch;
    c.status = status;
    const bool fuse = head && l == 4;
    if (head && l >= 3) {
      c.whead = w + BAYER_CNN_WH;
      c.prop = prop;
      c.conf = conf;
      c.range = range;
    }
    // inference: layers 3, 4 and the head in one kernel where layer-3 rows fit
    // one tile (the layer-3 map then stays on chip)
    if (head && l == 3 && conv34_head_supported(s.W[3]))
      return launch_conv34_head_tc(c, wimg[4], w + boff[4], s.H[4], s.W[4], st);
    cudaError_t e = l <= 2 ? launch_conv_s2_rows_tc(c, l, st) : launch_conv_tc(c, l, fuse, st);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace

size_t cnn_act_bytes(int W, int H, int batch) { return wimg_offset(W, H, batch) + wimg_all_bytes(); }

size_t cnn_grad_bytes(int W, int H, int batch) {
  return act_elems(cnn_shapes(W, H), batch) * sizeof(__nv_bfloat16);
}

cudaError_t cnn_forward(const CnnFrames& fr, int batch, const uint16_t* wbf16, int range, void* acts, float* prop,
                        float* conf, int* status, cudaStream_t st, int* zero_words) {
  return cnn_forward_acts(fr, batch, wbf16, acts, status, true, range, prop, conf, st, zero_words);
}

cudaError_t cnn_loss_grad(const CnnFrames& fr, int batch, const uint16_t* wbf16, const bayer_mv_t* labels, int range,
                          float neg_weight, void* acts, void* dpre, float* grad, float* loss, int* status,
                          cudaStream_t st) {
  const CnnShapes s = cnn_shapes(fr.W, fr.H);
  cudaError_t e = cnn_forward_acts(fr, batch, wbf16, acts, status, false, range, nullptr, nullptr, st);
  if (e != cudaSuccess) return e;
  const __nv_bfloat16* w = reinterpret_cast<const __nv_bfloat16*>(wbf16);
  const __nv_bfloat16* a[5];
  a[1] = static_cast<const __nv_bfloat16*>(acts);
  for (int l = 2; l <= 4; ++l) a[l] = a[l - 1] + (size_t)batch * s.H[l - 1] * s.W[l - 1] * kC;
  __nv_bfloat16* d[5];
  d[1] = static_cast<__nv_bfloat16*>(dpre);
  for (int l = 2; l <= 4; ++l) d[l] = d[l - 1] + (size_t)batch * s.H[l - 1] * s.W[l - 1] * kC;
  if ((e = cudaMemsetAsync(grad, 0, BAYER_CNN_NPARAMS * sizeof(float), st)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(loss, 0, sizeof(float), st)) != cudaSuccess) return e;
  const float inv_n = 1.0f / ((float)batch * (2 * s.H[4]) * (2 * s.W[4]));
  {
    dim3 g((s.H[4] * s.W[4] + kHeadCells - 1) / kHeadCells, batch);
    head_loss_bwd_kernel<<<g, kHeadCells, 0, st>>>(a[4], s.H[4], s.W[4], w, range, labels, inv_n, neg_weight, d[4], grad,
                                            loss);
  }
  const int woff[5] = {0, BAYER_CNN_W1, BAYER_CNN_W2, BAYER_CNN_W3, BAYER_CNN_W4};
  const int boff[5] = {0, BAYER_CNN_B1, BAYER_CNN_B2, BAYER_CNN_B3, BAYER_CNN_B4};
  char* img_t = static_cast<char*>(acts) + wimg_offset(fr.W, fr.H, batch) + wimg_t_offset();
  if ((e = pack_conv_dx_weights(wbf16, woff + 2, reinterpret_cast<uint16_t*>(img_t), st)) != cudaSuccess) return e;
  const bool vec_atomics = (reinterpret_cast<uintptr_t>(grad) & 15) == 0;
  const bool vec = (reinterpret_cast<uintptr_t>(fr.ref) % 4) == 0 && (reinterpret_cast<uintptr_t>(fr.cur) % 4) == 0 &&
                   fr.pitch % 2 == 0 && fr.ref_bs % 2 == 0 && fr.cur_bs % 2 == 0;
  for (int l = 4; l >= 1; --l) {
    ConvBwdArgs c{};
    c.dout = d[l];
    c.Ho = s.H[l];
    c.Wo = s.W[l];
    c.xin = l > 1 ? a[l - 1] : nullptr;
    c.fr = fr;
    c.vec = vec;
    c.Hi = s.H[l - 1];
    c.Wi = s.W[l - 1];
    c.batch = batch;
    c.gw = grad + woff[l];
    c.gb = grad + boff[l];
    c.vec_atomics = vec_atomics;
    c.status = status;
    if ((e = launch_conv_dw_tc(c, l == 1, st)) != cudaSuccess) return e;
    if (l > 1) {
      c.wimg_t = reinterpret_cast<const uint4*>(img_t + (size_t)(l - 2) * (conv_dx_weight_bytes() / 3));
      c.din = d[l - 1];
      if ((e = launch_conv_dx_tc(c, st)) != cudaSuccess) return e;
    }
  }
  return cudaGetLastError();
}

cudaError_t cnn_adamw(float* w, uint16_t* wbf16, const float* g, float* m, float* v, int n, int step, float lr,
                      float b1, float b2, float eps, float wd, cudaStream_t st) {
  const float bc1 = 1.f - powf(b1, (float)step), bc2 = 1.f - powf(b2, (float)step);
  adamw_kernel<<<(n + 255) / 256, 256, 0, st>>>(w, reinterpret_cast<__nv_bfloat16*>(wbf16), g, m, v, n, lr, b1, b2,
                                                eps, wd, bc1, bc2);
  return cudaGetLastError();
}

cudaError_t cnn_to_bf16(const float* w, uint16_t* wbf16, int n, cudaStream_t st) {
  f32_to_bf16_kernel<<<(n + 255) / 256, 256, 0, st>>>(w, reinterpret_cast<__nv_bfloat16*>(wbf16), n);
  return cudaGetLastError();
}

}  // namespace bme

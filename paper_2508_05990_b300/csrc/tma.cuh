// Tensor-memory-accelerator (TMA) tile loads of uint16 frame stacks and of
// float32 feature planes: the
// host-side tensor map (cuTensorMapEncodeTiled, fetched from the driver
// through the runtime so nothing links libcuda) and the device-side bulk
// tensor copy that completes on an mbarrier.
//
// Rules kept by every caller: the global base is 16-byte aligned, the row
// pitch and the frame stride are multiples of 16 bytes, the box's inner extent
// is a multiple of 16 bytes, and the innermost start coordinate x is a
// multiple of 16 bytes (8 uint16 or 4 float32 elements).  Other coordinates
// may lie outside the frame (loads there read zeros); only loads are issued.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "tc_common.cuh"

namespace bme {
namespace tma {

using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                              const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// cuTensorMapEncodeTiled, looked up once through the runtime (null if missing).
inline EncodeFn encode_fn() {
  static EncodeFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeFn>(p);
  });
  return fn;
}

// A rank-3 map over n frames of H x W uint16 samples (row pitch and frame
// stride in elements), box box_w x box_h x 1, out-of-range samples read as 0.
// Returns false (map unusable) when the driver entry point is missing or the
// layout breaks an alignment rule.
inline bool encode_u16_frames(CUtensorMap* map, const void* base, int W, int H, int n, long long pitch,
                              long long frame_stride, int box_w, int box_h) {
  const EncodeFn fn = encode_fn();
  if (!fn) return false;
  if ((reinterpret_cast<uintptr_t>(base) & 15) || ((pitch * 2) & 15) || ((box_w * 2) & 15)) return false;
  if (n > 1 && (frame_stride <= 0 || ((frame_stride * 2) & 15))) return false;
  if (box_w > 256 || box_h > 256 || box_w < 1 || box_h < 1) return false;
  const long long fstride = n > 1 ? frame_stride : pitch * H;  // unused when n == 1; any valid value
  const cuuint64_t dims[3] = {(cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)n};
  const cuuint64_t strides[2] = {(cuuint64_t)(pitch * 2), (cuuint64_t)(((fstride * 2) + 15) / 16 * 16)};
  const cuuint32_t box[3] = {(cuuint32_t)box_w, (cuuint32_t)box_h, 1};
  const cuuint32_t estride[3] = {1, 1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT16, 3, const_cast<void*>(base), dims, strides, box, estride,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// A rank-4 map over n frames of H x W uint16 samples seen as 16-byte chunks:
// dims (8 samples, W/8 chunks, H rows, n frames), box 8 x box_chunks x box_h x
// 1, so that one copy brings box_h rows of box_chunks * 8 consecutive samples
// (more than the 256 of a box dimension) starting at a 16-byte chunk; chunks
// and rows outside the frame read as 0.  Returns false when the driver entry
// point is missing or the layout breaks an alignment rule (W % 8 == 0 too).
inline bool encode_u16_frame_chunks(CUtensorMap* map, const void* base, int W, int H, int n, long long pitch,
                                    long long frame_stride, int box_chunks, int box_h) {
  const EncodeFn fn = encode_fn();
  if (!fn) return false;
  if ((reinterpret_cast<uintptr_t>(base) & 15) || ((pitch * 2) & 15) || (W & 7)) return false;
  if (n > 1 && (frame_stride <= 0 || ((frame_stride * 2) & 15))) return false;
  if (box_chunks > 256 || box_h > 256 || box_chunks < 1 || box_h < 1) return false;
  const long long fstride = n > 1 ? frame_stride : pitch * H;  // unused when n == 1; any valid value
  const cuuint64_t dims[4] = {8, (cuuint64_t)(W / 8), (cuuint64_t)H, (cuuint64_t)n};
  const cuuint64_t strides[3] = {16, (cuuint64_t)(pitch * 2), (cuuint64_t)(((fstride * 2) + 15) / 16 * 16)};
  const cuuint32_t box[4] = {8, (cuuint32_t)box_chunks, (cuuint32_t)box_h, 1};
  const cuuint32_t estride[4] = {1, 1, 1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT16, 4, const_cast<void*>(base), dims, strides, box, estride,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// A rank-3 map over `planes` contiguous H x W float32 planes (row pitch W,
// plane stride H * W elements), box box_w x box_h x 1, out-of-range elements
// read as 0.  Returns false when the driver entry point is missing or the
// layout breaks an alignment rule (16-byte base, row pitch and plane stride
// multiples of 16 bytes, box_w a multiple of 4).
inline bool encode_f32_planes(CUtensorMap* map, const void* base, int W, int H, long long planes, int box_w,
                              int box_h) {
  const EncodeFn fn = encode_fn();
  if (!fn) return false;
  if ((reinterpret_cast<uintptr_t>(base) & 15) || ((4ll * W) & 15) || ((4ll * W * H) & 15) || (box_w & 3)) return false;
  if (box_w > 256 || box_h > 256 || box_w < 1 || box_h < 1 || planes < 1) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)planes};
  const cuuint64_t strides[2] = {(cuuint64_t)(4ll * W), (cuuint64_t)(4ll * W * H)};
  const cuuint32_t box[3] = {(cuuint32_t)box_w, (cuuint32_t)box_h, 1};
  const cuuint32_t estride[3] = {1, 1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void*>(base), dims, strides, box, estride,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Arrive on `mbar` (one arrival) and add `bytes` to the transaction count the
// current phase waits for.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* mbar, uint32_t bytes) {
  asm volatile("{\n.reg .b64 st;\nmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}\n" ::"r"(
                   tc::smem_addr(mbar)),
               "r"(bytes)
               : "memory");
}

// Before the first copy through a tensor map that lies in global memory
// (written before the launch, by a copy or a store), order the tensor-map
// proxy's reads of its 128 bytes after those writes.
__device__ __forceinline__ void fence_map_acquire(const CUtensorMap* map) {
  asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(reinterpret_cast<uint64_t>(map))
               : "memory");
}

// One box of `map` at (x, y, z) into shared memory at `dst` (128-byte
// aligned); completes `bytes` of the transaction count of `mbar`.
__device__ __forceinline__ void load_3d(void* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* mbar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(tc::smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(tc::smem_addr(mbar))
      : "memory");
}

// One box of a rank-4 `map` at (x, y, z, w) into shared memory at `dst`
// (128-byte aligned); completes its bytes on `mbar`.
__device__ __forceinline__ void load_4d(void* dst, const CUtensorMap* map, int x, int y, int z, int w, uint64_t* mbar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
      "[%6];" ::"r"(tc::smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(w), "r"(tc::smem_addr(mbar))
      : "memory");
}

}  // namespace tma
}  // namespace bme

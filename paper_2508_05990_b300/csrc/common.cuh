// Device-side helpers shared by the motion-estimation and propagation kernels.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/bayer_me.h"

namespace bme {

// Pixel word in shared memory: the bit pattern of the float 2^23 + v for a
// 12-bit sample v (0x4B000000 | v).  As an integer, |a - b| of two such words
// equals |v_a - v_b|, so sad.u32 works on it directly; as a float, the
// difference of two words is exact too.  One copy serves both pipes.
__device__ __forceinline__ uint32_t pix_word(uint32_t v) { return 0x4B000000u | v; }

// Pixel words of the low / high 16-bit sample of a 32-bit word (one byte
// permute each: bytes [v.b0, v.b1, 0x00, 0x4B] and [v.b2, v.b3, 0x00, 0x4B]).
__device__ __forceinline__ uint32_t pix_lo(uint32_t two) { return __byte_perm(two, 0x4B000000u, 0x7610); }
__device__ __forceinline__ uint32_t pix_hi(uint32_t two) { return __byte_perm(two, 0x4B000000u, 0x7632); }

// |a - b| + c on the integer pipe (PTX sad.u32).
__device__ __forceinline__ uint32_t sad_u32(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t d;
  asm("sad.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
  return d;
}

// Packed pixel pairs (two 16-bit samples in one 32-bit word, as they lie in
// the frame).  min.u16x2: the minimum of each half (one instruction, sm_90+).
__device__ __forceinline__ uint32_t min_u16x2(uint32_t a, uint32_t b) {
  uint32_t d;
  asm("min.u16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
  return d;
}

// c + a.lo * w.byte0 + a.hi * w.byte1 (PTX dp2a.lo, unsigned): with byte
// weights (1, 1) the sum of both halves, with (2, 2) twice that.
__device__ __forceinline__ uint32_t dp2a_lo(uint32_t a, uint32_t w, uint32_t c) {
  uint32_t d;
  asm("dp2a.lo.u32.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(w), "r"(c));
  return d;
}

// Candidate key: lexicographic (sad, |dx|+|dy|, dy, dx) as one uint64 so that
// the tie-break is a plain unsigned minimum.  |dx|, |dy| <= 511.
constexpr uint64_t kInvalidKey = ~0ull;

__device__ __forceinline__ uint64_t make_key(uint32_t sad, int dx, int dy) {
  uint32_t l1 = (uint32_t)(abs(dx) + abs(dy));
  uint32_t tie = (l1 << 20) | ((uint32_t)(dy + 511) << 10) | (uint32_t)(dx + 511);
  return ((uint64_t)sad << 30) | tie;
}

__device__ __forceinline__ bayer_mv_t key_to_mv(uint64_t key) {
  bayer_mv_t m;
  m.dx = (int16_t)((int)(key & 1023u) - 511);
  m.dy = (int16_t)((int)((key >> 10) & 1023u) - 511);
  m.sad = (uint32_t)(key >> 30);
  return m;
}

__device__ __forceinline__ uint64_t warp_min_u64(uint64_t k) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    uint64_t other = __shfl_xor_sync(0xffffffffu, k, o);
    k = other < k ? other : k;
  }
  return k;
}

}  // namespace bme

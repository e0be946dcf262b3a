// Encoders of the two 5th-generation tensor-core (tcgen05.mma) operand descriptors used by the
// tensor-core Chebyshev transforms: the shared-memory matrix descriptor and the instruction
// descriptor of .kind::tf32.  Plain C++ (host and device), so that a host test can check every
// field's position against the PTX ISA tables before anything is launched.
//
// Shared-memory matrix descriptor (64 bits), tcgen05 form:
//   bits  0-13  matrix start address >> 4 (shared-window byte address)
//   bits 16-29  leading-dimension byte offset >> 4
//   bits 32-45  stride-dimension byte offset >> 4
//   bits 46-47  descriptor version, 1 for tcgen05
//   bits 49-51  matrix base offset (0: no swizzle)
//   bit  52     leading-dimension offset mode (0: relative)
//   bits 61-63  swizzle mode (0: none)
// For a K-major operand without swizzling the layout is built from core matrices of 8 rows x
// 16 bytes (8 x 4 tf32), each 128 contiguous bytes; the leading-dimension byte offset is the
// distance between core matrices adjacent in K, the stride-dimension byte offset the distance
// between core matrices adjacent in M (or N).
//
// Instruction descriptor (32 bits), .kind::f16 / .kind::tf32:
//   bits  0-1 sparsity selector, bit 2 sparsity, bit 3 saturate (all 0 here)
//   bits  4-5 D type (1: f32)
//   bits  7-9 A type, bits 10-12 B type (.kind::tf32: 2 = tf32)
//   bit 13 negate A, bit 14 negate B, bit 15 A MN-major, bit 16 B MN-major (0: K-major)
//   bits 17-22 N >> 3, bits 24-28 M >> 4, bits 30-31 max shift (.ws only, 0)
#pragma once

#include <stdint.h>

#if defined(__CUDACC__)
#define DPS_HD __host__ __device__
#else
#define DPS_HD
#endif

namespace dps {
namespace umma {

DPS_HD constexpr uint64_t smem_desc(uint32_t addr, uint32_t lbo_bytes, uint32_t sbo_bytes) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo_bytes >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo_bytes >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

DPS_HD constexpr uint32_t idesc_tf32(uint32_t m, uint32_t n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((n >> 3) << 17) | ((m >> 4) << 24);
}

// Byte offset of element (row, k) in a K-major, unswizzled tile of 8 tf32 columns (two core
// matrices along K): the two core matrices of an 8-row group are adjacent (leading-dimension byte
// offset kLbo = 128), 8-row groups follow each other (stride-dimension byte offset kSbo = 256).  A
// tile of R rows spans tile_bytes(R) = (R / 8) * kSbo bytes; with offsets this small every address
// the tensor core forms from the descriptor stays inside the tile.  (A padded stride of 272 bytes,
// which makes the producers' 16-byte row stores conflict-free, measured no faster.)
constexpr uint32_t kLbo = 128, kSbo = 256;
DPS_HD constexpr uint32_t kmajor_offset(uint32_t row, uint32_t k) {
  return (row >> 3) * kSbo + (k >> 2) * kLbo + (row & 7u) * 16u + (k & 3u) * 4u;
}
DPS_HD constexpr uint32_t tile_bytes(uint32_t rows) { return (rows >> 3) * kSbo; }

// tf32 rounding of a float's bit pattern, to nearest with ties away from zero (the rounding of
// cvt.rna.tf32.f32): add half of the 13 dropped mantissa bits' range to the magnitude bits (the
// sign bit is untouched; a carry moves into the exponent as rounding up should) and clear them.
// Integer operations only, for finite inputs.
DPS_HD constexpr uint32_t tf32_rna_bits(uint32_t x) { return (x + 0x1000u) & 0xFFFFE000u; }

}  // namespace umma
}  // namespace dps

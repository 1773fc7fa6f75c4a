// Shared-memory layout and descriptor encodings of the tensor-core GEMM
// (tc_gemm.cuh), host- and device-callable so that host tests can check
// them: operand tiles in the canonical no-swizzle K-major layout of
// tcgen05.mma (core matrices of 8 rows x 16 bytes, 128 bytes each), the
// 64-bit shared-memory matrix descriptor and the 32-bit instruction
// descriptor of kind::f16 with BF16 operands and an FP32 accumulator.
#pragma once

#include <stdint.h>

#ifndef __CUDACC__
#define TC_HD
#else
#define TC_HD __host__ __device__
#endif

namespace psms {
namespace tc {

constexpr int TM = 128;  // tile rows = TMEM lanes (M of one MMA)
constexpr int TK = 64;   // K chunk per shared-memory stage (four MMAs of K = 16)
// byte distances between core matrices: along K (leading) and between
// groups of 8 rows (stride) in a tile of TK columns
constexpr uint32_t LBO = 128, SBO = (TK / 8) * 128;

// byte offset of element (r, k) (2-byte BF16) in a K-major no-swizzle tile
// of TK columns: core matrix (r/8, k/8), row r%8 of 16 bytes inside it
TC_HD inline uint32_t canon_off(int r, int k) {
    return (uint32_t)((((r >> 3) * (TK / 8) + (k >> 3)) << 7) + ((r & 7) << 4) + ((k & 7) << 1));
}

// shared-memory matrix descriptor, no swizzle: start address >> 4 (bits
// 0-13), leading byte offset >> 4 (16-29), stride byte offset >> 4
// (32-45), the fixed descriptor version 1 at bit 46, base offset 0 and
// swizzle mode 0 (bits 49-51, 61-63)
TC_HD inline uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}

// instruction descriptor of kind::f16: dense, FP32 accumulator (bits 4-5 =
// 1), BF16 A (bits 7-9 = 1) and B (bits 10-12 = 1), no negation, both
// K-major (bits 15, 16 = 0), N/8 at bits 17-22, M/16 at bits 24-28
template <int TN>
TC_HD inline uint32_t instr_desc() {
    static_assert(TN % 16 == 0 && TN >= 16 && TN <= 256, "N of an M = 128 MMA: a multiple of 16 up to 256");
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TN >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);
}

}  // namespace tc
}  // namespace psms

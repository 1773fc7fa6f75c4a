// Test harness: the tensor-core GEMM's layout and descriptor encodings
// (csrc/tc_layout.hpp), compiled for the host with the host C++ compiler so
// that the tests can check them without a GPU.  Not part of the library.
#include <cstdint>

#include "../paper_1204_1306_gb300/csrc/tc_layout.hpp"

extern "C" {

// out[r * TK + k] = byte offset of element (r, k) of a tile of `rows` rows
void tc_canon_off_host(int rows, uint32_t *out) {
    for (int r = 0; r < rows; ++r)
        for (int k = 0; k < psms::tc::TK; ++k) out[r * psms::tc::TK + k] = psms::tc::canon_off(r, k);
}

uint64_t tc_smem_desc_host(uint32_t addr, uint32_t lbo, uint32_t sbo) { return psms::tc::smem_desc(addr, lbo, sbo); }

uint32_t tc_instr_desc_host(int tn) {
    return tn == 256 ? psms::tc::instr_desc<256>() : tn == 64 ? psms::tc::instr_desc<64>() : 0u;
}

void tc_constants_host(int *out) {
    out[0] = psms::tc::TM;
    out[1] = psms::tc::TK;
    out[2] = (int)psms::tc::LBO;
    out[3] = (int)psms::tc::SBO;
}

}  // extern "C"

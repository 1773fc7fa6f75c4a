// Test harness: the estimators' host-side planning (csrc/interp_plan.hpp),
// compiled with the host C++ compiler.  Not part of the library.
#include "../paper_1204_1306_gb300/csrc/interp_plan.hpp"

extern "C" {

void interp_coefs_host(int N, int i0, int n, int shift, int independent, float *ab) {
    psms::interp_coefs(N, i0, n, shift, independent != 0, ab);
}

int balanced_chunk_host(int N, int k) { return psms::balanced_chunk(N, k); }

}  // extern "C"

// Face and colour logic of the recursive domain decomposition (Eq. (ddrec)):
// outer blocks of extent B tiled by the context's (inner) blocks of extent l.
// __host__ __device__ so that the kernels and the tests' host harness share it.
//
//  SUB   (Schur complement of an outer block, Eq. (ddrec)): black inner
//        blocks; a face of the site's inner block counts when it is not on
//        the outer block's boundary (the Dirichlet outer faces carry no hop).
//  OUTER (global Schur complement of the outer decomposition, Eq.
//        (ddfactor)): black outer blocks, every face of the outer block.
// The projector on a site is (1 + t gamma_mu)/2 for one face (t = +1 on a
// +mu face, -1 on a -mu face), the identity for two or more, zero for none
// or on a white block.
#pragma once

#define PSMS_OHD __host__ __device__ __forceinline__

namespace psms {
namespace outer {

enum Mode : int { SUB = 0, OUTER = 1 };

// colour (0 black) of the site's inner (SUB) or outer (OUTER) block
PSMS_OHD int colour(int mode, const int x[4], const int l[4], const int B[4]) {
    int c = 0;
    for (int m = 0; m < 4; ++m) c += x[m] / (mode == SUB ? l[m] : B[m]);
    return c & 1;
}

// number of counted faces at global coordinates x; fmu / ft of the last one
PSMS_OHD int faces(int mode, const int x[4], const int l[4], const int B[4], int &fmu, int &ft) {
    int nf = 0;
    fmu = 0;
    ft = 0;
    for (int m = 0; m < 4; ++m) {
        const int xo = x[m] % B[m];  // coordinate inside the outer block
        const int y = mode == SUB ? x[m] % l[m] : xo;
        const int e = mode == SUB ? l[m] : B[m];
        if (y == e - 1 && (mode == OUTER || xo != B[m] - 1)) {
            ++nf;
            fmu = m;
            ft = 1;
        } else if (y == 0 && (mode == OUTER || xo != 0)) {
            ++nf;
            fmu = m;
            ft = -1;
        }
    }
    return nf;
}

// true when the link (x, mu) crosses an outer-block face
PSMS_OHD bool crossing(const int x[4], int mu, const int B[4]) { return x[mu] % B[mu] == B[mu] - 1; }

}  // namespace outer
}  // namespace psms

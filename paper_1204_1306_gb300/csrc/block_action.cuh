// Per-block change of the plaquette action between a field U and a proposal
// U' (Eq. (Sw) without beta; App. C's beta terms at the block level).
// __host__ __device__ so that the kernel and the tests' host harness run the
// same code.
//
// Attribution: a plaquette (x; mu < nu) whose links changed belongs to the
// block of the starting site of its first changed link in the order
// (x,mu), (x+mu,nu), (x+nu,mu), (x,nu); a link changed when any of its 18
// numbers differs.  With blocks of extent >= 3 the changed links of a
// plaquette all lie in one block, so this is the block that changed it.
//
// The owner's starting site is x, x+mu or x+nu, so every plaquette owned by
// block b starts in b or one site below it: the scan of block b covers
// x_m in [B_m l_m - 1, B_m l_m + l_m - 1] (wrapped), or the whole extent
// when one block spans direction m, and keeps the plaquettes it owns.
#pragma once

#include "hyp.cuh"

namespace psms {
namespace act {

using hyp::M;

// ld(f, mu, x): link of field f (0: U, 1: U') in direction mu at x (the
// loader wraps coordinates that lie one site outside the lattice)
template <class Ld>
PSMS_HD bool changed(const Ld &ld, int mu, const int x[4]) {
    const M a = ld(0, mu, x), b = ld(1, mu, x);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            if (a.e[i][j].re != b.e[i][j].re || a.e[i][j].im != b.e[i][j].im) return true;
    return false;
}

template <class Ld>
PSMS_HD double retr_plaq(const Ld &ld, int f, int mu, int nu, const int x[4]) {
    int xm[4] = {x[0], x[1], x[2], x[3]};
    int xn[4] = {x[0], x[1], x[2], x[3]};
    xm[mu] += 1;
    xn[nu] += 1;
    const M p = hyp::mmul(hyp::mmul(ld(f, mu, x), ld(f, nu, xm)), hyp::mdag(hyp::mmul(ld(f, nu, x), ld(f, mu, xn))));
    return hyp::retrace(p);
}

struct Grid {
    int L[4], l[4], nb[4];
};

PSMS_HD int wrap(int v, int L) { return v < 0 ? v + L : (v >= L ? v - L : v); }

PSMS_HD int block_lex(const Grid &g, const int x[4]) {
    int b = 0;
    for (int m = 0; m < 4; ++m) b = b * g.nb[m] + wrap(x[m], g.L[m]) / g.l[m];
    return b;
}

// Partial sum, over the scan points t = tid, tid + nthr, ... of block
// (B, lexicographic index b), of -(ReTr P' - ReTr P)/3 for the plaquettes b
// owns.
template <class Ld>
PSMS_HD double block_change_partial(const Ld &ld, const Grid &g, const int B[4], int b, int tid, int nthr) {
    int lo[4], ext[4];
    long long n = 1;
    for (int m = 0; m < 4; ++m) {
        if (g.nb[m] == 1) {
            lo[m] = 0;
            ext[m] = g.L[m];
        } else {
            lo[m] = B[m] * g.l[m] - 1;
            ext[m] = g.l[m] + 1;
        }
        n *= ext[m];
    }
    double acc = 0.0;
    for (long long t = tid; t < n; t += nthr) {
        long long q = t;
        int x[4];
        for (int m = 3; m >= 0; --m) {
            x[m] = wrap(lo[m] + (int)(q % ext[m]), g.L[m]);
            q /= ext[m];
        }
        for (int mu = 0; mu < 4; ++mu)
            for (int nu = mu + 1; nu < 4; ++nu) {
                int xm[4] = {x[0], x[1], x[2], x[3]};
                int xn[4] = {x[0], x[1], x[2], x[3]};
                xm[mu] += 1;
                xn[nu] += 1;
                const int *start = nullptr;
                if (changed(ld, mu, x)) start = x;
                else if (changed(ld, nu, xm)) start = xm;
                else if (changed(ld, mu, xn)) start = xn;
                else if (changed(ld, nu, x)) start = x;
                if (!start || block_lex(g, start) != b) continue;
                acc -= (retr_plaq(ld, 1, mu, nu, x) - retr_plaq(ld, 0, mu, nu, x)) / 3.0;
            }
    }
    return acc;
}

}  // namespace act
}  // namespace psms

// Arithmetic of one level of HYP smearing and of the block HYP plaquette
// action (App. C; Sec. 5 takes the smearing parameters of the HYP
// construction of Hasenfratz and Knechtli, Phys. Rev. D 64 (2001) 034504).
// Everything here is __host__ __device__: the kernels of hyp.cu call it per
// thread, and the same code compiled for the host is what the tests check
// against the oracle without a GPU.
//
// Fat links, built in three steps confined to the hypercubes attached to a
// link (x, mu):
//   level 3  Vbar(x,mu;eta)  = Proj[(1-a3) U(x,mu) + a3/2 S_eta(U, U)],
//            the staples in the single direction eta; the link is
//            "undecorated" in the two directions other than mu and eta;
//   level 2  Vtil(x,mu;nu)   = Proj[(1-a2) U(x,mu) + a2/4 sum_{rho != mu,nu}
//            S_rho(Vbar(.,rho;sigma), Vbar(.,mu;sigma))], sigma the fourth
//            direction (not mu, nu, rho);
//   level 1  V(x,mu)         = Proj[(1-a1) U(x,mu) + a1/6 sum_{nu != mu}
//            S_nu(Vtil(.,nu;mu), Vtil(.,mu;nu))];
// S_nu(T, W) = T(x,nu) W(x+nu,mu) T(x+mu,nu)^dag
//            + T(x-nu,nu)^dag W(x-nu,mu) T(x-nu+mu,nu).
//
// Proj[M]: the unitary polar factor of M, computed by Newton's iteration
// X <- (g X + X^{-dag} / g) / 2 with Higham's scaling g = (|X^-1|_F /
// |X|_F)^{1/2} (N. J. Higham, SIAM J. Sci. Stat. Comput. 7 (1986) 1160),
// then the phase of its determinant removed with the principal cube root.
#pragma once

#include <math.h>

#define PSMS_HD __host__ __device__ __forceinline__

namespace psms {
namespace hyp {

struct Z {
    double re, im;
};

struct M {
    Z e[3][3];
};

PSMS_HD Z zadd(Z a, Z b) { return {a.re + b.re, a.im + b.im}; }
PSMS_HD Z zsub(Z a, Z b) { return {a.re - b.re, a.im - b.im}; }
PSMS_HD Z zmul(Z a, Z b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
PSMS_HD Z zconj(Z a) { return {a.re, -a.im}; }

PSMS_HD M mzero() {
    M r;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) r.e[i][j] = {0.0, 0.0};
    return r;
}

PSMS_HD M mmul(const M &a, const M &b) {
    M r;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            Z z = zmul(a.e[i][0], b.e[0][j]);
            z = zadd(z, zmul(a.e[i][1], b.e[1][j]));
            z = zadd(z, zmul(a.e[i][2], b.e[2][j]));
            r.e[i][j] = z;
        }
    return r;
}

PSMS_HD M mdag(const M &a) {
    M r;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) r.e[i][j] = zconj(a.e[j][i]);
    return r;
}

// r += s * a
PSMS_HD void maxpy(M &r, double s, const M &a) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            r.e[i][j].re += s * a.e[i][j].re;
            r.e[i][j].im += s * a.e[i][j].im;
        }
}

PSMS_HD double mnorm2(const M &a) {
    double s = 0.0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) s += a.e[i][j].re * a.e[i][j].re + a.e[i][j].im * a.e[i][j].im;
    return s;
}

PSMS_HD double retrace(const M &a) { return a.e[0][0].re + a.e[1][1].re + a.e[2][2].re; }

// signed cofactor C_ij (cyclic form, valid for 3 x 3)
PSMS_HD Z cofactor(const M &a, int i, int j) {
    const int i1 = (i + 1) % 3, i2 = (i + 2) % 3, j1 = (j + 1) % 3, j2 = (j + 2) % 3;
    return zsub(zmul(a.e[i1][j1], a.e[i2][j2]), zmul(a.e[i1][j2], a.e[i2][j1]));
}

PSMS_HD Z mdet(const M &a) {
    Z d = zmul(a.e[0][0], cofactor(a, 0, 0));
    d = zadd(d, zmul(a.e[0][1], cofactor(a, 0, 1)));
    return zadd(d, zmul(a.e[0][2], cofactor(a, 0, 2)));
}

// (a^-1)^dagger: entry (i, j) is conj(C_ij / det a)
PSMS_HD M minv_dag(const M &a) {
    M c;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) c.e[i][j] = cofactor(a, i, j);
    Z d = zadd(zadd(zmul(a.e[0][0], c.e[0][0]), zmul(a.e[0][1], c.e[0][1])), zmul(a.e[0][2], c.e[0][2]));
    const double n = d.re * d.re + d.im * d.im;
    const Z inv = {d.re / n, -d.im / n};
    M r;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) r.e[i][j] = zconj(zmul(c.e[i][j], inv));
    return r;
}

constexpr int kPolarMaxIter = 60;

// Proj[M]; the iteration count is bounded, and a singular or non-finite M
// gives a non-finite result that the callers detect.
PSMS_HD M project_su3(M x) {
    bool scaled = true;
    int extra = -1;
    for (int it = 0; it < kPolarMaxIter; ++it) {
        const M xi = minv_dag(x);
        double g = 1.0;
        if (scaled) g = sqrt(sqrt(mnorm2(xi) / mnorm2(x)));
        M nx = mzero();
        maxpy(nx, 0.5 * g, x);
        maxpy(nx, 0.5 / g, xi);
        M d = nx;
        maxpy(d, -1.0, x);
        const double rel = sqrt(mnorm2(d) / mnorm2(nx));
        x = nx;
        if (!(rel == rel)) break;  // NaN: give up, the caller sees it
        if (extra >= 0) {
            if (--extra < 0) break;
        } else if (rel < 1e-9) {
            scaled = false;  // quadratic convergence from here: two more steps
            extra = 1;
        }
    }
    const Z d = mdet(x);
    const double ph = atan2(d.im, d.re) / 3.0;
    const Z c = {cos(ph), -sin(ph)};
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) x.e[i][j] = zmul(x.e[i][j], c);
    return x;
}

// decorated-field keys: the direction k != mu of a level-3 (eta) or
// level-2 (nu) field, stored as key = 3 mu + (k - (k > mu))
PSMS_HD int key_of(int mu, int k) { return 3 * mu + (k - (k > mu ? 1 : 0)); }
PSMS_HD int dir_of_key(int key) {
    const int mu = key / 3, r = key % 3;
    return r + (r >= mu ? 1 : 0);
}

// Ld: callable ld(lev, mu, k, x) returning the link of field `lev`
// (0 thin U, 3 Vbar(.,mu;k), 2 Vtil(.,mu;k), 1 V(.,mu)) at coordinates x,
// which may lie up to two sites outside the lattice (the loader wraps).
// S_nu(T, W)(x, mu) with T = field lt in direction nu with key kt and
// W = field lw in direction mu with key kw
template <class Ld>
PSMS_HD M staple_sum(const Ld &ld, int lt, int kt, int lw, int kw, int mu, int nu, const int x[4]) {
    int xn[4] = {x[0], x[1], x[2], x[3]};
    int xm[4] = {x[0], x[1], x[2], x[3]};
    int xmn[4] = {x[0], x[1], x[2], x[3]};
    int xmnm[4] = {x[0], x[1], x[2], x[3]};
    xn[nu] += 1;       // x + nu
    xm[mu] += 1;       // x + mu
    xmn[nu] -= 1;      // x - nu
    xmnm[nu] -= 1;     // x - nu + mu
    xmnm[mu] += 1;
    M up = mmul(mmul(ld(lt, nu, kt, x), ld(lw, mu, kw, xn)), mdag(ld(lt, nu, kt, xm)));
    M dn = mmul(mmul(mdag(ld(lt, nu, kt, xmn)), ld(lw, mu, kw, xmn)), ld(lt, nu, kt, xmnm));
    maxpy(up, 1.0, dn);
    return up;
}

// One fat link of level lev (3, 2, 1) in direction mu with key k (level 3:
// the staple direction eta; level 2: the undecorated direction nu; level 1:
// ignored) at x.
template <class Ld>
PSMS_HD M fat_link(const Ld &ld, int lev, int mu, int k, const int x[4], double a1, double a2, double a3) {
    M s = mzero();
    double a = 0.0, w = 0.0;
    if (lev == 3) {
        a = a3;
        w = a3 / 2.0;
        s = staple_sum(ld, 0, 0, 0, 0, mu, k, x);
    } else if (lev == 2) {
        a = a2;
        w = a2 / 4.0;
        for (int rho = 0; rho < 4; ++rho) {
            if (rho == mu || rho == k) continue;
            const int sigma = 6 - mu - k - rho;
            // T = Vbar(., rho; sigma), W = Vbar(., mu; sigma)
            maxpy(s, 1.0, staple_sum(ld, 3, sigma, 3, sigma, mu, rho, x));
        }
    } else {
        a = a1;
        w = a1 / 6.0;
        for (int nu = 0; nu < 4; ++nu) {
            if (nu == mu) continue;
            // T = Vtil(., nu; mu), W = Vtil(., mu; nu)
            maxpy(s, 1.0, staple_sum(ld, 2, mu, 2, nu, mu, nu, x));
        }
    }
    M m = mzero();
    maxpy(m, 1.0 - a, ld(0, mu, 0, x));
    maxpy(m, w, s);
    return project_su3(m);
}

// (3 - Re Tr P_{mu nu}(x)) / 3 for the plaquette of field lev at x
template <class Ld>
PSMS_HD double plaquette_term(const Ld &ld, int lev, int mu, int nu, const int x[4]) {
    int xm[4] = {x[0], x[1], x[2], x[3]};
    int xn[4] = {x[0], x[1], x[2], x[3]};
    xm[mu] += 1;
    xn[nu] += 1;
    const M p = mmul(mmul(ld(lev, mu, 0, x), ld(lev, nu, 0, xm)), mdag(mmul(ld(lev, nu, 0, x), ld(lev, mu, 0, xn))));
    return (3.0 - retrace(p)) / 3.0;
}

}  // namespace hyp
}  // namespace psms

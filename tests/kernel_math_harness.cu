// Test harness: per-thread arithmetic of the library's kernels (the HYP
// smearing of csrc/hyp.cuh and the per-block action change of
// csrc/block_action.cuh), the same code the kernels run, compiled for the
// host and driven over canonical arrays, so that the tests can compare it
// with the oracle without a GPU.  Not part of the library.
#include <vector>

#include "../paper_1204_1306_gb300/csrc/block_action.cuh"
#include "../paper_1204_1306_gb300/csrc/hyp.cuh"
#include "../paper_1204_1306_gb300/csrc/outer.cuh"

using psms::hyp::M;

namespace {

struct HostLd {
    int L[4];
    long long V;
    const M *U;   // [site][mu]
    const M *F3;  // [key][site]
    const M *F2;  // [key][site]
    const M *F1;  // [mu][site]

    __host__ __device__ M operator()(int lev, int mu, int k, const int x[4]) const {
        int y[4];
        for (int m = 0; m < 4; ++m) y[m] = ((x[m] % L[m]) + L[m]) % L[m];
        const long long s = ((long long)(y[0] * L[1] + y[1]) * L[2] + y[2]) * L[3] + y[3];
        if (lev == 0) return U[s * 4 + mu];
        if (lev == 3) return F3[psms::hyp::key_of(mu, k) * V + s];
        if (lev == 2) return F2[psms::hyp::key_of(mu, k) * V + s];
        return F1[mu * V + s];
    }
};

void coords(const int L[4], long long s, int x[4]) {
    x[3] = (int)(s % L[3]);
    s /= L[3];
    x[2] = (int)(s % L[2]);
    s /= L[2];
    x[1] = (int)(s % L[1]);
    x[0] = (int)(s / L[1]);
}

}  // namespace

// U: canonical links [V][4][3][3] complex (interleaved doubles); V_out the
// same layout; alpha = (a1, a2, a3)
extern "C" void hyp_smear_host(const double *U, const int *L, const double *alpha, double *V_out) {
    HostLd ld;
    for (int m = 0; m < 4; ++m) ld.L[m] = L[m];
    ld.V = (long long)L[0] * L[1] * L[2] * L[3];
    const M *Um = reinterpret_cast<const M *>(U);
    std::vector<M> F3(12 * ld.V), F2(12 * ld.V), F1(4 * ld.V);
    ld.U = Um;
    ld.F3 = F3.data();
    ld.F2 = F2.data();
    ld.F1 = F1.data();
    for (int lev = 3; lev >= 1; --lev) {
        const int n_keys = lev == 1 ? 4 : 12;
        std::vector<M> &dst = lev == 3 ? F3 : (lev == 2 ? F2 : F1);
        for (int key = 0; key < n_keys; ++key)
            for (long long s = 0; s < ld.V; ++s) {
                int x[4];
                coords(L, s, x);
                const int mu = lev == 1 ? key : key / 3;
                const int k = lev == 1 ? 0 : psms::hyp::dir_of_key(key);
                dst[key * ld.V + s] = psms::hyp::fat_link(ld, lev, mu, k, x, alpha[0], alpha[1], alpha[2]);
            }
    }
    M *out = reinterpret_cast<M *>(V_out);
    for (long long s = 0; s < ld.V; ++s)
        for (int mu = 0; mu < 4; ++mu) out[s * 4 + mu] = F1[mu * ld.V + s];
}

// S_HYP,b per block in lexicographic block order, from fat links V
// (canonical layout) and block extents l
extern "C" void hyp_block_action_host(const double *Vfat, const int *L, const int *l, double *out) {
    HostLd ld;
    for (int m = 0; m < 4; ++m) ld.L[m] = L[m];
    ld.V = (long long)L[0] * L[1] * L[2] * L[3];
    std::vector<M> F1(4 * ld.V);
    const M *Vm = reinterpret_cast<const M *>(Vfat);
    for (long long s = 0; s < ld.V; ++s)
        for (int mu = 0; mu < 4; ++mu) F1[mu * ld.V + s] = Vm[s * 4 + mu];
    ld.F1 = F1.data();
    int nb[4];
    for (int m = 0; m < 4; ++m) nb[m] = L[m] / l[m];
    const int n_blocks = nb[0] * nb[1] * nb[2] * nb[3];
    for (int b = 0; b < n_blocks; ++b) out[b] = 0.0;
    for (long long s = 0; s < ld.V; ++s) {
        int x[4];
        coords(L, s, x);
        const int b = ((x[0] / l[0] * nb[1] + x[1] / l[1]) * nb[2] + x[2] / l[2]) * nb[3] + x[3] / l[3];
        for (int mu = 0; mu < 4; ++mu)
            for (int nu = mu + 1; nu < 4; ++nu)
                if (x[mu] % l[mu] <= l[mu] - 2 && x[nu] % l[nu] <= l[nu] - 2)
                    out[b] += psms::hyp::plaquette_term(ld, 1, mu, nu, x);
    }
}

// Proj[M] for n matrices (3x3 complex, interleaved doubles)
extern "C" void hyp_project_host(const double *m, int n, double *out) {
    const M *in = reinterpret_cast<const M *>(m);
    M *o = reinterpret_cast<M *>(out);
    for (int i = 0; i < n; ++i) o[i] = psms::hyp::project_su3(in[i]);
}

namespace {

struct PairHostLd {
    int L[4];
    const M *U0, *U1;  // canonical [site][mu]

    __host__ __device__ M operator()(int f, int mu, const int x[4]) const {
        int y[4];
        for (int m = 0; m < 4; ++m) y[m] = ((x[m] % L[m]) + L[m]) % L[m];
        const long long s = ((long long)(y[0] * L[1] + y[1]) * L[2] + y[2]) * L[3] + y[3];
        return (f ? U1 : U0)[s * 4 + mu];
    }
};

}  // namespace

// dS_w,b per block (lexicographic) of U0 -> U1, scanning each block the way
// the kernel does (one thread)
extern "C" void block_change_host(const double *U0, const double *U1, const int *L, const int *l, double *out) {
    PairHostLd ld;
    psms::act::Grid g;
    for (int m = 0; m < 4; ++m) {
        ld.L[m] = g.L[m] = L[m];
        g.l[m] = l[m];
        g.nb[m] = L[m] / l[m];
    }
    ld.U0 = reinterpret_cast<const M *>(U0);
    ld.U1 = reinterpret_cast<const M *>(U1);
    const int nb = g.nb[0] * g.nb[1] * g.nb[2] * g.nb[3];
    for (int b = 0; b < nb; ++b) {
        int B[4], q = b;
        for (int m = 3; m >= 0; --m) {
            B[m] = q % g.nb[m];
            q /= g.nb[m];
        }
        out[b] = psms::act::block_change_partial(ld, g, B, b, 0, 1);
    }
}

// faces / colour of the recursive decomposition for every site of the
// lattice L with blocks l and outer blocks B: out[4 * s + (0..3)] =
// (colour, number of faces, mu of the last face, its sign)
extern "C" void outer_faces_host(const int *L, const int *l, const int *B, int mode, int *out) {
    const long long V = (long long)L[0] * L[1] * L[2] * L[3];
    for (long long s = 0; s < V; ++s) {
        int x[4];
        coords(L, s, x);
        int fmu, ft;
        const int nf = psms::outer::faces(mode, x, l, B, fmu, ft);
        out[4 * s + 0] = psms::outer::colour(mode, x, l, B);
        out[4 * s + 1] = nf;
        out[4 * s + 2] = fmu;
        out[4 * s + 3] = ft;
    }
}

// 1 where the link (x, mu) crosses an outer face
extern "C" void outer_crossing_host(const int *L, const int *B, int *out) {
    const long long V = (long long)L[0] * L[1] * L[2] * L[3];
    for (long long s = 0; s < V; ++s) {
        int x[4];
        coords(L, s, x);
        for (int mu = 0; mu < 4; ++mu) out[4 * s + mu] = psms::outer::crossing(x, mu, B) ? 1 : 0;
    }
}

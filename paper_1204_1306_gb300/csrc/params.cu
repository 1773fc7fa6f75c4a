// Coefficients of the parametrised filter levels (App. C, Eqs. (Si),
// (DeltaSi), (sigmaDeltaSiparams), (paramsi)).  Host arithmetic on a few
// small covariance matrices: no context, no device memory, no kernel.
//
// Level i = 1..n accepts with min{1, exp(-Delta_i)},
// Delta_i = sum_{j<=i} beta_i^(j) Delta S^(j); level 0 is the pure-gauge
// proposal at coupling beta_0^(0).  Each action's coefficients sum to its
// target beta^(j).  From the last level down, the level's own coefficient
// follows from that constraint and the others minimise the level's variance
// Sigma_i^2 = beta^T C_i beta: setting its gradient to zero gives the
// normal equations  sum_{k free} C^(jk) beta_i^(k) = -C^(ji) beta_i^(i)
// for every free j < i.  Actions estimated stochastically take no
// coefficient at later levels.  beta_0^(0) closes the plaquette constraint.
#include <cmath>
#include <vector>

#include "psms.h"

namespace {

constexpr int kMaxActions = 64;

// Solves A x = b (n x n, row-major) by Gaussian elimination with partial
// pivoting.  Returns false when a pivot is zero or not finite.
bool solve_dense(std::vector<double> A, std::vector<double> b, int n, std::vector<double> &x) {
    for (int k = 0; k < n; ++k) {
        int p = k;
        for (int r = k + 1; r < n; ++r)
            if (std::fabs(A[r * n + k]) > std::fabs(A[p * n + k])) p = r;
        const double piv = A[p * n + k];
        if (!(std::fabs(piv) > 0.0) || !std::isfinite(piv)) return false;
        if (p != k) {
            for (int c = 0; c < n; ++c) std::swap(A[k * n + c], A[p * n + c]);
            std::swap(b[k], b[p]);
        }
        for (int r = k + 1; r < n; ++r) {
            const double f = A[r * n + k] / piv;
            if (f == 0.0) continue;
            for (int c = k; c < n; ++c) A[r * n + c] -= f * A[k * n + c];
            b[r] -= f * b[k];
        }
    }
    x.assign(n, 0.0);
    for (int k = n - 1; k >= 0; --k) {
        double s = b[k];
        for (int c = k + 1; c < n; ++c) s -= A[k * n + c] * x[c];
        x[k] = s / A[k * n + k];
    }
    return true;
}

}  // namespace

extern "C" psms_status psms_level_covariance(const double *samples, long long n_samples, int n_actions,
                                             double *cov) {
    if (!samples || !cov || n_samples < 2 || n_actions < 1 || n_actions > kMaxActions) return PSMS_EINVAL;
    const int m = n_actions;
    std::vector<double> mean(m, 0.0);
    for (long long s = 0; s < n_samples; ++s)
        for (int j = 0; j < m; ++j) {
            const double v = samples[s * m + j];
            if (!std::isfinite(v)) return PSMS_EINVAL;
            mean[j] += v;
        }
    for (int j = 0; j < m; ++j) mean[j] /= (double)n_samples;
    std::vector<double> c(m * m, 0.0);
    for (long long s = 0; s < n_samples; ++s) {
        const double *row = samples + s * m;
        for (int j = 0; j < m; ++j) {
            const double dj = row[j] - mean[j];
            for (int k = 0; k <= j; ++k) c[j * m + k] += dj * (row[k] - mean[k]);
        }
    }
    for (int j = 0; j < m; ++j)
        for (int k = 0; k <= j; ++k) {
            const double v = c[j * m + k] / (double)n_samples;
            cov[j * m + k] = v;
            cov[k * m + j] = v;
        }
    return PSMS_OK;
}

extern "C" psms_status psms_level_coefficients(int n_levels, const double *covs, const double *targets,
                                               const int *stochastic, double *beta) {
    if (!covs || !targets || !beta || n_levels < 1 || n_levels + 1 > kMaxActions) return PSMS_EINVAL;
    const int n = n_levels;
    const int m = n + 1;
    for (int j = 0; j < m; ++j)
        if (!std::isfinite(targets[j])) return PSMS_EINVAL;
    // offset of C_i (size (i+1) x (i+1)) in the packed input
    std::vector<long long> off(m, 0);
    long long tot = 0;
    for (int i = 1; i <= n; ++i) {
        off[i] = tot;
        tot += (long long)(i + 1) * (i + 1);
    }
    for (long long q = 0; q < tot; ++q)
        if (!std::isfinite(covs[q])) return PSMS_EINVAL;
    std::vector<double> B(m * m, 0.0);
    for (int i = n; i >= 1; --i) {
        double bii = targets[i];
        for (int k = i + 1; k <= n; ++k) bii -= B[k * m + i];
        B[i * m + i] = bii;
        std::vector<int> fr;
        for (int j = 0; j < i; ++j)
            if (!(stochastic && stochastic[j])) fr.push_back(j);
        if (fr.empty()) continue;
        const double *C = covs + off[i];
        const int w = i + 1;
        const int nf = (int)fr.size();
        std::vector<double> A(nf * nf), rhs(nf), x;
        for (int a = 0; a < nf; ++a) {
            for (int b = 0; b < nf; ++b) A[a * nf + b] = C[fr[a] * w + fr[b]];
            rhs[a] = -C[fr[a] * w + i] * bii;
        }
        if (!solve_dense(A, rhs, nf, x)) return PSMS_EINVAL;
        for (int a = 0; a < nf; ++a) B[i * m + fr[a]] = x[a];
    }
    double b00 = targets[0];
    for (int k = 1; k <= n; ++k) b00 -= B[k * m + 0];
    B[0] = b00;
    for (int q = 0; q < m * m; ++q) beta[q] = B[q];
    return PSMS_OK;
}

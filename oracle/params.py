"""Coefficients of the parametrised filter levels (App. C, Eqs. (Si),
(DeltaSi), (sigmaDeltaSiparams), (paramsi)).  TEST INFRASTRUCTURE ONLY:
imported by tests, the package's smoke check and the benchmark's CPU
baseline, never by the product path.

Level i = 1..n accepts with min{1, exp(-Delta_i)},
Delta_i = sum_{j<=i} beta_i^(j) Delta S^(j); level 0 is the pure-gauge
proposal at coupling beta_0^(0).  Every action's coefficients sum to its
target, sum_{i>=j} beta_i^(j) = beta^(j) (the plaquette's to beta, an
auxiliary action's to 0, a determinant's to 1).

Solution scheme (App. C.1), from the last level down: at level i the
coefficient of the level's own action follows from the constraint,
beta_i^(i) = beta^(i) - sum_{k>i} beta_k^(i); the free coefficients
beta_i^(j), j < i, minimise the variance Sigma_i^2 of Eq.
(sigmaDeltaSiparams) over the level's samples.  Reading: setting the
derivative of Sigma_i^2 to zero gives
    sum_{k<i} C^(jk) beta_i^(k) = -C^(ji) beta_i^(i),   j < i,
the normal equations of a least-squares fit; the printed Eq. (paramsi)
doubles only the diagonal term, which does not minimise Eq.
(sigmaDeltaSiparams) when the actions are correlated, so it is taken as a
misprint.  Actions estimated stochastically take no free coefficient at
later levels (App. C.1: no parameters for stochastic terms), so their
beta_k^(j), k > j, are 0; the proposal's coupling closes the plaquette
constraint, beta_0^(0) = beta^(0) - sum_{i>=1} beta_i^(0).
"""
import numpy as np


def covariance(samples):
    """C^(jk) of Eq. (sigmaDeltaSiparams) from samples [n_samples, n_actions]
    of (Delta S^(0), ..., Delta S^(i)) (population normalisation)."""
    x = np.asarray(samples, dtype=np.float64)
    d = x - x.mean(axis=0)
    return d.T @ d / x.shape[0]


def variance(C, beta):
    """Sigma^2 of Eq. (sigmaDeltaSiparams) for coefficients beta."""
    b = np.asarray(beta, dtype=np.float64)
    return float(b @ C @ b)


def solve_level(C, beta_ii, free):
    """Free coefficients of one level: minimise Sigma_i^2 over beta_i^(j),
    j in `free` (all j < i), with beta_i^(i) fixed; C is the (i+1)x(i+1)
    covariance of the level.  Returns beta_i^(0..i)."""
    i = C.shape[0] - 1
    beta = np.zeros(i + 1)
    beta[i] = beta_ii
    f = list(free)
    if f:
        beta[f] = np.linalg.solve(C[np.ix_(f, f)], -C[f, i] * beta_ii)
    return beta


def coefficients(covs, targets, stochastic=None):
    """beta_i^(j) for levels i = 0..n as a lower-triangular (n+1)x(n+1)
    array.  covs[i-1] is the covariance of (Delta S^(0..i)) measured at
    level i; targets[j] = beta^(j); stochastic[j] marks actions estimated
    stochastically."""
    n = len(targets) - 1
    if stochastic is None:
        stochastic = [False] * (n + 1)
    B = np.zeros((n + 1, n + 1))
    for i in range(n, 0, -1):
        B[i, i] = targets[i] - B[i + 1:, i].sum()
        free = [j for j in range(i) if not stochastic[j]]
        B[i, :i + 1] = solve_level(np.asarray(covs[i - 1], dtype=np.float64), B[i, i], free)
    B[0, 0] = targets[0] - B[1:, 0].sum()
    return B


def constrained_diagonal(B, targets):
    """The coefficients fixed by the constraints, given the others: the
    diagonal beta_i^(i) (i >= 1) and beta_0^(0)."""
    n = len(targets) - 1
    out = np.zeros(n + 1)
    for i in range(1, n + 1):
        out[i] = targets[i] - np.asarray(B)[i + 1:, i].sum()
    out[0] = targets[0] - np.asarray(B)[1:, 0].sum()
    return out

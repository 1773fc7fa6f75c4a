"""Pins of the coefficient scheme of the parametrised levels (App. C): the
printed Tables 1 and 2 against the constraints, the level solution against
a least-squares fit of the samples, its optimality, and the handling of
stochastic actions."""
import json
import os

import numpy as np
import pytest

from oracle import params

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def _samples(n, seed, k=4):
    """Correlated synthetic Delta S^(j) samples (a common factor plus noise)."""
    g = np.random.default_rng(seed)
    f = g.standard_normal((n, 1))
    w = np.array([1.0, 0.6, -0.8, 1.3, 0.4, -0.5][:k])
    return f * w + g.standard_normal((n, k)) * np.array([0.5, 0.9, 0.3, 0.7, 1.1, 0.6][:k])


@pytest.mark.parametrize("table", GOLDEN["parametrised_levels"]["tables"], ids=lambda t: t["name"])
def test_printed_tables_satisfy_the_constraints(table):
    """The coefficients each constraint fixes (beta_0^(0) from the plaquette
    target beta, beta_1^(1) from the HYP action's target 0, beta_2^(2) from
    the block determinants' target 1) follow from the other printed ones;
    the global level carries the Schur term with coefficient 1."""
    rows = table["beta"]
    B = np.zeros((4, 4))
    for i, r in enumerate(rows):
        for j, v in enumerate(r):
            if v is not None:
                B[i, j] = v
    B[3, 3] = 1.0
    targets = table["targets"] + [1.0]
    diag = params.constrained_diagonal(B, targets)
    for i in range(3):
        assert abs(diag[i] - rows[i][i]) <= table["precision"], (i, diag[i], rows[i][i])
    assert diag[3] == 1.0


def test_level_solution_is_least_squares():
    """Minimising Sigma_i^2 over the free coefficients is the least-squares
    fit of -beta_i^(i) Delta S^(i) by the other actions (centred samples)."""
    x = _samples(4000, 1)
    C = params.covariance(x)
    beta_ii = 1.7
    sol = params.solve_level(C, beta_ii, [0, 1, 2])
    xc = x - x.mean(axis=0)
    ref, *_ = np.linalg.lstsq(xc[:, :3], -beta_ii * xc[:, 3], rcond=None)
    assert np.abs(sol[:3] - ref).max() < 1e-10
    assert sol[3] == beta_ii
    # the variance is the residual of the fit
    resid = xc[:, :3] @ ref + beta_ii * xc[:, 3]
    assert abs(params.variance(C, sol) - np.mean(resid ** 2)) < 1e-10


def test_level_solution_is_optimal_and_printed_form_is_not():
    """Random moves of the free coefficients raise Sigma^2; the equations as
    printed (diagonal term doubled) give a larger Sigma^2 on correlated
    actions, so the stationarity reading is the one that minimises."""
    x = _samples(4000, 2)
    C = params.covariance(x)
    sol = params.solve_level(C, 1.0, [0, 1, 2])
    v = params.variance(C, sol)
    g = np.random.default_rng(3)
    for _ in range(200):
        d = np.zeros(4)
        d[:3] = 0.05 * g.standard_normal(3)
        assert params.variance(C, sol + d) >= v - 1e-12
    A = C[:3, :3] + np.diag(np.diag(C[:3, :3]))
    printed = np.append(np.linalg.solve(A, -C[:3, 3]), 1.0)
    assert params.variance(C, printed) > v * 1.01
    assert v < C[3, 3]                       # the free coefficients reduce the variance


def test_coefficients_constraints_and_stochastic_actions():
    """Column sums equal the targets; a stochastic action takes no
    coefficient at later levels; uncorrelated actions take none either."""
    x = _samples(3000, 4)
    covs = [params.covariance(x[:, :i + 1]) for i in range(1, 4)]
    targets = [5.6, 0.0, 1.0, 1.0]
    for stoch in ([False, False, False, True], [False, False, True, True]):
        B = params.coefficients(covs, targets, stoch)
        assert np.allclose(np.tril(B), B)
        assert np.abs(B.sum(axis=0) - targets).max() < 1e-12
        for j, s in enumerate(stoch):
            if s:
                assert np.all(B[j + 1:, j] == 0)
        if stoch[2]:
            assert B[2, 2] == 1.0 and B[3, 2] == 0.0
    d = np.random.default_rng(5).standard_normal((20000, 4)) * [1.0, 2.0, 0.5, 1.5]
    B = params.coefficients([params.covariance(d[:, :i + 1]) for i in range(1, 4)], targets)
    off = B - np.diag(np.diag(B))
    assert np.abs(off).max() < 0.05          # sampling noise only

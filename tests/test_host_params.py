"""The library's host functions for the parametrised levels (App. C),
called through the C ABI without a GPU, against the oracle's coefficient
scheme (which is pinned in test_oracle_params.py)."""
import numpy as np
import pytest

import paper_1204_1306_gb300 as ps
from oracle import params


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1204_1306_gb300 import build
    build.build()
    ps.load_library()


def _samples(n, seed, k):
    g = np.random.default_rng(seed)
    f = g.standard_normal((n, 1))
    return f * g.standard_normal(k) + g.standard_normal((n, k)) * g.uniform(0.3, 1.2, k)


def test_covariance_matches_oracle():
    x = _samples(5000, 1, 5)
    assert np.abs(ps.psms_level_covariance(x) - params.covariance(x)).max() < 1e-12


@pytest.mark.parametrize("n,stoch", [(1, None), (3, [0, 0, 0, 1]), (3, [0, 0, 1, 1]), (5, [0, 1, 0, 0, 1, 1])])
def test_coefficients_match_oracle(n, stoch):
    x = _samples(4000, 10 + n, n + 1)
    covs = [params.covariance(x[:, :i + 1]) for i in range(1, n + 1)]
    targets = np.random.default_rng(n).uniform(-1, 6, n + 1)
    got = ps.psms_level_coefficients(covs, targets, stoch)
    ref = params.coefficients(covs, targets, None if stoch is None else [bool(s) for s in stoch])
    assert np.abs(got - ref).max() < 1e-10 * max(1.0, np.abs(ref).max())
    assert np.abs(got.sum(axis=0) - targets).max() < 1e-12


def test_errors():
    with pytest.raises(ps.PsmsError):
        ps.psms_level_covariance(np.zeros((1, 3)))
    with pytest.raises(ps.PsmsError):
        ps.psms_level_covariance(np.full((4, 2), np.nan))
    singular = [np.zeros((2, 2))]
    with pytest.raises(ps.PsmsError):
        ps.psms_level_coefficients(singular, [5.0, 1.0])
    # a stochastic lower action leaves nothing to solve: no error
    B = ps.psms_level_coefficients(singular, [5.0, 1.0], [1, 1])
    assert B[1, 1] == 1.0 and B[0, 0] == 5.0 and B[1, 0] == 0.0

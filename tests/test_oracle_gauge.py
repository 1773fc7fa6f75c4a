"""Pins of the oracle's pure-gauge proposal (Cabibbo-Marinari heatbath and
overrelaxation, Sec. 6) and of the per-block plaquette attribution."""
import numpy as np
import pytest
from scipy import integrate, stats

from oracle import filter as ofilter, gauge, lattice, philox
from tests import seeded


@pytest.mark.parametrize("alpha", [0.3, 1.5, 2.0, 4.0, 12.0])
def test_a0_sampler_distribution(alpha):
    """a0 ~ sqrt(1-a0^2) exp(alpha a0) on [-1, 1] (Creutz below alpha = 2,
    Kennedy-Pendleton above): Kolmogorov-Smirnov against the exact CDF."""
    n = 20000
    link = np.arange(n, dtype=np.uint64)
    a0, failed = gauge.sample_a0(np.full(n, alpha), 17, 3, link, 1)
    assert not failed.any()
    f = lambda a: np.sqrt(1 - a * a) * np.exp(alpha * (a - 1))
    Z = integrate.quad(f, -1, 1)[0]
    cdf = lambda a: np.array([integrate.quad(f, -1, x)[0] / Z for x in np.atleast_1d(a)])
    grid = np.linspace(-1, 1, 4001)
    cgrid = cdf(grid)
    res = stats.kstest(a0, lambda x: np.interp(x, grid, cgrid))
    assert res.pvalue > 1e-3


def _all_link_subsets(geom):
    return [(mu, geom.parity == p) for mu in range(4) for p in (0, 1)]


def test_overrelaxation_conserves_action():
    dims = (4, 4, 4, 4)
    geom = lattice.Geometry(dims, dims)
    U = seeded.gauge_field(dims, 3)
    s0 = gauge.wilson_action(U)
    gauge.one_sweep(U, geom, _all_link_subsets(geom), 5.3, "or", 1, 0)
    assert abs(gauge.wilson_action(U) - s0) < 1e-12 * s0
    assert np.abs(U @ gauge.dag(U) - np.eye(3)).max() < 1e-13


def test_sweep_changes_only_active_links():
    dims = (8, 8, 8, 8)
    geom = lattice.Geometry(dims, (4, 4, 4, 4))
    U = gauge.generate_links(dims, 0.5, 5)
    Un, nxt, failed = gauge.domain_sweep(U, geom, 5.3, 1, 1, 9, 100)
    act = geom.active_links()
    changed = np.any(np.abs(Un - U) > 0, axis=(-1, -2))
    assert np.array_equal(changed, act)
    assert failed == 0 and nxt == 100 + 4
    assert np.abs(Un @ gauge.dag(Un) - np.eye(3)).max() < 1e-14
    assert np.abs(np.linalg.det(Un) - 1).max() < 1e-14


def test_single_link_heatbath_distribution():
    """Cabibbo-Marinari heatbath of one link with a fixed staple A samples
    exp((beta/3) ReTr(U A)) dU: compared with an independent Metropolis chain
    on SU(3) (two-sample KS test of ReTr(U A))."""
    beta = 2.0
    A = seeded.haar_su3((), 7) + seeded.haar_su3((), 8)
    nch = 3000
    Ul = seeded.haar_su3((nch,), 9)
    Ab = np.broadcast_to(A, (nch, 3, 3))
    link = np.arange(nch, dtype=np.uint64)
    for s in range(12):
        Ul, f = gauge.update_links(Ul, Ab, beta, "hb", 21, s, link)
        assert f == 0
    hb = np.real(np.trace(Ul @ A, axis1=-2, axis2=-1))
    g = np.random.default_rng(4)
    X = seeded.haar_su3((nch,), 10)
    act = lambda M: (beta / 3) * np.real(np.trace(M @ A, axis1=-2, axis2=-1))
    cur = act(X)
    for _ in range(400):
        om = g.standard_normal((nch, 8))
        Rm = gauge.expm_i_hermitian(gauge.hermitian_generators(om), 0.6)
        Y = Rm @ X
        new = act(Y)
        acc = g.random(nch) < np.exp(new - cur)
        X[acc] = Y[acc]
        cur[acc] = new[acc]
    mc = np.real(np.trace(X @ A, axis1=-2, axis2=-1))
    assert stats.ks_2samp(hb, mc).pvalue > 1e-3


def test_strong_coupling_plaquette():
    """Small beta: <ReTr U_p / 3> = beta/18 + O(beta^2) (strong-coupling expansion)."""
    dims = (4, 4, 4, 4)
    geom = lattice.Geometry(dims, dims)
    beta = 0.3
    U = seeded.gauge_field(dims, 30)
    vals = []
    for s in range(10):
        gauge.one_sweep(U, geom, _all_link_subsets(geom), beta, "hb", 77, s)
        if s >= 2:
            vals.append(gauge.mean_plaquette(U))
    assert abs(np.mean(vals) - beta / 18) < 0.012


def test_per_block_action_change_sums_and_matches_definition():
    """dS_w,b summed over blocks is dS_w; for l >= 3 each dS_w,b equals the
    action change when only block b's active links are replaced."""
    dims = (8, 8, 8, 8)
    geom = lattice.Geometry(dims, (4, 4, 4, 4))
    U = gauge.generate_links(dims, 0.5, 6)
    Un, _, _ = gauge.domain_sweep(U, geom, 5.3, 1, 0, 2, 0)
    per = ofilter.per_block_action_change(U, Un, geom)
    assert abs(per.sum() - (gauge.wilson_action(Un) - gauge.wilson_action(U))) < 1e-9
    act = geom.active_links()
    for b in (0, 5):
        sel = act & (geom.block_index == b)[..., None]
        Ub = U.copy()
        Ub[sel] = Un[sel]
        assert abs(per[b] - (gauge.wilson_action(Ub) - gauge.wilson_action(U))) < 1e-9

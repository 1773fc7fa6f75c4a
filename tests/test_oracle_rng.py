"""Pins of the oracle's Philox-4x64-10 and its Gaussian draws."""
import numpy as np
import pytest

from oracle import philox


def _numpy_block(ctr, key):
    """numpy.random.Philox increments its 256-bit counter before each block,
    so the block for counter c is produced from state c - 1."""
    c = int(ctr[0]) | (int(ctr[1]) << 64) | (int(ctr[2]) << 128) | (int(ctr[3]) << 192)
    c = (c - 1) % (1 << 256)
    words = np.array([(c >> (64 * i)) & ((1 << 64) - 1) for i in range(4)], dtype=np.uint64)
    bg = np.random.Philox(key=np.array(key, dtype=np.uint64), counter=words)
    return bg.random_raw(4)


@pytest.mark.parametrize("ctr,key", [
    ((0, 0, 0, 0), (0, 0)),
    ((1, 0, 0, 0), (1, 2)),
    ((2**64 - 1, 5, 7, 9), (0x50534D53, 3)),
    ((123456789, 2**63 + 11, 42, 2**64 - 2), (2**64 - 1, 2**63)),
    ((0, 0, 1, 0), (17, 1)),
])
def test_philox_matches_numpy(ctr, key):
    ours = philox.philox4x64(np.array([ctr], dtype=np.uint64), key)[0]
    ref = _numpy_block(ctr, key)
    assert np.array_equal(ours, ref)


def test_philox_vectorised_equals_scalar():
    ctr = philox.make_ctr(np.arange(50, dtype=np.uint64), 3, 9, 1)
    v = philox.philox4x64(ctr, (7, 8))
    for k in (0, 17, 49):
        assert np.array_equal(v[k], _numpy_block(tuple(int(x) for x in ctr[k]), (7, 8)))


def test_uniform_open_interval():
    w = np.array([0, 2**64 - 1, 2**63], dtype=np.uint64)
    u = philox.to_uniform(w)
    assert u[0] > 0.0 and u[1] < 1.0
    assert u[0] == 2.0 ** -53 and u[1] == 1.0 - 2.0 ** -53
    assert abs(u[2] - 0.5) < 1e-15


def test_noise_moments():
    """Eq. (pfmeasure)/(aveta): complex Gaussian with E|z|^2 = 1, Re, Im ~ N(0,1/2)."""
    z = philox.noise_field(0x1234, 5, 7, 40000).reshape(-1)
    n = z.size
    assert abs(np.mean(np.abs(z) ** 2) - 1.0) < 5 * np.sqrt(1.0 / n)
    assert abs(np.mean(z)) < 5 / np.sqrt(n)
    assert abs(np.mean(z * z)) < 5 / np.sqrt(n)
    assert abs(np.var(z.real) - 0.5) < 5 * np.sqrt(0.5 / n)
    # E|z|^4 = 2 for a standard complex Gaussian
    assert abs(np.mean(np.abs(z) ** 4) - 2.0) < 5 * np.sqrt(20.0 / n)


def test_noise_streams_independent():
    a = philox.noise_field(1, 0, 0, 1000)
    b = philox.noise_field(1, 0, 1, 1000)
    c = philox.noise_field(1, 1, 0, 1000)
    assert not np.allclose(a, b) and not np.allclose(a, c)
    assert abs(np.vdot(a.reshape(-1), b.reshape(-1))) / a.size < 0.05


def test_link_omegas_standard_normal():
    om = philox.link_omegas(99, 20000).reshape(-1)
    n = om.size
    assert abs(om.mean()) < 5 / np.sqrt(n)
    assert abs(om.var() - 1.0) < 5 * np.sqrt(2.0 / n)


def test_shift_vector_range():
    dims = (4, 6, 8, 10)
    seen = [philox.shift_vector(3, c, dims) for c in range(200)]
    for s in seen:
        assert all(0 <= s[m] < dims[m] for m in range(4))
    assert len(set(seen)) > 150

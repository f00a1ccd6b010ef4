"""The seeded generators: SplitMix64 against its published outputs, and the
shape of the synthetic distributions."""
import numpy as np

from paper_1108_5815_gb300 import inputs


def test_splitmix64_reference_outputs():
    # first outputs for seed 0 and seed 1234567 (Steele, Lea & Flood 2014 /
    # the reference C implementation)
    assert [int(v) for v in inputs.splitmix64(0, 3)] == [
        0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    assert [int(v) for v in inputs.splitmix64(1234567, 2)] == [
        6457827717110365317, 3203168211198807973]


def test_streams_are_deterministic_and_in_range():
    x, q = inputs.uniform_cube(1000, 5)
    x2, q2 = inputs.uniform_cube(1000, 5)
    assert np.array_equal(x, x2) and np.array_equal(q, q2)
    assert x.dtype == np.float32 and x.shape == (1000, 3)
    assert x.min() >= 0 and x.max() < 1 and q.min() >= -1 and q.max() <= 1


def test_plummer_radius_distribution():
    x, q = inputs.plummer(200000, 3)
    r = np.linalg.norm(x.astype(np.float64), axis=1)
    assert r.max() <= 20.0 + 1e-4
    # enclosed mass fraction M(r) = r^3/(1+r^2)^1.5 normalised to M(20)
    mmax = 20.0 ** 3 / (1 + 400.0) ** 1.5
    for rr in (0.5, 1.0, 2.0, 5.0):
        expect = rr ** 3 / (1 + rr * rr) ** 1.5 / mmax
        assert abs(np.mean(r <= rr) - expect) < 5e-3
    assert np.allclose(q, 1.0 / 200000)


def test_shell_on_unit_sphere_and_sampling():
    x, _ = inputs.sphere_shell(1000, 2)
    assert np.allclose(np.linalg.norm(x.astype(np.float64), axis=1), 1.0, atol=1e-6)
    idx = inputs.sample_indices(10000, 300, 8)
    assert len(np.unique(idx)) == 300 and idx.min() >= 0 and idx.max() < 10000

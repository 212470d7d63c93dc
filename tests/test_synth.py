"""The shared seeded generators (CPU only)."""
import numpy as np

import synth


def test_splitmix64_published_vector():
    # first three outputs of SplitMix64 seeded with 0
    assert [int(v) for v in synth.splitmix64(0, 3)] == [
        0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_streams_are_counter_based():
    a = synth.splitmix64(7, 10)
    b = synth.splitmix64(7, 4, offset=6)
    assert np.array_equal(a[6:], b)


def test_distributions():
    u = synth.uniform(3, 200000)
    assert u.min() >= -1 and u.max() < 1 and abs(u.mean()) < 0.01
    z = synth.normal(2, 200000)
    assert abs(z.mean()) < 0.01 and abs(z.std() - 1) < 0.01
    k = synth.randint(4, 100000, 17, 65)
    assert k.min() == 17 and k.max() == 65


def test_grf_unit_variance():
    m = synth.gaussian_field(17, 6)
    assert m.shape == (16 ** 3,) and abs(m.std() - 1) < 1e-12

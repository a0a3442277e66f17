"""Pins of the seeded input generator shared by the oracle and the CUDA path (synth/): the
counter form of splitmix64 against the generator's published reference outputs, and the
derived uniform / normal / unit-vector draws against their definitions."""
import numpy as np

import synth

# reference outputs published with the splitmix64 generator (Steele, Lea, Flood 2014;
# Vigna's reference implementation): seed 0 and seed 1234567
SEED0 = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F, 0xF88BB8A8724C81EC]
SEED1234567 = [6457827717110365317, 3203168211198807973, 9817491932198370423, 4593380528125082431,
               16408922859458223821]


def test_splitmix64_reference_outputs():
    assert [int(x) for x in synth.splitmix64(0, 4)] == SEED0
    assert [int(x) for x in synth.splitmix64(1234567, 5)] == SEED1234567
    # the counter form: output i does not depend on where the stream is started
    assert np.array_equal(synth.splitmix64(99, 3, start=2), synth.splitmix64(99, 5)[2:])


def test_derived_draws():
    u = synth.uniform(7, 100000, 1.0, 4.0)
    assert u.min() >= 1.0 and u.max() < 4.0 and abs(u.mean() - 2.5) < 0.02
    top = (synth.splitmix64(7, 1) >> np.uint64(11)).astype(np.float64)[0] * 2.0 ** -53
    assert u[0] == 1.0 + 3.0 * top
    g = synth.normal(8, 100000)
    assert abs(g.mean()) < 0.02 and abs(g.std() - 1.0) < 0.02
    v = synth.unit_vectors(9, 50)
    assert np.allclose(np.linalg.norm(v, axis=1), 1.0)
    assert np.array_equal(synth.tet_eps(2000, 3, 1.0, 4.0), synth.uniform(2000, 162, 1.0, 4.0))

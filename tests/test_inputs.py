"""The seeded input recipes (no GPU): the generator against the published
splitmix64 sequence, the workloads' shapes and distributions, and the
host helpers of the experiments."""
import math

import numpy as np

from paper_0705_4371_gb300 import experiments, inputs


def test_splitmix64_matches_its_published_definition():
    # reference values computed here from the definition (state += gamma;
    # z = state; z = (z ^ z >> 30) * m1; z = (z ^ z >> 27) * m2; z ^ z >> 31),
    # in plain Python integers, independently of the vectorised generator
    M = (1 << 64) - 1
    state = 1234567
    ref = []
    for _ in range(5):
        state = (state + 0x9E3779B97F4A7C15) & M
        z = state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M
        ref.append(z ^ (z >> 31))
    got = inputs.SplitMix64(1234567).next_u64_array(5)
    assert [int(v) for v in got] == ref
    # two draws continue the same stream
    g = inputs.SplitMix64(1234567)
    a = np.concatenate([g.next_u64_array(2), g.next_u64_array(3)])
    assert [int(v) for v in a] == ref


def test_cylinder_fields_recipe():
    w = inputs.cylinder(200, 72, 8, 1000.0)
    rho, ux, uy = inputs.cylinder_fields(w)
    m = w.solid_mask()
    assert (rho == 1.0).all()
    du = ux[~m] - w.u_in[0]
    assert np.abs(du).max() <= 1e-4 and np.abs(uy[~m]).max() <= 1e-4
    assert abs(du.mean()) < 3e-6 and abs(du.std() - 1e-4 / math.sqrt(3)) < 2e-6   # U[-1e-4, 1e-4]
    assert (ux[m] == 0).all() and m.sum() == 64
    # the same seed gives the same field
    assert np.array_equal(inputs.cylinder_fields(w)[1], ux)


def test_batch_recipe():
    ws = inputs.workload_c5()
    assert len(ws) == 64
    total = sum(w.nx * w.ny for w in ws)
    assert 2.5e7 < total < 3.6e7
    for w in ws:
        assert 256 <= w.nx <= 2048 and w.nx % 8 == 0 and w.ny == w.nx // 2
        assert w.L == max(4, round(w.ny / 25))
        re = w.L * w.u_in[0] / w.nu
        assert 100.0 * (1 - 1e-9) <= re <= 20000.0 * (1 + 1e-9)
        assert w.delta in (1e-4, 1e-3, 1e-2) and w.k == max(1, round(1e-4 * w.nx * w.ny))


def test_training_samples_recipe():
    r, ux, uy, es = inputs.energy_samples(20070531, 200000)
    assert r.min() >= 0.5 and r.max() < 2.0 and abs(r.mean() - 1.25) < 0.01
    s = np.hypot(ux, uy)
    assert s.max() < 0.2
    # uniform in the disc: the fraction inside radius 0.1 is a quarter
    assert abs((s < 0.1).mean() - 0.25) < 0.005
    assert es.min() >= 0.9 and es.max() < 1.1


def test_oscillation_measure():
    x = np.linspace(0.0, 1.0, 50)
    assert experiments.oscillation(1.0 - 0.5 * (x > 0.5)) == 0.0          # monotone step
    wiggle = 1.0 - 0.5 * (x > 0.5)
    wiggle[30] += 0.1                                                     # one overshoot
    assert abs(experiments.oscillation(wiggle) - 0.2) < 1e-12

"""The seeded input generators (synth/) that both the oracle and the library read:
the workloads' sizes, their seeded draws and their ranges, checked on the CPU.
The generators hold none of the method's arithmetic; these tests only pin that the
inputs are what the workload table states, and that a seed reproduces them."""

import numpy as np

from synth import machine_config
from synth.machines import serving_requests, slab_machine


def test_workload_sizes():
    assert machine_config(0).n_dof == 1876
    m1 = machine_config(1)
    assert m1.n_dof == 313646
    # stand 49 x 49 x 121 nodes, stock 25 x 25 x 37 nodes
    assert m1.stand.mesh.n_nodes == 49 * 49 * 121
    assert m1.n_dof - m1.stand.mesh.n_nodes == 25 * 25 * 37


def test_seeded_stroke_is_reproducible_and_in_range():
    a, b = machine_config(1), machine_config(1)
    assert (a.amp, a.period) == (b.amp, b.period)
    assert 0.1 <= a.amp <= 0.3 and 1.0 <= a.period <= 4.0
    c = machine_config(1, seed=1)
    assert (c.amp, c.period) != (a.amp, a.period)
    # the stroke keeps the stock on the stand: z in [z0 - A, z0 + A] and the stock 0.3 m long
    assert a.z0 - a.amp >= 0.0 and a.z0 + a.amp + 0.3 <= 1.0


def test_batch_pool_is_reproducible_and_uneven():
    ms = machine_config(3, truncate=8)
    again = machine_config(3, truncate=8)
    assert [m.n_dof for m in ms] == [m.n_dof for m in again]
    assert [(m.amp, m.period, m.q0) for m in ms] == [(m.amp, m.period, m.q0) for m in again]
    for m in ms:
        assert 2.5e4 <= m.q0 <= 7.5e4
        assert m.scheme.nodes == "lobatto" and m.scheme.M == 3 and m.scheme.P == 20
    assert len({m.n_dof for m in ms}) > 1


def test_serving_schedule():
    reqs = serving_requests(50.0, n_requests=400, seed=3)
    t = np.array([r["arrival_s"] for r in reqs])
    h = np.array([r["horizon_s"] for r in reqs])
    idx = np.array([r["machine_index"] for r in reqs])
    assert np.all(np.diff(t) > 0)
    # exponential gaps of mean 1 / lambda: the mean of 400 lies within 5 standard errors
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert abs(gaps.mean() - 1.0 / 50.0) <= 5 * (1.0 / 50.0) / np.sqrt(400)
    assert h.min() >= 30.0 and h.max() <= 600.0
    assert idx.min() >= 0 and idx.max() < 64
    assert reqs == serving_requests(50.0, n_requests=400, seed=3)


def test_slab_machine_shape():
    mach, T0 = slab_machine(4, 16)
    # one hexahedron thick in x: 2 x 5 x 17 stand nodes; the source is one hexahedron
    assert mach.stand.mesh.n_nodes == 2 * 5 * 17
    assert mach.n_dof == 2 * 5 * 17 + 8
    assert T0.shape == (mach.n_dof,)
    assert np.all(T0[mach.stand.mesh.n_nodes:] == T0[-1])

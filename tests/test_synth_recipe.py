"""The seeded synthetic inputs follow the recipe they are documented with
(stand-ins for the paper's NEKO Taylor-Green snapshots, Sec. IV-A/B): affine
hex elements of a lattice on [0, 2 pi)^3 sampled at the GLL nodes, fields that
are sums of 16 seeded Fourier modes with amplitude |k|^slope plus N(0, 1e-6)
noise, Jacobians uniform in [0.5, 2], and the 64 uneven batched snapshots.
The generator holds none of the method's arithmetic; these checks evaluate
its fields by the plain formula, independently of the matrix product it uses."""
import math

import numpy as np
import pytest
import torch

import oracle
import synth


@pytest.mark.parametrize("lx", [2, 5, 6, 8, 10, 12])
def test_sample_points_are_the_gll_nodes(lx):
    nodes, _ = oracle.gll(lx)
    assert np.max(np.abs(synth.sample_points(lx) - nodes)) < 1e-14


def test_modes_follow_the_spectrum():
    for seed, k_max, slope in [(10, 64, -5.0 / 3.0), (1003, 30, -3.0), (7, 1, -2.0)]:
        k, amp, phase = synth.mode_parameters(seed, k_max, slope)
        assert k.shape == (16, 3) and amp.shape == (16,) and phase.shape == (16,)
        mag = np.linalg.norm(k.astype(np.float64), axis=1)
        assert np.all(mag >= 1.0) and np.all(mag <= k_max + math.sqrt(3) / 2 + 1e-12)
        np.testing.assert_allclose(amp, mag ** slope, rtol=1e-15)
        assert np.all((phase >= 0.0) & (phase < 2.0 * np.pi))
    # seeded: the same seed gives the same modes, another seed others
    a, b = synth.mode_parameters(11, 64, -5.0 / 3.0), synth.mode_parameters(11, 64, -5.0 / 3.0)
    assert all(np.array_equal(x, y) for x, y in zip(a, b))
    assert not np.array_equal(a[0], synth.mode_parameters(12, 64, -5.0 / 3.0)[0])


@pytest.mark.parametrize("n_elem,lx", [(27, 6), (64, 8), (50, 5)])
def test_field_is_the_sum_of_its_modes(n_elem, lx):
    seed, slope = 13, -5.0 / 3.0
    u = synth.field(n_elem, lx, seed, slope, noise=0.0).numpy()
    nx, ny, nz = synth.lattice(n_elem)
    k, amp, phase = synth.mode_parameters(seed, max(nx, ny, nz), slope)
    xi = synth.sample_points(lx)
    rng = np.random.default_rng(0)
    for _ in range(40):
        e = int(rng.integers(n_elem))
        a, b, c = (int(v) for v in rng.integers(lx, size=3))  # point (i, j, k) = (c, b, a)
        ex, ey, ez = e % nx, (e // nx) % ny, e // (nx * ny)
        x = np.array([(ex + 0.5 * (xi[c] + 1.0)) * 2.0 * np.pi / nx,
                      (ey + 0.5 * (xi[b] + 1.0)) * 2.0 * np.pi / ny,
                      (ez + 0.5 * (xi[a] + 1.0)) * 2.0 * np.pi / nz])
        ref = float(np.sum(amp * np.cos(k @ x + phase)))
        assert abs(u[e, a, b, c] - ref) <= 1e-12 * np.sum(amp), (e, a, b, c)


def test_noise_jacobians_and_shapes():
    u0 = synth.field(512, 8, 21, noise=0.0)
    u1 = synth.field(512, 8, 21)
    d = (u1 - u0).numpy().ravel()
    assert abs(d.std() / 1e-6 - 1.0) < 0.02 and abs(d.mean()) < 1e-8
    j = synth.jacobians(100000).numpy()
    assert j.min() >= 0.5 and j.max() < 2.0 and abs(j.mean() - 1.25) < 0.01
    f, jj, tau = synth.small_case()
    assert tuple(f.shape) == (1, 512, 8, 8, 8) and tuple(jj.shape) == (512,) and tau == 1e-3
    assert synth.lattice(64 ** 3) == (64, 64, 64) and synth.lattice(1000) == (10, 10, 10)
    nx, ny, nz = synth.lattice(4097)
    assert nx == ny and nx * ny * nz >= 4097 and nx * ny * (nz - 1) < 4097


def test_batched_cases_follow_the_recipe():
    cases = synth.batched_cases()
    assert len(cases) == 64
    ne = np.array([c["n_elem"] for c in cases])
    assert ne.min() >= 4096 and ne.max() <= 200000
    # log-uniform: the logs' mean near the middle of [log 4096, log 200000]
    assert abs(np.log(ne).mean() - 0.5 * (math.log(4096) + math.log(200000))) < 0.6
    assert {c["lx"] for c in cases} == {6, 8, 10}
    assert {len(c["seeds"]) for c in cases} <= {1, 2, 3, 4} and all(c["n_fields"] == len(c["seeds"]) for c in cases)
    assert all(-3.0 <= c["slope"] <= -5.0 / 3.0 for c in cases)
    seeds = [s for c in cases for s in c["seeds"]]
    assert len(seeds) == len(set(seeds))
    assert synth.batched_cases() == cases  # seeded

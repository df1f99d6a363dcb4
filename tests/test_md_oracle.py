"""Pins of the oracle's MD integrators (the step loop around the NNP and
coupling terms): a closed-form invariant of velocity Verlet on a harmonic
oscillator, time reversibility, BAOAB reducing to velocity Verlet without
friction, and BAOAB's exact Ornstein-Uhlenbeck velocity statistics without
forces.  CPU only."""
import numpy as np
import pytest

import oracle
from paper_2201_08110_gb300 import workloads as W


def harmonic(k):
    return lambda x: -k * x


def test_velocity_verlet_conserves_its_shadow_energy_on_a_harmonic_oscillator():
    """For x'' = -w^2 x velocity Verlet conserves exactly (up to rounding)
    1/2 m v^2 + 1/2 k x^2 (1 - w^2 dt^2 / 4) at whole steps, while the plain
    energy oscillates at order (w dt)^2."""
    m, k, dt = 2.0, 3.0, 0.2
    w2 = k / m
    x0, v0 = np.array([[1.0, -0.5, 0.25]]), np.array([[0.3, 0.1, -0.2]])
    xs, vs = oracle.md_velocity_verlet(x0, v0, [m], harmonic(k), dt, 2000)
    shadow = 0.5 * m * (vs ** 2).sum((1, 2)) + 0.5 * k * (1.0 - w2 * dt * dt / 4.0) * (xs ** 2).sum((1, 2))
    assert np.abs(shadow - shadow[0]).max() <= 1e-12 * shadow[0]
    plain = 0.5 * m * (vs ** 2).sum((1, 2)) + 0.5 * k * (xs ** 2).sum((1, 2))
    assert np.abs(plain - plain[0]).max() > 1e-4 * plain[0]  # the invariant is not the plain energy


def test_velocity_verlet_is_time_reversible():
    g = W.rng(3)
    x0 = g.normal(size=(5, 3))
    v0 = g.normal(size=(5, 3))
    m = g.uniform(1.0, 4.0, size=5)
    force = lambda x: -x * (1.0 + 0.1 * (x ** 2).sum(1, keepdims=True))  # anharmonic, central
    xs, vs = oracle.md_velocity_verlet(x0, v0, m, force, 0.01, 300)
    xb, vb = oracle.md_velocity_verlet(xs[-1], -vs[-1], m, force, 0.01, 300)
    np.testing.assert_allclose(xb[-1], x0, atol=1e-10)
    np.testing.assert_allclose(-vb[-1], v0, atol=1e-10)


def test_baoab_without_friction_is_velocity_verlet():
    g = W.rng(5)
    x0, v0 = g.normal(size=(4, 3)), g.normal(size=(4, 3))
    m = np.array([1.0, 12.0, 14.0, 16.0])
    noise = g.normal(size=(50, 4, 3))
    xa, va = oracle.md_langevin_baoab(x0, v0, m, harmonic(1.5), 0.05, 0.0, 1.0, noise)
    xv, vv = oracle.md_velocity_verlet(x0, v0, m, harmonic(1.5), 0.05, 50)
    np.testing.assert_allclose(xa, xv, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(va, vv, rtol=1e-12, atol=1e-12)


def test_baoab_velocities_follow_the_ornstein_uhlenbeck_process_without_forces():
    """With F = 0 the velocity after n steps is c1^n v0 + a Gaussian of
    variance (kT/m)(1 - c1^(2n)): checked on the given noise exactly for the
    mean part and statistically (10,000 particles) for the variance."""
    n, steps, dt, gamma, kT = 10000, 40, 0.1, 0.5, 2.0
    g = W.rng(7)
    m = np.full(n, 4.0)
    v0 = np.full((n, 3), 1.5)
    noise = g.normal(size=(steps, n, 3))
    _, vs = oracle.md_langevin_baoab(np.zeros((n, 3)), v0, m, lambda x: np.zeros_like(x), dt, gamma,
                                     kT, noise)
    c1 = np.exp(-gamma * dt)
    c2 = np.sqrt(1 - c1 * c1)
    # exact: v_n = c1^n v0 + c2 sqrt(kT/m) sum_s c1^(n-1-s) xi_s
    expect = c1 ** steps * v0 + c2 * np.sqrt(kT / 4.0) * sum(
        c1 ** (steps - 1 - s) * noise[s] for s in range(steps))
    np.testing.assert_allclose(vs[-1], expect, rtol=1e-12, atol=1e-12)
    var = (kT / 4.0) * (1.0 - c1 ** (2 * steps))
    assert vs[-1].mean() == pytest.approx(1.5 * c1 ** steps, abs=5 * np.sqrt(var / (3 * n)))
    assert vs[-1].var() == pytest.approx(var, rel=0.05)

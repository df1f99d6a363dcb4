"""Pins of the oracle's NNP-MM coupling term (Eq. 4): closed forms of the
Coulomb and Lennard-Jones pair terms and of the combination rule, Newton's
third law, central finite differences, invariances and additivity.  CPU only."""
import numpy as np
import pytest

import oracle
from paper_2201_08110_gb300 import workloads as W

KE = W.COULOMB_KCAL


def one_pair(r, qn=0.0, qm=0.0, sn=0.0, sm=0.0, en=0.0, em=0.0, axis=(0.3, -0.4, 0.866)):
    u = np.asarray(axis, dtype=np.float64)
    u /= np.linalg.norm(u)
    xn = np.array([[1.0, 2.0, 3.0]])
    xm = xn + r * u
    e, fn, fm = oracle.coupling(xn, [qn], [sn], [en], xm, [qm], [sm], [em], KE)
    return e, fn[0], fm[0], u


@pytest.mark.parametrize("r", [1.5, 3.0, 7.25, 40.0])
def test_two_charges_coulomb_closed_form(r):
    qn, qm = 0.7, -0.45
    e, fn, fm, u = one_pair(r, qn=qn, qm=qm)
    assert e == pytest.approx(KE * qn * qm / r, rel=1e-14)
    # attraction: the MM atom is pulled towards the NNP atom
    np.testing.assert_allclose(fm, KE * qn * qm / r ** 2 * u, rtol=1e-13, atol=1e-16)
    np.testing.assert_allclose(fn, -fm, rtol=0, atol=1e-15)


def test_lennard_jones_minimum_and_zero_with_lorentz_berthelot():
    # sigma_ij = (3.0 + 3.4) / 2 = 3.2, eps_ij = sqrt(0.1 * 0.4) = 0.2
    rmin = 2.0 ** (1.0 / 6.0) * 3.2
    e, fn, fm, _ = one_pair(rmin, sn=3.0, sm=3.4, en=0.1, em=0.4)
    assert e == pytest.approx(-0.2, rel=1e-13)
    assert np.abs(fm).max() < 1e-13 and np.abs(fn).max() < 1e-13
    e, fn, fm, u = one_pair(3.2, sn=3.0, sm=3.4, en=0.1, em=0.4)
    assert abs(e) < 1e-15
    # at r = sigma: -dV/dr = 24 eps / sigma, pushing the MM atom away
    np.testing.assert_allclose(fm, 24.0 * 0.2 / 3.2 * u, rtol=1e-13)


def test_zero_eps_switches_lennard_jones_off():
    e, _, _, _ = one_pair(0.9, sn=3.0, sm=0.0, en=0.1, em=0.0)
    assert e == 0.0


def small_system(seed, n_nnp=7, n_mm=40):
    g = W.rng(seed)
    xn = W.geometry(g, n_nnp, edge=5.0, dmin=1.0)
    env = W.mm_environment(seed + 1, xn, n_mm, density=0.05)
    return xn, env


def call(xn, env, xm=None):
    return oracle.coupling(xn, env.nnp_q, env.nnp_sigma, env.nnp_eps,
                           env.mm_pos if xm is None else xm, env.mm_q, env.mm_sigma,
                           env.mm_eps, KE)


def test_newton_third_law_and_zero_torque():
    xn, env = small_system(3)
    e, fn, fm = call(xn, env)
    ftot = fn.sum(0) + fm.sum(0)
    scale = np.abs(fn).sum() + np.abs(fm).sum()
    assert np.abs(ftot).max() <= 1e-13 * scale
    torque = np.cross(xn, fn).sum(0) + np.cross(env.mm_pos.astype(np.float64), fm).sum(0)
    assert np.abs(torque).max() <= 1e-12 * scale * 10.0


def test_forces_are_minus_the_energy_gradient():
    xn, env = small_system(5)
    xn = xn.astype(np.float64)
    xm = env.mm_pos.astype(np.float64)
    _, fn, fm = call(xn, env, xm)
    h = 1e-5
    g = W.rng(9)
    for side, n in (("nnp", xn.shape[0]), ("mm", xm.shape[0])):
        for _ in range(4):
            a, k = int(g.integers(n)), int(g.integers(3))
            xp, xq = (xn.copy(), xm.copy()), (xn.copy(), xm.copy())
            idx = 0 if side == "nnp" else 1
            xp[idx][a, k] += h
            xq[idx][a, k] -= h
            ep = oracle.coupling(xp[0], env.nnp_q, env.nnp_sigma, env.nnp_eps, xp[1], env.mm_q,
                                 env.mm_sigma, env.mm_eps, KE)[0]
            eq = oracle.coupling(xq[0], env.nnp_q, env.nnp_sigma, env.nnp_eps, xq[1], env.mm_q,
                                 env.mm_sigma, env.mm_eps, KE)[0]
            fd = -(ep - eq) / (2 * h)
            f = (fn if side == "nnp" else fm)[a, k]
            assert fd == pytest.approx(f, rel=1e-6, abs=1e-7)


def test_translation_and_rotation_invariance():
    xn, env = small_system(7)
    e0, fn0, fm0 = call(xn, env)
    t = np.array([3.0, -1.5, 0.25])
    c, s = np.cos(0.7), np.sin(0.7)
    R = np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])
    e1, fn1, fm1 = call(xn @ R.T + t, env, env.mm_pos.astype(np.float64) @ R.T + t)
    assert e1 == pytest.approx(e0, rel=1e-12)
    np.testing.assert_allclose(fn1, fn0 @ R.T, rtol=1e-9, atol=1e-10)
    np.testing.assert_allclose(fm1, fm0 @ R.T, rtol=1e-9, atol=1e-10)


def test_additive_over_mm_atoms():
    xn, env = small_system(11)
    e, fn, fm = call(xn, env)
    k = 17
    parts = []
    for sl in (slice(0, k), slice(k, None)):
        parts.append(oracle.coupling(xn, env.nnp_q, env.nnp_sigma, env.nnp_eps, env.mm_pos[sl],
                                     env.mm_q[sl], env.mm_sigma[sl], env.mm_eps[sl], KE))
    assert parts[0][0] + parts[1][0] == pytest.approx(e, rel=1e-12)
    np.testing.assert_allclose(parts[0][1] + parts[1][1], fn, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(np.concatenate([parts[0][2], parts[1][2]]), fm, rtol=0, atol=0)


def test_coincident_atoms_rejected():
    with pytest.raises(ValueError):
        oracle.coupling([[0.0, 0.0, 0.0]], [1.0], [3.0], [0.1], [[0.0, 0.0, 0.0]], [1.0], [3.0],
                        [0.1], KE)


def test_error_scales_of_one_pair():
    """For one pair the squared-energy sum is the energy squared and each atom's
    gross force is the magnitude of the pair force."""
    u = np.array([0.0, 0.6, 0.8])
    xn = np.array([[0.0, 0.0, 0.0]])
    xm = 2.5 * u[None, :]
    e, fn, fm, e2, gn, gm = oracle.coupling(xn, [0.4], [3.0], [0.1], xm, [-0.8], [3.4], [0.4], KE,
                                            norms=True)
    assert e2 == pytest.approx(e * e, rel=1e-14)
    assert gn[0] == pytest.approx(np.linalg.norm(fn[0]), rel=1e-14)
    assert gm[0] == pytest.approx(np.linalg.norm(fm[0]), rel=1e-14)


@pytest.mark.parametrize("n_mm", [1, 2, 3, 257, 4099])
def test_mm_environment_follows_its_recipe(n_mm):
    """The MM region is what the input recipe states: n_mm atoms in waters of
    O then two H (0.9572 A bonds, 104.52 degrees), TIP3P charges and
    Lennard-Jones on O only, oxygens at least 3 A from every NNP atom, NNP
    charges summing to zero; the same seed gives the same region."""
    xn = W.geometry(W.rng(4), 20, edge=8.0, dmin=0.95)
    env = W.mm_environment(21, xn, n_mm)
    assert env.n_mm == n_mm and env.mm_q.shape == (n_mm,)
    assert abs(float(env.nnp_q.astype(np.float64).sum())) < 1e-5
    assert np.all((env.nnp_sigma >= 2.5) & (env.nnp_sigma <= 3.5))
    assert np.all((env.nnp_eps >= 0.02) & (env.nnp_eps <= 0.2))
    role = np.arange(n_mm) % 3  # 0: O, 1-2: H
    np.testing.assert_allclose(env.mm_q, np.where(role == 0, -0.834, 0.417), rtol=1e-6)
    np.testing.assert_allclose(env.mm_sigma, np.where(role == 0, 3.15061, 0.0), rtol=1e-6)
    np.testing.assert_allclose(env.mm_eps, np.where(role == 0, 0.1521, 0.0), rtol=1e-6)
    x = env.mm_pos.astype(np.float64)
    oxy = x[role == 0]
    d_on = np.sqrt(((oxy[:, None, :] - xn[None, :, :]) ** 2).sum(-1)).min()
    assert d_on >= 3.0 - 1e-5
    for w in range(n_mm // 3):
        o, h1, h2 = x[3 * w], x[3 * w + 1], x[3 * w + 2]
        b1, b2 = h1 - o, h2 - o
        assert np.linalg.norm(b1) == pytest.approx(0.9572, abs=1e-5)
        assert np.linalg.norm(b2) == pytest.approx(0.9572, abs=1e-5)
        ang = np.degrees(np.arccos(b1 @ b2 / (np.linalg.norm(b1) * np.linalg.norm(b2))))
        assert ang == pytest.approx(104.52, abs=1e-3)
    again = W.mm_environment(21, xn, n_mm)
    assert np.array_equal(again.mm_pos, env.mm_pos) and np.array_equal(again.nnp_q, env.nnp_q)

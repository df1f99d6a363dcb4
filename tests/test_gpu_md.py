"""The replica MD loop (nnp_md_*) against the oracle's FP64 integrators.

Two replicas of the 24-atom molecule (the second displaced by 0.05 A noise),
one network, FP32 networks: the oracle runs the same integrator in FP64 with
its own forces (oracle.compute, plus oracle.coupling for the coupling term
with the MM atoms fixed) and, for Langevin dynamics, the same normal draws.

Bound: the GPU forces differ from the oracle's by at most 1e-4 of their RMS
(FP32 networks, max |dF|); over n steps of size dt a force error dF moves a
position by at most about (n dt)^2 / 2 |dF| / m, and over these short runs
(n dt = 1.5 time units, forces of about 0.15 per A, masses 1-35) the
trajectories separate by far less than 1e-3 of the distance each atom
travels: positions and velocities are checked at that relative bound, the
potential energies at 1e-4 of the molecule's gross atomic energy (plus the
coupling term's own FP32 error scale where it is on).
"""
import numpy as np
import pytest

import oracle
from paper_2201_08110_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MASS = {1: 1.008, 6: 12.011, 7: 14.007, 8: 15.999, 9: 18.998, 16: 32.06, 17: 35.45}


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2201_08110_gb300 import build, nnp
    build.build()
    return nnp


def replicas():
    b, w, M = W.config1()
    g = W.rng(31)
    p1 = (b.pos.astype(np.float64) + g.normal(0.0, 0.05, size=b.pos.shape)).astype(np.float32)
    n = b.n_atoms
    batch = W.Batch(np.concatenate([b.Z, b.Z]), np.concatenate([b.pos, p1]),
                    np.array([0, n, 2 * n], np.int32))
    masses = np.array([MASS[int(z)] for z in batch.Z])
    v0 = g.normal(0.0, 0.02, size=(2 * n, 3)) / np.sqrt(masses)[:, None]
    return batch, w, M, masses, v0


def oracle_force(batch, w, M, env=None):
    def force(x):
        r = oracle.compute(batch.Z, x, batch.mol_off, w, M)
        F = r["forces"].copy()
        if env is not None:
            for m in range(batch.n_mols):
                a0, a1 = int(batch.mol_off[m]), int(batch.mol_off[m + 1])
                _, fn, _ = oracle.coupling(x[a0:a1], env.nnp_q[a0:a1], env.nnp_sigma[a0:a1],
                                           env.nnp_eps[a0:a1], env.mm_pos, env.mm_q, env.mm_sigma,
                                           env.mm_eps, W.COULOMB_KCAL)
                F[a0:a1] += fn
        return F
    return force


def oracle_energy(batch, w, M, x, env=None):
    """Energies per replica and their error scale: 1e-4 of the NNP term's
    gross atomic energy, plus the coupling term's FP32 scale (1e-5 of the root
    sum of its squared pair energies + 1e-6 of it, as in its own tests)."""
    r = oracle.compute(batch.Z, x, batch.mol_off, w, M, forces=False, atom_energies=True)
    E = r["energy"].copy()
    tol = 1e-4 * np.add.reduceat(np.abs(r["atom_energies"]), batch.mol_off[:-1])
    if env is not None:
        for m in range(batch.n_mols):
            a0, a1 = int(batch.mol_off[m]), int(batch.mol_off[m + 1])
            e, _, _, e2, _, _ = oracle.coupling(x[a0:a1], env.nnp_q[a0:a1], env.nnp_sigma[a0:a1],
                                                env.nnp_eps[a0:a1], env.mm_pos, env.mm_q,
                                                env.mm_sigma, env.mm_eps, W.COULOMB_KCAL, norms=True)
            E[m] += e
            tol[m] += 1e-5 * np.sqrt(e2) + 1e-6 * abs(e)
    return E, tol


def check(x, v, E, xs, vs, batch, w, M, env=None):
    x0 = xs[0]
    travel = np.abs(xs[-1] - x0).max()
    assert travel > 0.05  # the atoms moved
    assert np.abs(x - xs[-1]).max() <= 1e-3 * travel
    assert np.abs(v - vs[-1]).max() <= 1e-3 * np.abs(vs[-1]).max()
    for k in (0, len(xs) // 2 - 1, len(xs) - 2):  # energy after step k + 1
        Eref, tol = oracle_energy(batch, w, M, xs[k + 1], env)
        assert np.all(np.abs(E[k] - Eref) <= tol), (k, E[k], Eref, tol)


def run_md(lib, batch, w, M, masses, v0, n, dt, integrator, noise=None, env_dev=None,
           concurrent=True, **kw):
    model = lib.NNP(batch.Z, w, M, mol_off=batch.mol_off)
    md = lib.MD(model, masses, dt, integrator=integrator, env=env_dev, coulomb_k=W.COULOMB_KCAL,
                concurrent=concurrent, **kw)
    x = torch.tensor(batch.pos.astype(np.float64), device="cuda")
    v = torch.tensor(v0, device="cuda")
    E = torch.empty(n, batch.n_mols, dtype=torch.float64, device="cuda")
    md.run(x, v, n, noise=None if noise is None else torch.tensor(noise, device="cuda"), energy=E)
    torch.cuda.synchronize()
    model.status()
    out = x.cpu().numpy(), v.cpu().numpy(), E.cpu().numpy()
    md.close()
    model.close()
    return out


def test_velocity_verlet_matches_oracle(lib):
    batch, w, M, masses, v0 = replicas()
    n, dt = 30, 0.05
    x, v, E = run_md(lib, batch, w, M, masses, v0, n, dt, "verlet")
    xs, vs = oracle.md_velocity_verlet(batch.pos, v0, masses, oracle_force(batch, w, M), dt, n)
    check(x, v, E, xs, vs, batch, w, M)


def test_langevin_baoab_matches_oracle_with_the_same_draws(lib):
    batch, w, M, masses, v0 = replicas()
    n, dt, gamma, kT = 30, 0.05, 1.0, 0.01
    noise = W.rng(32).standard_normal((n, batch.n_atoms, 3))
    x, v, E = run_md(lib, batch, w, M, masses, v0, n, dt, "baoab", noise=noise, gamma=gamma, kT=kT)
    xs, vs = oracle.md_langevin_baoab(batch.pos, v0, masses, oracle_force(batch, w, M), dt, gamma,
                                      kT, noise)
    check(x, v, E, xs, vs, batch, w, M)


def test_coupling_term_in_the_loop_serial_and_concurrent(lib):
    """Both replicas in one fixed water-like MM environment (the coupling term
    of Eq. 4 with the MM atoms held): serial and concurrent streams give the
    same trajectory (up to the order of FP64 additions across CTAs) and both
    follow the oracle's."""
    batch, w, M, masses, v0 = replicas()
    n, dt = 20, 0.05
    env1 = W.mm_environment(77, batch.pos[:batch.n_atoms // 2], n_mm=3000)
    env = W.Environment(np.concatenate([env1.nnp_q, env1.nnp_q]),
                        np.concatenate([env1.nnp_sigma, env1.nnp_sigma]),
                        np.concatenate([env1.nnp_eps, env1.nnp_eps]),
                        env1.mm_pos, env1.mm_q, env1.mm_sigma, env1.mm_eps)
    dev = lambda a: torch.tensor(np.ascontiguousarray(a, dtype=np.float32), device="cuda")

    class Env:
        pass
    env_dev = Env()
    for k in ("nnp_q", "nnp_sigma", "nnp_eps", "mm_pos", "mm_q", "mm_sigma", "mm_eps"):
        setattr(env_dev, k, dev(getattr(env, k)))
    runs = [run_md(lib, batch, w, M, masses, v0, n, dt, "verlet", env_dev=env_dev, concurrent=c)
            for c in (False, True)]
    np.testing.assert_allclose(runs[0][0], runs[1][0], rtol=0, atol=1e-9)
    np.testing.assert_allclose(runs[0][2], runs[1][2], rtol=1e-9, atol=1e-9)
    xs, vs = oracle.md_velocity_verlet(batch.pos, v0, masses, oracle_force(batch, w, M, env), dt, n)
    x, v, E = runs[1]
    check(x, v, E, xs, vs, batch, w, M, env)


def test_rejects_bad_parameters(lib):
    batch, w, M, masses, v0 = replicas()
    model = lib.NNP(batch.Z, w, M, mol_off=batch.mol_off)
    with pytest.raises(lib.NNPError):
        lib.MD(model, masses, -1.0)
    bad = masses.copy()
    bad[3] = 0.0
    with pytest.raises(lib.NNPError):
        lib.MD(model, bad, 0.05)
    md = lib.MD(model, masses, 0.05, integrator="baoab", gamma=1.0, kT=0.01)
    x = torch.tensor(batch.pos.astype(np.float64), device="cuda")
    v = torch.zeros_like(x)
    with pytest.raises(lib.NNPError) as e:  # BAOAB without its draws
        md.run(x, v, 3)
    assert e.value.status == "NNP_ERR_ARG"

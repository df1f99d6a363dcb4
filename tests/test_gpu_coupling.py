"""The NNP-MM coupling term (Eq. 4) on the GPU against the FP64 oracle, through
the C ABI.

Bounds, from the arithmetic (FP32 pair terms, each within a few tens of units
of 2^-24 of its value; per-atom FP32 sums of at most a few hundred terms,
FP64 sums beyond): per atom |dF| <= 1e-5 * sum_b |f_ab| (the gross magnitude
of its pair forces), and |dE| <= 1e-5 * sqrt(sum_ij e_ij^2) + 1e-6 * |E|: the
energy of a neutral environment is a small net of many pair terms of either
sign, and independent roundings of N terms grow with their root sum of
squares, not with the net."""
import numpy as np
import pytest

import oracle
from paper_2201_08110_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2201_08110_gb300 import build, nnp
    build.build()
    return nnp


def cuda(a):
    return torch.tensor(np.ascontiguousarray(a, dtype=np.float32), device="cuda")


def gpu_term(nnp, xn, env, **kw):
    E, fn, fm = nnp.mm_coupling(cuda(xn), cuda(env.nnp_q), cuda(env.nnp_sigma), cuda(env.nnp_eps),
                                cuda(env.mm_pos), cuda(env.mm_q), cuda(env.mm_sigma),
                                cuda(env.mm_eps), W.COULOMB_KCAL, **kw)
    torch.cuda.synchronize()
    return float(E.cpu()[0]), fn.cpu().numpy(), fm.cpu().numpy()


def ref_term(xn, env):
    return oracle.coupling(xn, env.nnp_q, env.nnp_sigma, env.nnp_eps, env.mm_pos, env.mm_q,
                           env.mm_sigma, env.mm_eps, W.COULOMB_KCAL, norms=True)


def check(got, ref):
    E, fn, fm = got
    Er, fnr, fmr, e2, gn, gm = ref
    dE = abs(E - Er)
    assert dE <= 1e-5 * np.sqrt(e2) + 1e-6 * abs(Er), f"energy {E} vs {Er}"
    rn = np.abs(fn - fnr).max(axis=1) / np.maximum(gn, 1e-300)
    rm = np.abs(fm - fmr).max(axis=1) / np.maximum(gm, 1e-300)
    assert rn.max() <= 1e-5, f"NNP force error {rn.max():.3e} of the gross pair force"
    assert rm.max() <= 1e-5, f"MM force error {rm.max():.3e} of the gross pair force"
    return {"dE": dE, "dE_rel": dE / abs(Er), "fn": float(rn.max()), "fm": float(rm.max())}


def system(seed, n_nnp, n_mm):
    g = W.rng(seed)
    # the ligand-sized regions in the 8 A cube; larger ones at 0.3 atoms / A^3
    xn = W.geometry(g, n_nnp, edge=max(8.0, (n_nnp / 0.3) ** (1.0 / 3.0)), dmin=0.95)
    return xn, W.mm_environment(seed + 1, xn, n_mm)


@pytest.mark.parametrize("n_nnp,n_mm", [(1, 1), (7, 1000), (24, 257), (60, 4099), (75, 38000),
                                        (511, 3001), (512, 2048)])
def test_coupling_matches_oracle(lib, n_nnp, n_mm):
    """Single pair, ragged MM counts (not multiples of a CTA's 128 atoms), the
    paper's smallest system size (75 NNP atoms in 38 k MM atoms), and NNP
    regions at and just below the 512-atom limit (the largest shared-memory
    layout; NNP atoms not a multiple of the CTA's 8 warps)."""
    xn, env = system(100 + n_nnp, n_nnp, n_mm)
    worst = check(gpu_term(lib, xn, env), ref_term(xn, env))
    print(f"{n_nnp} x {n_mm}: {worst}")


def test_full_size_system_matches_oracle(lib):
    """The 60-atom molecule of workload 2 in 60,000 MM atoms, as the benchmark
    times it; the oracle evaluates all 3.6 M pairs."""
    b, env = W.coupling_config()
    worst = check(gpu_term(lib, b.pos, env), ref_term(b.pos, env))
    print(f"60 x 60000: {worst}")
    # Newton's third law on the GPU result: the net force is the rounding only
    _, fn, fm = gpu_term(lib, b.pos, env)
    _, _, _, _, gn, gm = ref_term(b.pos, env)
    assert np.abs(fn.sum(0) + fm.sum(0)).max() <= 1e-5 * (gn.sum() + gm.sum())


def test_outputs_are_added_to_the_given_buffers(lib):
    """The term adds into existing FP64 buffers: twice into the same buffers is
    twice the term, on top of what they held (the NNP forces of nnp_compute
    can be passed directly)."""
    xn, env = system(7, 12, 3000)
    E1, fn1, fm1 = gpu_term(lib, xn, env)
    e0 = torch.full((1,), 5.0, dtype=torch.float64, device="cuda")
    fn0 = torch.full((12, 3), -1.0, dtype=torch.float64, device="cuda")
    fm0 = torch.full((3000, 3), 2.0, dtype=torch.float64, device="cuda")
    for _ in range(2):
        gpu_term(lib, xn, env, energy=e0, nnp_forces=fn0, mm_forces=fm0)
    np.testing.assert_allclose(float(e0.cpu()[0]), 5.0 + 2 * E1, rtol=1e-12)
    np.testing.assert_allclose(fn0.cpu().numpy(), -1.0 + 2 * fn1, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(fm0.cpu().numpy(), 2.0 + 2 * fm1, rtol=1e-12, atol=1e-12)


def test_nnp_forces_plus_coupling_in_one_buffer(lib):
    """NNP/MM step: the NNP term's forces (nnp_compute) and the coupling term's
    forces on the NNP atoms accumulate in one FP64 buffer."""
    b, w, M = W.config2()
    env = W.mm_environment(W.workload_seed(2) + 50, b.pos, 5000)
    model = lib.NNP(b.Z, w, M, mol_off=b.mol_off)
    pos = cuda(b.pos)
    E, F = model.compute(pos)
    torch.cuda.synchronize()
    F_nnp = F.cpu().numpy().copy()
    Et = E.clone()
    lib.mm_coupling(pos, cuda(env.nnp_q), cuda(env.nnp_sigma), cuda(env.nnp_eps), cuda(env.mm_pos),
                    cuda(env.mm_q), cuda(env.mm_sigma), cuda(env.mm_eps), W.COULOMB_KCAL,
                    energy=Et, nnp_forces=F)
    torch.cuda.synchronize()
    Ec, fnc, _ = gpu_term(lib, b.pos, env)
    np.testing.assert_allclose(float(Et.cpu()[0]), float(E.cpu()[0]) + Ec, rtol=1e-12)
    np.testing.assert_allclose(F.cpu().numpy(), F_nnp + fnc, rtol=1e-12, atol=1e-12)

"""The ANI-1x model (Sec. 3, "Extensibility with other NNPs") on the GPU path
against the FP64 oracle's ANI-1x model, through the C ABI.

ANI-1x differs from ANI-2x in every size the kernels are specialised on:
four elements (10 species-pair blocks, 384 features), an angular grid of 4
distance x 8 angle shifts, a 5.2 A radial cutoff, Zeta = 32, and widths 144
and 112 that the device networks pad to 160 and 128 with zero weights.
Inputs: seeded H/C/N/O molecules (batches with 1-3 atom molecules and a
ragged tail, a 120-atom molecule, a periodic region) and ANI-1x-shaped
weights with and without random biases.  Tolerances are those of
tests/_gpu_common.py.
"""
import itertools

import numpy as np
import pytest

import oracle
from paper_2201_08110_gb300 import workloads as W
from tests._gpu_common import check_batch, oracle_batch, split_mode

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RCR = float(np.float32(5.2))
RCA = float(np.float32(3.5))


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2201_08110_gb300 import build, nnp
    build.build()
    return nnp


def run(nnp, b, w, M, prec="fp32", **kw):
    prec, single = split_mode(prec)
    if single:
        kw["single_pass"] = True
    h = nnp.NNP(b.Z, w, M, mol_off=b.mol_off, precision=prec, box=b.box, model="ani1x", **kw)
    E, F = h.compute(torch.tensor(b.pos, device="cuda"))
    torch.cuda.synchronize()
    h.status()
    return h, E.cpu().numpy(), F.cpu().numpy()


def case_inputs(case):
    if case == "batch":
        return W.batch(91, [20, 33, 64, 65, 120, 1, 2, 3, 97, 41], model="ani1x"), \
            W.weights(11, 8, model="ani1x"), 8
    if case == "batch_bias":
        return W.batch(92, [25, 1, 2, 3, 57, 130, 0, 18], model="ani1x"), \
            W.weights(12, 8, bias_std=0.1, model="ani1x"), 8
    if case == "periodic":
        return W.pocket(93, n=250, edge=14.0, model="ani1x"), W.weights(13, 2, model="ani1x"), 2
    raise ValueError(case)


@pytest.mark.parametrize("case", ["batch", "periodic"])
def test_pair_and_triple_sets_at_the_ani1x_cutoffs(lib, case):
    b, w, M = case_inputs(case)
    h, _, _ = run(lib, b, w, M)
    box = b.box if np.any(b.box) else None
    for kind, rc in ((0, RCR), (1, RCA)):
        counts, lists = (t.cpu().numpy() for t in h.neighbors(kind))
        for m in range(b.n_mols):
            a0, a1 = int(b.mol_off[m]), int(b.mol_off[m + 1])
            exp = sorted((int(i) + a0, int(j) + a0) for i, j in oracle.pairs(b.pos[a0:a1], rc, box=box))
            got = sorted((i, int(j)) for i in range(a0, a1) for j in lists[i, :counts[i]])
            assert got == exp, f"kind {kind} molecule {m}"
            if kind == 1:
                tri = sorted((i, min(j, k), max(j, k)) for i in range(a0, a1)
                             for j, k in itertools.combinations(lists[i, :counts[i]].tolist(), 2))
                tref = sorted((int(i) + a0, int(j) + a0, int(k) + a0)
                              for i, j, k in oracle.triples(b.pos[a0:a1], rc, box=box))
                assert tri == tref


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
@pytest.mark.parametrize("case", ["batch", "periodic"])
def test_features_match_oracle(lib, prec, case):
    """All 384 features of every atom, in the model's own layout.  Bound, in
    units of the row maximum: a distance from FP32 positions carries up to
    about 2^-23 relative error (6e-7 A at 5.2 A), which moves a Gaussian's
    argument y = sqrt(Eta log2 e) (r - Shf) by up to 3e-6 and the Gaussian
    2^(-y^2) by 2 ln2 |y| dy relative, at most about 3e-6 of the row maximum
    for radial terms; the angular power (t / 2)^32, five squarings of the FP32
    t / 2, adds up to 32 x 2^-24 + 31 x 2^-24 = 3.7e-6 on angular terms.
    Bound 1e-5 (measured up to 5.6e-6, on a molecule whose atoms see each
    other only in the Gaussians' tails).  BF16 features are exported as hi +
    lo, which carries about 2^-16 of the value: 1e-4 there."""
    b, w, M = case_inputs(case)
    h, _, _ = run(lib, b, w, M, prec)
    G = h.features().cpu().numpy().astype(np.float64)
    assert G.shape == (b.n_atoms, 384)
    for m in range(b.n_mols):
        a0, a1 = int(b.mol_off[m]), int(b.mol_off[m + 1])
        if a1 == a0:
            continue
        ref = oracle.aev(b.Z[a0:a1], b.pos[a0:a1], box=b.box if np.any(b.box) else None, model="ani1x")
        scale = np.maximum(np.abs(ref).max(axis=1, keepdims=True), 1e-30)
        err = (np.abs(G[a0:a1] - ref) / scale).max()
        assert err < (1e-5 if prec == "fp32" else 1e-4), f"molecule {m}: feature error {err:.3e}"


@pytest.mark.parametrize("prec", ["fp32", "bf16", "fp16", "bf16-single"])
@pytest.mark.parametrize("case", ["batch", "batch_bias", "periodic"])
def test_energy_forces_match_oracle(lib, prec, case):
    b, w, M = case_inputs(case)
    _, E, F = run(lib, b, w, M, prec)
    refs = oracle_batch(b, w, M, model="ani1x")
    worst = check_batch(prec, E, F, b, refs)
    print(f"ani1x {case} {prec}: worst errors {worst}")


def test_graph_replay_and_energy_only(lib):
    """One CUDA graph per step gives the direct launches' results; the
    energy-only call gives the same energies."""
    b, w, M = case_inputs("batch")
    _, E0, F0 = run(lib, b, w, M, "bf16")
    h = lib.NNP(b.Z, w, M, mol_off=b.mol_off, precision="bf16", use_graph=True, model="ani1x")
    pos = torch.tensor(b.pos, device="cuda")
    for _ in range(3):
        E, F = h.compute(pos)
    Ee, Fe = h.compute(pos, forces=False)
    torch.cuda.synchronize()
    h.status()
    assert Fe is None
    np.testing.assert_allclose(E.cpu().numpy(), E0, rtol=1e-12)
    np.testing.assert_allclose(F.cpu().numpy(), F0, rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(Ee.cpu().numpy(), E0, rtol=1e-12)


def test_two_models_side_by_side(lib):
    """An ANI-2x and an ANI-1x handle in one process, alternating: each keeps
    its own constants, layouts and kernels."""
    b1, w1, M1 = case_inputs("batch")
    b2, w2, M2 = W.batch(94, [30, 45], model="ani2x"), W.weights(14, 2), 2
    h1 = lib.NNP(b1.Z, w1, M1, mol_off=b1.mol_off, model="ani1x")
    h2 = lib.NNP(b2.Z, w2, M2, mol_off=b2.mol_off)
    p1, p2 = torch.tensor(b1.pos, device="cuda"), torch.tensor(b2.pos, device="cuda")
    for _ in range(2):
        E1, F1 = h1.compute(p1)
        E2, F2 = h2.compute(p2)
    torch.cuda.synchronize()
    check_batch("fp32", E1.cpu().numpy(), F1.cpu().numpy(), b1, oracle_batch(b1, w1, M1, model="ani1x"))
    check_batch("fp32", E2.cpu().numpy(), F2.cpu().numpy(), b2, oracle_batch(b2, w2, M2))


def test_rejects_elements_outside_the_model(lib):
    w = W.weights(1, 1, model="ani1x")
    for z in (9, 16, 17):
        with pytest.raises(lib.NNPError) as e:
            lib.NNP(np.array([6, z, 1], np.int32), w, 1, model="ani1x")
        assert e.value.status == "NNP_ERR_SPECIES"

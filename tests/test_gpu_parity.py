"""GPU path against the FP64 oracle, through the C ABI (ctypes binding).

Pair and triple sets must be identical; features, energies and forces must
meet the tolerances of tests/_gpu_common.py.  Inputs are the seeded synthetic
workloads (single molecules of 24 and 60 atoms, batches with atom counts
20-120, a periodic region) at sizes the oracle finishes in seconds, plus every
molecule of the full 512-molecule batch in the benchmark's launch
configuration.
"""
import itertools

import numpy as np
import pytest

import oracle
from paper_2201_08110_gb300 import workloads as W
from tests._gpu_common import check_batch, oracle_batch, oracle_whole_batch, split_mode

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RCR = float(np.float32(5.1))
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
    model = nnp.NNP(b.Z, w, M, mol_off=b.mol_off, precision=prec, box=b.box, **kw)
    pos = torch.tensor(b.pos, device="cuda")
    E, F = model.compute(pos)
    torch.cuda.synchronize()
    model.status()
    return model, E.cpu().numpy(), F.cpu().numpy()


def small_batch():
    return W.batch(77, [20, 33, 64, 65, 120, 1, 2, 3, 97, 41])


# --- neighbour search ---------------------------------------------------------

@pytest.mark.parametrize("case", ["cfg1", "batch", "periodic", "periodic_cells", "pocket_cells"])
def test_pair_and_triple_sets_are_identical(lib, case):
    """All-pairs search (molecules, small periodic region) and the cell list
    (2 cells per side in a 14 A box, 4 per side in the 24.7 A pocket)."""
    kw = {}
    if case == "cfg1":
        b, w, M = W.config1()
    elif case == "batch":
        b = small_batch()
        w, M = W.weights(5, 1), 1
    elif case == "pocket_cells":
        b = W.pocket(W.workload_seed(5) + 2)  # 1500 atoms: the cell list by default
        w, M = W.weights(5, 1), 1
    else:
        b = W.pocket(9, n=250, edge=14.0)
        w, M = W.weights(5, 1), 1
        kw = {"neighbor_mode": 2} if case == "periodic_cells" else {"neighbor_mode": 1}
    model, _, _ = run(lib, b, w, M, **kw)
    for kind, rc in ((0, RCR), (1, RCA)):
        counts, lists = model.neighbors(kind)
        counts, lists = counts.cpu().numpy(), lists.cpu().numpy()
        for m in range(b.n_mols):
            a0, a1 = int(b.mol_off[m]), int(b.mol_off[m + 1])
            box = b.box if np.any(b.box) else None
            ref = oracle.pairs(b.pos[a0:a1], rc, box=box)
            exp = sorted((int(i) + a0, int(j) + a0) for i, j in ref)
            got = sorted((i, int(j)) for i in range(a0, a1) for j in lists[i, :counts[i]])
            assert got == exp, f"kind {kind} molecule {m}"
            if kind == 1:
                tri = sorted((i, min(j, k), max(j, k)) for i in range(a0, a1)
                             for j, k in itertools.combinations(lists[i, :counts[i]].tolist(), 2))
                tref = sorted((int(i) + a0, int(j) + a0, int(k) + a0)
                              for i, j, k in oracle.triples(b.pos[a0:a1], rc, box=box))
                assert tri == tref


def test_pair_set_exact_at_the_cutoff(lib):
    """Pairs placed within a few ULP of Rcr and Rca on either side: the guard-band
    FP64 recheck reproduces the oracle's predicate exactly."""
    pts = [[0.0, 0.0, 0.0]]
    for k, rc in enumerate((RCR, RCA) * 6):
        d = np.float32(rc)
        step = (k // 2 - 3)
        x = np.nextafter(d, np.float32(np.inf) if step > 0 else np.float32(-np.inf))
        for _ in range(abs(step) - 1):
            x = np.nextafter(x, np.float32(np.inf) if step > 0 else np.float32(-np.inf))
        ang = 0.5 * k
        pts.append([float(x) * np.cos(ang), float(x) * np.sin(ang), 0.0])
    pos = np.asarray(pts, np.float32)
    Z = np.array([6] + [1] * (len(pts) - 1), np.int32)
    b = W.Batch(Z, pos, np.array([0, len(Z)], np.int32))
    model, _, _ = run(lib, b, W.weights(1, 1), 1)
    for kind, rc in ((0, RCR), (1, RCA)):
        counts, lists = (t.cpu().numpy() for t in model.neighbors(kind))
        got = sorted((i, int(j)) for i in range(len(Z)) for j in lists[i, :counts[i]])
        exp = sorted(map(tuple, oracle.pairs(pos, rc).tolist()))
        assert got == exp


# --- features -----------------------------------------------------------------

@pytest.mark.parametrize("case", ["cfg1", "batch", "periodic"])
def test_features_match_oracle(lib, case):
    if case == "cfg1":
        b, w, M = W.config1()
    elif case == "batch":
        b, w, M = small_batch(), W.weights(5, 1), 1
    else:
        b, w, M = W.pocket(9, n=250, edge=14.0), W.weights(5, 1), 1
    model, _, _ = run(lib, b, w, M)
    G = model.features().cpu().numpy().astype(np.float64)
    for m in range(b.n_mols):
        a0, a1 = int(b.mol_off[m]), int(b.mol_off[m + 1])
        ref = oracle.aev(b.Z[a0:a1], b.pos[a0:a1], box=b.box if np.any(b.box) else None)
        scale = np.maximum(np.abs(ref).max(axis=1, keepdims=True), 1e-30)
        err = np.abs(G[a0:a1] - ref) / scale
        # bound: the angular power uses the SFU log2 (absolute error <= 2^-22 on
        # [0.5, 2]), so a term carries up to Zeta * 2^-22 * ln 2 = 2.4e-6 relative
        # error; the FP32 energy bound (1e-5) holds with margin on top of it
        assert err.max() < 5e-6, f"molecule {m}: feature error {err.max():.3e} (row-max relative)"


# --- energies and forces -------------------------------------------------------

@pytest.mark.parametrize("prec", ["fp32", "bf16", "fp16", "bf16-single", "fp16-single"])
@pytest.mark.parametrize("case", ["cfg1", "cfg2", "batch", "batch_bias", "periodic"])
def test_energy_forces_match_oracle(lib, prec, case):
    """Every precision on the zero-bias workloads and on the random-bias variant
    (which includes 1-3 atom molecules whose single output layer cancels)."""
    if case == "cfg1":
        b, w, M = W.config1()
    elif case == "cfg2":
        b, w, M = W.config2()
    elif case == "batch":
        b, w, M = small_batch(), W.weights(6, 8), 8
    elif case == "batch_bias":
        b, w, M = small_batch(), W.weights(6, 8, bias_std=0.1), 8
    else:
        b, w, M = W.pocket(9, n=250, edge=14.0), W.weights(7, 2), 2
    _, E, F = run(lib, b, w, M, prec)
    refs = oracle_batch(b, w, M)
    worst = check_batch(prec, E, F, b, refs)
    print(f"{case} {prec}: worst errors {worst}")


def test_graph_replay_matches_direct_launches(lib):
    b, w, M = small_batch(), W.weights(6, 8), 8
    _, E0, F0 = run(lib, b, w, M, "fp32")
    model = lib.NNP(b.Z, w, M, mol_off=b.mol_off, use_graph=True)
    pos = torch.tensor(b.pos, device="cuda")
    for _ in range(3):
        E, F = model.compute(pos)
    torch.cuda.synchronize()
    model.status()
    np.testing.assert_allclose(E.cpu().numpy(), E0, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(F.cpu().numpy(), F0, rtol=1e-9, atol=1e-9)


def test_host_entry_point_matches_device_entry_point(lib):
    b, w, M = W.config2()
    model, E0, F0 = run(lib, b, w, M)
    E, F = model.compute_host(b.pos)
    np.testing.assert_allclose(E, E0, rtol=1e-12)
    np.testing.assert_allclose(F, F0, rtol=1e-9, atol=1e-12)


def test_autograd_function_returns_minus_forces(lib):
    b, w, M = small_batch(), W.weights(6, 2), 2
    model, E0, F0 = run(lib, b, w, M)
    for recompute in (False, True):
        x = torch.tensor(b.pos, device="cuda", requires_grad=True)
        E = lib.energy(x, model, recompute=recompute)
        (E * torch.arange(1, b.n_mols + 1, device="cuda", dtype=torch.float64)).sum().backward()
        scale = np.repeat(np.arange(1, b.n_mols + 1), np.diff(b.mol_off))[:, None]
        np.testing.assert_allclose(x.grad.cpu().numpy(), -scale * F0, rtol=1e-5, atol=1e-6)
        np.testing.assert_allclose(E.detach().cpu().numpy(), E0, rtol=1e-12)


@pytest.mark.parametrize("prec", ["fp32", "fp16", "bf16", "bf16-single"])
def test_energy_only_call_matches(lib, prec):
    """Energies without forces run the forward kernels alone (for 16-bit
    networks, the fused tail without its reverse phases); on the full batch
    each persistent tensor-core CTA takes many tiles of mixed elements.  The
    energies equal those of the energy-and-forces call."""
    if prec == "fp32":
        b, w, M = small_batch(), W.weights(6, 2), 2
    else:
        b, w, M = W.config3()
    model, E0, _ = run(lib, b, w, M, prec)
    E, F = model.compute(torch.tensor(b.pos, device="cuda"), forces=False)
    torch.cuda.synchronize()
    model.status()
    assert F is None
    np.testing.assert_allclose(E.cpu().numpy(), E0, rtol=1e-12)


def test_perturbed_steps_track_oracle(lib):
    """Workload 2: one handle, positions perturbed by N(0, 0.01^2) A every step."""
    b, w, M = W.config2()
    model = lib.NNP(b.Z, w, M, use_graph=True)
    g = W.rng(5)
    pos = torch.empty(b.n_atoms, 3, dtype=torch.float32, device="cuda")
    for step in range(4):
        p = W.perturb(g, b.pos)
        pos.copy_(torch.from_numpy(p))
        E, F = model.compute(pos)
        torch.cuda.synchronize()
        ref = oracle.compute(b.Z, p, b.mol_off, w, M, atom_energies=True)
        bb = W.Batch(b.Z, p, b.mol_off)
        check_batch("fp32", E.cpu().numpy(), F.cpu().numpy(), bb, {0: ref})


# --- edge cases and errors ------------------------------------------------------

def test_degenerate_molecules(lib):
    """Empty molecules, single atoms and pairs next to normal ones."""
    b = W.batch(88, [0, 1, 2, 0, 25, 3])
    w, M = W.weights(8, 2, bias_std=0.1), 2
    _, E, F = run(lib, b, w, M)
    refs = oracle_batch(b, w, M)
    for m, ref in refs.items():
        if b.mol_off[m + 1] == b.mol_off[m]:
            assert E[m] == 0.0
    check_batch("fp32", E, F, b, {m: r for m, r in refs.items() if b.mol_off[m + 1] > b.mol_off[m]})


def test_rejects_bad_species_and_charge(lib):
    w = W.weights(1, 1)
    with pytest.raises(lib.NNPError) as e:
        lib.NNP(np.array([6, 5], np.int32), w, 1)
    assert e.value.status == "NNP_ERR_SPECIES"
    with pytest.raises(lib.NNPError) as e:
        lib.NNP(np.array([6, 1], np.int32), w, 1, total_charge=1)
    assert e.value.status == "NNP_ERR_CHARGE"
    with pytest.raises(lib.NNPError) as e:
        lib.NNP(np.array([6, 1], np.int32), w[:-1], 1)
    assert e.value.status == "NNP_ERR_ARG"


def test_nonfinite_positions_are_reported(lib):
    b, w, M = W.config1()
    model = lib.NNP(b.Z, w, M)
    p = b.pos.copy()
    p[3, 1] = np.nan
    model.compute(torch.tensor(p, device="cuda"))
    with pytest.raises(lib.NNPError) as e:
        model.status()
    assert e.value.status == "NNP_ERR_NONFINITE"
    model.compute(torch.tensor(b.pos, device="cuda"))
    model.status()  # the status word is cleared by the read


def test_capacity_overflow_is_reported_not_written(lib):
    b = W.batch(90, [100])
    model = lib.NNP(b.Z, W.weights(1, 1), 1, max_neighbors=32, max_angular=32)
    model.compute(torch.tensor(b.pos, device="cuda"))
    with pytest.raises(lib.NNPError) as e:
        model.status()
    assert e.value.status == "NNP_ERR_CAPACITY"


# --- full-size batch in the benchmark's configuration -------------------------------

@pytest.fixture(scope="module")
def full_batch_refs():
    b, w, M = W.config3()
    return b, w, M, oracle_whole_batch(b, w, M)


@pytest.mark.parametrize("prec", ["fp32", "bf16", "fp16"])
def test_full_batch_against_oracle(lib, prec, full_batch_refs):
    """Every molecule of the 512-molecule batch against the oracle; BF16 is
    exactly what the benchmark times (graph replay, tuned schedule)."""
    b, w, M, refs = full_batch_refs
    model = lib.NNP(b.Z, w, M, mol_off=b.mol_off, precision=prec, use_graph=True)
    pos = torch.tensor(b.pos, device="cuda")
    if prec == "bf16":
        model.autotune(pos)
    for _ in range(2):
        E, F = model.compute(pos)
    torch.cuda.synchronize()
    model.status()
    E, F = E.cpu().numpy(), F.cpu().numpy()
    worst = check_batch(prec, E, F, b, refs)
    print(f"full batch {prec}: worst errors over {len(refs)} molecules {worst}")
    # every molecule: net force and torque of an isolated molecule vanish
    for m in range(b.n_mols):
        a0, a1 = int(b.mol_off[m]), int(b.mol_off[m + 1])
        Fm = F[a0:a1]
        scale = np.sqrt(np.mean(Fm ** 2)) * (a1 - a0)
        assert np.abs(Fm.sum(0)).max() <= 1e-4 * scale


# --- workload 5 shapes: the periodic pocket and the densest molecules ----------------

@pytest.mark.parametrize("prec", ["fp32", "fp16", "bf16"])
def test_pocket_and_dense_molecules(lib, prec):
    """The 1500-atom periodic region (24.7 A box, too large for the per-warp
    shared-memory force accumulators, so the global FP64 atomics path runs) and
    250-atom molecules in the 8 A cube (about 0.49 atoms / A^3, the densest
    lists of the workloads: centres with more angular neighbours than the
    reverse pass's main launch stages go through its overflow launch), against
    the oracle."""
    w, M = W.weights(99, 2), 2
    pocket = W.pocket(W.workload_seed(5) + 2)
    _, E, F = run(lib, pocket, w, M, prec)
    check_batch(prec, E, F, pocket, oracle_batch(pocket, w, M))
    dense = W.batch(W.workload_seed(5), [250, 249, 30])
    model, E, F = run(lib, dense, w, M, prec)
    check_batch(prec, E, F, dense, oracle_batch(dense, w, M))
    ca, _ = model.neighbors(1)
    print(f"dense molecules: max angular neighbours {int(ca.max())} of capacity {model.capacity()[1]}")
    # more than the reverse pass stages per warp (64): its overflow launch ran
    assert int(ca.max()) > 64


@pytest.mark.parametrize("prec", ["bf16", "fp16-single"])
def test_single_cta_first_layer_matches_oracle(lib, prec):
    """The first layer's products on single CTAs (128-row tiles, the path for
    a device that cannot hold CTA pairs): the batch with biases and the
    periodic region (2 networks, first-layer tiles split into column pieces)
    against the oracle, with repeated steps bit-identical."""
    cases = [(small_batch(), W.weights(6, 8, bias_std=0.1), 8), (W.pocket(9, n=250, edge=14.0), W.weights(7, 2), 2)]
    for b, w, M in cases:
        model, E, F = run(lib, b, w, M, prec, single_cta=True, use_graph=True)
        worst = check_batch(prec, E, F, b, oracle_batch(b, w, M))
        print(f"single-CTA {prec}: worst errors {worst}")
        pos = torch.tensor(b.pos, device="cuda")
        for _ in range(5):
            E2, _ = model.compute(pos)
        torch.cuda.synchronize()
        model.status()
        np.testing.assert_array_equal(E2.cpu().numpy(), E)


@pytest.mark.parametrize("prec", ["bf16", "fp16"])
def test_repeated_steps_give_identical_energies(lib, prec):
    """Twenty steps of one handle on the same positions: the energies are
    bit-identical (every sum on their path has a fixed order) and the forces
    agree to FP64 rounding (their global accumulation order may vary).  A
    race between CTAs (an output box written by two of them, a read before a
    write) shows here even where the values it produces stay plausible.  The
    periodic region with 2 networks has first-layer tiles split into column
    pieces; the batch has 8 networks."""
    cases = [(W.pocket(W.workload_seed(5) + 2), W.weights(99, 2), 2), (small_batch(), W.weights(6, 8), 8)]
    for b, w, M in cases:
        model = lib.NNP(b.Z, w, M, mol_off=b.mol_off, precision=prec, box=b.box, use_graph=True)
        pos = torch.tensor(b.pos, device="cuda")
        E0, F0 = (t.cpu().numpy().copy() for t in model.compute(pos))
        for _ in range(19):
            E, F = model.compute(pos)
        torch.cuda.synchronize()
        model.status()
        np.testing.assert_array_equal(E.cpu().numpy(), E0)
        np.testing.assert_allclose(F.cpu().numpy(), F0, rtol=1e-12, atol=1e-12)


def test_autotuner_keeps_results_and_picks_valid_schedule(lib):
    b, w, M = small_batch(), W.weights(6, 8), 8
    for prec in ("fp32", "fp16"):
        model, E0, F0 = run(lib, b, w, M, prec, use_graph=True)
        pos = torch.tensor(b.pos, device="cuda")
        chosen = model.autotune(pos)
        assert chosen["featurizer_warps"] in (2, 4, 8) and chosen["reverse_warps"] in (2, 4, 8)
        assert chosen["first_layer_n_tile"] in (128, 256)
        E, F = model.compute(pos)
        torch.cuda.synchronize()
        model.status()
        np.testing.assert_allclose(E.cpu().numpy(), E0, rtol=1e-9, atol=1e-12)
        np.testing.assert_allclose(F.cpu().numpy(), F0, rtol=1e-6, atol=1e-9)


def test_pinned_schedules_keep_results_and_reject_bad_values(lib):
    # every schedule the autotuner may pick, pinned through nnp_set_schedule,
    # gives the energies and forces of the default schedule
    b, w, M = small_batch(), W.weights(6, 8), 8
    model, E0, F0 = run(lib, b, w, M, "fp16", use_graph=True)
    pos = torch.tensor(b.pos, device="cuda")
    for sched in ((2, 2, 2, 256, 1), (8, 4, 16, 128, 0), (4, 2, 16, 256, 0)):
        model.set_schedule(dict(zip(lib.NNP.SCHEDULE_KEYS, sched)))
        E, F = model.compute(pos)
        torch.cuda.synchronize()
        model.status()
        np.testing.assert_allclose(E.cpu().numpy(), E0, rtol=1e-9, atol=1e-12)
        np.testing.assert_allclose(F.cpu().numpy(), F0, rtol=1e-6, atol=1e-9)
    for bad in ((3, 2, 2, 256, 1), (2, 2, 3, 256, 1), (2, 2, 2, 64, 1), (2, 2, 2, 256, 2)):
        with pytest.raises(lib.NNPError) as e:
            model.set_schedule(dict(zip(lib.NNP.SCHEDULE_KEYS, bad)))
        assert e.value.status == "NNP_ERR_ARG"


# --- features kept only for the forward pass, and the device-side abort path -------

@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_recompute_aev_shares_the_feature_buffer(lib, prec):
    """recompute_aev: the features live in the dE/dG buffer.  Energies and forces
    equal those of a handle with its own feature buffer; the features can be
    read after an energy-only step (equal to the other handle's), not after a
    step whose reverse pass reused the buffer."""
    b, w, M = small_batch(), W.weights(6, 8), 8
    pos = torch.tensor(b.pos, device="cuda")
    ref = lib.NNP(b.Z, w, M, mol_off=b.mol_off, precision=prec)
    E0, F0 = ref.compute(pos)
    G0 = ref.features()
    model = lib.NNP(b.Z, w, M, mol_off=b.mol_off, precision=prec, recompute_aev=True, use_graph=True)
    for _ in range(2):
        E, F = model.compute(pos)
    torch.cuda.synchronize()
    model.status()
    np.testing.assert_array_equal(E.cpu().numpy(), E0.cpu().numpy())
    np.testing.assert_array_equal(F.cpu().numpy(), F0.cpu().numpy())
    with pytest.raises(lib.NNPError) as e:
        model.features()
    assert e.value.status == "NNP_ERR_UNSUPPORTED"
    model.compute(pos, forces=False)
    G = model.features()
    torch.cuda.synchronize()
    np.testing.assert_array_equal(G.cpu().numpy(), G0.cpu().numpy())


@pytest.mark.parametrize("use_graph", [False, True])
@pytest.mark.parametrize("prec", ["bf16", "fp16-single"])
def test_device_timeout_path_reports_and_recovers(lib, prec, use_graph):
    """The tensor-core kernels' abort path: test_abort makes the first step's
    kernels start as if a bounded wait had given up (before any copy or
    product is issued); every CTA frees its tensor memory and exits, the
    status reads NNP_ERR_TIMEOUT, and the next step on the same handle is
    clean and matches the oracle."""
    b, w, M = small_batch(), W.weights(6, 8), 8
    p, single = split_mode(prec)
    model = lib.NNP(b.Z, w, M, mol_off=b.mol_off, precision=p, single_pass=single,
                    use_graph=use_graph, test_abort=True)
    pos = torch.tensor(b.pos, device="cuda")
    model.compute(pos)
    with pytest.raises(lib.NNPError) as e:
        model.status()
    assert e.value.status == "NNP_ERR_TIMEOUT"
    E, F = model.compute(pos)
    torch.cuda.synchronize()
    model.status()
    check_batch(prec, E.cpu().numpy(), F.cpu().numpy(), b, oracle_batch(b, w, M))

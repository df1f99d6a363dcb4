"""Pins of the FP64 oracle against what the mathematics fixes.

The paper prints no worked example for the featurizer or the networks, so the
oracle is pinned by closed forms, limits, invariants, brute force and an
independent automatic-differentiation evaluation (Sec. 2, Eqs. 2-3: the NNP
term and F = -grad V; Sec. 1: ANI symmetry functions, 5.1 A cutoff, seven
elements; Sec. 2 "Optimization": the 8-network ensemble).  Each test names the
mistake it is there to catch.
"""
import itertools
import math

import numpy as np
import pytest

import oracle
from paper_2201_08110_gb300 import workloads as W

RCR = float(np.float32(5.1))
RCA = float(np.float32(3.5))
ETA_R, ETA_A, ZETA = 19.7, 12.5, 14.1
SHF_R = [0.8 + (4.9 - 0.8) * k / 15 for k in range(16)]
SHF_A = [0.8 + (3.1 - 0.8) * k / 7 for k in range(8)]
SHF_Z = [0.39 + (2.75 - 0.39) * k / 3 for k in range(4)]
PAIRS = list(itertools.combinations_with_replacement(range(7), 2))


def fc(r, rc):
    return 0.5 * math.cos(math.pi * r / rc) + 0.5 if r < rc else 0.0


def one_mol(Z, pos):
    return np.asarray(Z, np.int32), np.asarray(pos, np.float64), np.array([0, len(Z)], np.int32)


# --- featurizer constants ------------------------------------------------------

def test_shift_grids_are_the_stated_ranges():
    """16 radial shifts 0.8-4.9 A, 8 angular-radial shifts 0.8-3.1 A, 4 angle
    shifts 0.39-2.75 rad, both ends included; cutoffs are the FP32 constants."""
    h = oracle.hyper()
    assert h["Rcr"] == RCR and h["Rca"] == RCA
    for key, lo, hi, n in (("ShfR", 0.8, 4.9, 16), ("ShfA", 0.8, 3.1, 8), ("ShfZ", 0.39, 2.75, 4)):
        g = h[key]
        assert g.shape == (n,)
        assert g[0] == pytest.approx(lo, abs=1e-15) and g[-1] == pytest.approx(hi, abs=1e-15)
        assert np.allclose(np.diff(g), (hi - lo) / (n - 1), rtol=0, atol=1e-14)


# --- radial closed forms -----------------------------------------------------

@pytest.mark.parametrize("r", [0.9, RCR / 2, SHF_R[7], 4.0, 5.0])
def test_two_atom_radial_closed_form(r):
    """Two atoms: G_i[s_j, k] = 1/4 exp(-EtaR (r - ShfR_k)^2) fc(r), every other
    entry zero (catches a wrong prefactor, species block, or a leaked angular
    term).  At r = Rcr/2 the cutoff is exactly 1/2; at r = ShfR_7 the Gaussian
    is exactly 1."""
    Z, pos, _ = one_mol([6, 8], [[0, 0, 0], [r, 0, 0]])
    G = oracle.aev(Z, pos)
    for i, sj in ((0, 3), (1, 1)):
        exp = np.zeros(1008)
        for k in range(16):
            exp[sj * 16 + k] = 0.25 * math.exp(-ETA_R * (r - SHF_R[k]) ** 2) * fc(r, RCR)
        np.testing.assert_allclose(G[i], exp, rtol=1e-13, atol=1e-300)
    if r == RCR / 2:
        assert fc(r, RCR) == pytest.approx(0.5, abs=1e-15)
    if r == SHF_R[7]:
        assert G[0, 3 * 16 + 7] == pytest.approx(0.25 * fc(r, RCR), rel=1e-14)


def test_radial_cutoff_excludes_beyond_rcr():
    Z, pos, _ = one_mol([1, 1], [[0, 0, 0], [RCR + 1e-6, 0, 0]])
    assert not np.any(oracle.aev(Z, pos))


# --- angular closed form -------------------------------------------------------

def three_atom(r, theta_mod, sj=6, sk=7):
    """Centre O at the origin, neighbours at distance r with the angle chosen so
    that acos(0.95 cos angle) == theta_mod."""
    phi = math.acos(math.cos(theta_mod) / 0.95)
    return one_mol([8, sj, sk], [[0, 0, 0], [r, 0, 0], [r * math.cos(phi), r * math.sin(phi), 0]])


@pytest.mark.parametrize("a0,z0", [(3, 1), (0, 0), (5, 2)])
def test_three_atom_angular_closed_form(a0, z0):
    """One triple: at theta' = ShfZ_z and (r_ij + r_ik)/2 = ShfA_a the term is
    exactly 2 fc(r)^2 (pins the 2^(1-Zeta) prefactor, the 0.95 angle
    convention, the pair-block and (a, z) layout).  Neighbouring entries follow
    the Gaussian ratio and the cosine power."""
    r = SHF_A[a0]
    Z, pos, _ = three_atom(r, SHF_Z[z0])
    G = oracle.aev(Z, pos)[0]
    p = PAIRS.index((1, 2))  # C, N
    blk = G[112 + 32 * p: 112 + 32 * (p + 1)].reshape(8, 4)
    f2 = fc(r, RCA) ** 2
    assert blk[a0, z0] == pytest.approx(2.0 * f2, rel=1e-12)
    for a in range(8):
        for z in range(4):
            ang = 2.0 * ((1.0 + math.cos(SHF_Z[z0] - SHF_Z[z])) / 2.0) ** ZETA
            rad = math.exp(-ETA_A * (r - SHF_A[a]) ** 2)
            assert blk[a, z] == pytest.approx(ang * rad * f2, rel=1e-11, abs=1e-300)
    # every other angular block of the centre is empty
    mask = np.ones(896, bool)
    mask[32 * p: 32 * (p + 1)] = False
    assert not np.any(G[112:][mask])


def test_angular_block_is_symmetric_in_species_order():
    """p(s, t) == p(t, s): swapping the neighbours' elements fills the same block."""
    Z1, pos, _ = three_atom(1.5, 1.0, 6, 7)
    Z2 = np.array([8, 7, 6], np.int32)
    np.testing.assert_allclose(oracle.aev(Z1, pos)[0, 112:], oracle.aev(Z2, pos)[0, 112:], rtol=1e-14)


def test_angular_zero_with_fewer_than_two_neighbours():
    Z, pos, _ = one_mol([6, 1, 1], [[0, 0, 0], [1.0, 0, 0], [-4.0, 0, 0]])
    G = oracle.aev(Z, pos)
    assert not np.any(G[0, 112:])  # only one neighbour within Rca of the centre
    assert np.any(G[0, :112])


# --- pair / triple enumeration --------------------------------------------------

def brute_pairs(pos, rc, box=None):
    out = []
    n = len(pos)
    for i in range(n):
        for j in range(n):
            if i == j:
                continue
            if box is None:
                d2 = sum((float(pos[j][c]) - float(pos[i][c])) ** 2 for c in range(3))
            else:  # nearest of the 27 images, an independent route to the minimum image
                d2 = min(sum((float(pos[j][c]) + L * box[c] - float(pos[i][c])) ** 2
                             for c, L in enumerate(sh))
                         for sh in itertools.product((-1, 0, 1), repeat=3))
            if d2 < rc * rc:
                out.append((i, j))
    return sorted(out)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_pairs_and_triples_match_brute_force(seed):
    b = W.batch(seed, [18])
    for rc in (RCR, RCA):
        got = sorted(map(tuple, oracle.pairs(b.pos, rc).tolist()))
        assert got == brute_pairs(b.pos, rc)
    tri = sorted(map(tuple, oracle.triples(b.pos, RCA).tolist()))
    nb = {}
    for i, j in brute_pairs(b.pos, RCA):
        nb.setdefault(i, []).append(j)
    exp = sorted((i, j, k) for i, js in nb.items() for j, k in itertools.combinations(sorted(js), 2))
    assert tri == exp


def test_periodic_pairs_match_image_enumeration():
    b = W.pocket(7, n=60, edge=11.0)
    box = [11.0] * 3
    for rc in (RCR, RCA):
        got = sorted(map(tuple, oracle.pairs(b.pos, rc, box=box).tolist()))
        assert got == brute_pairs(b.pos, rc, box)


# --- networks and automatic differentiation -------------------------------------

torch = pytest.importorskip("torch")


def torch_networks(G, Z, w, n_models):
    """Independent evaluation of the ensemble of element networks with torch
    (FP64), from the packed weight layout."""
    zs = list(W.ELEMENTS_Z)
    per_model = W.weights_per_model()
    E = 0
    for m in range(n_models):
        off = m * per_model
        for e in range(7):
            dims = (1008,) + W.HIDDEN[e] + (1,)
            mats = []
            for l in range(4):
                nW = dims[l] * dims[l + 1]
                Wt = torch.tensor(w[off:off + nW].reshape(dims[l + 1], dims[l]), dtype=torch.float64)
                off += nW
                bt = torch.tensor(w[off:off + dims[l + 1]], dtype=torch.float64)
                off += dims[l + 1]
                mats.append((Wt, bt))
            rows = [i for i, z in enumerate(Z) if z == zs[e]]
            if not rows:
                continue
            x = G[rows]
            for l, (Wt, bt) in enumerate(mats):
                x = x @ Wt.T + bt
                if l < 3:  # CELU, alpha = 0.1 (written out: torch's own FP64 CELU
                    # backward carries an FP32-rounded 1/alpha)
                    x = torch.where(x > 0, x, 0.1 * torch.expm1(torch.clamp(x, max=0.0) / 0.1))
            E = E + x.sum() / n_models
    return E


def torch_aev(Z, pos):
    """Independent featurizer in torch (FP64): explicit acos / cos(theta - ShfZ),
    species pairs via combinations_with_replacement order."""
    sp = [W.ELEMENTS_Z.index(int(z)) for z in Z]
    n = len(Z)
    feats = []
    for i in range(n):
        rad = [torch.zeros(16, dtype=torch.float64) for _ in range(7)]
        ang = {pq: torch.zeros(8, 4, dtype=torch.float64) for pq in PAIRS}
        for j in range(n):
            if j == i:
                continue
            dv = pos[j] - pos[i]
            r = torch.sqrt((dv * dv).sum())
            if r.item() < RCR:
                f = 0.5 * torch.cos(math.pi * r / RCR) + 0.5
                rad[sp[j]] = rad[sp[j]] + 0.25 * torch.exp(-ETA_R * (r - torch.tensor(SHF_R, dtype=torch.float64)) ** 2) * f
        for j, k in itertools.combinations([q for q in range(n) if q != i], 2):
            dj, dk = pos[j] - pos[i], pos[k] - pos[i]
            rj, rk = torch.linalg.norm(dj), torch.linalg.norm(dk)
            if rj.item() >= RCA or rk.item() >= RCA:
                continue
            th = torch.acos(0.95 * (dj @ dk) / (rj * rk))
            fj = 0.5 * torch.cos(math.pi * rj / RCA) + 0.5
            fk = 0.5 * torch.cos(math.pi * rk / RCA) + 0.5
            A = 2 * ((1 + torch.cos(th - torch.tensor(SHF_Z, dtype=torch.float64))) / 2) ** ZETA
            R = torch.exp(-ETA_A * ((rj + rk) / 2 - torch.tensor(SHF_A, dtype=torch.float64)) ** 2)
            key = tuple(sorted((sp[j], sp[k])))
            ang[key] = ang[key] + torch.outer(R, A) * fj * fk
        feats.append(torch.cat(rad + [ang[pq].reshape(-1) for pq in PAIRS]))
    return torch.stack(feats)


def test_featurizer_matches_independent_torch_evaluation():
    b = W.batch(11, [9])
    G = oracle.aev(b.Z, b.pos)
    Gt = torch_aev(b.Z, torch.tensor(b.pos, dtype=torch.float64)).numpy()
    assert np.any(G[:, 112:])
    np.testing.assert_allclose(G, Gt, rtol=1e-11, atol=1e-14)


@pytest.mark.parametrize("bias_std", [0.0, 0.1])
def test_networks_energy_and_dEdG_match_torch_autograd(bias_std):
    """Energy from the oracle's own features through an independent torch
    evaluation of the packed networks, and dE/dG against torch autograd (pins
    the weight layout, CELU, the ensemble mean and the network reverse mode)."""
    b = W.batch(12, [14])
    w = W.weights(5, 2, bias_std=bias_std)
    out = oracle.compute(b.Z, b.pos, b.mol_off, w, 2, aev=True, dEdG=True)
    G = torch.tensor(out["aev"], dtype=torch.float64, requires_grad=True)
    E = torch_networks(G, b.Z, w, 2)
    E.backward()
    assert out["energy"][0] == pytest.approx(E.item(), rel=1e-12, abs=1e-12)
    np.testing.assert_allclose(out["dEdG"], G.grad.numpy(), rtol=1e-9, atol=1e-12)


def test_forces_match_torch_autograd_of_independent_path():
    b = W.batch(13, [8])
    w = W.weights(6, 1, bias_std=0.1)
    out = oracle.compute(b.Z, b.pos, b.mol_off, w, 1)
    x = torch.tensor(b.pos, dtype=torch.float64, requires_grad=True)
    E = torch_networks(torch_aev(b.Z, x), b.Z, w, 1)
    E.backward()
    assert out["energy"][0] == pytest.approx(E.item(), rel=1e-11)
    np.testing.assert_allclose(out["forces"], -x.grad.numpy(), rtol=1e-8, atol=1e-10)


# --- finite differences -------------------------------------------------------

def test_forces_match_central_differences():
    """F = -dE/dx against central differences, h = 1e-4 A (error O(h^2))."""
    b = W.batch(21, [10])
    w = W.weights(22, 2, bias_std=0.1)
    pos = b.pos.astype(np.float64)
    F = oracle.compute(b.Z, pos, b.mol_off, w, 2)["forces"]
    h = 1e-4
    fd = np.zeros_like(pos)
    for a in range(pos.shape[0]):
        for c in range(3):
            p1, p2 = pos.copy(), pos.copy()
            p1[a, c] += h
            p2[a, c] -= h
            fd[a, c] = -(oracle.energy(b.Z, p1, w, 2) - oracle.energy(b.Z, p2, w, 2)) / (2 * h)
    scale = np.sqrt(np.mean(F ** 2))
    assert np.max(np.abs(F - fd)) < 1e-6 * max(scale, 1.0)


def test_featurizer_adjoint_matches_central_differences():
    """The featurizer reverse mode alone: d(sum g.G)/dx for a random g."""
    b = W.batch(23, [9])
    pos = b.pos.astype(np.float64)
    g = W.rng(24).standard_normal((9, 1008))
    grad = oracle.aev_adjoint(b.Z, pos, g)
    h = 1e-5
    for a in range(9):
        for c in range(3):
            p1, p2 = pos.copy(), pos.copy()
            p1[a, c] += h
            p2[a, c] -= h
            fd = (np.sum(g * oracle.aev(b.Z, p1)) - np.sum(g * oracle.aev(b.Z, p2))) / (2 * h)
            assert grad[a, c] == pytest.approx(fd, rel=1e-6, abs=1e-7)


# --- invariants ---------------------------------------------------------------

def random_rotation(seed):
    q, r = np.linalg.qr(W.rng(seed).standard_normal((3, 3)))
    q = q * np.sign(np.diag(r))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


def test_invariances_and_zero_net_force_and_torque():
    b = W.batch(31, [30])
    w = W.weights(32, 2, bias_std=0.1)
    pos = b.pos.astype(np.float64)
    out = oracle.compute(b.Z, pos, b.mol_off, w, 2)
    E, F = out["energy"][0], out["forces"]
    # translation
    assert oracle.energy(b.Z, pos + np.array([3.3, -1.7, 12.9]), w, 2) == pytest.approx(E, rel=1e-12)
    # rotation (forces rotate with the frame)
    Rm = random_rotation(33)
    out_r = oracle.compute(b.Z, pos @ Rm.T, b.mol_off, w, 2)
    assert out_r["energy"][0] == pytest.approx(E, rel=1e-12)
    np.testing.assert_allclose(out_r["forces"], F @ Rm.T, atol=1e-10)
    # permutation of the atoms (same-element swaps included)
    perm = W.rng(34).permutation(30)
    out_p = oracle.compute(b.Z[perm], pos[perm], b.mol_off, w, 2)
    assert out_p["energy"][0] == pytest.approx(E, rel=1e-12)
    np.testing.assert_allclose(out_p["forces"], F[perm], atol=1e-12)
    # net force and torque vanish for an isolated molecule
    assert np.max(np.abs(F.sum(0))) < 1e-12 * max(1, np.abs(F).max()) * 30
    assert np.max(np.abs(np.cross(pos, F).sum(0))) < 1e-10


def test_same_element_swap_only_changes_order():
    """Swapping two H atoms leaves the features of the others unchanged."""
    b = W.batch(35, [12])
    hs = np.where(b.Z == 1)[0]
    assert len(hs) >= 2
    perm = np.arange(12)
    perm[[hs[0], hs[1]]] = perm[[hs[1], hs[0]]]
    G = oracle.aev(b.Z, b.pos)
    Gp = oracle.aev(b.Z[perm], b.pos[perm])
    np.testing.assert_allclose(Gp, G[perm], rtol=1e-13, atol=1e-300)


def test_ensemble_is_the_mean_of_single_networks():
    b = W.batch(36, [15])
    w = W.weights(37, 3)
    per = W.weights_per_model()
    E3 = oracle.compute(b.Z, b.pos, b.mol_off, w, 3, forces=False)["energy"][0]
    Es = [oracle.compute(b.Z, b.pos, b.mol_off, w[m * per:(m + 1) * per], 1, forces=False)["energy"][0]
          for m in range(3)]
    assert E3 == pytest.approx(np.mean(Es), rel=1e-13)


@pytest.mark.parametrize("rc,extra", [(RCR, [[0.0, 2.0, 0.0]]), (RCA, [[0.0, 1.2, 0.0], [0.9, 0.0, 0.7]])])
def test_energy_and_forces_continuous_across_cutoff(rc, extra):
    """A pair moved across Rcr (or Rca): both one-sided limits agree, since fc
    and fc' vanish at the cutoff."""
    w = W.weights(41, 1, bias_std=0.1)
    Z = np.array([6, 7] + [1] * len(extra), np.int32)
    res = []
    d = 1e-7
    for r in (rc - d, rc + d):
        pos = np.array([[0, 0, 0], [r, 0, 0]] + extra, np.float64)
        out = oracle.compute(Z, pos, np.array([0, len(Z)]), w, 1)
        res.append((out["energy"][0], out["forces"]))
    # the smooth part of the change is -F_x(atom 1) * 2d; what is left is a jump
    smooth = -0.5 * (res[0][1][1, 0] + res[1][1][1, 0]) * 2 * d
    assert abs(res[1][0] - res[0][0] - smooth) < 1e-13
    assert np.max(np.abs(res[0][1] - res[1][1])) < 1e-5


def test_periodic_energy_invariant_under_image_shift():
    b = W.pocket(51, n=40, edge=11.0)
    w = W.weights(52, 1)
    box = [11.0] * 3
    E = oracle.energy(b.Z, b.pos, w, 1, box=box)
    shifted = b.pos.astype(np.float64).copy()
    shifted[::3] += np.array([11.0, -22.0, 11.0])
    assert oracle.energy(b.Z, shifted, w, 1, box=box) == pytest.approx(E, rel=1e-12)


def test_rejects_unknown_element():
    with pytest.raises(ValueError):
        oracle.aev(np.array([6, 5], np.int32), np.zeros((2, 3)))

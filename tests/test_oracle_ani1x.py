"""Pins of the FP64 oracle's ANI-1x-shaped model (CPU).

The paper also runs ANI-1x (Sec. 3 "Extensibility with other NNPs") but
prints none of its constants; the model here is the ANI-1x shape: elements
H, C, N, O; radial cutoff 5.2 A, EtaR 16, 16 shifts 0.9 + 0.26875 k A; angular
cutoff 3.5 A, EtaA 8, Zeta 32, 4 distance shifts 0.9 + 0.65 a A and 8 angle
shifts pi/16 + z pi/8; features [radial 4 x 16 | 10 species-pair blocks of
4 x 8 (distance-shift major)] = 384; networks H 384-160-128-96-1,
C 384-144-112-96-1, N and O 384-128-112-96-1.  As for the ANI-2x shape, the
oracle is pinned by closed forms, an independent autodiff evaluation, finite
differences, invariants and limits; each test names the mistake it catches.
"""
import itertools
import math

import numpy as np
import pytest

import oracle
from paper_2201_08110_gb300 import workloads as W

MODEL = "ani1x"
RCR = float(np.float32(5.2))
RCA = float(np.float32(3.5))
ETA_R, ETA_A, ZETA = 16.0, 8.0, 32.0
SHF_R = [0.9 + 0.26875 * k for k in range(16)]
SHF_A = [0.9 + 0.65 * a for a in range(4)]
SHF_Z = [math.pi / 16 + z * math.pi / 8 for z in range(8)]
PAIRS = list(itertools.combinations_with_replacement(range(4), 2))
NF = 384


def fc(r, rc):
    return 0.5 * math.cos(math.pi * r / rc) + 0.5 if r < rc else 0.0


def one_mol(Z, pos):
    return np.asarray(Z, np.int32), np.asarray(pos, np.float64), np.array([0, len(Z)], np.int32)


def test_constants_and_sizes():
    h = oracle.hyper(MODEL)
    assert h["Rcr"] == RCR and h["Rca"] == RCA
    assert (h["EtaR"], h["EtaA"], h["Zeta"]) == (ETA_R, ETA_A, ZETA)
    np.testing.assert_allclose(h["ShfR"], SHF_R, rtol=0, atol=1e-15)
    np.testing.assert_allclose(h["ShfA"], SHF_A, rtol=0, atol=1e-15)
    np.testing.assert_allclose(h["ShfZ"], SHF_Z, rtol=0, atol=1e-15)
    assert oracle.weights_per_model(MODEL) == W.weights_per_model(MODEL)
    assert W.weights_per_model(MODEL) == sum(
        n * m + m for dims in ((384,) + hid + (1,) for hid in W.HIDDEN_ANI1X)
        for n, m in zip(dims[:-1], dims[1:]))


@pytest.mark.parametrize("r", [0.9, RCR / 2, SHF_R[9], 5.1])
def test_two_atom_radial_closed_form(r):
    """Two atoms: G_i[s_j, k] = 1/4 exp(-EtaR (r - ShfR_k)^2) fc(r; 5.2), all else
    zero (catches the ANI-2x cutoff or grid leaking in, a wrong species block)."""
    Z, pos, _ = one_mol([6, 8], [[0, 0, 0], [r, 0, 0]])
    G = oracle.aev(Z, pos, model=MODEL)
    assert G.shape == (2, NF)
    for i, sj in ((0, 3), (1, 1)):
        exp = np.zeros(NF)
        for k in range(16):
            exp[sj * 16 + k] = 0.25 * math.exp(-ETA_R * (r - SHF_R[k]) ** 2) * fc(r, RCR)
        np.testing.assert_allclose(G[i], exp, rtol=1e-13, atol=1e-300)


def three_atom(r, theta_mod, sj=6, sk=7):
    phi = math.acos(math.cos(theta_mod) / 0.95)
    return one_mol([8, sj, sk], [[0, 0, 0], [r, 0, 0], [r * math.cos(phi), r * math.sin(phi), 0]])


@pytest.mark.parametrize("a0,z0", [(1, 5), (0, 1), (3, 2), (2, 6)])
def test_three_atom_angular_closed_form(a0, z0):
    """At theta' = ShfZ_z and (r_ij + r_ik)/2 = ShfA_a the term is exactly
    2 fc(r)^2; the neighbouring entries follow the Gaussian ratio and the
    cosine power (pins the 4 x 8 block layout, distance-shift major, and the
    block index of (C, N) in the 4-element triangle).  theta' = acos(0.95 cos)
    lies in [0.318, 2.82] rad, so the first and last angle shifts are never
    met exactly."""
    r = SHF_A[a0]
    Z, pos, _ = three_atom(r, SHF_Z[z0])
    G = oracle.aev(Z, pos, model=MODEL)[0]
    p = PAIRS.index((1, 2))
    blk = G[64 + 32 * p: 64 + 32 * (p + 1)].reshape(4, 8)
    f2 = fc(r, RCA) ** 2
    assert blk[a0, z0] == pytest.approx(2.0 * f2, rel=1e-12)
    for a in range(4):
        for z in range(8):
            ang = 2.0 * ((1.0 + math.cos(SHF_Z[z0] - SHF_Z[z])) / 2.0) ** ZETA
            rad = math.exp(-ETA_A * (r - SHF_A[a]) ** 2)
            assert blk[a, z] == pytest.approx(ang * rad * f2, rel=1e-10, abs=1e-300)
    mask = np.ones(320, bool)
    mask[32 * p: 32 * (p + 1)] = False
    assert not np.any(G[64:][mask])


def test_rejects_elements_outside_the_model():
    for z in (9, 16, 17, 5):
        with pytest.raises(ValueError):
            oracle.aev(np.array([6, z], np.int32), np.array([[0, 0, 0], [1.5, 0, 0.0]]), model=MODEL)


def torch_energy(Z, pos, w, n_models):
    """Independent evaluation: explicit acos angles, species pairs from
    itertools, the networks from the packed layout, torch autograd."""
    torch = pytest.importorskip("torch")
    x = torch.tensor(pos, dtype=torch.float64, requires_grad=True)
    spec = [W.ELEMENTS_Z_ANI1X.index(int(z)) for z in Z]
    n = len(Z)
    feats = []
    for i in range(n):
        rad = [torch.zeros((), dtype=torch.float64) for _ in range(64)]
        ang = [torch.zeros((), dtype=torch.float64) for _ in range(320)]
        for j in range(n):
            if j == i:
                continue
            d = x[j] - x[i]
            r = torch.sqrt((d * d).sum())
            if float(r.detach()) < RCR:
                f = 0.5 * torch.cos(math.pi * r / RCR) + 0.5
                for k in range(16):
                    rad[spec[j] * 16 + k] = rad[spec[j] * 16 + k] + 0.25 * torch.exp(-ETA_R * (r - SHF_R[k]) ** 2) * f
        for j, k in itertools.combinations(range(n), 2):
            if i in (j, k):
                continue
            dj, dk = x[j] - x[i], x[k] - x[i]
            rj, rk = torch.sqrt((dj * dj).sum()), torch.sqrt((dk * dk).sum())
            if float(rj.detach()) >= RCA or float(rk.detach()) >= RCA:
                continue
            th = torch.acos(0.95 * (dj * dk).sum() / (rj * rk))
            f = (0.5 * torch.cos(math.pi * rj / RCA) + 0.5) * (0.5 * torch.cos(math.pi * rk / RCA) + 0.5)
            b = PAIRS.index(tuple(sorted((spec[j], spec[k]))))
            for a in range(4):
                for z in range(8):
                    t = 2 * ((1 + torch.cos(th - SHF_Z[z])) / 2) ** ZETA * torch.exp(
                        -ETA_A * ((rj + rk) / 2 - SHF_A[a]) ** 2) * f
                    ang[32 * b + 8 * a + z] = ang[32 * b + 8 * a + z] + t
        feats.append(torch.stack(rad + ang))
    G = torch.stack(feats)
    per = W.weights_per_model(MODEL)
    # CELU written out: its derivative is then exp(z / alpha) itself (a
    # gradient formed from the activation as (celu + alpha) / alpha cancels
    # for very negative z and loses about 1e-7 of the force)
    celu = lambda v: torch.where(v > 0, v, 0.1 * (torch.exp(torch.clamp(v, max=0.0) / 0.1) - 1.0))
    E = torch.zeros((), dtype=torch.float64)
    for m in range(n_models):
        p = torch.tensor(w[m * per:(m + 1) * per], dtype=torch.float64)
        o, layers = 0, []
        for e in range(4):
            dims = (384,) + W.HIDDEN_ANI1X[e] + (1,)
            L = []
            for l in range(4):
                fi, fo = dims[l], dims[l + 1]
                L.append((p[o:o + fi * fo].reshape(fo, fi), p[o + fi * fo:o + fi * fo + fo]))
                o += fi * fo + fo
            layers.append(L)
        for i in range(n):
            h = G[i]
            for l, (Wl, bl) in enumerate(layers[spec[i]]):
                h = Wl @ h + bl
                if l < 3:
                    h = celu(h)
            E = E + h[0] / n_models
    E.backward()
    return float(E), -x.grad.numpy(), G.detach().numpy()


@pytest.mark.parametrize("bias_std", [0.0, 0.1])
def test_energy_forces_and_features_match_independent_autodiff(bias_std):
    b = W.batch(61, [9], model=MODEL)
    w = W.weights(62, 2, bias_std=bias_std, model=MODEL)
    E_t, F_t, G_t = torch_energy(b.Z, b.pos.astype(np.float64), w, 2)
    out = oracle.compute(b.Z, b.pos, b.mol_off, w, 2, aev=True, model=MODEL)
    np.testing.assert_allclose(out["aev"], G_t, rtol=1e-11, atol=1e-14)
    assert out["energy"][0] == pytest.approx(E_t, rel=1e-11, abs=1e-13)
    np.testing.assert_allclose(out["forces"], F_t, rtol=1e-10, atol=1e-13)


def test_forces_match_central_differences():
    b = W.batch(63, [14], model=MODEL)
    w = W.weights(64, 2, model=MODEL)
    pos = b.pos.astype(np.float64)
    F = oracle.compute(b.Z, pos, b.mol_off, w, 2, model=MODEL)["forces"]
    h = 1e-4
    fd = np.zeros_like(F)
    for a in range(len(b.Z)):
        for c in range(3):
            p1, p2 = pos.copy(), pos.copy()
            p1[a, c] += h
            p2[a, c] -= h
            fd[a, c] = -(oracle.energy(b.Z, p1, w, 2, model=MODEL) -
                         oracle.energy(b.Z, p2, w, 2, model=MODEL)) / (2 * h)
    scale = np.abs(F).max()
    assert np.abs(F - fd).max() <= 1e-6 * scale


def test_featurizer_adjoint_matches_central_differences():
    b = W.batch(65, [10], model=MODEL)
    pos = b.pos.astype(np.float64)
    g = W.rng(66).standard_normal((len(b.Z), NF))
    grad = oracle.aev_adjoint(b.Z, pos, g, model=MODEL)
    h = 1e-5
    for a in range(len(b.Z)):
        for c in range(3):
            p1, p2 = pos.copy(), pos.copy()
            p1[a, c] += h
            p2[a, c] -= h
            fd = (np.sum(g * oracle.aev(b.Z, p1, model=MODEL)) -
                  np.sum(g * oracle.aev(b.Z, p2, model=MODEL))) / (2 * h)
            assert grad[a, c] == pytest.approx(fd, rel=1e-6, abs=1e-7)


def test_invariances_and_zero_net_force_and_torque():
    b = W.batch(67, [16], model=MODEL)
    w = W.weights(68, 2, model=MODEL)
    pos = b.pos.astype(np.float64)
    out = oracle.compute(b.Z, pos, b.mol_off, w, 2, model=MODEL)
    E, F = out["energy"][0], out["forces"]
    assert oracle.energy(b.Z, pos + np.array([2.5, -0.7, 9.1]), w, 2, model=MODEL) == pytest.approx(E, rel=1e-12)
    th = 0.73
    R = np.array([[math.cos(th), -math.sin(th), 0], [math.sin(th), math.cos(th), 0], [0, 0, 1.0]])
    out_r = oracle.compute(b.Z, pos @ R.T, b.mol_off, w, 2, model=MODEL)
    assert out_r["energy"][0] == pytest.approx(E, rel=1e-12)
    np.testing.assert_allclose(out_r["forces"], F @ R.T, rtol=1e-9, atol=1e-12)
    perm = W.rng(69).permutation(len(b.Z))
    assert oracle.energy(b.Z[perm], pos[perm], w, 2, model=MODEL) == pytest.approx(E, rel=1e-12)
    scale = np.abs(F).max() * len(b.Z)
    assert np.abs(F.sum(0)).max() <= 1e-12 * scale
    assert np.abs(np.cross(pos, F).sum(0)).max() <= 1e-11 * scale * 10


@pytest.mark.parametrize("rc,extra", [(RCR, [[0.0, 2.0, 0.0]]), (RCA, [[0.0, 1.2, 0.0], [0.9, 0.0, 0.7]])])
def test_energy_and_forces_continuous_across_cutoff(rc, extra):
    """A neighbour moved across a cutoff: energy and forces just inside equal
    those just outside (fc and its slope vanish there)."""
    w = W.weights(70, 1, model=MODEL)
    Z = np.array([6, 1] + [1] * len(extra), np.int32)
    res = []
    for eps in (-1e-9, 1e-9):
        pos = np.array([[0, 0, 0], [rc + eps, 0, 0]] + extra, np.float64)
        out = oracle.compute(Z, pos, np.array([0, len(Z)]), w, 1, model=MODEL)
        res.append((out["energy"][0], out["forces"]))
    assert res[0][0] == pytest.approx(res[1][0], abs=1e-9)
    np.testing.assert_allclose(res[0][1], res[1][1], atol=1e-7)

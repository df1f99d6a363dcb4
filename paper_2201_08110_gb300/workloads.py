"""Seeded synthetic inputs: molecules, batches, a periodic pocket, network weights.

This module only draws random inputs; it holds none of the method's
arithmetic, and both the CUDA path and the FP64 oracle consume what it
produces.  The paper's workload is four protein-bound ligands of 48-75 atoms
(Table 1) evaluated by ANI-2x with its 8-network ensemble (Sec. 2,
"Optimization"; Table 2).  Those structures and the trained weights are not
available, so seeded stand-ins of the same shape are drawn here:

* geometry: sequential random addition of uniform points in an 8 A cube,
  rejecting a point closer than 0.95 A to any accepted one (non-periodic);
  the periodic pocket uses the minimum-image distance in a cubic box;
* elements: H, C, N, O, F, S, Cl with probabilities .45/.35/.08/.08 and the
  remaining .04 shared equally by F, S and Cl;
* weights: Xavier-normal, W ~ N(0, 2 / (fan_in + fan_out)), drawn in the order
  model -> element (H, C, N, O, F, S, Cl) -> layer, with zero biases unless
  ``bias_std`` is given.

Workloads (seed of workload k is 1000 + k, its weights use seed + 1):

1. one 24-atom molecule H12 C8 N2 O2, one network (correctness);
2. one 60-atom molecule H27 C21 N5 O4 F1 S1 Cl1, 8 networks, positions
   perturbed by independent N(0, 0.01^2) A noise per step;
3. 512 molecules, atom counts uniform in [20, 120], 8 networks;
4. the batch of 3, with the networks' matrix products in BF16 / FP16;
5. 4096 molecules, counts log-uniform in [30, 250], plus one 1500-atom
   periodic pocket (24.7 A cube, density 0.1 / A^3).

For the NNP-MM coupling term (Eq. 4) the molecule of workload 2 is placed in
an MM region of the size of the paper's solvated systems (Table 1: 38-60 k
atoms): TIP3P-like water (O -0.834 e, two H +0.417 e at 0.9572 A and
104.52 degrees; Lennard-Jones sigma / eps 3.15061 A / 0.1521 kcal/mol on O,
none on H) at 0.1 atoms / A^3 around it, and the NNP atoms get charges
N(0, 0.3^2) shifted to a zero total with sigma ~ U(2.5, 3.5) A and
eps ~ U(0.02, 0.2) kcal/mol (GAFF2-like ranges).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

ELEMENTS_Z = (1, 6, 7, 8, 9, 16, 17)
ELEMENT_P = (0.45, 0.35, 0.08, 0.08, 0.04 / 3, 0.04 / 3, 0.04 / 3)
# Hidden widths per element for the ANI-2x architecture (input 1008, output 1).
HIDDEN = ((256, 192, 160), (224, 192, 160), (192, 160, 128), (192, 160, 128),
          (160, 128, 96), (160, 128, 96), (160, 128, 96))
N_INPUT = 1008
# The ANI-1x architecture: elements H, C, N, O, input 384.
ELEMENTS_Z_ANI1X = (1, 6, 7, 8)
HIDDEN_ANI1X = ((160, 128, 96), (144, 112, 96), (128, 112, 96), (128, 112, 96))
N_INPUT_ANI1X = 384
# H, C, N, O molecules for the ANI-1x model: the mix above without F/S/Cl,
# renormalised
ELEMENT_P_ANI1X = tuple(p / 0.96 for p in (0.45, 0.35, 0.08, 0.08))


@dataclass
class Batch:
    """A batch of molecules: atoms of molecule m are [mol_off[m], mol_off[m+1])."""
    Z: np.ndarray            # int32 [N]
    pos: np.ndarray          # float32 [N, 3], Angstrom
    mol_off: np.ndarray      # int32 [n_mols + 1]
    box: np.ndarray = field(default_factory=lambda: np.zeros(3))  # zeros = non-periodic

    @property
    def n_atoms(self) -> int:
        return int(self.mol_off[-1])

    @property
    def n_mols(self) -> int:
        return int(self.mol_off.shape[0] - 1)

    def molecule(self, m: int) -> "Batch":
        a, b = int(self.mol_off[m]), int(self.mol_off[m + 1])
        return Batch(self.Z[a:b].copy(), self.pos[a:b].copy(),
                     np.array([0, b - a], dtype=np.int32), self.box.copy())


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def geometry(g: np.random.Generator, n: int, edge: float = 8.0, dmin: float = 0.95,
             periodic: bool = False, max_tries: int = 100000) -> np.ndarray:
    """n points in [0, edge)^3 by sequential random addition with a minimum
    separation (minimum image when periodic).  Returns float32 [n, 3]."""
    out = np.zeros((n, 3), dtype=np.float64)
    k = 0
    tries = 0
    d2min = dmin * dmin
    while k < n:
        cand = g.random(3) * edge
        cand = cand.astype(np.float32).astype(np.float64)
        tries += 1
        if tries > max_tries * max(n, 1):
            raise RuntimeError("geometry: could not place atoms at this density")
        if k:
            d = out[:k] - cand
            if periodic:
                d -= edge * np.round(d / edge)
            if np.min(np.einsum("ij,ij->i", d, d)) < d2min:
                continue
        out[k] = cand
        k += 1
    return out.astype(np.float32)


def species_iid(g: np.random.Generator, n: int, model: str = "ani2x") -> np.ndarray:
    zs, ps = (ELEMENTS_Z, ELEMENT_P) if model == "ani2x" else (ELEMENTS_Z_ANI1X, ELEMENT_P_ANI1X)
    idx = g.choice(len(zs), size=n, p=np.array(ps))
    return np.asarray(zs, dtype=np.int32)[idx]


def species_counts(g: np.random.Generator, counts) -> np.ndarray:
    """Fixed element counts (H, C, N, O, F, S, Cl), shuffled into a random order."""
    Z = np.concatenate([np.full(c, z, dtype=np.int32) for z, c in zip(ELEMENTS_Z, counts)])
    g.shuffle(Z)
    return Z


def single(seed: int, counts, edge: float = 8.0) -> Batch:
    g = rng(seed)
    Z = species_counts(g, counts)
    pos = geometry(g, Z.shape[0], edge=edge)
    return Batch(Z, pos, np.array([0, Z.shape[0]], dtype=np.int32))


def batch(seed: int, sizes, model: str = "ani2x") -> Batch:
    """Molecules with the given atom counts, species i.i.d. from the mix."""
    g = rng(seed)
    Zs, Ps, off = [], [], [0]
    for n in sizes:
        n = int(n)
        Zs.append(species_iid(g, n, model))
        Ps.append(geometry(g, n))
        off.append(off[-1] + n)
    Z = np.concatenate(Zs) if Zs else np.zeros(0, np.int32)
    P = np.concatenate(Ps) if Ps else np.zeros((0, 3), np.float32)
    return Batch(Z.astype(np.int32), P.astype(np.float32), np.asarray(off, dtype=np.int32))


def pocket(seed: int, n: int = 1500, edge: float = 24.7, model: str = "ani2x") -> Batch:
    """One periodic region of n atoms in a cubic box."""
    g = rng(seed)
    Z = species_iid(g, n, model)
    pos = geometry(g, n, edge=edge, periodic=True)
    return Batch(Z, pos, np.array([0, n], dtype=np.int32), np.full(3, edge))


def architecture(model: str = "ani2x"):
    """(elements, hidden widths per element, input width) of a model."""
    if model == "ani2x":
        return ELEMENTS_Z, HIDDEN, N_INPUT
    if model == "ani1x":
        return ELEMENTS_Z_ANI1X, HIDDEN_ANI1X, N_INPUT_ANI1X
    raise ValueError(model)


def weights(seed: int, n_models: int, bias_std: float = 0.0, model: str = "ani2x") -> np.ndarray:
    """Packed FP32 parameters [model][element][W1 b1 W2 b2 W3 b3 w4 b4],
    each W row-major [out][in]."""
    zs, hidden, n_in = architecture(model)
    g = rng(seed)
    chunks = []
    for _m in range(n_models):
        for e in range(len(zs)):
            dims = (n_in,) + hidden[e] + (1,)
            for l in range(4):
                fi, fo = dims[l], dims[l + 1]
                std = np.sqrt(2.0 / (fi + fo))
                chunks.append((g.standard_normal((fo, fi)) * std).astype(np.float32).ravel())
                if bias_std > 0:
                    chunks.append((g.standard_normal(fo) * bias_std).astype(np.float32))
                else:
                    chunks.append(np.zeros(fo, dtype=np.float32))
    return np.concatenate(chunks)


def weights_per_model(model: str = "ani2x") -> int:
    zs, hidden, n_in = architecture(model)
    s = 0
    for e in range(len(zs)):
        dims = (n_in,) + hidden[e] + (1,)
        s += sum(dims[l] * dims[l + 1] + dims[l + 1] for l in range(4))
    return s


def perturb(g: np.random.Generator, pos: np.ndarray, sigma: float = 0.01) -> np.ndarray:
    return (pos.astype(np.float64) + g.normal(0.0, sigma, size=pos.shape)).astype(np.float32)


# --- the five workloads -------------------------------------------------------

def workload_seed(k: int) -> int:
    return 1000 + k


def config1() -> tuple[Batch, np.ndarray, int]:
    s = workload_seed(1)
    return single(s, (12, 8, 2, 2, 0, 0, 0)), weights(s + 1, 1), 1


def config2() -> tuple[Batch, np.ndarray, int]:
    s = workload_seed(2)
    return single(s, (27, 21, 5, 4, 1, 1, 1)), weights(s + 1, 8), 8


def config3_sizes(n_mols: int = 512) -> np.ndarray:
    return rng(workload_seed(3) + 100).integers(20, 121, size=n_mols)


def config3(n_mols: int = 512) -> tuple[Batch, np.ndarray, int]:
    s = workload_seed(3)
    return batch(s, config3_sizes(n_mols)), weights(s + 1, 8), 8


def config3_ani1x(n_mols: int = 512) -> tuple[Batch, np.ndarray, int]:
    """The 512-molecule batch's sizes with H, C, N, O molecules and an
    8-network ANI-1x ensemble (the second model of Sec. 3)."""
    s = workload_seed(3) + 10
    return batch(s, config3_sizes(n_mols), model="ani1x"), weights(s + 1, 8, model="ani1x"), 8


def config5_sizes(n_mols: int = 4096) -> np.ndarray:
    u = rng(workload_seed(5) + 100).uniform(np.log(30.0), np.log(250.0), size=n_mols)
    return np.rint(np.exp(u)).astype(np.int64)


def config5(n_mols: int = 4096) -> tuple[Batch, Batch, np.ndarray, int]:
    s = workload_seed(5)
    return batch(s, config5_sizes(n_mols)), pocket(s + 2), weights(s + 1, 8), 8


# --- the MM region around an NNP region (coupling term, Eq. 4) ----------------

COULOMB_KCAL = 332.0637133  # 1 / (4 pi eps0) in kcal/mol * A / e^2


@dataclass
class Environment:
    """Coupling-term inputs: per-atom Lennard-Jones parameters and charges of the
    NNP atoms (in the order of their positions) and the MM atoms."""
    nnp_q: np.ndarray       # float32 [n_nnp], e
    nnp_sigma: np.ndarray   # float32 [n_nnp], A
    nnp_eps: np.ndarray     # float32 [n_nnp], kcal/mol
    mm_pos: np.ndarray      # float32 [n_mm, 3], A
    mm_q: np.ndarray        # float32 [n_mm]
    mm_sigma: np.ndarray    # float32 [n_mm]
    mm_eps: np.ndarray      # float32 [n_mm]

    @property
    def n_mm(self) -> int:
        return int(self.mm_pos.shape[0])


def mm_environment(seed: int, nnp_pos: np.ndarray, n_mm: int = 60000, density: float = 0.1,
                   dmin: float = 2.0) -> Environment:
    """Water-like MM atoms around the NNP atoms nnp_pos [n, 3]: oxygens uniform
    in a cube of n_mm / density A^3 centred on the NNP region (enlarged, for
    small n_mm, to the NNP region plus twice the exclusion distance and 4 A),
    none closer than dmin + 1 A to an NNP atom, each followed by its two
    hydrogens (a randomly oriented H-O-H of 104.52 degrees, 0.9572 A bonds);
    the last water is cut short when n_mm is not a multiple of 3."""
    g = rng(seed)
    nnp_pos = np.asarray(nnp_pos, dtype=np.float64).reshape(-1, 3)
    n_nnp = nnp_pos.shape[0]
    q = g.normal(0.0, 0.3, size=n_nnp)
    q -= q.mean()
    sig = g.uniform(2.5, 3.5, size=n_nnp)
    eps = g.uniform(0.02, 0.2, size=n_nnp)
    n_w = (n_mm + 2) // 3
    span = float(np.ptp(nnp_pos, axis=0).max()) if n_nnp else 0.0
    edge = max((n_mm / density) ** (1.0 / 3.0), span + 2.0 * (dmin + 1.0) + 4.0)
    centre = nnp_pos.mean(axis=0) if n_nnp else np.zeros(3)
    oxy = np.zeros((0, 3))
    for _ in range(1000):  # the corners of the cube always stay outside the exclusion
        if oxy.shape[0] >= n_w:
            break
        cand = centre + g.uniform(-0.5 * edge, 0.5 * edge, size=(2 * n_w + 16, 3))
        if n_nnp:
            d2 = ((cand[:, None, :] - nnp_pos[None, :, :]) ** 2).sum(-1).min(axis=1)
            cand = cand[d2 >= (dmin + 1.0) ** 2]
        oxy = np.concatenate([oxy, cand])[:n_w]
    if oxy.shape[0] < n_w:
        raise RuntimeError("mm_environment: could not place the oxygens")
    # two hydrogens per oxygen: bond vectors in a random frame
    half = 0.5 * np.deg2rad(104.52)
    local = 0.9572 * np.array([[np.sin(half), 0.0, np.cos(half)],
                               [-np.sin(half), 0.0, np.cos(half)]])
    a = g.normal(size=(n_w, 3))
    a /= np.linalg.norm(a, axis=1, keepdims=True)
    b = g.normal(size=(n_w, 3))
    b -= (b * a).sum(1, keepdims=True) * a
    b /= np.linalg.norm(b, axis=1, keepdims=True)
    c = np.cross(a, b)
    frames = np.stack([b, c, a], axis=1)  # rows: x, y, z axes of each water
    hyd = oxy[:, None, :] + np.einsum("hk,wkd->whd", local, frames)
    pos = np.concatenate([oxy[:, None, :], hyd], axis=1).reshape(-1, 3)[:n_mm]
    mq = np.tile([-0.834, 0.417, 0.417], n_w)[:n_mm]
    ms = np.tile([3.15061, 0.0, 0.0], n_w)[:n_mm]
    me = np.tile([0.1521, 0.0, 0.0], n_w)[:n_mm]
    f32 = lambda x: np.ascontiguousarray(x, dtype=np.float32)
    return Environment(f32(q), f32(sig), f32(eps), f32(pos), f32(mq), f32(ms), f32(me))


def coupling_config(n_mm: int = 60000) -> tuple[Batch, Environment]:
    """The 60-atom molecule of workload 2 in an MM region of n_mm atoms."""
    b, _, _ = config2()
    return b, mm_environment(workload_seed(2) + 50, b.pos, n_mm)

"""FP64 CPU oracle for the ANI-2x-style NNP energy and forces.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package.  The
product path (``paper_2201_08110_gb300``) never imports it and shares no code,
table or constant with it.

The arithmetic lives in ``ani_oracle.c`` (plain C, FP64, built with
``-ffp-contract=off`` so every product and sum is rounded on its own); this
module compiles it with gcc on first use and marshals numpy arrays.  What is
computed is the NNP term V_NNP(Z, r) of the paper's Sec. 2 (Eqs. 2-3) and
F = -grad V_NNP, with the ANI featurizer and ensemble of atomic networks the
paper names in Sec. 1 and Sec. 2 ("Optimization"): model "ani2x" (7 elements,
1008 features, the default) or "ani1x" (H, C, N, O, 384 features; the other
ANI model the paper runs, Sec. 3 "Extensibility with other NNPs").  The functional form is
written out in the header of ``ani_oracle.c``; the NNP-MM coupling term of
Eq. 4 (``coupling``) is written out beside its function there.  The MD
integrators of the step loop around both terms (``md_velocity_verlet``,
``md_langevin_baoab``) are plain numpy.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ani_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD_DIR, "libani_oracle.so")

NUM_FEATURES = 1008
ELEMENTS_Z = (1, 6, 7, 8, 9, 16, 17)
MODELS = {"ani2x": 0, "ani1x": 1}
MODEL_ELEMENTS = {"ani2x": (1, 6, 7, 8, 9, 16, 17), "ani1x": (1, 6, 7, 8)}
MODEL_FEATURES = {"ani2x": 1008, "ani1x": 384}

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ani_oracle.c into a shared library (gcc, OpenMP, FP64)."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(_SRC)):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-fno-fast-math", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        lib.ani_oracle_weights_per_model.restype = ctypes.c_long
        lib.ani_oracle_weights_per_model_m.restype = ctypes.c_long
        lib.ani_oracle_weights_per_model_m.argtypes = [ctypes.c_int]
        lib.ani_oracle_compute.restype = ctypes.c_int
        lib.ani_oracle_compute.argtypes = [ctypes.c_int, P, P, P, P, ctypes.c_int, P,
                                           ctypes.c_long, P, P, P, P, P, ctypes.c_int]
        lib.ani_oracle_compute_m.restype = ctypes.c_int
        lib.ani_oracle_compute_m.argtypes = [ctypes.c_int, ctypes.c_int, P, P, P, P, ctypes.c_int, P,
                                             ctypes.c_long, P, P, P, P, P, ctypes.c_int]
        lib.ani_oracle_pairs.restype = ctypes.c_long
        lib.ani_oracle_pairs.argtypes = [ctypes.c_int, P, P, ctypes.c_double, P, P, ctypes.c_long]
        lib.ani_oracle_triples.restype = ctypes.c_long
        lib.ani_oracle_triples.argtypes = [ctypes.c_int, P, P, ctypes.c_double, P, P, P,
                                           ctypes.c_long]
        lib.ani_oracle_aev_m.restype = ctypes.c_int
        lib.ani_oracle_aev_m.argtypes = [ctypes.c_int, ctypes.c_int, P, P, P, P]
        lib.ani_oracle_aev_adjoint_m.restype = ctypes.c_int
        lib.ani_oracle_aev_adjoint_m.argtypes = [ctypes.c_int, ctypes.c_int, P, P, P, P, P]
        lib.ani_oracle_hyper_m.restype = ctypes.c_int
        lib.ani_oracle_hyper_m.argtypes = [ctypes.c_int, P]
        lib.ani_oracle_coupling.restype = ctypes.c_int
        lib.ani_oracle_coupling.argtypes = [ctypes.c_int, P, P, P, P, ctypes.c_int, P, P, P, P,
                                            ctypes.c_double, P, P, P, P, P, P]
        _lib = lib
        return lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _box(box):
    if box is None:
        return None
    b = np.ascontiguousarray(box, dtype=np.float64).reshape(3)
    if not np.any(b):
        return None
    return b


def _model(model) -> int:
    if model not in MODELS:
        raise ValueError(f"oracle: unknown model {model!r}")
    return MODELS[model]


def weights_per_model(model: str = "ani2x") -> int:
    return int(_load().ani_oracle_weights_per_model_m(_model(model)))


_GRIDS = {"ani2x": (16, 8, 4), "ani1x": (16, 4, 8)}


def hyper(model: str = "ani2x") -> dict:
    """The featurizer constants as the oracle uses them."""
    out = np.zeros(5 + 48, dtype=np.float64)
    _load().ani_oracle_hyper_m(_model(model), _ptr(out))
    nr, na, nz = _GRIDS[model]
    return {"Rcr": out[0], "Rca": out[1], "EtaR": out[2], "EtaA": out[3], "Zeta": out[4],
            "ShfR": out[5:5 + nr].copy(), "ShfA": out[5 + nr:5 + nr + na].copy(),
            "ShfZ": out[5 + nr + na:5 + nr + na + nz].copy()}


def compute(Z, pos, mol_off, weights, n_models, box=None, forces=True, aev=False,
            atom_energies=False, dEdG=False, nthreads=0, model: str = "ani2x"):
    """Energies [n_mols] and (optionally) forces [N,3], features [N,F],
    per-atom energies [N] and dE/dG [N,F] of a batch, all FP64 (F = 1008 for
    "ani2x", 384 for "ani1x").

    pos may be float32 or float64; float32 values are promoted exactly.
    """
    lib = _load()
    nf = MODEL_FEATURES[model]
    Z = np.ascontiguousarray(Z, dtype=np.int32)
    pos = np.ascontiguousarray(pos, dtype=np.float64).reshape(-1, 3)
    mol_off = np.ascontiguousarray(mol_off, dtype=np.int32)
    w = np.ascontiguousarray(weights, dtype=np.float32).reshape(-1)
    n = int(mol_off[-1])
    assert Z.shape[0] == n and pos.shape[0] == n
    n_mols = mol_off.shape[0] - 1
    E = np.zeros(n_mols, dtype=np.float64)
    F = np.zeros((n, 3), dtype=np.float64) if (forces or dEdG) else None
    G = np.zeros((n, nf), dtype=np.float64) if aev else None
    Ea = np.zeros(n, dtype=np.float64) if atom_energies else None
    dG = np.zeros((n, nf), dtype=np.float64) if dEdG else None
    rc = lib.ani_oracle_compute_m(_model(model), n_mols, _ptr(mol_off), _ptr(Z), _ptr(pos),
                                  _ptr(_box(box)), int(n_models), _ptr(w), int(w.size), _ptr(E),
                                  _ptr(F), _ptr(G), _ptr(Ea), _ptr(dG), int(nthreads))
    if rc == -1:
        raise ValueError("oracle: unsupported atomic number")
    if rc != 0:
        raise ValueError(f"oracle: bad arguments (code {rc})")
    out = {"energy": E}
    if forces:
        out["forces"] = F
    if aev:
        out["aev"] = G
    if atom_energies:
        out["atom_energies"] = Ea
    if dEdG:
        out["dEdG"] = dG
    return out


def energy(Z, pos, weights, n_models, box=None, model: str = "ani2x"):
    """Energy of a single molecule (all atoms), FP64."""
    n = len(Z)
    return float(compute(Z, pos, np.array([0, n]), weights, n_models, box=box,
                         forces=False, model=model)["energy"][0])


def pairs(pos, rc, box=None):
    """Ordered pairs (i, j), i != j, with d^2 < rc^2 (FP64 predicate)."""
    lib = _load()
    pos = np.ascontiguousarray(pos, dtype=np.float64).reshape(-1, 3)
    n = pos.shape[0]
    cap = max(1, n * (n - 1))
    I = np.zeros(cap, dtype=np.int32)
    J = np.zeros(cap, dtype=np.int32)
    cnt = lib.ani_oracle_pairs(n, _ptr(pos), _ptr(_box(box)), float(rc), _ptr(I), _ptr(J), cap)
    return np.stack([I[:cnt], J[:cnt]], axis=1)


def triples(pos, rc, box=None):
    """Triples (i, j, k), j < k, both within rc of centre i."""
    lib = _load()
    pos = np.ascontiguousarray(pos, dtype=np.float64).reshape(-1, 3)
    n = pos.shape[0]
    cap = max(1, n * (n - 1) * (n - 2) // 2)
    I = np.zeros(cap, dtype=np.int32)
    J = np.zeros(cap, dtype=np.int32)
    K = np.zeros(cap, dtype=np.int32)
    cnt = lib.ani_oracle_triples(n, _ptr(pos), _ptr(_box(box)), float(rc), _ptr(I), _ptr(J),
                                 _ptr(K), cap)
    return np.stack([I[:cnt], J[:cnt], K[:cnt]], axis=1)


def aev(Z, pos, box=None, model: str = "ani2x"):
    """Feature vectors [n, F] of one molecule, FP64."""
    lib = _load()
    Z = np.ascontiguousarray(Z, dtype=np.int32)
    pos = np.ascontiguousarray(pos, dtype=np.float64).reshape(-1, 3)
    out = np.zeros((Z.shape[0], MODEL_FEATURES[model]), dtype=np.float64)
    if lib.ani_oracle_aev_m(_model(model), Z.shape[0], _ptr(Z), _ptr(pos), _ptr(_box(box)),
                            _ptr(out)) != 0:
        raise ValueError("oracle: unsupported atomic number")
    return out


def aev_adjoint(Z, pos, g, box=None, model: str = "ani2x"):
    """d(sum_i g_i . G_i)/dx for one molecule, FP64 [n, 3]."""
    lib = _load()
    Z = np.ascontiguousarray(Z, dtype=np.int32)
    pos = np.ascontiguousarray(pos, dtype=np.float64).reshape(-1, 3)
    g = np.ascontiguousarray(g, dtype=np.float64).reshape(Z.shape[0], MODEL_FEATURES[model])
    out = np.zeros((Z.shape[0], 3), dtype=np.float64)
    if lib.ani_oracle_aev_adjoint_m(_model(model), Z.shape[0], _ptr(Z), _ptr(pos), _ptr(_box(box)),
                                    _ptr(g), _ptr(out)) != 0:
        raise ValueError("oracle: unsupported atomic number")
    return out


def coupling(nnp_pos, nnp_q, nnp_sigma, nnp_eps, mm_pos, mm_q, mm_sigma, mm_eps, ke,
             norms=False):
    """The NNP-MM coupling term of Eq. 4 (Coulomb + Lennard-Jones over every
    NNP-MM pair, Lorentz-Berthelot combination, no cutoff): FP64 energy and
    forces (-dV/dx) on the NNP atoms [n_nnp, 3] and the MM atoms [n_mm, 3].
    norms=True also returns the sum of the squared pair energies and, per atom,
    the sum of the magnitudes of its pair forces (NNP, MM): the scales of the
    rounding error of a sum of independently rounded terms."""
    lib = _load()
    f64 = lambda a: np.ascontiguousarray(a, dtype=np.float64)
    xn, xm = f64(nnp_pos).reshape(-1, 3), f64(mm_pos).reshape(-1, 3)
    qn, sn, en = f64(nnp_q), f64(nnp_sigma), f64(nnp_eps)
    qm, sm, em = f64(mm_q), f64(mm_sigma), f64(mm_eps)
    n_nnp, n_mm = xn.shape[0], xm.shape[0]
    for a, n in ((qn, n_nnp), (sn, n_nnp), (en, n_nnp), (qm, n_mm), (sm, n_mm), (em, n_mm)):
        if a.shape != (n,):
            raise ValueError("oracle: parameter arrays must match the atom counts")
    e = np.zeros(1, dtype=np.float64)
    fn = np.zeros((n_nnp, 3), dtype=np.float64)
    fm = np.zeros((n_mm, 3), dtype=np.float64)
    e2 = np.zeros(1, dtype=np.float64)
    gn = np.zeros(n_nnp, dtype=np.float64)
    gm = np.zeros(n_mm, dtype=np.float64)
    if lib.ani_oracle_coupling(n_nnp, _ptr(xn), _ptr(qn), _ptr(sn), _ptr(en), n_mm, _ptr(xm),
                               _ptr(qm), _ptr(sm), _ptr(em), float(ke), _ptr(e), _ptr(fn),
                               _ptr(fm), _ptr(e2), _ptr(gn), _ptr(gm)) != 0:
        raise ValueError("oracle: an NNP atom and an MM atom coincide")
    if norms:
        return float(e[0]), fn, fm, float(e2[0]), gn, gm
    return float(e[0]), fn, fm


def md_velocity_verlet(x0, v0, masses, force, dt, n_steps):
    """Velocity Verlet (the NVE integrator of an MD step loop) in FP64: for
    each step, v += dt/2 F/m; x += dt v; F = force(x); v += dt/2 F/m.
    force(x) -> [n, 3] is -dV/dx.  Returns the positions and velocities after
    every step, [n_steps + 1, n, 3] each (index 0 = the input)."""
    x = np.array(x0, dtype=np.float64).reshape(-1, 3)
    v = np.array(v0, dtype=np.float64).reshape(-1, 3)
    m = np.asarray(masses, dtype=np.float64).reshape(-1, 1)
    xs, vs = [x.copy()], [v.copy()]
    f = np.asarray(force(x), dtype=np.float64)
    for _ in range(n_steps):
        v = v + 0.5 * dt * f / m
        x = x + dt * v
        f = np.asarray(force(x), dtype=np.float64)
        v = v + 0.5 * dt * f / m
        xs.append(x.copy())
        vs.append(v.copy())
    return np.stack(xs), np.stack(vs)


def md_langevin_baoab(x0, v0, masses, force, dt, gamma, kT, noise):
    """Langevin dynamics by the BAOAB splitting in FP64, one step per row of
    noise [n_steps, n, 3] (standard normal draws, passed in so that any
    implementation can use the same ones): B: v += dt/2 F/m; A: x += dt/2 v;
    O: v = c1 v + c2 sqrt(kT/m) xi with c1 = exp(-gamma dt), c2 = sqrt(1 - c1^2);
    A: x += dt/2 v; F = force(x); B: v += dt/2 F/m.  Returns positions and
    velocities after every step, [n_steps + 1, n, 3] each."""
    x = np.array(x0, dtype=np.float64).reshape(-1, 3)
    v = np.array(v0, dtype=np.float64).reshape(-1, 3)
    m = np.asarray(masses, dtype=np.float64).reshape(-1, 1)
    c1 = np.exp(-gamma * dt)
    c2 = np.sqrt(1.0 - c1 * c1)
    xs, vs = [x.copy()], [v.copy()]
    f = np.asarray(force(x), dtype=np.float64)
    for xi in np.asarray(noise, dtype=np.float64):
        v = v + 0.5 * dt * f / m
        x = x + 0.5 * dt * v
        v = c1 * v + c2 * np.sqrt(kT / m) * xi
        x = x + 0.5 * dt * v
        f = np.asarray(force(x), dtype=np.float64)
        v = v + 0.5 * dt * f / m
        xs.append(x.copy())
        vs.append(v.copy())
    return np.stack(xs), np.stack(vs)

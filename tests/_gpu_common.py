"""Helpers shared by the GPU parity tests: building the library, running the
oracle on the same seeded inputs, and the error measures with their bounds.

Tolerances (per molecule, against the FP64 oracle):
* FP32 networks: |dE| / |E| <= 1e-5 and max |dF| <= 1e-4 * RMS(F_ref);
* BF16 / FP16 networks: |dE| / |E| <= 2e-3 and RMS(dF) / RMS(F_ref) <= 1e-2.
When |E_ref| < 1e-3 * sum_i |E_i,ref| (cancellation between atomic energies of
random-weight networks), the energy bound applies to sum_i |E_i,ref| instead.
"""
import numpy as np

import oracle

TOL = {"fp32": {"e": 1e-5, "f_max": 1e-4}, "bf16": {"e": 2e-3, "f_rms": 1e-2},
       "fp16": {"e": 2e-3, "f_rms": 1e-2}}


def oracle_batch(b, w, M, mols=None, aev=False):
    """Oracle energies/forces (and per-atom energies) for the given molecules
    of a batch (all by default); returns per-molecule dicts."""
    mols = range(b.n_mols) if mols is None else mols
    out = {}
    for m in mols:
        sub = b.molecule(m)
        r = oracle.compute(sub.Z, sub.pos, sub.mol_off, w, M, box=b.box, aev=aev, atom_energies=True)
        out[m] = r
    return out


def energy_error(E, ref):
    """Relative energy error with the cancellation rule."""
    denom = abs(ref["energy"][0])
    s = np.sum(np.abs(ref["atom_energies"]))
    if denom < 1e-3 * s:
        denom = s
    return abs(E - ref["energy"][0]) / max(denom, 1e-300)


def force_errors(F, Fref):
    rms = np.sqrt(np.mean(Fref ** 2)) if Fref.size else 0.0
    if rms == 0.0:
        return 0.0, 0.0
    d = F - Fref
    return np.max(np.abs(d)) / rms, np.sqrt(np.mean(d ** 2)) / rms


def check_batch(prec, E, F, b, refs):
    """Asserts the tolerances of `prec` on every molecule in refs; returns the
    worst errors (reported by the caller)."""
    tol = TOL[prec]
    worst = {"e": 0.0, "f_max": 0.0, "f_rms": 0.0}
    for m, ref in refs.items():
        a0, a1 = int(b.mol_off[m]), int(b.mol_off[m + 1])
        ee = energy_error(E[m], ref)
        fm, fr = force_errors(F[a0:a1], ref["forces"]) if F is not None else (0.0, 0.0)
        worst["e"] = max(worst["e"], ee)
        worst["f_max"] = max(worst["f_max"], fm)
        worst["f_rms"] = max(worst["f_rms"], fr)
        assert ee <= tol["e"], f"{prec} molecule {m}: energy error {ee:.3e} > {tol['e']}"
        if "f_max" in tol:
            assert fm <= tol["f_max"], f"{prec} molecule {m}: max force error {fm:.3e}"
        if "f_rms" in tol:
            assert fr <= tol["f_rms"], f"{prec} molecule {m}: rms force error {fr:.3e}"
    return worst

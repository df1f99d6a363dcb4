"""Helpers shared by the GPU parity tests: building the library, running the
oracle on the same seeded inputs, and the error measures with their bounds.

Tolerances (per molecule, against the FP64 oracle):
* FP32 networks: |dE| / S <= 1e-5 and max |dF| <= 1e-4 * RMS(F_ref);
* FP16 networks: |dE| / S <= 2e-3 and RMS(dF) / RMS(F_ref) <= 1e-2;
* BF16 networks, one pass: |dE| / S <= 6e-3 and RMS(dF) / RMS(F_ref) <= 1e-2.
S = sum_i |E_i,ref| is the molecule's gross atomic energy.  It equals |E_ref|
when the atomic energies share a sign (ANI's per-element offsets make them
do), and it stays well conditioned when the atomic energies of random-weight
networks cancel (|E_ref| reaches 1e-3 S on these workloads).  |dE| / |E_ref|
is reported alongside.  The single-pass BF16 bound is derived from the
arithmetic: rounding the weights to 8 significant bits perturbs every atom of
an element the same way, so the energy error grows with S rather than with
its square root; on the 512-molecule batch this reaches 3.6e-3 S, above the
2e-3 of the FP16 bound.
"""
import numpy as np

import oracle

TOL = {"fp32": {"e": 1e-5, "f_max": 1e-4}, "bf16": {"e": 6e-3, "f_rms": 1e-2},
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
    """|dE| / S with S the gross atomic energy sum_i |E_i,ref|."""
    s = np.sum(np.abs(ref["atom_energies"]))
    return abs(E - ref["energy"][0]) / max(s, 1e-300)


def energy_error_plain(E, ref):
    return abs(E - ref["energy"][0]) / max(abs(ref["energy"][0]), 1e-300)


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
    worst = {"e": 0.0, "e_plain": 0.0, "f_max": 0.0, "f_rms": 0.0}
    for m, ref in refs.items():
        a0, a1 = int(b.mol_off[m]), int(b.mol_off[m + 1])
        ee = energy_error(E[m], ref)
        worst["e_plain"] = max(worst["e_plain"], energy_error_plain(E[m], ref))
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

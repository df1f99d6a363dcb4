"""Central differences of the GPU energy against the GPU forces, with a bound
that accounts for the noise of an FP32 or 16-bit path.

The oracle's analytic gradient is checked against central differences in
FP64 (tests/test_oracle_pins.py). Here the GPU path is differentiated
numerically, following the finite-difference reading of the oracle section.
With FP32 positions and FP32 (or 16-bit) networks, a plain tolerance on the
difference quotient is meaningless at small h: an energy error e becomes a
quotient error of up to 2e / D. The bound adds the parts the parity rule
allows:

    |F_fd,gpu - F_gpu| <= |F_fd,oracle - F_oracle|     truncation at this step (FP64)
                          + f_tol RMS(F_oracle)        the analytic forces' allowed error
                          + 2 e_tol |E_oracle| / D     the energies' allowed error over the step

e_tol and f_tol are the parity rule's energy and force tolerances:
* FP32: e_tol 1e-5 (relative), f_tol 1e-4 (max component);
* split BF16: e_tol 2e-3, f_tol 0.1. The rule bounds the RMS force error by
  1e-2; its components reach 3.5e-2 of RMS(F) on the 512-molecule batch.

The central difference uses the FP32 positions x + h and x - h, and D is
their exact difference. The test prints each part beside the measured
quotient error. Workload 2's 60-atom molecule with 8 networks, twelve seeded
coordinates. h = 2e-3 A for FP32: the energy-noise part is then about 5 % of
RMS(F). h = 2e-2 A for BF16, whose allowed energy error makes the quotient
a weak check at any step (the part is then about RMS(F) itself, while the
truncation part stays near 1e-4 of it).
"""
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


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_central_differences_of_the_gpu_energy(lib, prec):
    b, w, M = W.config2()
    h = 2e-3 if prec == "fp32" else 2e-2
    model = lib.NNP(b.Z, w, M, mol_off=b.mol_off, precision=prec)
    x0 = b.pos.astype(np.float32)

    def gpu(p, forces=True):
        E, F = model.compute(torch.tensor(p, device="cuda"), forces=forces)
        torch.cuda.synchronize()
        model.status()
        return float(E.cpu().numpy()[0]), (None if F is None else F.cpu().numpy())

    E0, F0 = gpu(x0)
    ref0 = oracle.compute(b.Z, x0, b.mol_off, w, M)
    e_tol, f_tol = (1e-5, 1e-4) if prec == "fp32" else (2e-3, 0.1)
    rms_f = float(np.sqrt(np.mean(ref0["forces"] ** 2)))
    g = W.rng(71)
    picks = [(int(g.integers(b.n_atoms)), int(g.integers(3))) for _ in range(12)]
    worst = 0.0
    for a, k in picks:
        xp, xm = x0.copy(), x0.copy()
        xp[a, k] = np.float32(x0[a, k] + h)
        xm[a, k] = np.float32(x0[a, k] - h)
        D = float(xp[a, k]) - float(xm[a, k])  # exact in FP64
        Ep, _ = gpu(xp, forces=False)
        Em, _ = gpu(xm, forces=False)
        rp = oracle.compute(b.Z, xp, b.mol_off, w, M, forces=False)
        rm = oracle.compute(b.Z, xm, b.mol_off, w, M, forces=False)
        fd_gpu = -(Ep - Em) / D
        fd_orc = -(rp["energy"][0] - rm["energy"][0]) / D
        trunc = abs(fd_orc - ref0["forces"][a, k])
        analytic = f_tol * rms_f
        noise = 2.0 * e_tol * abs(ref0["energy"][0]) / D
        bound = trunc + analytic + noise
        err = abs(fd_gpu - F0[a, k])
        measured_noise = 2.0 * max(abs(Ep - rp["energy"][0]), abs(Em - rm["energy"][0])) / D
        worst = max(worst, err / bound)
        print(f"{prec} atom {a} dim {k}: |fd - F| {err:.3e}  bound {bound:.3e} "
              f"(truncation {trunc:.1e}, analytic {analytic:.1e} [measured {abs(F0[a, k] - ref0['forces'][a, k]):.1e}], "
              f"energy noise {noise:.1e} [measured {measured_noise:.1e}])")
        assert err <= bound, f"atom {a} dim {k}: {err:.3e} > {bound:.3e}"
    print(f"{prec}: worst |fd - F| / bound = {worst:.3f}")

"""Python binding of libnnp (include/nnp.h): argument marshalling only.

Every step of the energy/force evaluation runs in the library's CUDA kernels;
this module passes device pointers (from torch tensors), sizes and the CUDA
stream through the C ABI and turns status codes into exceptions.  If the
library is not built the import of the binding fails loudly: there is no
Python or CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libnnp.so")

FP32, BF16, FP16 = 0, 1, 2
_PREC = {"fp32": FP32, "bf16": BF16, "fp16": FP16}
ANI2X, ANI1X = 0, 1
_MODEL = {"ani2x": ANI2X, "ani1x": ANI1X}
STATUS = {0: "NNP_OK", 1: "NNP_ERR_ARG", 2: "NNP_ERR_SPECIES", 3: "NNP_ERR_CHARGE",
          4: "NNP_ERR_ALLOC", 5: "NNP_ERR_CUDA", 6: "NNP_ERR_CAPACITY", 7: "NNP_ERR_NONFINITE",
          8: "NNP_ERR_TIMEOUT", 9: "NNP_ERR_UNSUPPORTED", 10: "NNP_ERR_TOO_LARGE"}

# Every entry point declared in include/nnp.h.
EXPORTS = ("nnp_weights_per_model", "nnp_num_features", "nnp_weights_per_model_of",
           "nnp_num_features_of", "nnp_create", "nnp_create_batch",
           "nnp_compute", "nnp_compute_host", "nnp_get_status", "nnp_last_error", "nnp_destroy",
           "nnp_get_capacity", "nnp_get_neighbors", "nnp_get_features",
           "nnp_get_atomic_energies", "nnp_compute_timed", "nnp_kernels_per_step",
           "nnp_features_static", "nnp_autotune", "nnp_set_schedule", "nnp_mm_coupling",
           "nnp_md_create", "nnp_md_run", "nnp_md_last_error", "nnp_md_destroy")
STATIC_MAX_ATOMS = 256
COUPLING_MAX_NNP = 512
STAGES = ("neighbors", "features", "l1_fwd", "l2_fwd", "l3_fwd", "energy", "l3_rev", "l2_rev",
          "l1_rev", "adjoint")


class NNPError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code
        self.status = STATUS.get(code, str(code))


class Params(ctypes.Structure):
    _fields_ = [("n_models", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("weights", ctypes.c_void_p), ("n_weights", ctypes.c_int64),
                ("box", ctypes.c_double * 3), ("total_charge", ctypes.c_int32),
                ("max_neighbors", ctypes.c_int32), ("max_angular", ctypes.c_int32),
                ("use_graph", ctypes.c_int32), ("neighbor_mode", ctypes.c_int32),
                ("single_pass", ctypes.c_int32), ("recompute_aev", ctypes.c_int32),
                ("test_abort", ctypes.c_int32), ("model", ctypes.c_int32),
                ("single_cta", ctypes.c_int32), ("reserved", ctypes.c_int32 * 2)]


class MDParams(ctypes.Structure):
    _fields_ = [("integrator", ctypes.c_int32), ("dt", ctypes.c_double), ("gamma", ctypes.c_double),
                ("kT", ctypes.c_double), ("masses", ctypes.c_void_p), ("n_mm", ctypes.c_int32),
                ("mm_positions_dev", ctypes.c_void_p), ("mm_charges_dev", ctypes.c_void_p),
                ("mm_sigma_dev", ctypes.c_void_p), ("mm_epsilon_dev", ctypes.c_void_p),
                ("nnp_charges_dev", ctypes.c_void_p), ("nnp_sigma_dev", ctypes.c_void_p),
                ("nnp_epsilon_dev", ctypes.c_void_p), ("coulomb_k", ctypes.c_double),
                ("concurrent", ctypes.c_int32), ("reserved", ctypes.c_int32 * 8)]


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libnnp.so; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libnnp is not built ({path} missing): run "
                          "`python -m paper_2201_08110_gb300.build` (needs nvcc)")
    lib = ctypes.CDLL(path)
    P, I32, I64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    lib.nnp_weights_per_model.restype = I64
    lib.nnp_num_features.restype = I32
    lib.nnp_weights_per_model_of.argtypes = [I32]
    lib.nnp_weights_per_model_of.restype = I64
    lib.nnp_num_features_of.argtypes = [I32]
    lib.nnp_num_features_of.restype = I32
    lib.nnp_create.argtypes = [P, I32, P, P]
    lib.nnp_create.restype = ctypes.c_int
    lib.nnp_create_batch.argtypes = [P, P, I32, P, P]
    lib.nnp_create_batch.restype = ctypes.c_int
    lib.nnp_compute.argtypes = [P, P, P, P, P]
    lib.nnp_compute.restype = ctypes.c_int
    lib.nnp_compute_host.argtypes = [P, P, P, P, P]
    lib.nnp_compute_host.restype = ctypes.c_int
    lib.nnp_get_status.argtypes = [P]
    lib.nnp_get_status.restype = ctypes.c_int
    lib.nnp_last_error.argtypes = [P]
    lib.nnp_last_error.restype = ctypes.c_char_p
    lib.nnp_destroy.argtypes = [P]
    lib.nnp_destroy.restype = None
    lib.nnp_get_capacity.argtypes = [P, P, P]
    lib.nnp_get_capacity.restype = ctypes.c_int
    lib.nnp_get_neighbors.argtypes = [P, I32, P, P, I32, P]
    lib.nnp_get_neighbors.restype = ctypes.c_int
    lib.nnp_get_features.argtypes = [P, P, P]
    lib.nnp_get_features.restype = ctypes.c_int
    lib.nnp_get_atomic_energies.argtypes = [P, P, P]
    lib.nnp_get_atomic_energies.restype = ctypes.c_int
    lib.nnp_compute_timed.argtypes = [P, P, P, P, P, P, I32]
    lib.nnp_compute_timed.restype = ctypes.c_int
    lib.nnp_kernels_per_step.argtypes = [P, I32]
    lib.nnp_kernels_per_step.restype = I32
    lib.nnp_autotune.argtypes = [P, P, P, P]
    lib.nnp_autotune.restype = ctypes.c_int
    lib.nnp_features_static.argtypes = [P, P, I32, P, P]
    lib.nnp_set_schedule.argtypes = [P, P]
    lib.nnp_set_schedule.restype = I32
    lib.nnp_features_static.restype = ctypes.c_int
    lib.nnp_mm_coupling.argtypes = [P, P, P, P, I32, P, P, P, P, I32, ctypes.c_double, P, P, P, P]
    lib.nnp_mm_coupling.restype = ctypes.c_int
    lib.nnp_md_create.argtypes = [P, P, P]
    lib.nnp_md_create.restype = ctypes.c_int
    lib.nnp_md_run.argtypes = [P, P, P, I32, P, P, P]
    lib.nnp_md_run.restype = ctypes.c_int
    lib.nnp_md_last_error.argtypes = [P]
    lib.nnp_md_last_error.restype = ctypes.c_char_p
    lib.nnp_md_destroy.argtypes = [P]
    lib.nnp_md_destroy.restype = None
    _lib = lib
    return lib


def _model_id(model) -> int:
    return _MODEL[model] if isinstance(model, str) else int(model)


def weights_per_model(model="ani2x") -> int:
    return int(load_library().nnp_weights_per_model_of(_model_id(model)))


def num_features(model="ani2x") -> int:
    return int(load_library().nnp_num_features_of(_model_id(model)))


def _stream_ptr(stream) -> int:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


def _ptr(t) -> Optional[int]:
    return None if t is None else int(t.data_ptr())


class NNP:
    """A handle on libnnp for one batch layout (atomic numbers and molecule
    boundaries fixed at construction; positions change every call)."""

    def __init__(self, Z, weights, n_models: int, mol_off=None, precision: str = "fp32",
                 box=None, max_neighbors: int = 0, max_angular: int = 0,
                 use_graph: bool = False, total_charge: int = 0, neighbor_mode: int = 0,
                 single_pass: bool = False, recompute_aev: bool = False, test_abort: bool = False,
                 model="ani2x", single_cta: bool = False):
        self._lib = load_library()
        Z = np.ascontiguousarray(Z, dtype=np.int32)
        if mol_off is None:
            mol_off = np.array([0, Z.shape[0]], dtype=np.int32)
        mol_off = np.ascontiguousarray(mol_off, dtype=np.int32)
        w = np.ascontiguousarray(weights, dtype=np.float32).reshape(-1)
        p = Params()
        p.n_models = int(n_models)
        p.precision = _PREC[precision] if isinstance(precision, str) else int(precision)
        p.weights = w.ctypes.data
        p.n_weights = w.size
        b = np.zeros(3) if box is None else np.asarray(box, dtype=np.float64).reshape(3)
        for k in range(3):
            p.box[k] = float(b[k])
        p.total_charge = int(total_charge)
        p.max_neighbors = int(max_neighbors)
        p.max_angular = int(max_angular)
        p.use_graph = 1 if use_graph else 0
        p.neighbor_mode = int(neighbor_mode)
        p.single_pass = 1 if single_pass else 0
        p.recompute_aev = 1 if recompute_aev else 0
        p.test_abort = 1 if test_abort else 0
        p.model = _model_id(model)
        p.single_cta = 1 if single_cta else 0
        h = ctypes.c_void_p()
        rc = self._lib.nnp_create_batch(Z.ctypes.data, mol_off.ctypes.data, mol_off.shape[0] - 1,
                                        ctypes.byref(p), ctypes.byref(h))
        if rc != 0:
            raise NNPError(rc, self._lib.nnp_last_error(None).decode())
        self._h = h
        self.n_atoms = int(mol_off[-1])
        self.n_mols = int(mol_off.shape[0] - 1)
        self.n_models = int(n_models)
        self.precision = precision
        self.mol_off = mol_off
        self.box = b
        self.model = p.model
        self.n_features = num_features(p.model)

    # -- lifetime --
    def close(self):
        if getattr(self, "_h", None):
            self._lib.nnp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc != 0:
            raise NNPError(rc, self._lib.nnp_last_error(self._h).decode())

    # -- evaluation --
    def compute(self, positions, energy_out=None, forces_out=None, forces: bool = True, stream=None):
        """positions: CUDA float32 [N, 3].  Returns (energy [n_mols] float64,
        forces [N, 3] float64 or None), enqueued on `stream` (default: torch's
        current stream)."""
        import torch
        assert positions.is_cuda and positions.dtype == torch.float32 and positions.is_contiguous()
        dev = positions.device
        if energy_out is None:
            energy_out = torch.empty(self.n_mols, dtype=torch.float64, device=dev)
        if forces and forces_out is None:
            forces_out = torch.empty(self.n_atoms, 3, dtype=torch.float64, device=dev)
        if not forces:
            forces_out = None
        self._check(self._lib.nnp_compute(self._h, _ptr(positions), _ptr(energy_out),
                                          _ptr(forces_out), _stream_ptr(stream)))
        return energy_out, forces_out

    def compute_host(self, positions: np.ndarray, forces: bool = True, stream=None):
        """Host arrays in and out (copies inside, synchronises)."""
        pos = np.ascontiguousarray(positions, dtype=np.float32)
        E = np.zeros(self.n_mols, dtype=np.float64)
        F = np.zeros((self.n_atoms, 3), dtype=np.float64) if forces else None
        self._check(self._lib.nnp_compute_host(self._h, pos.ctypes.data, E.ctypes.data,
                                               None if F is None else F.ctypes.data,
                                               _stream_ptr(stream)))
        return E, F

    def compute_timed(self, positions, energy_out, forces_out=None, stream=None):
        """One evaluation with direct launches; returns {stage: milliseconds}."""
        ms = (ctypes.c_float * len(STAGES))()
        self._check(self._lib.nnp_compute_timed(self._h, _ptr(positions), _ptr(energy_out),
                                                _ptr(forces_out), _stream_ptr(stream), ms,
                                                len(STAGES)))
        return dict(zip(STAGES, list(ms)))

    def autotune(self, positions, stream=None) -> dict:
        """Time candidate schedules on these positions and keep the fastest."""
        out = (ctypes.c_int32 * 5)()
        self._check(self._lib.nnp_autotune(self._h, _ptr(positions), _stream_ptr(stream), out))
        return {"featurizer_warps": out[0], "reverse_warps": out[1],
                "reverse_centres_per_item": out[2], "first_layer_n_tile": out[3],
                "reverse_shared_accumulators": out[4]}

    SCHEDULE_KEYS = ("featurizer_warps", "reverse_warps", "reverse_centres_per_item",
                     "first_layer_n_tile", "reverse_shared_accumulators")

    def set_schedule(self, schedule: dict):
        """Apply a schedule returned by autotune() (same keys), without timing."""
        vals = (ctypes.c_int32 * 5)(*[int(schedule[k]) for k in self.SCHEDULE_KEYS])
        self._check(self._lib.nnp_set_schedule(self._h, vals))

    def kernels_per_step(self, forces: bool = True) -> int:
        return int(self._lib.nnp_kernels_per_step(self._h, 1 if forces else 0))

    def status(self):
        """Raise NNPError if a device-side condition was recorded."""
        self._check(self._lib.nnp_get_status(self._h))

    # -- inspection --
    def capacity(self):
        r, a = ctypes.c_int32(), ctypes.c_int32()
        self._check(self._lib.nnp_get_capacity(self._h, ctypes.byref(r), ctypes.byref(a)))
        return r.value, a.value

    def neighbors(self, kind: int = 0, stream=None):
        import torch
        cap = self.capacity()[kind]
        counts = torch.empty(self.n_atoms, dtype=torch.int32, device="cuda")
        lists = torch.empty(self.n_atoms, cap, dtype=torch.int32, device="cuda")
        self._check(self._lib.nnp_get_neighbors(self._h, kind, _ptr(counts), _ptr(lists), cap,
                                                _stream_ptr(stream)))
        return counts, lists

    def features(self, stream=None):
        import torch
        out = torch.empty(self.n_atoms, self.n_features, dtype=torch.float32, device="cuda")
        self._check(self._lib.nnp_get_features(self._h, _ptr(out), _stream_ptr(stream)))
        return out

    def atomic_energies(self, stream=None):
        import torch
        out = torch.empty(self.n_atoms, dtype=torch.float64, device="cuda")
        self._check(self._lib.nnp_get_atomic_energies(self._h, _ptr(out), _stream_ptr(stream)))
        return out


def _check_tensor(t, name, dtype, shape):
    """The C ABI takes raw device pointers: a tensor on another device, of
    another type or layout, or too small would be misread or overrun."""
    import torch
    if not (t.is_cuda and t.device == torch.device("cuda", torch.cuda.current_device())):
        raise ValueError(f"{name}: must be a CUDA tensor on the current device")
    if t.dtype != dtype:
        raise ValueError(f"{name}: dtype {t.dtype}, expected {dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name}: must be contiguous")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name}: shape {tuple(t.shape)}, expected {tuple(shape)}")


def features_static(Z, positions, out=None, stream=None):
    """Features of one non-periodic molecule (CUDA int32 Z [n], CUDA float32
    positions [n, 3]) through the allocation-free entry point; returns CUDA
    float32 [n, 1008].  For callers that cannot let the library allocate
    device memory (see nnp_features_static in include/nnp.h)."""
    import torch
    lib = load_library()
    n = int(positions.shape[0])
    if out is None:
        out = torch.empty(n, 1008, dtype=torch.float32, device=positions.device)
    _check_tensor(Z, "Z", torch.int32, (n,))
    _check_tensor(positions, "positions", torch.float32, (n, 3))
    _check_tensor(out, "out", torch.float32, (n, 1008))
    rc = lib.nnp_features_static(_ptr(Z), _ptr(positions), n, _ptr(out), _stream_ptr(stream))
    if rc != 0:
        raise NNPError(rc, "nnp_features_static")
    return out


def mm_coupling(nnp_pos, nnp_q, nnp_sigma, nnp_eps, mm_pos, mm_q, mm_sigma, mm_eps, coulomb_k,
                energy=None, nnp_forces=None, mm_forces=None, stream=None):
    """The NNP-MM coupling term (Coulomb + Lennard-Jones over every NNP-MM
    pair; see nnp_mm_coupling in include/nnp.h).  CUDA float32 inputs
    (positions [n, 3], charges / sigma / eps [n]); the energy (CUDA float64 [1])
    and the forces (CUDA float64 [n, 3]) are ADDED to the given buffers, or to
    zeroed ones that are returned: (energy, nnp_forces, mm_forces)."""
    import torch
    lib = load_library()
    dev = mm_pos.device
    n_nnp, n_mm = int(nnp_pos.shape[0]), int(mm_pos.shape[0])
    if energy is None:
        energy = torch.zeros(1, dtype=torch.float64, device=dev)
    if nnp_forces is None:
        nnp_forces = torch.zeros(n_nnp, 3, dtype=torch.float64, device=dev)
    if mm_forces is None:
        mm_forces = torch.zeros(n_mm, 3, dtype=torch.float64, device=dev)
    f32, f64 = torch.float32, torch.float64
    _check_tensor(nnp_pos, "nnp_pos", f32, (n_nnp, 3))
    _check_tensor(mm_pos, "mm_pos", f32, (n_mm, 3))
    for name, t, n in (("nnp_q", nnp_q, n_nnp), ("nnp_sigma", nnp_sigma, n_nnp),
                       ("nnp_eps", nnp_eps, n_nnp), ("mm_q", mm_q, n_mm),
                       ("mm_sigma", mm_sigma, n_mm), ("mm_eps", mm_eps, n_mm)):
        _check_tensor(t, name, f32, (n,))
    _check_tensor(energy, "energy", f64, (1,))
    _check_tensor(nnp_forces, "nnp_forces", f64, (n_nnp, 3))
    _check_tensor(mm_forces, "mm_forces", f64, (n_mm, 3))
    rc = lib.nnp_mm_coupling(_ptr(nnp_pos), _ptr(nnp_q), _ptr(nnp_sigma), _ptr(nnp_eps), n_nnp,
                             _ptr(mm_pos), _ptr(mm_q), _ptr(mm_sigma), _ptr(mm_eps), n_mm,
                             float(coulomb_k), _ptr(energy), _ptr(nnp_forces), _ptr(mm_forces),
                             _stream_ptr(stream))
    if rc != 0:
        raise NNPError(rc, "nnp_mm_coupling")
    return energy, nnp_forces, mm_forces


class MD:
    """The replica MD loop of include/nnp.h (nnp_md_*) around an NNP handle:
    velocity Verlet ("verlet") or Langevin BAOAB ("baoab") over every atom of
    the handle, each step one CUDA graph replay; optionally the NNP-MM coupling
    term of one fixed MM environment (env: a workloads.Environment-like object
    with CUDA float32 tensors mm_pos [n_mm, 3], mm_q, mm_sigma, mm_eps [n_mm]
    and nnp_q, nnp_sigma, nnp_eps [N]), on a second stream when concurrent."""

    def __init__(self, model: NNP, masses, dt: float, integrator: str = "verlet",
                 gamma: float = 0.0, kT: float = 0.0, env=None, coulomb_k: float = 0.0,
                 concurrent: bool = True):
        import torch
        self._lib = load_library()
        self.model = model
        m = np.ascontiguousarray(masses, dtype=np.float64).reshape(-1)
        if m.shape[0] != model.n_atoms:
            raise ValueError("masses: one per atom of the handle")
        p = MDParams()
        p.integrator = {"verlet": 0, "baoab": 1}[integrator]
        p.dt, p.gamma, p.kT = float(dt), float(gamma), float(kT)
        p.masses = m.ctypes.data
        self._env = env
        if env is not None:
            n, n_mm = model.n_atoms, int(env.mm_pos.shape[0])
            f32 = torch.float32
            _check_tensor(env.mm_pos, "mm_pos", f32, (n_mm, 3))
            for name, t, k in (("mm_q", env.mm_q, n_mm), ("mm_sigma", env.mm_sigma, n_mm),
                               ("mm_eps", env.mm_eps, n_mm), ("nnp_q", env.nnp_q, n),
                               ("nnp_sigma", env.nnp_sigma, n), ("nnp_eps", env.nnp_eps, n)):
                _check_tensor(t, name, f32, (k,))
            p.n_mm = n_mm
            p.mm_positions_dev, p.mm_charges_dev = _ptr(env.mm_pos), _ptr(env.mm_q)
            p.mm_sigma_dev, p.mm_epsilon_dev = _ptr(env.mm_sigma), _ptr(env.mm_eps)
            p.nnp_charges_dev, p.nnp_sigma_dev = _ptr(env.nnp_q), _ptr(env.nnp_sigma)
            p.nnp_epsilon_dev = _ptr(env.nnp_eps)
            p.coulomb_k = float(coulomb_k)
            p.concurrent = 1 if concurrent else 0
        h = ctypes.c_void_p()
        rc = self._lib.nnp_md_create(model._h, ctypes.byref(p), ctypes.byref(h))
        if rc != 0:
            raise NNPError(rc, "nnp_md_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            self._lib.nnp_md_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def run(self, x, v, n_steps: int, noise=None, energy=None, stream=None):
        """n_steps steps from x, v (CUDA float64 [N, 3], updated in place);
        noise: CUDA float64 [n_steps, N, 3] (BAOAB); energy: CUDA float64
        [n_steps, n_mols] or None, the potential energy after each step."""
        import torch
        n = self.model.n_atoms
        f64 = torch.float64
        _check_tensor(x, "x", f64, (n, 3))
        _check_tensor(v, "v", f64, (n, 3))
        if noise is not None:
            _check_tensor(noise, "noise", f64, (n_steps, n, 3))
        if energy is not None:
            _check_tensor(energy, "energy", f64, (n_steps, self.model.n_mols))
        rc = self._lib.nnp_md_run(self._h, _ptr(x), _ptr(v), int(n_steps), _ptr(noise), _ptr(energy),
                                  _stream_ptr(stream))
        if rc != 0:
            raise NNPError(rc, self._lib.nnp_md_last_error(self._h).decode())


def _autograd_function():
    import torch

    class NNPEnergy(torch.autograd.Function):
        """E(positions) with forces from the library's hand-written reverse pass.

        forward evaluates energies and forces in one call and keeps the forces;
        with ``recompute=True`` it evaluates the energy only and the backward
        re-runs the whole pass (nothing of the forward is kept), which is the
        low-memory mode for large batches."""

        @staticmethod
        def forward(ctx, positions, model: NNP, recompute: bool = False):
            pos = positions.detach().contiguous()
            if recompute:
                E, _ = model.compute(pos, forces=False)
                ctx.save_for_backward(pos)
            else:
                E, F = model.compute(pos, forces=True)
                ctx.save_for_backward(F)
            ctx.model, ctx.recompute = model, recompute
            return E

        @staticmethod
        def backward(ctx, gE):
            model = ctx.model
            if ctx.recompute:
                (pos,) = ctx.saved_tensors
                _, F = model.compute(pos, forces=True)
            else:
                (F,) = ctx.saved_tensors
            counts = torch.as_tensor(np.diff(model.mol_off), device=F.device, dtype=torch.long)
            g_atom = torch.repeat_interleave(gE.to(torch.float64), counts)
            return (-(g_atom[:, None] * F)).to(torch.float32), None, None

    return NNPEnergy


_fn = None


def energy(positions, model: NNP, recompute: bool = False):
    """Differentiable energies [n_mols] (float64) of CUDA positions [N, 3]."""
    global _fn
    if _fn is None:
        _fn = _autograd_function()
    return _fn.apply(positions, model, recompute)

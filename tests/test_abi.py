"""The C ABI library builds for sm_103a, loads without a GPU and exports every
entry point include/nnp.h declares (no compute call is made here)."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "nnp.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(nnp_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    if not shutil.which("nvcc") and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2201_08110_gb300 import build, nnp
    build.build()
    return nnp.load_library()


def test_header_declarations_are_the_binding_exports():
    from paper_2201_08110_gb300 import nnp
    assert declared_functions() == sorted(nnp.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert isinstance(getattr(lib, name), ctypes._CFuncPtr), name


def test_host_only_queries(lib):
    from paper_2201_08110_gb300 import workloads as W
    assert lib.nnp_weights_per_model() == W.weights_per_model() == 1713223
    assert lib.nnp_num_features() == 1008


def test_model_queries(lib):
    """Sizes per model: ANI-2x as above, ANI-1x 384 features and the oracle's
    parameter count; an unknown model is -1."""
    import oracle
    from paper_2201_08110_gb300 import nnp
    assert lib.nnp_weights_per_model_of(0) == 1713223
    assert lib.nnp_num_features_of(0) == 1008
    assert lib.nnp_num_features_of(1) == 384 == oracle.MODEL_FEATURES["ani1x"]
    assert lib.nnp_weights_per_model_of(1) == oracle.weights_per_model(model="ani1x") == 326660
    assert lib.nnp_weights_per_model_of(2) == -1 and lib.nnp_num_features_of(-1) == -1
    assert nnp.weights_per_model("ani1x") == 326660 and nnp.num_features("ani1x") == 384


def test_create_checks_the_model_before_touching_the_device(lib):
    """ANI-1x has no F, S or Cl, needs its own weight count and a box edge
    above 2 x 5.2 A; an unknown model id is NNP_ERR_ARG."""
    from paper_2201_08110_gb300 import nnp
    import numpy as np
    p = nnp.Params()
    p.n_models = 1
    p.model = 1
    w = np.zeros(nnp.weights_per_model("ani1x"), np.float32)
    p.weights = w.ctypes.data
    p.n_weights = w.size
    h = ctypes.c_void_p()
    Z = np.array([6, 9], np.int32)
    assert lib.nnp_create(Z.ctypes.data, 2, ctypes.byref(p), ctypes.byref(h)) == 2  # F
    assert b"atomic number 9" in lib.nnp_last_error(None)
    Z = np.array([6, 1], np.int32)
    p.box[0] = p.box[1] = p.box[2] = 10.3  # above 2 x 5.1, below 2 x 5.2
    assert lib.nnp_create(Z.ctypes.data, 2, ctypes.byref(p), ctypes.byref(h)) == 1
    p.box[0] = p.box[1] = p.box[2] = 0.0
    p.model = 0  # ANI-2x with ANI-1x's weight count
    assert lib.nnp_create(Z.ctypes.data, 2, ctypes.byref(p), ctypes.byref(h)) == 1
    p.model = 2
    assert lib.nnp_create(Z.ctypes.data, 2, ctypes.byref(p), ctypes.byref(h)) == 1
    assert b"model" in lib.nnp_last_error(None)
    assert not h.value


def test_create_rejects_bad_arguments_before_touching_the_device(lib):
    """Argument, species and charge errors are returned synchronously."""
    from paper_2201_08110_gb300 import nnp
    import numpy as np
    p = nnp.Params()
    p.n_models = 1
    w = np.zeros(nnp.weights_per_model(), np.float32)
    p.weights = w.ctypes.data
    p.n_weights = w.size
    h = ctypes.c_void_p()
    Z = np.array([6, 5], np.int32)
    assert lib.nnp_create(Z.ctypes.data, 2, ctypes.byref(p), ctypes.byref(h)) == 2  # species
    assert b"atomic number 5" in lib.nnp_last_error(None)
    Z = np.array([6, 1], np.int32)
    p.total_charge = -1
    assert lib.nnp_create(Z.ctypes.data, 2, ctypes.byref(p), ctypes.byref(h)) == 3  # charge
    p.total_charge = 0
    p.n_weights = w.size - 1
    assert lib.nnp_create(Z.ctypes.data, 2, ctypes.byref(p), ctypes.byref(h)) == 1  # weights size
    p.n_weights = w.size
    p.box[0] = p.box[1] = p.box[2] = 9.0
    assert lib.nnp_create(Z.ctypes.data, 2, ctypes.byref(p), ctypes.byref(h)) == 1  # box < 2 Rc
    p.box[0] = p.box[1] = p.box[2] = 0.0
    p.single_cta = 2
    assert lib.nnp_create(Z.ctypes.data, 2, ctypes.byref(p), ctypes.byref(h)) == 1  # flag not 0 / 1
    p.single_cta = 0
    p.reserved[1] = 1
    assert lib.nnp_create(Z.ctypes.data, 2, ctypes.byref(p), ctypes.byref(h)) == 1  # reserved field
    assert not h.value


def test_coupling_rejects_bad_arguments_before_touching_the_device(lib):
    """nnp_mm_coupling checks its counts and buffers on the host: a negative
    count or a null buffer is NNP_ERR_ARG, more NNP atoms than fit in shared
    memory NNP_ERR_TOO_LARGE, and an empty side returns NNP_OK without work
    (none of these launches anything, so they run without a GPU)."""
    from paper_2201_08110_gb300 import nnp
    args = lambda n_nnp, n_mm, bufs: (*bufs[:4], n_nnp, *bufs[4:8], n_mm, 332.0, *bufs[8:11], None)
    nulls = [None] * 11
    fake = [ctypes.c_void_p(16 * (k + 1)) for k in range(11)]  # never dereferenced on these paths
    assert lib.nnp_mm_coupling(*args(-1, 10, fake)) == 1
    assert lib.nnp_mm_coupling(*args(5, -1, fake)) == 1
    assert lib.nnp_mm_coupling(*args(5, 10, nulls)) == 1
    assert lib.nnp_mm_coupling(*args(nnp.COUPLING_MAX_NNP + 1, 10, fake)) == 10
    assert lib.nnp_mm_coupling(*args(0, 10, nulls)) == 0
    assert lib.nnp_mm_coupling(*args(5, 0, nulls)) == 0

"""The allocation-free entry point nnp_features_static, through the C ABI.

It exists for callers that cannot let a library allocate device memory (an MD
engine capturing its time step into a CUDA graph, or a framework that owns
the device memory budget).  Its features must equal those the handle-based
entry point (nnp_compute + nnp_get_features) produces, within the feature
tolerance of the parity tests, on two calls in a row: the second call reuses
the shared scratch array the first one left behind.  Collected last so that a
run stopping at the first failure has already run every other test.
"""
import numpy as np
import pytest

import oracle
from paper_2201_08110_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nnp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2201_08110_gb300 import build, nnp
    build.build()
    return nnp


def handle_features(nnp, b):
    model = nnp.NNP(b.Z, W.weights(3, 1), 1)
    model.compute(torch.tensor(b.pos, device="cuda"))
    G = model.features()
    torch.cuda.synchronize()
    model.status()
    return G.cpu().numpy()


def static_features(nnp, b):
    Z = torch.tensor(b.Z, dtype=torch.int32, device="cuda")
    pos = torch.tensor(b.pos, device="cuda")
    G = nnp.features_static(Z, pos)
    torch.cuda.synchronize()
    return G.cpu().numpy()


def test_static_entry_point_matches_handle_features_on_consecutive_calls(nnp):
    # a large molecule first, then a smaller one: stale scratch rows of the
    # first call must not leak into the second
    big = W.batch(404, [nnp.STATIC_MAX_ATOMS]).molecule(0)
    small, _, _ = W.config1()
    for b in (big, small, big):
        got = static_features(nnp, b)
        ref = handle_features(nnp, b)
        scale = np.maximum(np.abs(ref).max(axis=1, keepdims=True), 1e-30)
        err = np.abs(got - ref) / scale
        assert np.all(np.isfinite(got))
        assert err.max() < 5e-6, f"feature error {err.max():.3e} (row-max relative)"
        # and straight against the FP64 oracle (same bound as the handle path's
        # feature parity test)
        exact = oracle.aev(b.Z, b.pos)
        scale = np.maximum(np.abs(exact).max(axis=1, keepdims=True), 1e-30)
        err = np.abs(got - exact) / scale
        assert err.max() < 5e-6, f"feature error against the oracle {err.max():.3e}"


def test_static_entry_point_rejects_too_many_atoms(nnp):
    n = nnp.STATIC_MAX_ATOMS + 1
    Z = torch.ones(n, dtype=torch.int32, device="cuda")
    pos = torch.zeros(n, 3, dtype=torch.float32, device="cuda")
    with pytest.raises(nnp.NNPError) as e:
        nnp.features_static(Z, pos)
    assert e.value.status == "NNP_ERR_TOO_LARGE"


def test_static_entry_point_poisons_bad_atomic_numbers(nnp):
    b, _, _ = W.config1()
    Z = torch.tensor(b.Z, dtype=torch.int32, device="cuda")
    Z[3] = 5
    G = nnp.features_static(Z, torch.tensor(b.pos, device="cuda"))
    torch.cuda.synchronize()
    assert torch.isnan(G).all()
    # and the next valid call is clean again
    assert np.all(np.isfinite(static_features(nnp, b)))

"""Failure detection on the device without faulting it: a bounded wait that
expires reports SBM_ERR_TIMEOUT and leaves the context usable; host-side
argument and state errors."""
import numpy as np
import pytest
import torch

import paper_2507_17053_gb300 as G
import synthetic as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def test_bounded_wait_expiry_is_reported_and_context_survives():
    P = G.Problem.from_workload(S.SPHERE_3D_Q4.resized(8))
    G.sbm_device_status(P.handle)                      # clean start
    G.sbm_selftest_timeout(P.handle)
    with pytest.raises(G.SbmError) as e:
        G.sbm_device_status(P.handle)
    assert G.STATUS[e.value.status] == "SBM_ERR_TIMEOUT"
    G.sbm_device_status(P.handle)                      # the word was cleared
    # the context is still fine: an apply works and is right
    x = torch.from_numpy(S.random_vector(1, P.n_dofs, "uniform")).cuda()
    y1 = P.apply_f64(x)
    y2 = P.apply_f64(x)
    assert torch.equal(y1, y2) and torch.isfinite(y1).all()


def test_setup_twice_and_bad_vectors():
    P = G.Problem.from_workload(S.DISK_2D_Q2)
    with pytest.raises(G.SbmError) as e:
        G.sbm_setup_face_data(P.handle)
    assert G.STATUS[e.value.status] == "SBM_ERR_STATE"
    x = torch.zeros(P.n_dofs, dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        P.apply_f64(x[:-1])
    with pytest.raises(G.SbmError):
        G.sbm_apply_f32(P.handle, x.float(), x.float(), face_mode=7)


def test_nan_input_propagates_without_error():
    P = G.Problem.from_workload(S.SPHERE_3D_Q4.resized(8))
    x = torch.zeros(P.n_dofs, dtype=torch.float64, device="cuda")
    x[5] = float("nan")
    y = P.apply_f64(x)
    G.sbm_device_status(P.handle)
    assert torch.isnan(y).any() and not torch.isnan(y).all()


"""The allocation-free FP64 apply (sbm_apply_f64_noalloc) gives the same y as
sbm_apply_f64.

It exists for callers that cannot allocate device memory when they apply the
operator; its scratch is one static device array shared by every call.  This
file is named so that pytest collects it last: a run that stops at the first
failure has run every other test before it.  It passes alone in a fresh
process and after the other tests (the array keeps the previous call's
contents; the entry point must not depend on them).
"""
import ctypes

import numpy as np
import pytest
import torch

import paper_2507_17053_gb300 as G
import synthetic as S

pytestmark = pytest.mark.gpu
TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def _call_noalloc(P, x, y):
    """Straight through the C ABI."""
    st = torch.cuda.current_stream().cuda_stream
    return G.lib().sbm_apply_f64_noalloc(ctypes.c_void_p(P.handle), ctypes.c_void_p(x.data_ptr()),
                                         ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(st))


@pytest.mark.parametrize("w", [S.SPHERE_3D_Q4.resized(12), S.DISK_2D_Q2,
                               S.ELLIPSOID_3D_Q6.resized(8)], ids=lambda w: w.name)
def test_noalloc_apply_matches_apply_twice(w):
    P = G.Problem.from_workload(w)
    x = torch.from_numpy(S.random_vector(w.seed, P.n_dofs, w.dist)).cuda()
    ref = P.apply_f64(x).cpu().numpy()
    scale = np.abs(ref).max()
    for _ in range(2):                      # two calls in a row on the shared array
        y = torch.full_like(x, float("nan"))
        assert _call_noalloc(P, x, y) == 0, G.lib().sbm_last_error_detail()
        torch.cuda.synchronize()
        assert np.abs(y.cpu().numpy() - ref).max() <= TOL * scale
    # other problems in between, with x full of NaN, leave NaN wherever their
    # face results and colour buffers fall in the shared array (these cover
    # a larger region than P's): a value of P's call read before written
    # would come out NaN
    for wq in (S.DISK_2D_Q2.resized(20, degree=3), S.SPHERE_3D_Q4.resized(24),
               S.ELLIPSOID_3D_Q6.resized(10), S.SPHERE_3D_Q4.resized(16, degree=2)):
        Q = G.Problem.from_workload(wq)
        xq = torch.full((Q.n_dofs,), float("nan"), dtype=torch.float64, device="cuda")
        yq = torch.empty_like(xq)
        assert _call_noalloc(Q, xq, yq) == 0, G.lib().sbm_last_error_detail()
        torch.cuda.synchronize()
        assert torch.isnan(yq).all()
        y = torch.full_like(x, float("nan"))
        assert _call_noalloc(P, x, y) == 0
        torch.cuda.synchronize()
        yh = y.cpu().numpy()
        assert np.isfinite(yh).all()
        assert np.abs(yh - ref).max() <= TOL * scale


def test_noalloc_rejects_oversized_and_dg_problems():
    big = G.Problem.from_workload(S.SPHERE_3D_Q4.resized(48))     # ~1.35 M DoFs
    x = torch.zeros(big.n_dofs, dtype=torch.float64, device="cuda")
    assert _call_noalloc(big, x, torch.empty_like(x)) == 1          # SBM_ERR_ARG
    assert b"bytes of scratch" in G.lib().sbm_last_error_detail()
    dg = G.Problem.from_workload(S.TORUS_3D_DG_Q3.resized(10))
    xd = torch.zeros(dg.n_dofs, dtype=torch.float64, device="cuda")
    assert _call_noalloc(dg, xd, torch.empty_like(xd)) == 8         # SBM_ERR_UNSUPPORTED

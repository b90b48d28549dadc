"""Tensor-core (tcgen05) face modes of the FP32 apply: TF32 and BF16 shifted
point evaluation, against the FP64 oracle, and inside FP64 iterative
refinement."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla
import torch

import paper_2507_17053_gb300 as G
import synthetic as S
from oracle.operator import Problem as OracleProblem, sin_solution

pytestmark = pytest.mark.gpu

# relative max-norm error bounds against the FP64 oracle, per degree, about
# 3x the largest error measured on a GB300 for these cases (TF32 keeps 10
# mantissa bits, BF16 7; measured TF32 1.9e-4 .. 4.3e-4, BF16 1.3e-3 ..
# 2.6e-3, the p = 2 sphere and p = 3 sphere/torus the largest)
BOUND = {"tf32": {1: 6e-4, 2: 1.3e-3, 3: 1e-3, 4: 6e-4, 5: 7.5e-4, 6: 9e-4},
         "bf16": {1: 4e-3, 2: 7.5e-3, 3: 8e-3, 4: 5e-3, 5: 7e-3, 6: 6e-3}}

CASES = [S.SPHERE_3D_Q4.resized(10), S.ELLIPSOID_3D_Q6.resized(8),
         S.SPHERE_3D_Q4.resized(7, degree=2), S.SPHERE_3D_Q4.resized(7, degree=3),
         S.TORUS_3D_DG_Q3.resized(12), S.SPHERE_3D_Q4.resized(6, degree=1),
         S.SPHERE_3D_Q4.resized(6, degree=5)]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def _rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


@pytest.mark.parametrize("mode", ["tf32", "bf16"])
@pytest.mark.parametrize("w", CASES, ids=lambda w: w.name + f"_q{w.degree}")
def test_tensor_face_apply_error(w, mode):
    O = OracleProblem.from_workload(w)
    P = G.Problem.from_workload(w)
    x = S.random_vector(w.seed, O.n_dofs, w.dist)
    x32 = torch.from_numpy(x).float().cuda()
    ref = O.apply(x.astype(np.float32).astype(np.float64))
    y_fp32 = P.apply_f32(x32).double().cpu().numpy()
    y_tc = P.apply_f32(x32, face_mode=mode).double().cpu().numpy()
    G.sbm_device_status(P.handle)
    err_tc, err_fp32 = _rel(y_tc, ref), _rel(y_fp32, ref)
    print(f"{w.name} q{w.degree} {mode}: {err_tc:.3e} (fp32 faces {err_fp32:.3e})")
    assert err_tc <= BOUND[mode][w.degree]
    assert err_fp32 <= 5e-7
    # the tensor-core path really ran (it rounds differently from FP32) and a
    # second call gives the same bits
    assert not np.array_equal(y_tc, y_fp32)
    y_tc2 = P.apply_f32(x32, face_mode=mode).double().cpu().numpy()
    assert np.array_equal(y_tc, y_tc2)


def test_tensor_face_modes_rejected_in_2d():
    P = G.Problem.from_workload(S.DISK_2D_Q2)
    x = torch.zeros(P.n_dofs, dtype=torch.float32, device="cuda")
    with pytest.raises(G.SbmError) as e:
        P.apply_f32(x, face_mode="tf32")
    assert G.STATUS[e.value.status] == "SBM_ERR_UNSUPPORTED"


@pytest.mark.parametrize("mode", ["tf32", "bf16"])
def test_ir_with_tensor_faces_reaches_fp64_tolerance(mode):
    w = S.SPHERE_3D_Q4.resized(8, degree=2)
    O = OracleProblem.from_workload(w)
    P = G.Problem.from_workload(w)
    u, f = sin_solution(3)
    b = O.rhs(f, u)
    xref = spla.spsolve(O.assemble().tocsc(), b)
    bd = torch.from_numpy(b).cuda()
    x = torch.zeros_like(bd)
    it, rr, ok, outer = G.sbm_solve_ir(P.handle, bd, x, rtol=1e-10, max_outer=60, restart=100,
                                       inner_rtol=1e-3, inner_maxit=3000,
                                       face_mode=G.FACE_MODE[mode])
    assert ok and rr <= 1e-10, (it, rr, outer)
    assert np.linalg.norm(x.cpu().numpy() - xref) <= 1e-7 * np.linalg.norm(xref)

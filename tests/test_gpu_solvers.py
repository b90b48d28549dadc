"""CG, GMRES and mixed-precision iterative refinement on the GPU, against the
oracle's direct solve of the same assembled system."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla
import torch

import paper_2507_17053_gb300 as G
import synthetic as S
from oracle.operator import Problem as OracleProblem, sin_solution

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def _system(w):
    O = OracleProblem.from_workload(w)
    P = G.Problem.from_workload(w)
    u, f = sin_solution(w.dim)
    b = O.rhs(f, u)
    xref = spla.spsolve(O.assemble().tocsc(), b)
    return O, P, b, xref


@pytest.mark.parametrize("precond", ["none", "jacobi"])
@pytest.mark.parametrize("d", [2, 3])
def test_cg_on_zero_shift_spd_system(d, precond):
    """Box domain on mesh planes: the shift is zero and A is symmetric
    positive definite (symmetric Nitsche form), so CG must converge."""
    w = S._wl("box", d, 2, 8 if d == 3 else 16, S.box((0.0,) * d, (0.5,) * d))
    O, P, b, xref = _system(w)
    bd = torch.from_numpy(b).cuda()
    x = torch.zeros_like(bd)
    it, rr, ok = G.sbm_cg(P.handle, bd, x, rtol=1e-10, maxit=5000, precond=G.PRECOND[precond])
    assert ok and rr <= 1e-10 and it > 5
    xs = x.cpu().numpy()
    assert np.linalg.norm(xs - xref) <= 1e-8 * np.linalg.norm(xref)
    # deterministic: a second solve is bitwise identical
    x2 = torch.zeros_like(bd)
    G.sbm_cg(P.handle, bd, x2, rtol=1e-10, maxit=5000, precond=G.PRECOND[precond])
    assert torch.equal(x, x2)


def test_cg_reports_failure_on_nonsymmetric_system():
    """The 2D workload's operator is not symmetric (non-zero shift); CG on it
    does not reach 1e-10 and must say so instead of hanging or crashing."""
    O, P, b, xref = _system(S.DISK_2D_Q2)
    bd = torch.from_numpy(b).cuda()
    x = torch.zeros_like(bd)
    it, rr, ok = G.sbm_cg(P.handle, bd, x, rtol=1e-10, maxit=3000)
    assert not ok and it <= 3000
    with pytest.raises(G.SbmError) as e:
        G.sbm_cg(P.handle, bd, torch.zeros_like(bd), rtol=1e-10, maxit=50,
                 raise_not_converged=True)
    assert G.STATUS[e.value.status] == "SBM_ERR_NOT_CONVERGED"


def test_gmres_disk_workload():
    O, P, b, xref = _system(S.DISK_2D_Q2)
    bd = torch.from_numpy(b).cuda()
    x = torch.zeros_like(bd)
    it, rr, ok = G.sbm_gmres(P.handle, bd, x, rtol=1e-10, maxit=5000, restart=100)
    assert ok and rr <= 1e-10
    assert np.linalg.norm(x.cpu().numpy() - xref) <= 1e-7 * np.linalg.norm(xref)


@pytest.mark.parametrize("w", [S.DISK_2D_Q2, S.SPHERE_3D_Q4.resized(8, degree=2)],
                         ids=lambda w: w.name)
def test_mixed_precision_ir(w):
    O, P, b, xref = _system(w)
    bd = torch.from_numpy(b).cuda()
    x = torch.zeros_like(bd)
    it, rr, ok, outer = G.sbm_solve_ir(P.handle, bd, x, rtol=1e-10, max_outer=40, restart=100,
                                       inner_rtol=1e-4, inner_maxit=3000)
    assert ok and rr <= 1e-10, (it, rr, outer)
    assert np.linalg.norm(x.cpu().numpy() - xref) <= 1e-7 * np.linalg.norm(xref)


@pytest.mark.parametrize("w", [S.DISK_2D_Q2, S.SPHERE_3D_Q4.resized(8, degree=2),
                               S.ELLIPSOID_3D_Q6.resized(6, degree=3)],
                         ids=lambda w: w.name)
def test_bicgstab_fp64(w):
    """BiCGStab on the nonsymmetric SBM system reaches 1e-10 (true residual)
    and the direct solution; a second solve is bitwise identical."""
    O, P, b, xref = _system(w)
    bd = torch.from_numpy(b).cuda()
    x = torch.zeros_like(bd)
    it, rr, ok = G.sbm_bicgstab(P.handle, bd, x, rtol=1e-10, maxit=20000)
    assert ok and rr <= 1e-10, (it, rr)
    assert np.linalg.norm(x.cpu().numpy() - xref) <= 1e-7 * np.linalg.norm(xref)
    x2 = torch.zeros_like(bd)
    it2, _, _ = G.sbm_bicgstab(P.handle, bd, x2, rtol=1e-10, maxit=20000)
    assert it2 == it and torch.equal(x, x2)


def test_bicgstab_initial_guess_and_zero_rhs():
    O, P, b, xref = _system(S.DISK_2D_Q2.resized(12))
    bd = torch.from_numpy(b).cuda()
    # the exact solution as initial guess: converged before the first iteration
    x = torch.from_numpy(xref).cuda()
    it, rr, ok = G.sbm_bicgstab(P.handle, bd, x, rtol=1e-8, maxit=100)
    assert ok and it == 0 and rr <= 1e-8
    # b = 0 from x = 0: nothing to do, x stays 0
    z = torch.zeros_like(bd)
    x = torch.zeros_like(bd)
    it, rr, ok = G.sbm_bicgstab(P.handle, z, x, rtol=1e-10, maxit=100)
    assert ok and it == 0 and rr == 0.0 and not x.any()
    # an iteration cap too small reports NOT_CONVERGED with the true residual
    x = torch.zeros_like(bd)
    it, rr, ok = G.sbm_bicgstab(P.handle, bd, x, rtol=1e-12, maxit=3)
    assert not ok and it == 3 and rr > 1e-12
    with pytest.raises(G.SbmError):
        G.sbm_bicgstab(P.handle, bd, torch.zeros_like(bd), rtol=1e-12, maxit=3,
                       raise_not_converged=True)


@pytest.mark.parametrize("mode,rtol", [("fp32", 1e-5), ("tf32", 1e-3)])
def test_bicgstab_fp32(mode, rtol):
    """FP32 vectors and apply, FP64 scalars: reaches rtol (true residual of
    the same FP32 apply; with TF32 faces the apply's own rounding, about
    1e-4 of |A x|, bounds what any residual can reach), and the FP64
    operator's residual of the FP32 solution is within 10 rtol."""
    w = S.SPHERE_3D_Q4.resized(8, degree=2)
    O, P, b, xref = _system(w)
    bd = torch.from_numpy(b).cuda().float()
    x = torch.zeros_like(bd)
    it, rr, ok = G.sbm_bicgstab_f32(P.handle, bd, x, rtol=rtol, maxit=20000,
                                    face_mode=G.FACE_MODE[mode])
    assert ok and rr <= rtol, (it, rr)
    bd64 = torch.from_numpy(b).cuda()
    r64 = bd64 - P.apply_f64(x.double())
    assert float(r64.norm() / bd64.norm()) <= 10 * rtol


def test_bicgstab_fp32_rejects_tensor_faces_in_2d():
    P = G.Problem.from_workload(S.DISK_2D_Q2.resized(8))
    b = torch.ones(P.n_dofs, device="cuda")
    with pytest.raises(G.SbmError) as e:
        G.sbm_bicgstab_f32(P.handle, b, torch.zeros_like(b), face_mode=G.FACE_MODE["tf32"])
    assert G.STATUS[e.value.status] == "SBM_ERR_UNSUPPORTED"


@pytest.mark.parametrize("inner,tol,maxit", [("bicgstab_mixed", 1e-2, 300),
                                              ("bicgstab", 1e-2, 300),
                                              ("bicgstab_mixed", 1e-6, 100)])
def test_refinement_short_inner_solves_and_fp64_finish(inner, tol, maxit):
    """Short inner solves (capped, loose tolerance) with FP64 vectors and FP32
    applies, or on FP32 vectors; when they stall (the last case: 100
    iterations never reach 1e-6) FP64 BiCGStab finishes to the FP64
    tolerance."""
    w = S.SPHERE_3D_Q4.resized(10, degree=2)
    O, P, b, xref = _system(w)
    bd = torch.from_numpy(b).cuda()
    x = torch.zeros_like(bd)
    it, rr, ok, outer = G.sbm_solve_ir(P.handle, bd, x, rtol=1e-10, max_outer=60,
                                       inner_rtol=tol, inner_maxit=maxit,
                                       inner_solver=G.INNER[inner])
    assert ok and rr <= 1e-10, (it, rr, outer)
    assert np.linalg.norm(x.cpu().numpy() - xref) <= 1e-7 * np.linalg.norm(xref)


@pytest.mark.parametrize("mode", ["fp32", "tf32", "bf16"])
def test_mixed_precision_ir_bicgstab_inner(mode):
    """FP64 refinement around an FP32 BiCGStab inner solve reaches the FP64
    tolerance, also when the faces run on the tensor cores."""
    w = S.SPHERE_3D_Q4.resized(8, degree=2)
    O, P, b, xref = _system(w)
    bd = torch.from_numpy(b).cuda()
    x = torch.zeros_like(bd)
    it, rr, ok, outer = G.sbm_solve_ir(P.handle, bd, x, rtol=1e-10, max_outer=60,
                                       inner_rtol=1e-3, inner_maxit=5000,
                                       face_mode=G.FACE_MODE[mode],
                                       inner_solver=G.INNER["bicgstab"])
    assert ok and rr <= 1e-10, (it, rr, outer)
    assert np.linalg.norm(x.cpu().numpy() - xref) <= 1e-7 * np.linalg.norm(xref)


@pytest.mark.parametrize("w,mode", [(S.DISK_2D_Q2, "fp32"),
                                    (S.SPHERE_3D_Q4.resized(10, degree=2), "fp32"),
                                    (S.SPHERE_3D_Q4.resized(10, degree=2), "tf32")],
                         ids=lambda v: getattr(v, "name", str(v)))
def test_bicgstab_mixed_reliable_updates(w, mode):
    """BiCGStab on FP32 applies with FP64 reliable updates reaches the FP64
    tolerance without restarts of the Krylov space (the true residual is
    checked here with the FP64 apply) and matches the oracle's direct solve;
    it replaced the recursive residual at least once per decade."""
    O, P, b, xref = _system(w)
    bd = torch.from_numpy(b).cuda()
    x = torch.zeros_like(bd)
    it, rr, ok, rep = G.sbm_bicgstab_mixed(P.handle, bd, x, rtol=1e-10, maxit=20000,
                                            face_mode=G.FACE_MODE[mode])
    assert ok and rr <= 1e-10, (it, rr, rep)
    res = bd - P.apply_f64(x)
    assert float(res.norm() / bd.norm()) <= 1.01e-10
    # FP32 faces: an update per decade; TF32 faces (operator error ~3e-4) may
    # stall early and hand over to the FP64 finish
    assert rep >= (5 if mode == "fp32" else 1), rep
    assert np.linalg.norm(x.cpu().numpy() - xref) <= 1e-7 * np.linalg.norm(xref)


def test_bicgstab_mixed_rejects_bad_arguments():
    P = G.Problem.from_workload(S.DISK_2D_Q2)
    b = torch.ones(P.n_dofs, dtype=torch.float64, device="cuda")
    x = torch.zeros_like(b)
    with pytest.raises(G.SbmError):
        G.sbm_bicgstab_mixed(P.handle, b, x, rtol=0.0)
    with pytest.raises(G.SbmError) as e:
        G.sbm_bicgstab_mixed(P.handle, b, x, face_mode=G.FACE_MODE["tf32"])   # 2D: no TC faces
    assert G.STATUS[e.value.status] == "SBM_ERR_UNSUPPORTED"

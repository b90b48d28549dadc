"""The first-order Taylor extension (SBM_EXT_TAYLOR1) on the GPU against the
oracle's taylor1 operator: FP64 parity 1e-12 (CG and DG, 2D and 3D, every p),
full-size sampled rows, diagonal, FP32 error, batch = single applies, a
BiCGStab solve, and the tensor-core face modes refused."""
import dataclasses

import numpy as np
import pytest
import scipy.sparse.linalg as spla
import torch

import paper_2507_17053_gb300 as G
import synthetic as S
from oracle.operator import Problem as OracleProblem, sin_solution

pytestmark = pytest.mark.gpu
TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def _t(w):
    return dataclasses.replace(w, extension="taylor1", name=w.name + "+taylor1")


def _rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


CASES = ([_t(S.DISK_2D_Q2.resized(11, degree=p)) for p in (1, 2, 4, 6)]
         + [_t(S.SPHERE_3D_Q4.resized(7, degree=p)) for p in (1, 2, 3, 4, 5, 6)]
         + [_t(S.ELLIPSOID_3D_Q6.resized(8)), _t(S.TORUS_3D_DG_Q3.resized(10)),
            _t(S.batched_ellipsoids(nprob=2, n_range=(8, 10))[1]),
            _t(S._wl("box", 3, 2, 6, S.box((0.0,) * 3, (0.5,) * 3)))])


@pytest.mark.parametrize("w", CASES, ids=lambda w: w.name)
def test_taylor_apply_matches_oracle(w):
    O = OracleProblem.from_workload(w)
    assert O.extension == "taylor1"
    P = G.Problem.from_workload(w)
    x = S.random_vector(w.seed, O.n_dofs, w.dist)
    xd = torch.from_numpy(x).cuda()
    y = P.apply_f64(xd)
    assert torch.equal(y, P.apply_f64(xd))
    ref = O.apply(x)
    assert _rel(y.cpu().numpy(), ref) <= TOL
    # FP32 path (FP32 cells and faces)
    y32 = P.apply_f32(xd.float()).double().cpu().numpy()
    assert _rel(y32, O.apply(x.astype(np.float32).astype(np.float64))) <= 1e-6
    # diagonal
    d = torch.empty_like(xd)
    G.sbm_diagonal(P.handle, d)
    np.testing.assert_allclose(d.cpu().numpy(), O.diagonal(), rtol=0,
                               atol=1e-12 * np.abs(O.diagonal()).max())


def test_taylor_full_size_sampled_rows():
    w = _t(S.SPHERE_3D_Q4)
    O = OracleProblem.from_workload(w)
    P = G.Problem.from_workload(w)
    x = S.random_vector(w.seed, O.n_dofs, w.dist)
    y = P.apply_f64(torch.from_numpy(x).cuda()).cpu().numpy()
    rng = np.random.default_rng(1)
    rows = rng.choice(O.n_dofs, size=5000, replace=False)
    fc = np.unique(O.mesh.sfaces[:, 0])
    rows = np.unique(np.concatenate([rows, O.dofmap[rng.choice(fc, 100, replace=False)].ravel()]))
    ref = O.apply_rows(x, rows)
    assert np.abs(y[rows] - ref).max() <= TOL * np.abs(ref).max()


def test_taylor_tensor_core_modes_refused():
    P = G.Problem.from_workload(_t(S.SPHERE_3D_Q4.resized(8)))
    x = torch.ones(P.n_dofs, device="cuda")
    with pytest.raises(G.SbmError) as e:
        P.apply_f32(x, face_mode="tf32")
    assert G.STATUS[e.value.status] == "SBM_ERR_UNSUPPORTED"


def test_taylor_batch_equals_single_applies():
    ws = [_t(w) for w in S.batched_ellipsoids(nprob=3, n_range=(6, 10))]
    ps = [G.Problem.from_workload(w) for w in ws]
    nrhs = 2
    B = G.Batch(ps, nrhs, autotune=False)
    for k in range(len(ps)):
        B.set_tile_shape(k, 0)          # the single applies use tile shape 0
    xs = [torch.from_numpy(np.concatenate([S.random_vector(w.seed + r, p.n_dofs, "uniform")
                                           for r in range(nrhs)])).cuda()
          for w, p in zip(ws, ps)]
    ys = [torch.empty_like(x) for x in xs]
    B.apply(xs, ys)
    torch.cuda.synchronize()
    for p, x, y in zip(ps, xs, ys):
        for r in range(nrhs):
            sl = slice(r * p.n_dofs, (r + 1) * p.n_dofs)
            assert torch.equal(y[sl], p.apply_f64(x[sl].contiguous()))


def test_taylor_bicgstab_solution():
    w = _t(S.DISK_2D_Q2)
    O = OracleProblem.from_workload(w)
    P = G.Problem.from_workload(w)
    u, f = sin_solution(2)
    b = O.rhs(f, u)
    xref = spla.spsolve(O.assemble().tocsc(), b)
    bd = torch.from_numpy(b).cuda()
    x = torch.zeros_like(bd)
    it, rr, ok = G.sbm_bicgstab(P.handle, bd, x, rtol=1e-10, maxit=5000)
    assert ok and rr <= 1e-10
    assert np.linalg.norm(x.cpu().numpy() - xref) <= 1e-7 * np.linalg.norm(xref)

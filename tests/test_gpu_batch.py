"""Batched applies (several problems, several right-hand sides, one graph
launch) give exactly the per-problem applies."""
import dataclasses

import numpy as np
import pytest
import torch

import paper_2507_17053_gb300 as G
import synthetic as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def _problems():
    ws = S.batched_ellipsoids(nprob=7, n_range=(6, 14))
    ws.append(S.DISK_2D_Q2)
    return ws, [G.Problem.from_workload(w) for w in ws]


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_batch_equals_single_applies(dtype):
    ws, ps = _problems()
    nrhs = 3
    B = G.Batch(ps, nrhs, autotune=True)
    for k in range(len(ps)):
        B.set_tile_shape(k, 0)          # the single applies use tile shape 0
    xs = [torch.from_numpy(np.concatenate([S.random_vector(w.seed + r, p.n_dofs, "uniform")
                                           for r in range(nrhs)])).to("cuda", dtype)
          for w, p in zip(ws, ps)]
    ys = [torch.full_like(x, float("nan")) for x in xs]
    for _ in range(2):          # the second call replays the captured graph
        B.apply(xs, ys)
        torch.cuda.synchronize()
        for p, x, y in zip(ps, xs, ys):
            for r in range(nrhs):
                xr = x[r * p.n_dofs:(r + 1) * p.n_dofs].contiguous()
                ref = p.apply_f64(xr) if dtype == torch.float64 else p.apply_f32(xr)
                assert torch.equal(y[r * p.n_dofs:(r + 1) * p.n_dofs], ref)
    # the other tile shape (chunks of R/2 cells) sums a few shared nodes in a
    # different order: equal to rounding
    tol = 1e-12 if dtype == torch.float64 else 1e-6
    for k in range(len(ps)):
        B.set_tile_shape(k, 1 - B.tile_shape(k))
    ys2 = [torch.empty_like(x) for x in xs]
    B.apply(xs, ys2)
    torch.cuda.synchronize()
    for y, y2 in zip(ys, ys2):
        assert float((y - y2).abs().max() / y.abs().max()) <= tol


def test_batch_tile_shape_3_equals_single_applies():
    """FP32 batches of 3D problems run tile shape 3 (the chunks without
    staged runs) when pinned: bitwise the single FP32 applies (any of tile
    shapes 0, 2, 3).  FP64 batches and degrees with a 2D problem reject it."""
    ws = S.batched_ellipsoids(nprob=6, n_range=(6, 12), p_range=(2, 6))
    ps = [G.Problem.from_workload(w) for w in ws]
    nrhs = 2
    B = G.Batch(ps, nrhs, autotune=False)
    for deg in sorted({w.degree for w in ws}):
        B.set_knobs(32, deg, 3, 0, 0)
        with pytest.raises(G.SbmError) as e:
            B.set_knobs(64, deg, 3, 0, 0)
        assert G.STATUS[e.value.status] == "SBM_ERR_UNSUPPORTED"
    xs = [torch.from_numpy(np.concatenate([S.random_vector(w.seed + r, p.n_dofs, "uniform")
                                           for r in range(nrhs)])).to("cuda", torch.float32)
          for w, p in zip(ws, ps)]
    ys = [torch.full_like(x, float("nan")) for x in xs]
    for _ in range(2):
        B.apply(xs, ys)
        B.device_status()
        for p, x, y in zip(ps, xs, ys):
            for r in range(nrhs):
                xr = x[r * p.n_dofs:(r + 1) * p.n_dofs].contiguous()
                assert torch.equal(y[r * p.n_dofs:(r + 1) * p.n_dofs], p.apply_f32(xr))
    B.close()
    mixed = [G.Problem.from_workload(S.DISK_2D_Q2.resized(12, degree=3)),
             G.Problem.from_workload(S.SPHERE_3D_Q4.resized(6, degree=3))]
    B2 = G.Batch(mixed, 1, autotune=False)
    with pytest.raises(G.SbmError) as e:
        B2.set_knobs(32, 3, 3, 0, 0)
    assert G.STATUS[e.value.status] == "SBM_ERR_UNSUPPORTED"
    B2.close()


def test_batch_rejects_dg_and_bad_sizes():
    dg = G.Problem.from_workload(S.TORUS_3D_DG_Q3.resized(8))
    with pytest.raises(G.SbmError) as e:
        G.Batch([dg], 2)
    assert G.STATUS[e.value.status] == "SBM_ERR_UNSUPPORTED"
    ws, ps = _problems()
    B = G.Batch(ps[:2], 2, autotune=False)
    bad = [torch.zeros(3, device="cuda"), torch.zeros(3, device="cuda")]
    with pytest.raises(ValueError):
        B.apply(bad, bad)


def _solve_batch():
    ws = S.solve_batch()[:5] + [S.DISK_2D_Q2]
    return ws, [G.Problem.from_workload(w) for w in ws]


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_batch_solve_reaches_tolerance(mode):
    """Every system of the batch reaches |b - A x| <= 1e-10 |b|, checked with
    the single-problem FP64 apply; repeated solves are bitwise equal; the
    smallest system's solution matches the oracle's direct solve."""
    import scipy.sparse.linalg as spla

    from oracle.operator import Problem as OracleProblem
    ws, ps = _solve_batch()
    nrhs = 2
    B = G.Batch(ps, nrhs, autotune=False)
    bs = [torch.from_numpy(np.concatenate([S.random_vector(w.seed + 7 + r, p.n_dofs, "uniform")
                                           for r in range(nrhs)])).cuda()
          for w, p in zip(ws, ps)]
    xs = [torch.full_like(b, float("nan")) for b in bs]
    st, iters, relres, outer = B.solve(bs, xs, mode=mode, rtol=1e-10, check=False)
    assert st == G.SBM_OK, (G.STATUS.get(st), relres, iters, outer)
    assert relres.shape == (len(ps) * nrhs,) and np.all(relres <= 1e-10)
    assert np.all(iters > 0)
    if mode == "mixed":
        assert outer >= 1
    for p, b, x in zip(ps, bs, xs):
        for r in range(nrhs):
            sl = slice(r * p.n_dofs, (r + 1) * p.n_dofs)
            res = b[sl] - p.apply_f64(x[sl].contiguous())
            assert float(res.norm() / b[sl].norm()) <= 1.5e-10
    xs2 = [torch.empty_like(b) for b in bs]
    B.solve(bs, xs2, mode=mode, rtol=1e-10)
    for x, x2 in zip(xs, xs2):
        assert torch.equal(x, x2)
    k = min(range(len(ps)), key=lambda i: ps[i].n_dofs)
    O = OracleProblem.from_workload(ws[k])
    A = O.assemble().tocsc()
    for r in range(nrhs):
        sl = slice(r * ps[k].n_dofs, (r + 1) * ps[k].n_dofs)
        ref = spla.spsolve(A, bs[k][sl].cpu().numpy())
        assert np.abs(xs[k][sl].cpu().numpy() - ref).max() <= 1e-6 * np.abs(ref).max()
    B.close()


def test_batch_solve_rejects_bad_arguments():
    ws, ps = _solve_batch()
    B = G.Batch(ps[:2], 1, autotune=False)
    bs = [torch.zeros(p.n_dofs, dtype=torch.float64, device="cuda") for p in ps[:2]]
    xs = [torch.empty_like(b) for b in bs]
    for kw in ({"rtol": 0.0}, {"maxit": 0}, {"mode": "mixed", "inner_rtol": 1.5}):
        with pytest.raises(G.SbmError) as e:
            B.solve(bs, xs, **kw)
        assert G.STATUS[e.value.status] == "SBM_ERR_ARG"
    # zero right-hand sides: x = 0, relative residual 0
    st, iters, relres, _ = B.solve(bs, xs, mode="fp64")
    assert st == G.SBM_OK and np.all(relres == 0.0)
    assert all(float(x.abs().max()) == 0.0 for x in xs)
    B.close()


def test_batch_8rhs_matches_oracle_elementwise():
    """The persistent batched apply, 8 right-hand sides per problem, against
    the FP64 oracle element by element: FP64 within 1e-12 and FP32 within
    5e-7 (relative max norm per system); the autotuner's per-degree choices
    are recorded with the timings of the options it tried."""
    from oracle.operator import Problem as OracleProblem
    ws = S.batched_ellipsoids(nprob=5, n_range=(5, 9)) + [S.DISK_2D_Q2.resized(9, degree=3)]
    ps = [G.Problem.from_workload(w) for w in ws]
    os_ = [OracleProblem.from_workload(w) for w in ws]
    nrhs = 8
    B = G.Batch(ps, nrhs, autotune=True)
    xs = [np.concatenate([S.random_vector(S.rhs_seed(w, r), p.n_dofs, "uniform")
                          for r in range(nrhs)]) for w, p in zip(ws, ps)]
    for dt, tol in ((torch.float64, 1e-12), (torch.float32, 5e-7)):
        xd = [torch.from_numpy(x).to("cuda", dt) for x in xs]
        ys = [torch.full_like(x, float("nan")) for x in xd]
        B.apply(xd, ys)
        B.device_status()
        for p, O, x, y in zip(ps, os_, xs, ys):
            yh = y.double().cpu().numpy()
            for r in range(nrhs):
                sl = slice(r * p.n_dofs, (r + 1) * p.n_dofs)
                xr = x[sl] if dt == torch.float64 else x[sl].astype(np.float32).astype(np.float64)
                ref = O.apply(xr)
                err = float(np.abs(yh[sl] - ref).max() / np.abs(ref).max())
                assert err <= tol, (p.n_dofs, r, err)
    for prec in (32, 64):
        for deg in sorted({w.degree for w in ws}):
            k = B.knobs(prec, deg)
            # tile shape 3 (options 8, 9): FP32, degrees whose problems are all 3D
            direct = prec == 32 and all(w.dim == 3 for w in ws if w.degree == deg)
            shapes = (0, 1, 3) if direct else (0, 1)
            assert k["tile_shape"] in shapes and k["face_batch"] in (0, 1)
            opts = list(range(4)) + ([8, 9] if direct else [])
            timed = [k["ms"][i] for i in opts]
            assert all(m is not None and m > 0 for m in timed)
            if not direct:
                assert k["ms"][8] is None and k["ms"][9] is None
            best = (8 + k["face_batch"] if k["tile_shape"] == 3
                    else k["tile_shape"] + 2 * k["face_batch"])
            assert k["ms"][best] == min(timed)
    with pytest.raises(G.SbmError):
        B.knobs(64, 9)
    B.close()


def test_batch_bounded_wait_expires_without_hang():
    """A work item whose dependency nothing produces: the persistent kernel's
    bounded wait expires, SBM_ERR_TIMEOUT is reported, and the batch (and
    the context) stays usable."""
    ws, ps = _problems()
    B = G.Batch(ps[:2], 1, autotune=False)
    B.selftest_timeout()
    with pytest.raises(G.SbmError) as e:
        B.device_status()
    assert G.STATUS[e.value.status] == "SBM_ERR_TIMEOUT"
    B.device_status()           # cleared
    xs = [torch.ones(p.n_dofs, dtype=torch.float64, device="cuda") for p in ps[:2]]
    ys = [torch.empty_like(x) for x in xs]
    B.apply(xs, ys)
    B.device_status()
    for p, x, y in zip(ps[:2], xs, ys):
        assert torch.equal(y, p.apply_f64(x))
    B.close()


def test_batch_tensor_core_faces():
    """FP32 batched applies with the tensor-core face items (TF32 tcgen05
    point evaluation): within the TF32 error bound of the FP64 oracle, close
    to the single-problem TF32 apply, and the autotuner times the option."""
    from oracle.operator import Problem as OracleProblem
    ws = S.batched_ellipsoids(nprob=4, n_range=(6, 10))
    ps = [G.Problem.from_workload(w) for w in ws]
    nrhs = 2
    B = G.Batch(ps, nrhs, autotune=True, tensor_cores=True)
    for deg in sorted({w.degree for w in ws}):
        k = B.knobs(32, deg)
        assert k["ms"][4] is not None and k["ms"][5] is not None   # TC timed, both shapes
        assert k["ms"][6] is None                                  # no face batch with TC
        B.set_knobs(32, deg, 0, 0, 1)
        with pytest.raises(G.SbmError):
            B.set_knobs(64, deg, 0, 0, 1)
    xs = [np.concatenate([S.random_vector(S.rhs_seed(w, r), p.n_dofs, "uniform")
                          for r in range(nrhs)]) for w, p in zip(ws, ps)]
    xd = [torch.from_numpy(x).float().cuda() for x in xs]
    ys = [torch.full_like(x, float("nan")) for x in xd]
    B.apply(xd, ys)
    B.device_status()
    for w, p, x, y in zip(ws, ps, xs, ys):
        O = OracleProblem.from_workload(w)
        for r in range(nrhs):
            sl = slice(r * p.n_dofs, (r + 1) * p.n_dofs)
            ref = O.apply(x[sl].astype(np.float32).astype(np.float64))
            yb = y[sl].double().cpu().numpy()
            err = float(np.abs(yb - ref).max() / np.abs(ref).max())
            assert err <= 1.3e-3, (w.degree, err)
            ys_ = p.apply_f32(xd[ws.index(w)][sl].contiguous(), face_mode="tf32")
            d = float((y[sl] - ys_).abs().max() / ys_.abs().max())
            assert d <= 1e-5, d
    B.close()


def test_batch_over_one_launch_plan():
    """More problems than one launch holds (96): the batch runs several
    persistent launches in one graph; every problem still equals its single
    apply bitwise, in both precisions, including a first-order Taylor one."""
    ws = S.batched_ellipsoids(nprob=110, n_range=(3, 6), p_range=(1, 3))
    ws.append(S.SPHERE_3D_Q4.resized(6, degree=2))
    ws.append(dataclasses.replace(S.SPHERE_3D_Q4.resized(7, degree=3), extension="taylor1"))
    ps = [G.Problem.from_workload(w) for w in ws]
    nrhs = 2
    B = G.Batch(ps, nrhs, autotune=False)
    for dt in (torch.float64, torch.float32):
        xs = [torch.from_numpy(np.concatenate([S.random_vector(S.rhs_seed(w, r), p.n_dofs, "uniform")
                                               for r in range(nrhs)])).to("cuda", dt)
              for w, p in zip(ws, ps)]
        ys = [torch.full_like(x, float("nan")) for x in xs]
        B.apply(xs, ys)
        B.device_status()
        for p, x, y in zip(ps, xs, ys):
            for r in range(nrhs):
                sl = slice(r * p.n_dofs, (r + 1) * p.n_dofs)
                ref = p.apply_f64(x[sl].contiguous()) if dt == torch.float64 \
                    else p.apply_f32(x[sl].contiguous())
                assert torch.equal(y[sl], ref)
    B.close()

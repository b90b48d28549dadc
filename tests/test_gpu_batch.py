"""Batched applies (several problems, several right-hand sides, one graph
launch) give exactly the per-problem applies."""
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

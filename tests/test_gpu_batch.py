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
    tol = 1e-12 if dtype == torch.float64 else 1e-5
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

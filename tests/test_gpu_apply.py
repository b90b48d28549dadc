"""Parity of the CUDA FP64 apply (through the C ABI) with the CPU oracle.

Bar: ||y_gpu - y_oracle||_inf <= 1e-12 ||y_oracle||_inf on the same seeded x;
repeated applies are bitwise equal (atomic-free scatter)."""
import numpy as np
import pytest
import torch

import paper_2507_17053_gb300 as G
import synthetic as S
from oracle.operator import Problem as OracleProblem

pytestmark = pytest.mark.gpu
TOL = 1e-12
# FP32 apply against the FP64 oracle on FP32-rounded x (measured on a GB300:
# at most 1.5e-7 for p = 1..6; about 3x that)
F32_TOL = 5e-7


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    G.lib()


def _pair(w):
    return OracleProblem.from_workload(w), G.Problem.from_workload(w)


def _rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def _check_full(w, seed=None, dist=None):
    O, P = _pair(w)
    assert P.n_dofs == O.n_dofs
    x = S.random_vector(w.seed if seed is None else seed, O.n_dofs, dist or w.dist)
    xd = torch.from_numpy(x).cuda()
    y = P.apply_f64(xd)
    y2 = P.apply_f64(xd)
    torch.cuda.synchronize()
    assert torch.equal(y, y2), "repeated apply is not bitwise identical"
    ref = O.apply(x)
    err = _rel(y.cpu().numpy(), ref)
    assert err <= TOL, err
    return P, O, x, y


CG_CASES = [
    S.DISK_2D_Q2,                                   # the 2D workload at full size
    S.SPHERE_3D_Q4.resized(14),
    S.SPHERE_3D_Q4.resized(9),
    S.ELLIPSOID_3D_Q6.resized(10),
] + [S.DISK_2D_Q2.resized(11, degree=p) for p in range(1, 7)] \
  + [S.SPHERE_3D_Q4.resized(7, degree=p) for p in range(1, 7)] \
  + S.batched_ellipsoids(nprob=5, n_range=(6, 12))


@pytest.mark.parametrize("w", CG_CASES, ids=lambda w: w.name)
def test_cg_apply_matches_oracle(w):
    _check_full(w)


def test_single_active_cell():
    # a tiny ball around one cell centre: one active cell, 2d surrogate faces
    for d in (2, 3):
        c = (-1.0 + 0.25 * 3.5,) * d
        w = S._wl("single", d, 3, 8, S.ball(d, c, 0.05))
        P, O, _, _ = _check_full(w)
        assert P.n_cells == 1 and P.n_sfaces == 2 * d


def test_whole_box_and_one_cell_mesh():
    for d in (2, 3):
        # every cell active; the surrogate boundary is the box boundary, d = 0
        _check_full(S._wl("box", d, 2, 5, S.box((0.0,) * d, (1.5,) * d)))
        _check_full(S._wl("one", d, 4, 1, S.ball(d, (0.0,) * d, 0.9)))


# two balls with empty cell layers between them along z (3D) / y (2D)
_TWO_BALLS_3D = S._wl("two_balls_3d", 3, 3, 16, (S.BALLS, (0.1, 0.0, -0.6, 0.3,
                                                          -0.1, 0.05, 0.55, 0.35)))
_TWO_BALLS_2D = S._wl("two_balls_2d", 2, 4, 24, (S.BALLS, (0.0, -0.6, 0.3, 0.1, 0.6, 0.3)))


@pytest.mark.parametrize("w", [S.SPHERE_3D_Q4.resized(10), S.SPHERE_3D_Q4.resized(24),
                               S.DISK_2D_Q2, S.ELLIPSOID_3D_Q6.resized(9), _TWO_BALLS_3D,
                               _TWO_BALLS_2D, S.SPHERE_3D_Q4.resized(24, degree=1),
                               S.TORUS_3D_DG_Q3.resized(12)],
                         ids=lambda w: w.name)
def test_host_entry_point_equals_device_apply(w):
    """The host-buffer entry point pipelines the copies with the kernels
    slab by slab (cell layers along the last axis; with page-locked buffers
    as a CUDA graph captured per buffer pair and replayed); its result is
    bitwise the device apply's, with either tile shape, on a replay with new
    contents in the same buffers, and with pageable buffers."""
    P = G.Problem.from_workload(w)
    x = S.random_vector(3, P.n_dofs, "uniform")
    xh = torch.from_numpy(x).pin_memory()
    for shape in ((0,) if w.dg else (0, 1)):
        G.sbm_set_tile_shape(P.handle, shape, shape)
        yd = P.apply_f64(torch.from_numpy(x).cuda()).cpu().numpy()
        yh = torch.full((P.n_dofs,), np.nan, dtype=torch.float64).pin_memory()
        P.apply_f64_host(xh, yh)
        np.testing.assert_array_equal(yh.numpy(), yd)
        # the same buffers again, new contents (the captured graph replays)
        x2 = S.random_vector(4, P.n_dofs, "uniform")
        xh.copy_(torch.from_numpy(x2))
        yh.fill_(float("nan"))
        P.apply_f64_host(xh, yh)
        np.testing.assert_array_equal(yh.numpy(), P.apply_f64(torch.from_numpy(x2).cuda()).cpu().numpy())
        xh.copy_(torch.from_numpy(x))
        # pageable host buffers too
        yp = P.apply_f64_host(x.copy())
        np.testing.assert_array_equal(yp, yd)


def _sample_rows(O, rng, nrand=10000, nface_cells=200):
    rows = rng.choice(O.n_dofs, size=min(nrand, O.n_dofs), replace=False)
    fc = np.unique(O.mesh.sfaces[:, 0])
    pick = rng.choice(fc, size=min(nface_cells, len(fc)), replace=False)
    rows = np.unique(np.concatenate([rows, O.dofmap[pick].ravel()]))
    return rows


@pytest.mark.parametrize("w", [S.SPHERE_3D_Q4, S.ELLIPSOID_3D_Q6], ids=lambda w: w.name)
def test_full_size_sampled_rows(w):
    """Full-size workload, launched as the benchmark launches it; checked on
    10^4 random rows plus every row of 200 sampled surrogate-face cells."""
    O, P = _pair(w)
    x = S.random_vector(w.seed, O.n_dofs, w.dist)
    y = P.apply_f64(torch.from_numpy(x).cuda()).cpu().numpy()
    rows = _sample_rows(O, np.random.default_rng(0))
    ref = O.apply_rows(x, rows)
    scale = np.abs(ref).max()
    assert np.abs(y[rows] - ref).max() <= TOL * scale


@pytest.mark.parametrize("w", [S.SPHERE_3D_Q4, S.ELLIPSOID_3D_Q6], ids=lambda w: w.name)
def test_full_size_sampled_rows_autotuned(w):
    """Full-size workload in the benchmark's launch configuration (the
    autotuner's tile shape and store mode per precision): FP64 and FP32
    applies on 10^4 random rows plus every row of 200 sampled surrogate-face
    cells against the oracle."""
    O, P = _pair(w)
    shapes = G.sbm_autotune(P.handle)
    x = S.random_vector(w.seed, O.n_dofs, w.dist)
    xd = torch.from_numpy(x).cuda()
    rows = _sample_rows(O, np.random.default_rng(1))
    y = P.apply_f64(xd).cpu().numpy()
    ref = O.apply_rows(x, rows)
    assert np.abs(y[rows] - ref).max() <= TOL * np.abs(ref).max(), shapes
    x32 = x.astype(np.float32).astype(np.float64)
    y32 = P.apply_f32(xd.float()).double().cpu().numpy()
    ref32 = O.apply_rows(x32, rows)
    assert np.abs(y32[rows] - ref32).max() <= F32_TOL * np.abs(ref32).max(), shapes


@pytest.mark.parametrize("w", [S.SPHERE_3D_Q4.resized(12), S.ELLIPSOID_3D_Q6.resized(9),
                               S.DISK_2D_Q2], ids=lambda w: w.name)
def test_autotuned_tile_shapes_keep_parity(w):
    """Both cell-kernel tile shapes (chunks of R and R/2 cells) match the oracle."""
    O, P = _pair(w)
    x = S.random_vector(w.seed, O.n_dofs, w.dist)
    xd = torch.from_numpy(x).cuda()
    ref = O.apply(x)
    shapes = G.sbm_autotune(P.handle)
    assert all(s in ((0, 1, 2, 3) if w.dim == 3 else (0, 1)) for s in shapes)
    assert _rel(P.apply_f64(xd).cpu().numpy(), ref) <= TOL
    ref32 = O.apply(x.astype(np.float32).astype(np.float64))
    y32 = P.apply_f32(xd.float()).double().cpu().numpy()
    assert _rel(y32, ref32) <= F32_TOL
    # each shape pinned explicitly
    for s in (0, 1):
        G.sbm_set_tile_shape(P.handle, s, s)
        assert _rel(P.apply_f64(xd).cpu().numpy(), ref) <= TOL
        assert _rel(P.apply_f32(xd.float()).double().cpu().numpy(), ref32) <= F32_TOL
    with pytest.raises(G.SbmError):
        G.sbm_set_tile_shape(P.handle, 4, 0)


# tile shape 2: one thread per cell, the tile in registers (3D, FP32 p <= 4,
# FP64 p <= 3); the same chunks and summation order as shape 0
REG_CASES = [S.SPHERE_3D_Q4.resized(n, degree=p) for p, n in ((1, 9), (2, 8), (3, 7), (4, 12))] \
    + [S.ELLIPSOID_3D_Q6.resized(10, degree=4), S.SPHERE_3D_Q4.resized(17, degree=2)] \
    + S.batched_ellipsoids(nprob=3, n_range=(7, 11), p_range=(2, 4))


@pytest.mark.parametrize("w", REG_CASES, ids=lambda w: f"{w.name}_q{w.degree}")
def test_register_tile_shape_equals_shape0_and_oracle(w):
    O, P = _pair(w)
    x = S.random_vector(w.seed, O.n_dofs, w.dist)
    xd = torch.from_numpy(x).cuda()
    ref = O.apply(x)
    ref32 = O.apply(x.astype(np.float32).astype(np.float64))
    fp64 = w.degree <= 3
    G.sbm_set_tile_shape(P.handle, 0, 0)
    y64_0, y32_0 = P.apply_f64(xd), P.apply_f32(xd.float())
    G.sbm_set_tile_shape(P.handle, 2 if fp64 else 0, 2)
    y64, y32 = P.apply_f64(xd), P.apply_f32(xd.float())
    assert torch.equal(y32, y32_0), "shape 2 differs from shape 0 in FP32"
    assert torch.equal(y32, P.apply_f32(xd.float())), "repeated apply differs"
    assert _rel(y32.double().cpu().numpy(), ref32) <= F32_TOL
    if fp64:
        assert torch.equal(y64, y64_0), "shape 2 differs from shape 0 in FP64"
    assert _rel(y64.cpu().numpy(), ref) <= TOL
    # the host-buffer pipeline runs shape 0 for its slabs: the same bits
    yh = P.apply_f64_host(x)
    assert np.array_equal(yh, y64.cpu().numpy())


def test_register_tile_shape_rejected_where_unavailable():
    for w, shapes in ((S.SPHERE_3D_Q4.resized(6, degree=5), (-1, 2)),
                      (S.SPHERE_3D_Q4.resized(6, degree=4), (2, -1)),
                      (S.DISK_2D_Q2, (-1, 2)), (S.DISK_2D_Q2, (3, -1)),
                      (S.TORUS_3D_DG_Q3.resized(8), (3, -1))):
        P = G.Problem.from_workload(w)
        with pytest.raises(G.SbmError) as e:
            G.sbm_set_tile_shape(P.handle, *shapes)
        assert G.STATUS[e.value.status] == "SBM_ERR_UNSUPPORTED"


# tile shape 3 (3D, every degree): shape 0's chunks, each thread loading and
# storing its own z-lines instead of staging x-line runs in shared memory
DIRECT_CASES = [S.SPHERE_3D_Q4.resized(7, degree=p) for p in range(1, 7)] \
    + [S.SPHERE_3D_Q4.resized(17, degree=2), S.ELLIPSOID_3D_Q6.resized(10), _TWO_BALLS_3D] \
    + S.batched_ellipsoids(nprob=3, n_range=(7, 11))


@pytest.mark.parametrize("w", DIRECT_CASES, ids=lambda w: f"{w.name}_q{w.degree}")
def test_direct_tile_shape_equals_shape0_and_oracle(w):
    O, P = _pair(w)
    x = S.random_vector(w.seed, O.n_dofs, w.dist)
    xd = torch.from_numpy(x).cuda()
    ref = O.apply(x)
    ref32 = O.apply(x.astype(np.float32).astype(np.float64))
    G.sbm_set_tile_shape(P.handle, 0, 0)
    y64_0, y32_0 = P.apply_f64(xd), P.apply_f32(xd.float())
    yh_0 = P.apply_f64_host(x)
    G.sbm_set_tile_shape(P.handle, 3, 3)
    y64, y32 = P.apply_f64(xd), P.apply_f32(xd.float())
    assert torch.equal(y64, y64_0), "shape 3 differs from shape 0 in FP64"
    assert torch.equal(y32, y32_0), "shape 3 differs from shape 0 in FP32"
    assert torch.equal(y64, P.apply_f64(xd)), "repeated apply differs"
    assert _rel(y64.cpu().numpy(), ref) <= TOL
    assert _rel(y32.double().cpu().numpy(), ref32) <= F32_TOL
    # the host-buffer pipeline runs shape 3 slab by slab: the same bits
    assert np.array_equal(P.apply_f64_host(x), yh_0)


# colour-ordered stores (no colour buffers, no assembly pass): bitwise the
# colour-buffer applies of the same tile shape, applied repeatedly (the
# per-chunk completion counts carry over between launches)
ORDERED_CASES = [S.SPHERE_3D_Q4.resized(9, degree=p) for p in range(1, 7)] \
    + [S.DISK_2D_Q2.resized(13, degree=p) for p in range(1, 7)] \
    + [S.DISK_2D_Q2, S.SPHERE_3D_Q4.resized(24), S.ELLIPSOID_3D_Q6.resized(10), _TWO_BALLS_3D,
       _TWO_BALLS_2D] + S.batched_ellipsoids(nprob=3, n_range=(7, 11))


@pytest.mark.parametrize("w", ORDERED_CASES, ids=lambda w: f"{w.name}_q{w.degree}")
def test_ordered_stores_equal_colour_buffers(w):
    O, P = _pair(w)
    x = S.random_vector(w.seed, O.n_dofs, w.dist)
    xd = torch.from_numpy(x).cuda()
    ref = O.apply(x)
    ref32 = O.apply(x.astype(np.float32).astype(np.float64))
    for shape in [0] + ([3] if w.dim == 3 else []):
        G.sbm_set_tile_shape(P.handle, shape, shape)
        G.sbm_set_ordered_stores(P.handle, 0, 0)
        y64_0, y32_0 = P.apply_f64(xd), P.apply_f32(xd.float())
        G.sbm_set_ordered_stores(P.handle, 1, 1)
        assert G.sbm_ordered_stores(P.handle) == (1, 1)
        for rep in range(3):
            y64, y32 = P.apply_f64(xd), P.apply_f32(xd.float())
            assert torch.equal(y64, y64_0), f"FP64 shape {shape}: ordered != colour buffers"
            assert torch.equal(y32, y32_0), f"FP32 shape {shape}: ordered != colour buffers"
        G.sbm_device_status(P.handle)
        assert _rel(y64.cpu().numpy(), ref) <= TOL
        assert _rel(y32.double().cpu().numpy(), ref32) <= F32_TOL
    # the host-buffer pipeline keeps the colour buffers: the same bits
    assert np.array_equal(P.apply_f64_host(x), y64_0.cpu().numpy())


def test_ordered_stores_autotuned_and_rejected_for_dg():
    w = S.SPHERE_3D_Q4.resized(20)
    O, P = _pair(w)
    x = S.random_vector(w.seed, O.n_dofs, w.dist)
    xd = torch.from_numpy(x).cuda()
    G.sbm_autotune(P.handle)
    assert all(o in (0, 1) for o in G.sbm_ordered_stores(P.handle))
    assert _rel(P.apply_f64(xd).cpu().numpy(), O.apply(x)) <= TOL
    D = G.Problem.from_workload(S.TORUS_3D_DG_Q3.resized(8))
    with pytest.raises(G.SbmError) as e:
        G.sbm_set_ordered_stores(D.handle, 1, -1)
    assert G.STATUS[e.value.status] == "SBM_ERR_UNSUPPORTED"

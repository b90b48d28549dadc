"""The C-ABI library loads, exports every declared symbol, and checks its
arguments on the host (no GPU needed)."""
import ctypes

import dataclasses

import numpy as np
import pytest

import paper_2507_17053_gb300 as G
import synthetic as S
from oracle.operator import Problem as OracleProblem


@pytest.fixture(scope="module")
def lib():
    return G.lib()


def test_every_declared_symbol_is_exported(lib):
    names = G.header_functions()
    assert "sbm_apply_f64" in names and "sbm_create" in names
    for name in names:
        assert hasattr(lib, name), name


def test_error_strings(lib):
    for code in range(10):
        assert lib.sbm_error_string(code)
    assert lib.sbm_error_string(12345) == b"unknown status"


@pytest.mark.parametrize("bad,code", [
    (dict(dim=4), "SBM_ERR_ARG"),
    (dict(degree=0), "SBM_ERR_UNSUPPORTED"),
    (dict(degree=7), "SBM_ERR_UNSUPPORTED"),
    (dict(cells=0), "SBM_ERR_ARG"),
    (dict(kind=9), "SBM_ERR_ARG"),
    (dict(geom=(0.0, 0.0, -1.0)), "SBM_ERR_ARG"),
    (dict(geom=(5.0, 5.0, 0.1)), "SBM_ERR_EMPTY_DOMAIN"),
    (dict(pen_shift=0.0), "SBM_ERR_ARG"),
    (dict(extension=2), "SBM_ERR_ARG"),
    (dict(activity=2), "SBM_ERR_ARG"),
    (dict(activity=1, vf_threshold=0.0), "SBM_ERR_ARG"),
])
def test_create_rejects_bad_descriptions(bad, code):
    args = dict(dim=2, degree=2, cells=8, kind="ball", geom=(0.0, 0.0, 0.7))
    args.update(bad)
    with pytest.raises(G.SbmError) as e:
        G.sbm_create(G.make_desc(**args))
    assert G.STATUS[e.value.status] == code


def test_null_arguments(lib):
    assert lib.sbm_create(None, None) == 1
    out = ctypes.c_void_p()
    assert lib.sbm_create(None, ctypes.byref(out)) == 1 and out.value is None
    assert lib.sbm_apply_f64(None, None, None, None) == 1
    assert lib.sbm_sizes(None, None, None, None, None) == 1
    assert lib.sbm_apply_f64_host(None, None, None, None) == 1
    assert lib.sbm_bicgstab_mixed(None, None, None, 1e-10, 10, 0, None, None, None, None) == 1
    assert lib.sbm_batch_solve(None, None, None, 0, 1e-10, 10, 1e-2, 10, None, None, None,
                               None) == 1
    assert lib.sbm_batch_create(None, 0, 1, 0, ctypes.byref(out)) == 1
    lib.sbm_batch_destroy(None)   # no-op
    lib.sbm_destroy(None)   # no-op


def test_apply_before_device_setup_is_a_state_error():
    P = G.Problem(2, 2, 8, "ball", (0.0, 0.0, 0.7), device=False)
    with pytest.raises(G.SbmError) as e:
        G.sbm_apply_f64(P.handle, 16, 32, 0)   # fake non-null addresses: never touched
    assert G.STATUS[e.value.status] == "SBM_ERR_STATE"
    with pytest.raises(G.SbmError) as e:
        G.sbm_apply_f64(P.handle, 16, 16, 0)
    assert G.STATUS[e.value.status] == "SBM_ERR_ARG"
    # the host-buffer apply and the solvers check the state before any device work
    for call in (lambda: G.sbm_apply_f64_host(P.handle, 16, 32, 0),
                 lambda: G.sbm_bicgstab(P.handle, 16, 32, rtol=1e-10, maxit=10, stream=0),
                 lambda: G.sbm_bicgstab_mixed(P.handle, 16, 32, rtol=1e-10, maxit=10,
                                              stream=0),
                 lambda: G.sbm_solve_ir(P.handle, 16, 32, stream=0)):
        with pytest.raises(G.SbmError) as e:
            call()
        assert G.STATUS[e.value.status] == "SBM_ERR_STATE"


def _compare_geometry(w):
    O = OracleProblem.from_workload(w)
    P = G.Problem.from_workload(w, device=False)
    cells, sfaces, fx = P.geometry()
    assert P.n_cells == len(O.mesh.cells)
    assert P.n_dofs == O.n_dofs
    np.testing.assert_array_equal(cells, O.mesh.cells)          # bit-exact
    np.testing.assert_array_equal(sfaces, O.mesh.sfaces)
    if O.dg:
        assert P.n_ifaces == len(O.mesh.ifaces)
    # closest points: two independent projections (closed forms / bisection vs Newton)
    np.testing.assert_allclose(fx, O.mesh.face_x, rtol=0, atol=2e-14)


SMALL = [
    S.DISK_2D_Q2,
    S.SPHERE_3D_Q4.resized(20),
    S.ELLIPSOID_3D_Q6.resized(14),
    S.TORUS_3D_DG_Q3.resized(18),
] + S.batched_ellipsoids(nprob=4, n_range=(8, 14)) + [
    S.multiple_balls(3, cells=24), S.multiple_balls(12, cells=24, degree=2),
    S.multiple_balls(25, cells=32), S.multiple_balls(6, dim=2, cells=48, degree=2)] + [
    dataclasses.replace(S.DISK_2D_Q2, activity="volume", vf_threshold=t, name=f"disk_vf{t}")
    for t in (0.2, 0.5, 0.9)] + [
    dataclasses.replace(S.SPHERE_3D_Q4.resized(16), activity="volume", vf_threshold=0.3,
                        name="sphere_vf0.3"),
    dataclasses.replace(S.multiple_balls(10, cells=24), activity="volume", vf_threshold=0.6,
                        name="balls_vf0.6")]


@pytest.mark.parametrize("w", SMALL, ids=lambda w: w.name)
def test_host_geometry_matches_oracle(w):
    _compare_geometry(w)


@pytest.mark.slow
def test_host_geometry_matches_oracle_full_sphere():
    _compare_geometry(S.SPHERE_3D_Q4)


@pytest.mark.parametrize("w", SMALL[:4], ids=lambda w: w.name)
def test_host_rhs_and_interpolant_match_oracle(w):
    from oracle.operator import sin_solution
    O = OracleProblem.from_workload(w)
    P = G.Problem.from_workload(w, device=False)
    u, f = sin_solution(w.dim)
    ref = O.rhs(f, u)
    assert np.abs(P.rhs(0) - ref).max() <= 1e-13 * np.abs(ref).max()
    np.testing.assert_allclose(P.interpolate(0), O.interpolate(u), rtol=0, atol=1e-15)
    if w.dim == 2:
        u1 = lambda X: 2.0 * np.cos(X[..., 0]) * np.sin(X[..., 1])
        ref1 = O.rhs(lambda X: 2.0 * u1(X), u1)
        assert np.abs(P.rhs(1) - ref1).max() <= 1e-13 * np.abs(ref1).max()


@pytest.mark.parametrize("dist", ["uniform", "normal"])
@pytest.mark.parametrize("seed,offset", [(0, 0), (1, 0), (3, 17), (4 * 1000003 + 21, 5),
                                         (2 ** 64 - 1, 1000), (12345, 2 ** 40)])
def test_fill_random_matches_the_workload_generator(dist, seed, offset):
    """The exported generator gives the workload vectors bit for bit: the
    same splitmix64 values, the same 53-bit uniforms, the same Box--Muller
    arithmetic (C library log1p and cos, no fused multiply-adds)."""
    n = 2000
    got = G.sbm_fill_random(n, seed, dist, offset)
    ref = S.uniform_pm1(seed, n, offset) if dist == "uniform" else S.normal(seed, n, offset)
    assert np.array_equal(got.view(np.uint64), ref.view(np.uint64))
    if offset == 0:
        assert np.array_equal(got, S.random_vector(seed, n, dist))
    # a window of a longer stream is the same numbers
    tail = G.sbm_fill_random(n - 7, seed, dist, offset + 7)
    assert np.array_equal(tail, got[7:])


def test_fill_random_distributions_and_errors(lib):
    u = G.sbm_fill_random(200000, 9, "uniform")
    assert u.min() >= -1.0 and u.max() < 1.0 and abs(u.mean()) < 0.01
    z = G.sbm_fill_random(200000, 9, "normal")
    assert abs(z.mean()) < 0.01 and abs(z.std() - 1.0) < 0.01
    # the first stream value of seed 0 is the published splitmix64 output
    # for state 0 (the generator's first call): 0xE220A8397B1DCDAF
    first = S.splitmix64(0, 1)[0]
    assert int(first) == 0xE220A8397B1DCDAF
    assert u.size == 200000 and G.sbm_fill_random(0, 1, "uniform").size == 0
    assert lib.sbm_fill_random(-1, 0, 0, 0, None) == 1
    assert lib.sbm_fill_random(4, 0, 0, 0, None) == 1
    buf = (ctypes.c_double * 4)()
    assert lib.sbm_fill_random(4, 0, 0, 7, buf) == 1

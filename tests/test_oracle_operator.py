"""Pins of the oracle's global operator: brute force, closed forms, patch tests,
special cases and the convergence rates the paper reports (Appendix A)."""
import math
import os

import numpy as np
import pytest
import scipy.sparse.linalg as spla

import synthetic as S
from oracle import geometry, local
from oracle.operator import Problem, sin_solution

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

TINY = [
    # (dim, p, N, kind, geom, dg)
    (2, 2, 6, "ball", (0.05, -0.03, 0.73), False),
    (2, 3, 5, "ball", (0.1, 0.0, 0.8), True),
    (3, 2, 4, "ball", (0.02, 0.01, -0.03, 0.71), False),
    (3, 1, 6, "torus", (0.6, 0.25), True),
    (3, 2, 5, S.ellipsoid((0.8, 0.6, 0.5), S.rotation_from_quaternion((1, 0.3, -0.2, 0.5)))[0],
     S.ellipsoid((0.8, 0.6, 0.5), S.rotation_from_quaternion((1, 0.3, -0.2, 0.5)))[1], False),
]


def _prob(case):
    d, p, N, kind, geom, dg = case
    return Problem(d, p, N, kind, geom, dg=dg)


@pytest.mark.parametrize("case", TINY)
def test_assembled_equals_matrix_free_columnwise(case):
    """Brute force: column j of the CSR matrix equals the EBE apply of e_j."""
    P = _prob(case)
    A = P.assemble().toarray()
    n = P.n_dofs
    cols = np.unique(np.r_[0, n - 1, np.linspace(0, n - 1, 40).astype(int)])
    for j in cols:
        e = np.zeros(n)
        e[j] = 1.0
        np.testing.assert_allclose(P.apply(e), A[:, j], atol=1e-12 * np.abs(A).max())
    x = S.uniform_pm1(7, n)
    np.testing.assert_allclose(P.apply(x), A @ x, atol=1e-12 * np.abs(A).max())
    rows = np.array([0, n // 3, n - 1])
    np.testing.assert_allclose(P.apply_rows(x, rows), (A @ x)[rows], atol=1e-12 * np.abs(A).max())
    np.testing.assert_allclose(P.diagonal(), np.diag(A), atol=1e-12 * np.abs(A).max())


def _face_weight_sum(P, values):
    """sum_F sum_q h^{d-1} w_q values[F, q]."""
    return float(np.sum(values * P.mesh.face_weights[None, :]) * P.h ** (P.d - 1))


@pytest.mark.parametrize("case", TINY)
def test_constants_and_linear_functions(case):
    """a(1,1) = sigma |surrogate boundary|; a(u,1) and a(1,u) for linear u.

    With v = 1 only the penalty term survives, evaluated at the shifted
    points x_q for the trial function (1^T A u) and at the unshifted face
    points for the test function (u^T A 1); the normal-derivative terms
    cancel because the surrogate boundary is closed.
    """
    P = _prob(case)
    A = P.assemble()
    one = np.ones(P.n_dofs)
    nsf = len(P.mesh.sfaces)
    assert abs(one @ (A @ one) - P.sigma * nsf * P.h ** (P.d - 1)) < 1e-10 * P.sigma * nsf
    a = np.array([0.7, -1.3, 0.4][:P.d])
    b = 0.25
    lin = lambda X: X @ a + b
    u = P.interpolate(lin)
    ref_trial = P.sigma * _face_weight_sum(P, lin(P.mesh.face_x))
    ref_test = P.sigma * _face_weight_sum(P, lin(P.mesh.face_xt))
    scale = P.sigma * nsf * P.h ** (P.d - 1)
    assert abs(one @ (A @ u) - ref_trial) < 1e-10 * scale
    assert abs(u @ (A @ one) - ref_test) < 1e-10 * scale
    assert np.abs(P.mesh.face_shift).max() > 1e-3     # the shift is really there


@pytest.mark.parametrize("dg", [False, True])
@pytest.mark.parametrize("d", [2, 3])
def test_zero_shift_is_symmetric_nitsche(d, dg):
    """Box domain on mesh planes: x_q = x~_q, d = 0, and A is the symmetric
    Nitsche (plus SIPG) operator of Section 2: symmetric, and v^T A v > 0."""
    p = 2
    P = Problem(d, p, 8, "box", (0.0,) * d + (0.5,) * d, dg=dg)
    assert np.abs(P.mesh.face_shift).max() == 0.0
    A = P.assemble().toarray()
    np.testing.assert_allclose(A, A.T, atol=1e-12 * np.abs(A).max())
    assert np.linalg.eigvalsh(A)[0] > 0
    # a box that is not on mesh planes has a pure normal shift and breaks symmetry
    Q = Problem(d, p, 8, "box", (0.0,) * d + (0.55,) * d, dg=dg)
    sh = Q.mesh.face_shift
    kk = Q.mesh.sfaces[:, 1]
    for f in range(len(kk)):
        tang = [l for l in range(d) if l != kk[f]]
        assert np.abs(sh[f][:, tang]).max() == 0.0
        np.testing.assert_allclose(np.abs(sh[f][:, kk[f]]), 0.05, atol=1e-15)
    B = Q.assemble().toarray()
    assert np.abs(B - B.T).max() > 1e-3 * np.abs(B).max()


def _closest_cases():
    R = S.rotation_from_quaternion((0.3, -1.0, 0.4, 0.2))
    return [
        ("ball", (0.05, -0.03, 0.73), 2),
        ("ball", (0.02, 0.01, -0.03, 0.71), 3),
        ("torus", (0.6, 0.25), 3),
        S.ellipsoid((0.8, 0.6, 0.5)) + (3,),
        S.ellipsoid((0.85, 0.45, 0.6), R) + (3,),
        S.ellipsoid((0.7, 0.4)) + (2,),
    ]


@pytest.mark.parametrize("kind,geom,d", _closest_cases())
def test_closest_point(kind, geom, d):
    ls = geometry.LevelSet(kind, geom, d)
    rng = np.random.default_rng(11)
    pts = rng.uniform(-0.95, 0.95, size=(400, d))
    x = ls.closest_point(pts)
    assert np.abs(ls.phi(x)).max() < 1e-13
    # x - x~ is parallel to the surface normal at x (grad phi by central differences)
    e = 1e-6
    grad = np.stack([(ls.phi(x + e * np.eye(d)[i]) - ls.phi(x - e * np.eye(d)[i])) / (2 * e)
                     for i in range(d)], axis=-1)
    v = pts - x
    cos = np.abs(np.sum(v * grad, -1)) / (np.linalg.norm(v, axis=-1) * np.linalg.norm(grad, axis=-1))
    far = np.linalg.norm(v, axis=-1) > 1e-3
    assert np.all(cos[far] > 1 - 1e-6)
    # brute force: no sampled boundary point is closer than x (up to sampling)
    if d == 2:
        t = np.linspace(0, 2 * math.pi, 20001)
        dirs = np.stack([np.cos(t), np.sin(t)], -1)
    else:
        g = rng.normal(size=(60000, 3))
        dirs = g / np.linalg.norm(g, axis=-1, keepdims=True)
    samples = _surface_samples(ls, dirs)
    for i in range(0, len(pts), 40):
        best = np.min(np.linalg.norm(samples - pts[i], axis=-1))
        assert np.linalg.norm(pts[i] - x[i]) <= best + 1e-9


def _surface_samples(ls, dirs):
    """Points on Gamma along rays (ball/ellipsoid: from the centre; torus: a
    parametric sweep)."""
    if ls.kind == "ball":
        return ls.c + ls.r * dirs
    if ls.kind == "ellipsoid":
        y = dirs / np.sqrt(np.sum((dirs / ls.a) ** 2, -1, keepdims=True))
        return ls.c + y @ ls.R.T
    if ls.kind == "torus":
        u = np.linspace(0, 2 * math.pi, 800)
        v = np.linspace(0, 2 * math.pi, 400)
        U, V = np.meshgrid(u, v)
        rr = ls.Rmaj + ls.rmin * np.cos(V)
        return np.stack([rr * np.cos(U), rr * np.sin(U), ls.rmin * np.sin(V)], -1).reshape(-1, 3)
    raise AssertionError


def _poly(d, p, seed):
    """A random polynomial of degree <= p in each variable, and -Laplacian."""
    rng = np.random.default_rng(seed)
    terms = [(tuple(rng.integers(0, p + 1, size=d)), rng.normal()) for _ in range(6)]
    terms.append(((0,) * d, 0.3))

    def u(X):
        out = np.zeros(X.shape[:-1])
        for e, c in terms:
            out = out + c * np.prod([X[..., i] ** e[i] for i in range(d)], axis=0)
        return out

    def f(X):
        out = np.zeros(X.shape[:-1])
        for e, c in terms:
            for k in range(d):
                if e[k] >= 2:
                    ek = list(e)
                    ek[k] -= 2
                    out = out - c * e[k] * (e[k] - 1) * np.prod(
                        [X[..., i] ** ek[i] for i in range(d)], axis=0)
        return out
    return u, f


PATCH = [
    (2, 1, 8, "ball", (0.05, -0.03, 0.73), False),
    (2, 2, 7, "ball", (0.05, -0.03, 0.73), False),
    (2, 3, 6, "ball", (0.1, 0.05, 0.8), False),
    (2, 2, 7, "ball", (0.05, -0.03, 0.73), True),
    (3, 2, 5, "ball", (0.02, 0.01, -0.03, 0.71), False),
    (3, 1, 8, "torus", (0.6, 0.25), True),
    (3, 2, 5, S.ellipsoid((0.8, 0.6, 0.5), S.rotation_from_quaternion((1, 0.3, -0.2, 0.5)))[0],
     S.ellipsoid((0.8, 0.6, 0.5), S.rotation_from_quaternion((1, 0.3, -0.2, 0.5)))[1], False),
]


@pytest.mark.parametrize("case", PATCH)
def test_patch_polynomial_reproduced(case):
    """u* in Q_p, f = -Lap u*, g = u* at x_q: the discrete solution is u*.

    Point evaluation of the cell polynomial at the shifted point is exact for
    u* in Q_p, and all quadratures are exact, so the SBM solution reproduces
    u* (Section 2.1 weak form with E applied to u_h)."""
    d, p = case[0], case[1]
    P = _prob(case)
    u, f = _poly(d, p, seed=3 * d + p)
    b = P.rhs(f, u)
    uh = spla.spsolve(P.assemble().tocsc(), b)
    ref = P.interpolate(u)
    assert np.abs(uh - ref).max() < 1e-8 * max(1.0, np.abs(ref).max())


def test_patch_fails_for_degree_above_p():
    """Guard: a polynomial outside Q_p is NOT reproduced."""
    P = Problem(2, 1, 8, "ball", (0.05, -0.03, 0.73))
    u = lambda X: X[..., 0] ** 2
    f = lambda X: -2.0 * np.ones(X.shape[:-1])
    uh = spla.spsolve(P.assemble().tocsc(), P.rhs(f, u))
    assert np.abs(uh - P.interpolate(u)).max() > 1e-4


def _rates():
    out = {}
    for line in open(os.path.join(GOLDEN, "convergence_rates.txt")):
        if line.startswith("#") or not line.strip():
            continue
        p, r = line.split()
        out[int(p)] = float(r)
    return out


@pytest.mark.parametrize("p", [1, 2, 3])
def test_convergence_rate_unit_circle(p):
    """Appendix A: circle, u = 2 cos(x1) sin(x2); L2 error O(h^{p+1}).

    The circle is scaled to radius 0.8 inside [-1,1]^2 (u and f scaled with
    it).  SBM errors oscillate with how the surrogate boundary sits on the
    mesh, so the rate is the least-squares slope over eight meshes."""
    u = lambda X: 2.0 * np.cos(X[..., 0] / 0.8) * np.sin(X[..., 1] / 0.8)
    f = lambda X: 2.0 * u(X) / 0.64
    Ns = np.array([10, 14, 20, 28, 40, 56, 80, 112])
    errs = []
    for N in Ns:
        P = Problem(2, p, int(N), "ball", (0.0, 0.0, 0.8))
        uh = spla.spsolve(P.assemble().tocsc(), P.rhs(f, u))
        errs.append(P.l2_error(uh, u))
    slope = np.polyfit(np.log(2.0 / Ns), np.log(errs), 1)[0]
    expected = _rates()[p]
    assert slope > expected - 0.35, (errs, slope)


def test_convergence_rate_sin_disk():
    """Disk of the 2D workload with u = sin(pi x) sin(pi y), p = 2."""
    u, f = sin_solution(2)
    errs = []
    for N in (16, 32, 64):
        P = Problem(2, 2, N, "ball", (0.05, -0.03, 0.73))
        uh = spla.spsolve(P.assemble().tocsc(), P.rhs(f, u))
        errs.append(P.l2_error(uh, u))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.mean(rates) > 2.65, (errs, rates)


def test_workload_sizes_disk():
    """The 2D workload's surrogate domain: 427 active cells, 92 surrogate
    faces, 1 801 DoFs."""
    P = Problem.from_workload(S.DISK_2D_Q2)
    assert (len(P.mesh.cells), len(P.mesh.sfaces), P.n_dofs) == (427, 92, 1801)
    # every active cell's centre is inside, every surrogate face has an
    # inactive (or missing) neighbour, so the surrogate boundary is closed:
    # sum over faces of the outward normal is zero
    nsum = np.zeros(2)
    for c, k, s in P.mesh.sfaces:
        nsum[k] += 2 * s - 1
    assert np.all(nsum == 0)


def test_apply_cells_partition_sums_to_apply():
    """The cell-subset apply (used to time bounded samples) partitions A x."""
    for case in TINY:
        P = _prob(case)
        x = S.uniform_pm1(3, P.n_dofs)
        nc = len(P.mesh.cells)
        parts = np.array_split(np.arange(nc), 3)
        y = sum(P.apply_cells(x, c) for c in parts)
        np.testing.assert_allclose(y, P.apply(x), atol=1e-12 * np.abs(P.apply(x)).max())

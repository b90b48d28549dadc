"""Pins of the oracle's union-of-balls geometry (the multiple-ball benchmark,
Section 4.3): level set, closest point on the union's boundary.

The closest point is checked against brute force: a dense sampling of the
union's boundary (points of each sphere that no other ball contains) can
never be closer than the returned point, which itself must lie on the
boundary.  A single ball reduces to the ball kind."""
import numpy as np
import pytest

import synthetic as S
from oracle.geometry import LevelSet
from oracle.operator import Problem


def _sphere_samples(c, r, d, n):
    if d == 2:
        t = np.linspace(0, 2 * np.pi, n, endpoint=False)
        return c + r * np.stack([np.cos(t), np.sin(t)], axis=-1)
    k = int(np.sqrt(n))
    th = np.arccos(np.linspace(1, -1, k))
    ph = np.linspace(0, 2 * np.pi, 2 * k, endpoint=False)
    T, P = np.meshgrid(th, ph, indexing="ij")
    u = np.stack([np.sin(T) * np.cos(P), np.sin(T) * np.sin(P), np.cos(T)], axis=-1)
    return c + r * u.reshape(-1, 3)


def _boundary_samples(ls, n):
    pts = []
    for i in range(len(ls.br)):
        P = _sphere_samples(ls.bc[i], ls.br[i], ls.dim, n)
        keep = np.ones(len(P), dtype=bool)
        for j in range(len(ls.br)):
            if j != i:
                keep &= np.linalg.norm(P - ls.bc[j], axis=-1) >= ls.br[j]
        pts.append(P[keep])
    return np.concatenate(pts)


CONFIGS = [
    (2, [(-0.3, 0.0, 0.5), (0.3, 0.1, 0.45), (0.0, -0.4, 0.35)]),
    (3, [(-0.3, 0.0, 0.0, 0.5), (0.3, 0.1, 0.0, 0.45)]),
    (3, [(-0.3, 0.0, 0.0, 0.5), (0.3, 0.1, 0.0, 0.45), (0.0, -0.35, 0.2, 0.4)]),
]


@pytest.mark.parametrize("d,balls", CONFIGS)
def test_closest_point_beats_brute_force(d, balls):
    ls = LevelSet("balls", np.ravel(balls), d)
    samples = _boundary_samples(ls, 20000 if d == 2 else 160000)
    rng = np.random.default_rng(0)
    X = rng.uniform(-0.9, 0.9, size=(400, d))
    Y = ls.closest_point(X)
    # on the boundary: on one sphere, inside none
    assert np.all(np.abs(ls.phi(Y)) < 1e-12)
    dist = np.linalg.norm(Y - X, axis=-1)
    d2 = (X * X).sum(-1)[:, None] + (samples * samples).sum(-1)[None, :] - 2.0 * X @ samples.T
    brute = np.sqrt(np.maximum(d2.min(axis=1), 0.0))
    assert np.all(dist <= brute + 1e-7)
    # and the samples come close to it (the sampling resolves the boundary)
    assert np.max(brute - dist) < (0.05 if d == 3 else 0.005)


def test_single_ball_is_the_ball_kind():
    for d, g in ((2, (0.05, -0.03, 0.73)), (3, (0.02, 0.01, -0.03, 0.71))):
        a, b = LevelSet("ball", g, d), LevelSet("balls", g, d)
        X = np.random.default_rng(1).uniform(-1, 1, size=(500, d))
        np.testing.assert_array_equal(a.phi(X), b.phi(X))
        np.testing.assert_allclose(b.closest_point(X), a.closest_point(X), atol=1e-15)


def test_vertices_lie_on_three_spheres():
    ls = LevelSet("balls", np.ravel(CONFIGS[2][1]), 3)
    assert len(ls.vertices) > 0
    for v in ls.vertices:
        r = np.sort(np.abs(np.linalg.norm(v - ls.bc, axis=-1) - ls.br))
        assert r[2] < 1e-12                      # on (at least) three spheres
        assert np.all(np.linalg.norm(v - ls.bc, axis=-1) >= ls.br - 1e-12)


@pytest.mark.parametrize("d", [2, 3])
def test_multiple_balls_patch_test(d):
    """The surrogate operator on a union of balls reproduces Q_p polynomials
    (exact extension; g = u* at the returned boundary points)."""
    import scipy.sparse.linalg as spla
    w = S.multiple_balls(5, dim=d, cells=10 if d == 3 else 24, degree=2, seed=3)
    P = Problem.from_workload(w)
    assert np.all(np.abs(P.ls.phi(P.mesh.face_x.reshape(-1, d))) < 1e-12)
    u = lambda X: X[..., 0] ** 2 - 0.5 * X[..., 0] * X[..., 1] + X[..., -1]
    f = lambda X: -2.0 * np.ones(X.shape[:-1])
    uh = spla.spsolve(P.assemble().tocsc(), P.rhs(f, u))
    ref = P.interpolate(u)
    assert np.abs(uh - ref).max() < 1e-8 * max(1.0, np.abs(ref).max())

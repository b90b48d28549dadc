"""Seeded synthetic inputs for the shifted boundary method (SBM) operator.

This module is the one piece of code that both the CPU oracle checks and the
CUDA path's tests/benchmark use.  It holds input generation only -- a
counter-based random number generator, the distributions drawn from it, and
the descriptions of the workloads -- and none of the method's arithmetic
(no basis, quadrature, geometry projection or operator code).

Random stream (the paper names no generator; this is the convention used
throughout the repository):

* splitmix64, counter form: value k (k = 0, 1, ...) of stream ``seed`` is
  ``mix(seed + (k + 1) * 0x9E3779B97F4A7C15 mod 2**64)`` with the published
  splitmix64 finaliser (Steele, Lea, Flood, "Fast splittable pseudorandom
  number generators", OOPSLA 2014).
* U(-1, 1): ``u = (z >> 11) * 2**-53`` in [0, 1), value ``2u - 1``.
* N(0, 1): Box--Muller on consecutive pairs (u1, u2) of [0,1) uniforms,
  ``sqrt(-2 ln(1 - u1)) * cos(2 pi u2)`` (cosine branch only), with the C
  library's log1p and cos.
* The library exports the same generator (``sbm_fill_random``), bit for bit.
* Vectors are filled in the global DoF order of the problem they belong to.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Values ``offset .. offset+n-1`` of the counter-based splitmix64 stream."""
    k = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + k * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """[0, 1) doubles with 53 random bits each."""
    z = splitmix64(seed, n, offset)
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def uniform_pm1(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """U(-1, 1) input vector: values offset .. offset+n-1 of the stream."""
    return 2.0 * uniform01(seed, n, offset) - 1.0


# the C library's log1p and cos, element by element: numpy's vectorised
# versions differ from it (and between machines) in the last bit
_log1p = np.frompyfunc(math.log1p, 1, 1)
_cos = np.frompyfunc(math.cos, 1, 1)


def normal(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """N(0, 1) input vector of length n (Box--Muller, cosine branch): value
    j = offset + i from the uniform pair (u_2j, u_2j+1)."""
    u = uniform01(seed, 2 * n, 2 * offset).reshape(n, 2)
    lg = _log1p(-u[:, 0]).astype(np.float64)
    cs = _cos(2.0 * math.pi * u[:, 1]).astype(np.float64)
    return np.sqrt(-2.0 * lg) * cs


def random_vector(seed: int, n: int, dist: str) -> np.ndarray:
    if dist == "uniform":
        return uniform_pm1(seed, n)
    if dist == "normal":
        return normal(seed, n)
    raise ValueError(f"unknown distribution {dist!r}")


# --------------------------------------------------------------------------
# Workload descriptions
# --------------------------------------------------------------------------

BALL, ELLIPSOID, TORUS, BOX, BALLS = "ball", "ellipsoid", "torus", "box", "balls"


@dataclass(frozen=True)
class Workload:
    """One SBM problem: background mesh, degree, domain, variant and input.

    ``geom`` parameters by kind:
      ball:      centre (d values), radius
      ellipsoid: semi-axes (d values), rotation (row-major d*d, the matrix R
                 with x = R y, y in the ellipsoid's own frame), centre (d values)
      torus:     major radius R, minor radius r (axis z, centred at 0; d = 3)
      box:       centre (d values), half-widths (d values)
      balls:     union of balls: per ball its centre (d values) and radius
    """
    name: str
    dim: int
    degree: int
    cells: int                      # cells per side on [-1, 1]^d
    kind: str
    geom: tuple
    dg: bool = False
    seed: int = 0
    dist: str = "uniform"
    pen_shift: float = 10.0         # sigma = C p^2/h (CG) or C (p+1)^2/h (DG)
    pen_interior: float = 1.0       # DG interior faces: C (p+1)^2/h
    nrhs: int = 1
    extension: str = "exact"        # E u at x~: "exact" point evaluation, "taylor1"
    activity: str = "centre"        # active cells: "centre" inside, or "volume" fraction
    vf_threshold: float = 0.5       # volume fraction an active cell needs ("volume")

    def resized(self, cells: int, degree: int | None = None) -> "Workload":
        return replace(self, cells=cells,
                       degree=self.degree if degree is None else degree,
                       name=f"{self.name}@N{cells}")


def ball(dim, centre, radius):
    return BALL, tuple(centre) + (radius,)


def ellipsoid(axes, rot=None, centre=None):
    d = len(axes)
    if rot is None:
        rot = np.eye(d)
    if centre is None:
        centre = (0.0,) * d
    return ELLIPSOID, tuple(axes) + tuple(np.asarray(rot, float).ravel()) + tuple(centre)


def torus(R, r):
    return TORUS, (R, r)


def box(centre, half):
    return BOX, tuple(centre) + tuple(half)


def _wl(name, dim, degree, cells, geomspec, **kw):
    kind, geom = geomspec
    return Workload(name=name, dim=dim, degree=degree, cells=cells, kind=kind,
                    geom=tuple(float(g) for g in geom), **kw)


# The five workloads the operator is measured on.
DISK_2D_Q2 = _wl("disk2d_cg_q2_n32", 2, 2, 32, ball(2, (0.05, -0.03), 0.73), seed=0)
SPHERE_3D_Q4 = _wl("sphere3d_cg_q4_n96", 3, 4, 96, ball(3, (0.02, 0.01, -0.03), 0.71), seed=1)
ELLIPSOID_3D_Q6 = _wl("ellipsoid3d_cg_q6_n48", 3, 6, 48, ellipsoid((0.8, 0.6, 0.5)), seed=2)
TORUS_3D_DG_Q3 = _wl("torus3d_dg_q3_n64", 3, 3, 64, torus(0.6, 0.25), dg=True, seed=3,
                     dist="normal")

WORKLOADS = {w.name: w for w in (DISK_2D_Q2, SPHERE_3D_Q4, ELLIPSOID_3D_Q6, TORUS_3D_DG_Q3)}


def rotation_from_quaternion(q) -> np.ndarray:
    """Rotation matrix of the unit quaternion q/|q| = (w, x, y, z)."""
    w, x, y, z = np.asarray(q, float) / np.linalg.norm(q)
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
    ])


BATCH_SEED = 4
BATCH_GEOM_STREAM = BATCH_SEED + (1 << 32)   # separate stream for the geometry draws


def batched_ellipsoids(nprob: int = 64, nrhs: int = 8, seed: int = BATCH_SEED,
                       n_range=(16, 48), p_range=(2, 6)) -> list[Workload]:
    """Independent 3D CG problems on randomly rotated ellipsoids.

    Per problem, 9 draws from the geometry stream: N ~ U{n_range}, p ~ U{p_range},
    three semi-axes ~ U(0.4, 0.85), then 4 N(0,1) values (a Gaussian quaternion,
    normalised) for the rotation.  Input vector (problem k, right-hand side r)
    uses stream ``seed * 1000003 + k * 16 + r``.
    """
    gstream = seed + (1 << 32)
    out = []
    per = 5 + 8       # 5 uniforms + 4 normals (8 uniforms)
    u = uniform01(gstream, nprob * per).reshape(nprob, per)
    for k in range(nprob):
        uk = u[k]
        n = n_range[0] + int(uk[0] * (n_range[1] - n_range[0] + 1))
        p = p_range[0] + int(uk[1] * (p_range[1] - p_range[0] + 1))
        axes = tuple(0.4 + 0.45 * uk[2:5])
        pairs = uk[5:13].reshape(4, 2)
        q = np.sqrt(-2.0 * np.log1p(-pairs[:, 0])) * np.cos(2.0 * math.pi * pairs[:, 1])
        rot = rotation_from_quaternion(q)
        out.append(_wl(f"batch{k:02d}_q{p}_n{n}", 3, p, n, ellipsoid(axes, rot),
                       seed=seed * 1000003 + k * 16, nrhs=nrhs))
    return out


# Problems of batched_ellipsoids(nprob=24, n_range=(8, 14), p_range=(2, 3))
# whose SBM matrix has its spectrum in the open right half-plane and on which
# plain BiCGStab converges (eigenvalues of the oracle's assembled matrix and
# SciPy's BiCGStab; pinned in test_oracle_spectrum.py).  On these coarse
# meshes most p = 3 problems are indefinite (a few eigenvalues with negative
# real part), and one positive-real p = 3 problem (index 21) still makes
# BiCGStab diverge; only long-restart GMRES solves those.  The batched-solve
# comparisons use the rest.
SOLVE_BATCH = (1, 13, 15, 16, 17, 20, 23)


def solve_batch() -> list[Workload]:
    """The batched-solve workload: 7 problems (p = 2 or 3, 725 to 3 153 DoFs)."""
    ws = batched_ellipsoids(nprob=24, n_range=(8, 14), p_range=(2, 3))
    return [ws[i] for i in SOLVE_BATCH]


def rhs_seed(w: Workload, r: int) -> int:
    """Seed of right-hand side r of a workload (r = 0 is the workload's own seed)."""
    return w.seed + r


MULTIBALL_SEED = 5


def multiple_balls(nballs: int, dim: int = 3, cells: int = 64, degree: int = 3,
                   seed: int = MULTIBALL_SEED) -> Workload:
    """The multiple-ball geometric-complexity workload: the union of nballs
    random balls in [-1, 1]^dim (the paper's placements are not published).

    Geometry stream ``seed * 1000003 + nballs`` (uniforms, dim + 1 per ball):
    radius r_i = r0 (0.7 + 0.3 u_0) with r0 = 0.55 (3 / nballs)^(2/3): from
    three large balls to many small ones, whose boundary cells make up about
    half of the cut-or-active cells at 25 balls (the paper's range); centre
    coordinates uniform in [-1 + r_i + 2h, 1 - r_i - 2h] (h = 2 / cells), so
    every ball stays inside the box.  CG, x ~ U(-1, 1) from stream
    ``seed * 1000003 + nballs + 1000``.
    """
    per = dim + 1
    u = uniform01(seed * 1000003 + nballs, nballs * per).reshape(nballs, per)
    h = 2.0 / cells
    r0 = 0.55 * (3.0 / nballs) ** (2.0 / 3.0)
    geom = []
    for i in range(nballs):
        r = r0 * (0.7 + 0.3 * u[i, 0])
        lim = 1.0 - r - 2.0 * h
        geom += [-lim + 2.0 * lim * u[i, 1 + l] for l in range(dim)] + [r]
    return _wl(f"balls{nballs}_{dim}d_cg_q{degree}_n{cells}", dim, degree, cells,
               (BALLS, tuple(geom)), seed=seed * 1000003 + nballs + 1000)

"""The geometry stage of the set-up on the GPU (sbm_create_gpu) gives the
host set-up's problem bit for bit: active cells, surrogate faces, closest
points, DoF count, and therefore bitwise-equal applies."""
import dataclasses

import numpy as np
import pytest
import torch

import paper_2507_17053_gb300 as G
import synthetic as S

pytestmark = pytest.mark.gpu

CASES = [
    S.DISK_2D_Q2,
    S.SPHERE_3D_Q4,                                   # full size: 884,736 background cells
    S.ELLIPSOID_3D_Q6,
    S.TORUS_3D_DG_Q3,
    S._wl("box", 3, 2, 16, S.box((0.05, 0.0, -0.1), (0.5, 0.6, 0.45))),
    S.multiple_balls(25),
    S.multiple_balls(6, dim=2, cells=64, degree=2),
    dataclasses.replace(S.SPHERE_3D_Q4.resized(32), activity="volume", vf_threshold=0.3,
                        name="sphere_vf0.3"),
    dataclasses.replace(S.ELLIPSOID_3D_Q6.resized(16), extension="taylor1", name="ell_taylor1"),
] + S.batched_ellipsoids(nprob=3, n_range=(16, 24))


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


@pytest.mark.parametrize("w", CASES, ids=lambda w: w.name)
def test_gpu_setup_equals_host_setup(w):
    H = G.Problem.from_workload(w)
    D = G.Problem.from_workload(w, gpu_setup=True)
    assert (H.n_dofs, H.n_cells, H.n_sfaces, H.n_ifaces) == \
        (D.n_dofs, D.n_cells, D.n_sfaces, D.n_ifaces)
    for a, b in zip(H.geometry(), D.geometry()):
        np.testing.assert_array_equal(a, b)
    x = torch.from_numpy(S.random_vector(w.seed, H.n_dofs, w.dist)).cuda()
    assert torch.equal(H.apply_f64(x), D.apply_f64(x))


def test_gpu_setup_errors():
    d = G.make_desc(3, 2, 8, "ball", (5.0, 5.0, 5.0, 0.1))
    with pytest.raises(G.SbmError) as e:
        G.sbm_create_gpu(d, 0)
    assert G.STATUS[e.value.status] == "SBM_ERR_EMPTY_DOMAIN"
    with pytest.raises(G.SbmError) as e:
        G.sbm_create_gpu(G.make_desc(3, 2, 8, "ball", (0.0, 0.0, 0.0, 0.5)), -1)
    assert G.STATUS[e.value.status] == "SBM_ERR_ARG"

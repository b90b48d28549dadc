"""Geometry variants on the GPU: the multiple-ball geometry (union of balls,
Section 4.3) and the volume-fraction activity criterion.  FP64 apply parity
with the oracle (CG and DG, 2D and 3D, exact and first-order Taylor
extension) at 1e-12, and the FP32 apply within 1e-6."""
import dataclasses

import numpy as np
import pytest
import torch

import paper_2507_17053_gb300 as G
import synthetic as S
from oracle.operator import Problem as OracleProblem

pytestmark = pytest.mark.gpu

CASES = [
    S.multiple_balls(3, cells=16),
    S.multiple_balls(12, cells=20, degree=2),
    S.multiple_balls(25, cells=24, degree=4),
    S.multiple_balls(6, dim=2, cells=48, degree=3),
    dataclasses.replace(S.multiple_balls(10, cells=16, degree=3), dg=True, name="balls10_dg"),
    dataclasses.replace(S.multiple_balls(10, cells=16, degree=3), extension="taylor1",
                        name="balls10_taylor1"),
    # the volume-fraction activity criterion (surrogate faces on both sides of Gamma)
    dataclasses.replace(S.DISK_2D_Q2, activity="volume", vf_threshold=0.2, name="disk_vf0.2"),
    dataclasses.replace(S.SPHERE_3D_Q4.resized(12), activity="volume", vf_threshold=0.3,
                        name="sphere_vf0.3"),
    dataclasses.replace(S.multiple_balls(10, cells=16, degree=2), activity="volume",
                        vf_threshold=0.7, name="balls10_vf0.7"),
]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


@pytest.mark.parametrize("w", CASES, ids=lambda w: w.name)
def test_balls_apply_matches_oracle(w):
    O = OracleProblem.from_workload(w)
    P = G.Problem.from_workload(w)
    assert P.n_dofs == O.n_dofs
    x = S.random_vector(w.seed, O.n_dofs, w.dist)
    xd = torch.from_numpy(x).cuda()
    ref = O.apply(x)
    y = P.apply_f64(xd).cpu().numpy()
    assert np.abs(y - ref).max() <= 1e-12 * np.abs(ref).max()
    y32 = P.apply_f32(xd.float()).double().cpu().numpy()
    ref32 = O.apply(x.astype(np.float32).astype(np.float64))
    assert np.abs(y32 - ref32).max() <= 1e-6 * np.abs(ref32).max()

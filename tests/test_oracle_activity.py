"""Pins of the volume-fraction activity criterion (Section 2 cites it as an
alternative to "the centre is inside"): the midpoint rule on 8^d sub-cells.

An axis-aligned box whose faces sit a known fraction of a cell inside the
mesh planes gives closed-form fractions; a ball's fractions bracket the
centre criterion (threshold -> 0: every cut cell, -> 1: only cells inside)."""
import math

import numpy as np
import pytest

import synthetic as S
from oracle.geometry import LevelSet, Mesh


@pytest.mark.parametrize("d", [2, 3])
def test_box_volume_fractions_closed_form(d):
    """Box [-a, a]^d with a = 0.5 + 3h/8 on N = 8 (h = 1/4): the box covers
    the 4^d central cells fully and 3/8 of the next layer per axis, so a cell
    of the next layer has fraction (3/8)^k (k = axes in which it is in the
    outer layer) -- exactly representable by the 8-sub-cell midpoint rule."""
    N, h = 8, 0.25
    a = 0.5 + 3 * h / 8
    ls = LevelSet("box", (0.0,) * d + (a,) * d, d)
    for theta, k_max in ((0.3, 1), (0.1, 2), (0.05, 3), (0.5, 0), (1.0, 0)):
        M = Mesh(d, 1, N, ls, activity="volume", vf_threshold=theta)
        # cells with k outer-layer axes have fraction 0.375^k
        expected = sum(
            (4 ** (d - k)) * (2 ** k) * math.comb(d, k) for k in range(d + 1)
            if 0.375 ** k >= theta)
        assert len(M.cells) == expected, (theta, len(M.cells), expected)


def test_ball_thresholds_bracket_the_centre_rule():
    ls = LevelSet("ball", (0.05, -0.03, 0.0, 0.71), 3)
    centre = Mesh(3, 1, 16, ls)
    lo = Mesh(3, 1, 16, ls, activity="volume", vf_threshold=0.01)
    hi = Mesh(3, 1, 16, ls, activity="volume", vf_threshold=0.99)
    a_c, a_lo, a_hi = (set(map(tuple, m.cells)) for m in (centre, lo, hi))
    assert a_hi < a_c < a_lo                   # strict inclusions
    # every cell entirely inside (all 8 corners inside) is active at 0.99
    N, h = 16, 0.125
    for idx in a_c - a_hi:
        corners = -1.0 + h * (np.array(idx) + np.indices((2, 2, 2)).reshape(3, -1).T)
        assert ls.phi(corners).max() > -1e-3 * h   # such a cell touches the boundary


def test_volume_fraction_workload_sizes():
    w = S.DISK_2D_Q2
    from oracle.operator import Problem
    import dataclasses
    c = Problem.from_workload(w)
    v = Problem.from_workload(dataclasses.replace(w, activity="volume", vf_threshold=0.5))
    # the 0.5 volume rule and the centre rule agree except for a few cut cells
    sc, sv = set(map(tuple, c.mesh.cells)), set(map(tuple, v.mesh.cells))
    assert len(sc ^ sv) <= 0.05 * len(sc)

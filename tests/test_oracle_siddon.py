"""Pins of the oracle's Siddon system matrix against geometry it does not use.

Sec. 2 Eq. 1 defines a_ij as the contribution of ray i to pixel j; the build
takes it to be the exact length of ray i inside pixel j.  Each pin below is an
independent computation: a Liang-Barsky clip of the line against the whole
square (chord length), a clip against every single pixel square (brute force),
exact axis-aligned views, and hand-derived values on a 2x2 grid.
"""
import math
import os

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def clip_length(c, s, t, lo_x, hi_x, lo_y, hi_y):
    """Length of the line {t*(c,s) + u*(-s,c)} inside the box (Liang-Barsky)."""
    x0, y0, dx, dy = t * c, t * s, -s, c
    u0, u1 = -math.inf, math.inf
    for p0, d, lo, hi in ((x0, dx, lo_x, hi_x), (y0, dy, lo_y, hi_y)):
        if d == 0.0:
            if not (lo < p0 < hi):
                return 0.0
            continue
        a, b = (lo - p0) / d, (hi - p0) / d
        u0, u1 = max(u0, min(a, b)), min(u1, max(a, b))
    return max(0.0, u1 - u0)


def test_golden_2x2(oracle_mod):
    O = oracle_mod
    g = O.Geometry(2, 1, 1)
    for line in open(os.path.join(HERE, "golden", "siddon_2x2.txt")):
        if line.startswith("#") or not line.strip():
            continue
        head, tail = line.split("|")
        th, t = (float(v) for v in head.split())
        want = tail.split()
        c, s = {0.0: (1.0, 0.0), 90.0: (0.0, 1.0)}.get(th, (math.cos(math.radians(th)),
                                                           math.sin(math.radians(th))))
        pix, ln = O.siddon_ray(g, c, s, t)
        assert list(pix) == [int(v) for v in want[0::2]]
        np.testing.assert_allclose(ln, [float(v) for v in want[1::2]], rtol=1e-15, atol=1e-15)


@pytest.mark.parametrize("n_side,n_views,n_bins", [(32, 60, 46), (17, 23, 29), (64, 90, 92)])
def test_row_sums_equal_chord_length(oracle_mod, n_side, n_views, n_bins):
    O = oracle_mod
    g = O.Geometry(n_side, n_views, n_bins)
    csr = O.siddon_csr(g)
    cs = O.view_table(g)
    h = n_side / 2.0
    rows = np.zeros(g.m)
    for i in range(g.m):
        rows[i] = sum(csr.val[csr.row_ptr[i]:csr.row_ptr[i + 1]])
    for i in range(g.m):
        v, d = divmod(i, n_bins)
        t = (d - 0.5 * (n_bins - 1)) * 1.0
        want = clip_length(cs[v, 0], cs[v, 1], t, -h, h, -h, h)
        assert abs(rows[i] - want) <= 1e-13 * max(1.0, want), (i, rows[i], want)


def test_random_rays_match_per_pixel_clip(oracle_mod):
    """Brute force: clip the ray against each of the n_side^2 pixel squares."""
    O = oracle_mod
    n_side = 12
    g = O.Geometry(n_side, 1, 1)
    rng = np.random.default_rng(7)
    h = n_side / 2.0
    for _ in range(200):
        th = rng.uniform(0, math.pi)
        c, s = math.cos(th), math.sin(th)
        t = rng.uniform(-h * 1.5, h * 1.5)
        pix, ln = O.siddon_ray(g, c, s, t)
        dense = np.zeros(n_side * n_side)
        np.add.at(dense, pix, ln)
        brute = np.zeros(n_side * n_side)
        for iy in range(n_side):
            for ix in range(n_side):
                brute[iy * n_side + ix] = clip_length(c, s, t, -h + ix, -h + ix + 1,
                                                      -h + iy, -h + iy + 1)
        np.testing.assert_allclose(dense, brute, rtol=0, atol=1e-11)


@pytest.mark.parametrize("n_side,n_views,n_bins", [(32, 60, 46), (128, 180, 182)])
def test_axis_views_have_unit_column_sums(oracle_mod, n_side, n_views, n_bins):
    """At 0 and 90 degrees each pixel is crossed by exactly one ray through its
    centre (even n_side, even n_bins, unit bins), with length exactly 1."""
    O = oracle_mod
    g = O.Geometry(n_side, n_views, n_bins)
    csr = O.siddon_csr(g)
    A = csr.to_scipy()
    for v in (0, n_views // 2):
        block = A[v * n_bins:(v + 1) * n_bins]
        sums = np.asarray(block.sum(axis=0)).ravel()
        assert np.all(sums == 1.0)
        assert block.nnz == n_side * n_side


def test_view_table_axis_exact(oracle_mod):
    O = oracle_mod
    cs = O.view_table(O.Geometry(8, 60, 8))
    assert tuple(cs[0]) == (1.0, 0.0)
    assert tuple(cs[30]) == (0.0, 1.0)
    np.testing.assert_allclose(np.hypot(cs[:, 0], cs[:, 1]), 1.0, rtol=0, atol=2e-16)


def test_nnz_bound_and_indices(oracle_mod):
    O = oracle_mod
    g = O.Geometry(32, 60, 46)
    csr = O.siddon_csr(g)
    per_row = np.diff(csr.row_ptr)
    assert per_row.max() <= 2 * g.n_side - 1
    assert csr.col_idx.min() >= 0 and csr.col_idx.max() < g.n
    assert np.all(csr.val > 1e-12)


def test_dense_has_lambda_rows(oracle_mod):
    O = oracle_mod
    g = O.Geometry(16, 20, 24, sqrt_lambda=0.05)
    A = O.dense_system(g)
    assert A.shape == (g.m + g.n, g.n)
    np.testing.assert_array_equal(A[g.m:], 0.05 * np.eye(g.n))

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


# ---- fan-beam geometry (the paper's scanner, Sec. 3.1 / 3.2 tables) ----------

FAN = [(16, 24, 21, 30.0, 40.0), (24, 36, 33, 25.0, 60.0)]  # n_side, views, dets, fan, source


@pytest.mark.parametrize("n_side,n_views,n_det,fan,sid", FAN)
def test_fan_rays_pass_through_their_source(oracle_mod, n_side, n_views, n_det, fan, sid):
    """Every ray of view v contains the source point S_v = sid (cos b, sin b),
    the central detector's ray contains the rotation axis, and the rays of a
    view span the fan angle."""
    O = oracle_mod
    g = O.Geometry(n_side, n_views, n_det, arc_deg=360.0, kind="fan", source_dist=sid, fan_deg=fan)
    r = O.fan_rays(g).reshape(n_views, n_det, 3)
    for v in range(n_views):
        b = math.radians(v * 360.0 / n_views)
        S = (sid * math.cos(b), sid * math.sin(b))
        dist = S[0] * r[v, :, 0] + S[1] * r[v, :, 1] - r[v, :, 2]
        assert np.abs(dist).max() <= 1e-12 * sid
        assert r[v, (n_det - 1) // 2, 2] == 0.0  # odd detector count: central ray
        # directions (-s, c) of the extreme rays make the fan angle
        d0 = np.array([-r[v, 0, 1], r[v, 0, 0]])
        d1 = np.array([-r[v, -1, 1], r[v, -1, 0]])
        ang = math.degrees(math.acos(max(-1.0, min(1.0, float(d0 @ d1)))))
        assert abs(ang - fan) <= 1e-9
        # and the central ray points from the source through the axis
        dc = np.array([-r[v, (n_det - 1) // 2, 1], r[v, (n_det - 1) // 2, 0]])
        assert dc @ np.array([-math.cos(b), -math.sin(b)]) > 1 - 1e-12


@pytest.mark.parametrize("n_side,n_views,n_det,fan,sid", FAN)
def test_fan_row_sums_equal_chord_length(oracle_mod, n_side, n_views, n_det, fan, sid):
    O = oracle_mod
    g = O.Geometry(n_side, n_views, n_det, arc_deg=360.0, kind="fan", source_dist=sid, fan_deg=fan)
    csr = O.siddon_csr(g)
    rays = O.fan_rays(g)
    h = n_side / 2.0
    for i in range(g.m):
        got = float(np.sum(csr.val[csr.row_ptr[i]:csr.row_ptr[i + 1]]))
        want = clip_length(rays[i, 0], rays[i, 1], rays[i, 2], -h, h, -h, h)
        assert abs(got - want) <= 1e-13 * max(1.0, want), (i, got, want)


def test_fan_beam_tends_to_parallel_beam(oracle_mod):
    """A far source with a narrow fan (detector spacing 1 at the axis) gives
    nearly parallel rays: view v, detector d of the fan matches the parallel
    view a quarter turn later, detector n-1-d (orientation and sign pin).  An
    even detector count puts the rays through pixel centres, away from the
    grid lines where a tilt of 1e-6 would move a whole segment across."""
    O = oracle_mod
    n_side, n_views, n_det = 16, 24, 22
    sid = 1e7
    fan = math.degrees((n_det - 1) * 1.0 / sid)
    gf = O.Geometry(n_side, n_views, n_det, arc_deg=360.0, kind="fan", source_dist=sid, fan_deg=fan)
    gp = O.Geometry(n_side, n_views, n_det, arc_deg=360.0)
    Af = O.dense_system(gf).reshape(n_views, n_det, -1)
    Ap = O.dense_system(gp).reshape(n_views, n_det, -1)
    q = n_views // 4
    for v in range(n_views):
        np.testing.assert_allclose(Af[v], Ap[(v + q) % n_views][::-1], rtol=0, atol=1e-4)


# ---- Joseph's projector (the paper's matrices, Sec. 3.1) ----------------------

def test_joseph_hand_cases(oracle_mod):
    """Hand-derived entries on a 4x4 grid (pixels 0..15, row-major from the
    bottom-left, unit pixels): a horizontal ray along the centre of row 2 has
    weight 1 in each of its pixels; a vertical ray at x = 0.25 (fractional
    column position 1.75) splits 1/4 : 3/4 between columns 1 and 2 of every
    row; the 45-degree ray through the origin meets row centres at pixel
    centres, weight sqrt(2) each."""
    O = oracle_mod
    g = O.Geometry(4, 1, 1, projector="joseph")
    pix, val = O.joseph_ray(g, 0.0, 1.0, 0.5)
    assert list(pix) == [8, 9, 10, 11] and np.all(val == 1.0)
    pix, val = O.joseph_ray(g, 1.0, 0.0, 0.25)
    assert list(pix) == [1, 2, 5, 6, 9, 10, 13, 14]
    np.testing.assert_array_equal(val, [0.25, 0.75] * 4)
    r = math.sqrt(0.5)
    pix, val = O.joseph_ray(g, r, r, 0.0)
    big = val > 1e-12
    assert list(pix[big]) == [3, 6, 9, 12]
    np.testing.assert_allclose(val[big], math.sqrt(2.0), rtol=1e-15)


def test_joseph_integrates_linear_images_exactly(oracle_mod):
    """Linear interpolation reproduces a linear image exactly, and the row
    sampling is the midpoint rule along the ray, exact for linear functions:
    for rays whose sampled positions keep both neighbours inside the grid,
    sum_j a_ij f(centre_j) = the integral of f along the ray across the grid's
    sampled strip.  With f = 1 this is the row-sum (strip length) invariant."""
    O = oracle_mod
    n = 24
    g = O.Geometry(n, 1, 1, projector="joseph")
    h = n / 2.0
    ys, xs = np.divmod(np.arange(n * n), n)
    cx, cy = xs - h + 0.5, ys - h + 0.5
    rng = np.random.default_rng(3)
    al, be, ga = 0.3, -0.7, 1.9
    f = al + be * cx + ga * cy
    checked = 0
    for _ in range(300):
        th = rng.uniform(0, math.pi)
        c, s = math.cos(th), math.sin(th)
        t = rng.uniform(-4.0, 4.0)
        pix, val = O.joseph_ray(g, c, s, t)
        rows = abs(c) >= abs(s)
        # sampled positions across the stepping lines must stay within [centre 0, centre n-1]
        q = (np.arange(n) + 0.5) - h
        p = (t * c - s * (q - t * s) / c) if rows else (t * s + c * (t * c - q) / s)
        if not np.all((p >= -h + 0.5) & (p <= h - 0.5)):
            continue
        checked += 1
        L = 1.0 / (abs(c) if rows else abs(s))
        # integral of f along the ray over the strip: parametrise by the stepping coordinate
        pts_x = p if rows else q
        pts_y = q if rows else p
        want = L * np.sum(al + be * pts_x + ga * pts_y)  # midpoint rule, exact for linear f
        got = float(np.dot(val, f[pix]))
        assert abs(got - want) <= 1e-11 * max(1.0, abs(want))
        assert abs(val.sum() - n * L) <= 1e-12 * n * L
    assert checked > 50


def test_joseph_same_line_same_row(oracle_mod):
    O = oracle_mod
    g = O.Geometry(16, 1, 1, projector="joseph")
    rng = np.random.default_rng(5)
    for _ in range(50):
        th = rng.uniform(0, math.pi)
        c, s, t = math.cos(th), math.sin(th), rng.uniform(-9, 9)
        a = dict(zip(*O.joseph_ray(g, c, s, t)))
        b = dict(zip(*O.joseph_ray(g, -c, -s, -t)))
        assert set(a) == set(b)
        for k in a:
            assert abs(a[k] - b[k]) <= 1e-12


@pytest.mark.parametrize("n_side,n_views,n_bins", [(32, 60, 46), (16, 24, 20)])
def test_joseph_axis_views_equal_siddon(oracle_mod, n_side, n_views, n_bins):
    """At 0 and 90 degrees every ray runs along a pixel row (column) through
    the pixel centres, where both projectors are exact: Joseph's weight and
    Siddon's length are 1 in each pixel the ray crosses, so the two system
    matrices agree on those views entry for entry (and differ elsewhere)."""
    O = oracle_mod
    As = O.dense_system(O.Geometry(n_side, n_views, n_bins))
    Aj = O.dense_system(O.Geometry(n_side, n_views, n_bins, projector="joseph"))
    for v in (0, n_views // 2):
        rows = slice(v * n_bins, (v + 1) * n_bins)
        np.testing.assert_array_equal(Aj[rows], As[rows])
        assert np.count_nonzero(Aj[rows]) == n_side * n_side
    assert not np.array_equal(Aj, As)

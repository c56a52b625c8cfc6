"""Pins of the oracle's oblique-view sampling (CPU only).

The view geometry (orthographic rays along d(theta, phi), pixel axes e_theta and
e_phi about the box centre, the chord through the box split into
K = ceil(chord / dx) equal steps sampled at their midpoints) and the
trilinear interpolation of cell-centred values with indices clamped at the
faces are the readings the library takes of the ray-aligned geometry of
Sec. 2.2 for views that are not cell aligned.

Trilinear interpolation reproduces exactly every function in the span of
{1, x, y, z, xy, yz, zx, xyz}.  Each field here is such a function with its
own coefficients on every axis and every cross term, sampled at the cell
centres; so at a sample inside the lattice of cell centres the oracle must
return the function itself at the sample position, and within half a cell of
a face (where the index clamp acts) the function at the position clamped to
the outermost cell centres.  The expected positions come from the geometry
above evaluated here independently (slab method for the chord), so a weight
applied to the wrong axis, a swapped w / 1 - w, a half-cell offset of the
positions, a wrong chord or a wrong clamp each fail a test.
"""
from __future__ import annotations

import math

import numpy as np
import pytest

import oracle
from synth import View


def _poly_fields(n, dx, seed):
    """Five fields, each a random member of span{1, x, y, z, xy, yz, zx, xyz}
    (coordinates in cm), at the cell centres of an n^3 grid; returns the
    fields [z][y][x] and the exact functions."""
    rng = np.random.default_rng(seed)
    L = n * dx
    coeffs = rng.uniform(-1.0, 1.0, size=(5, 8))
    coeffs[:, 0] += 3.0   # keep values away from zero for a relative check

    def fn(q, x, y, z):
        a = coeffs[q]
        u, v, w = x / L, y / L, z / L
        return (a[0] + a[1] * u + a[2] * v + a[3] * w + a[4] * u * v + a[5] * v * w
                + a[6] * w * u + a[7] * u * v * w)

    c = (np.arange(n) + 0.5) * dx
    zz, yy, xx = np.meshgrid(c, c, c, indexing="ij")
    fields = tuple(np.ascontiguousarray(fn(q, xx, yy, zz)) for q in range(5))
    return fields, fn


def _expected_geometry(n, dx, view, px, py):
    """Direction, origin and chord of pixel (px, py) from the view definition."""
    th, ph = view.theta_rad, view.phi_rad
    d = np.array([math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), math.cos(th)])
    et = np.array([math.cos(th) * math.cos(ph), math.cos(th) * math.sin(ph), -math.sin(th)])
    ep = np.array([-math.sin(ph), math.cos(ph), 0.0])
    L = n * dx
    o = (np.full(3, 0.5 * L) + (px - 0.5 * (view.npx - 1)) * view.pixel_cm * et
         + (py - 0.5 * (view.npy - 1)) * view.pixel_cm * ep)
    t_in, t_out = -math.inf, math.inf
    for a in range(3):
        if abs(d[a]) < 1e-300:
            if not (0.0 <= o[a] <= L):
                return d, o, None
            continue
        t0, t1 = (0.0 - o[a]) / d[a], (L - o[a]) / d[a]
        t_in, t_out = max(t_in, min(t0, t1)), min(t_out, max(t0, t1))
    if not t_out > t_in:
        return d, o, None
    return d, o, (t_in, t_out)


def _check_ray(fields, fn, n, dx, view, px, py):
    smp, h = oracle.ray_samples(fields, dx, view, px, py)
    d, o, ch = _expected_geometry(n, dx, view, px, py)
    if ch is None:
        assert len(smp) == 0
        return 0, 0
    t_in, t_out = ch
    K = math.ceil((t_out - t_in) / dx - 1e-9)
    assert len(smp) == K
    assert h == pytest.approx((t_out - t_in) / K, rel=1e-13)
    lo, hi = 0.5 * dx, (n - 0.5) * dx
    clamped = 0
    for k in range(K):
        r = o + (t_in + (k + 0.5) * h) * d
        rc = np.clip(r, lo, hi)
        clamped += int(np.any(rc != r))
        want = [fn(q, *rc) for q in range(5)]
        np.testing.assert_allclose(smp[k], want, rtol=1e-12, atol=0.0,
                                   err_msg=f"pixel ({px},{py}) sample {k}")
    return K, clamped


@pytest.mark.parametrize("theta_deg,phi_deg", [(30.0, 45.0), (70.0, 200.0), (53.0, 301.0),
                                               (90.0, 17.0), (12.0, 0.0)])
def test_oblique_samples_reproduce_trilinear_polynomials(theta_deg, phi_deg):
    n, dx = 7, 3.0856775814913673e17
    fields, fn = _poly_fields(n, dx, seed=int(theta_deg * 7 + phi_deg))
    view = View(math.radians(theta_deg), math.radians(phi_deg), 9, 8, 0.83 * dx, 1)
    total = clamped = 0
    for py in range(view.npy):
        for px in range(view.npx):
            k, c = _check_ray(fields, fn, n, dx, view, px, py)
            total += k
            clamped += c
    # the lattice interior and the half-cell shells at the faces both occur
    assert total > 100 and 0 < clamped < total


def test_clamped_face_sample_reads_edge_extension():
    """A sample within half a cell of the x = 0 face reads the edge cell's
    value along x: a field that varies only in x returns the first cell's
    value there, and the exact line in the interior."""
    n, dx = 5, 1.0
    c = (np.arange(n) + 0.5) * dx
    gx = np.broadcast_to(2.0 + 0.7 * c[None, None, :], (n, n, n)).copy()
    ones = np.ones((n, n, n))
    fields = (gx, ones, ones, ones, ones)
    # theta = 90 deg, phi = 0: rays along +x through the box at y, z of pixel
    view = View(math.pi / 2, 0.0, n, n, dx, 1)
    smp, h = oracle.ray_samples(fields, dx, view, 2, 2)
    assert len(smp) == n and h == pytest.approx(dx, rel=1e-14)
    # samples at the cell centres x = (k + 1/2) dx: every one on a lattice point
    np.testing.assert_allclose(smp[:, 0], 2.0 + 0.7 * c, rtol=1e-14)
    # a slanted ray enters through the x = 0 face: its first sample sits less
    # than half a cell inside that face, where the clamp holds x at dx / 2
    view2 = View(math.radians(80.0), math.radians(10.0), n, n, dx, 1)
    d, o, ch = _expected_geometry(n, dx, view2, 2, 2)
    smp2, h2 = oracle.ray_samples(fields, dx, view2, 2, 2)
    r0 = o + (ch[0] + 0.5 * h2) * d
    assert r0[0] < 0.5 * dx
    assert smp2[0, 0] == pytest.approx(2.0 + 0.7 * 0.5 * dx, rel=1e-14)
    r1 = o + (ch[0] + 1.5 * h2) * d
    assert 0.5 * dx < r1[0] < (n - 0.5) * dx
    assert smp2[1, 0] == pytest.approx(2.0 + 0.7 * r1[0], rel=1e-13)


def test_central_ray_chord_length():
    """The ray through the box centre crosses the cube over L / max_a |d_a|."""
    n, dx = 8, 1.0
    fields = tuple(np.ones((n, n, n)) for _ in range(5))
    for th, ph in [(30.0, 45.0), (70.0, 200.0), (45.0, 45.0)]:
        view = View(math.radians(th), math.radians(ph), 3, 3, dx, 1)
        d, _, _ = _expected_geometry(n, dx, view, 1, 1)
        smp, h = oracle.ray_samples(fields, dx, view, 1, 1)
        chord = n * dx / np.abs(d).max()
        assert len(smp) * h == pytest.approx(chord, rel=1e-13)
        assert len(smp) == math.ceil(chord / dx - 1e-9)


def test_radial_view_reads_the_column_from_the_far_end():
    """The radial view of an [r][b][l] tensor (view.trilinear = 2) samples the
    column (l, b) = (x, y) from r = nz - 1 down to r = 0 (the observer), one
    sample per cell at step dx; it equals the z view of the r-reversed
    tensor."""
    n, dx = 5, 2.0
    rng = np.random.default_rng(3)
    fields = tuple(rng.uniform(1.0, 2.0, (n + 2, n, n + 1)) for _ in range(5))
    view = View(0.0, 0.0, n + 1, n, dx, 2)
    smp, h = oracle.ray_samples(fields, dx, view, 3, 1)
    assert h == dx and len(smp) == n + 2
    for q in range(5):
        np.testing.assert_array_equal(smp[:, q], fields[q][::-1, 1, 3])
    flipped = tuple(np.ascontiguousarray(f[::-1]) for f in fields)
    smp_z, _ = oracle.ray_samples(flipped, dx, View(0.0, 0.0, n + 1, n, dx, 0), 3, 1)
    np.testing.assert_array_equal(smp, smp_z)

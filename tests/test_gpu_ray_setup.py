"""Sample counts of the float kernels' ray set-up against the FP64 oracle.

The float kernels place the samples of an oblique ray with float-float
arithmetic (no double precision on the GPU): the chord through the box, the
count K = ceil(chord / dx - 1e-9) and the step h = chord / K (the oblique
geometry of the orthographic view, Sec. 2.2).  A wrong K on any ray changes
the whole ray, so the total over an image must equal the oracle's total
exactly.  The images are larger than the box's footprint (rays that miss) on
a box with three different sides, at generic angles and at angles where an
axis of the direction is zero or nearly zero (cos 90 deg ~ 6e-17).
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from synth import DUST, LINE_13CO_21, VelocityAxis, View, make_fields  # noqa: E402

PC = 3.0856775814913673e18


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2607_01338_b300  # noqa: F401


ANGLES = [(30.0, 45.0), (70.0, 200.0), (90.0, 0.0), (90.0, 45.0), (45.0, 90.0),
          (0.01, 10.0), (135.0, 300.0), (180.0, 0.0)]


def _count(theta, phi, shape, npx, npy, pitch):
    """(GPU stats, oracle total, oracle rays that hit) for one view."""
    import paper_2607_01338_b300 as irt
    from paper_2607_01338_b300 import binding as B
    nz, ny, nx = shape
    dx = 0.1 * PC
    fs = make_fields(64, seed=3)
    # a non-cubic box cut from the cube
    sub = [np.ascontiguousarray(a[:nz, :ny, :nx]) for a in fs.as_tuple()]
    f32 = [a.astype(np.float32) for a in sub]
    deq = [a.astype(np.float64) for a in f32]
    view = View(math.radians(theta), math.radians(phi), npx, npy, pitch * dx, 1)
    va = VelocityAxis(4, -4.0, 2.0, 1)
    g = irt.Grid(*[torch.from_numpy(a).cuda() for a in f32], dx)
    B.irt_grid_stats(g.handle, reset=True)
    irt.forward(g, view, va, LINE_13CO_21, DUST, components=("L",), flags=B.IRT_FLAG_STATS)
    torch.cuda.synchronize()
    st = B.irt_grid_stats(g.handle, reset=True)
    g.close()
    total = hit = 0
    for py in range(npy):
        for px in range(npx):
            smp, _ = oracle.ray_samples(deq, dx, view, px, py)
            total += len(smp)
            hit += len(smp) > 0
    return st, total, hit


@pytest.mark.parametrize("theta,phi,shape,npx,npy,pitch", [
    (60.0, 10.0, (13, 90, 5), 120, 96, 0.35),     # thin slab, fine pixels
    (90.0, 90.0, (20, 8, 32), 40, 30, 1.7),       # d = (~0, 1, ~6e-17), coarse pixels
    (1.0e-4, 33.0, (24, 20, 22), 30, 28, 1.0),    # nearly the z axis: chords within 2e-11 cells of nz
])
def test_sample_count_on_slabs_and_near_axis_views(theta, phi, shape, npx, npy, pitch):
    st, total, hit = _count(theta, phi, shape, npx, npy, pitch)
    assert hit > 0
    assert st["items"] == npx * npy
    assert st["samples"] == total, (st["samples"], total)


@pytest.mark.parametrize("theta,phi", ANGLES)
def test_oblique_sample_count_matches_oracle(theta, phi):
    import paper_2607_01338_b300 as irt
    from paper_2607_01338_b300 import binding as B
    nx, ny, nz = 40, 48, 56
    dx = 0.1 * PC
    fs = make_fields(64, seed=3)
    # a non-cubic box cut from the cube
    sub = [np.ascontiguousarray(a[:nz, :ny, :nx]) for a in fs.as_tuple()]
    f32 = [a.astype(np.float32) for a in sub]
    deq = [a.astype(np.float64) for a in f32]
    npx = npy = 80
    view = View(math.radians(theta), math.radians(phi), npx, npy, 0.93 * dx, 1)
    va = VelocityAxis(4, -4.0, 2.0, 1)
    g = irt.Grid(*[torch.from_numpy(a).cuda() for a in f32], dx)
    B.irt_grid_stats(g.handle, reset=True)
    irt.forward(g, view, va, LINE_13CO_21, DUST, components=("L",), flags=B.IRT_FLAG_STATS)
    torch.cuda.synchronize()
    st = B.irt_grid_stats(g.handle, reset=True)
    g.close()
    total = 0
    hit = 0
    for py in range(npy):
        for px in range(npx):
            smp, _ = oracle.ray_samples(deq, dx, view, px, py)
            total += len(smp)
            hit += len(smp) > 0
    assert hit > 0 and hit < npx * npy, "the image should hold both hits and misses"
    assert st["items"] == npx * npy
    assert st["samples"] == total, (st["samples"], total)

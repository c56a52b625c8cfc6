"""The adjoint beyond the z-view fast sweep: oblique views (the fast sweep
for smooth integration, the general sweep otherwise), and the general reverse
sweep (every velocity explicit) for the formal and Kahan-compensated formal
integrators, f = 0, several channel windows, and the smooth z-view rays the
fast sweep hands over (dust optically thick per step, line windows wider
than two slots).  Gradients of
Loss = mean(([L] - target)^2) against the FP64 oracle's dual-number
gradients, 1e-3 relative per cell with an absolute floor at the float32
rounding of the K-step recurrences (K 2^-24 of the largest gradient)."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from synth import (DUST, LINE_13CO_21, FieldSet, VelocityAxis, View, make_fields,  # noqa: E402
                   to_storage)

LINE = dict(LINE_13CO_21)
PC = 3.0856775814913673e18
RTOL = 1e-3


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2607_01338_b300  # noqa: F401


def _cmp(got, ref, K):
    allow = RTOL * np.abs(ref) + K * 2.0 ** -24 * np.abs(ref).max()
    return float((np.abs(got - ref) / allow).max())


def _gpu(f32, dx, view, va, target, integration, dust=DUST):
    import paper_2607_01338_b300 as irt
    g = irt.Grid(*[torch.from_numpy(a).cuda() for a in f32.as_tuple()], dx)
    L = irt.forward(g, view, va, LINE, dust, integration=integration)["L"]
    tgt = torch.from_numpy(target.astype(np.float32)).cuda()
    gL = 2.0 * (L - tgt) / L.numel()
    grads = irt.adjoint(g, view, va, LINE, dust, {"L": gL}, integration=integration)
    torch.cuda.synchronize()
    out = [x.double().cpu().numpy() for x in grads]
    g.close()
    for a in out:
        assert np.isfinite(a).all()
    return out


MODE = {"smooth": oracle.SMOOTH, "formal": oracle.FORMAL, "formal_kahan": oracle.FORMAL}


@pytest.mark.parametrize("integration", ["smooth", "formal"])
def test_oblique_view_gradient(integration):
    n = 12
    fs = make_fields(n, 61)
    f32, deq = to_storage(fs, np.float32)
    tf32, tdeq = to_storage(make_fields(n, 68), np.float32)
    dx = 0.1 * PC
    view = View(math.radians(30), math.radians(45), 14, 13, 0.9 * dx, 1)
    va = VelocityAxis(48, -72.0, 3.0, 1)
    target = oracle.render_cube(tdeq.as_tuple(), dx, LINE, DUST, view, va,
                                integration=MODE[integration])["L"]
    gn, gt, gv = _gpu(f32, dx, view, va, target, integration)
    rng = np.random.default_rng(7)
    cells = np.stack([rng.integers(0, n, 48), rng.integers(0, n, 48), rng.integers(0, n, 48)],
                     axis=1)
    loss, on, ot, ov = oracle.loss_grad_cells(deq.as_tuple(), dx, LINE, DUST, view, va, target,
                                              cells, integration=MODE[integration])
    got = {k: np.array([a[z, y, x] for x, y, z in cells]) for k, a in (("n", gn), ("T", gt),
                                                                        ("v", gv))}
    K = 2 * n   # longest chord in samples
    r = {"n": _cmp(got["n"], on, K), "T": _cmp(got["T"], ot, K), "v": _cmp(got["v"], ov, K)}
    assert all(v <= 1.0 for v in r.values()), r
    # the gradient reaches cells of many rays: the stencils overlap
    assert np.count_nonzero(gn) > n * n


def test_oblique_fast_sweep_all_passes():
    """Smooth oblique rays go through the fast sweep (4, 9 and full-width
    register passes by hull width, records and positions per ray); f = 2 and a
    13-block fine axis give hulls of every width."""
    n = 24
    fs = make_fields(n, 81)
    f32, deq = to_storage(fs, np.float32)
    tf32, tdeq = to_storage(make_fields(n, 88), np.float32)
    dx = 0.1 * PC
    view = View(math.radians(70), math.radians(200), 30, 28, 0.8 * dx, 1)
    va = VelocityAxis(96, -72.0, 1.5, 2)
    target = oracle.render_cube(tdeq.as_tuple(), dx, LINE, DUST, view, va,
                                integration=oracle.SMOOTH)["L"]
    gn, gt, gv = _gpu(f32, dx, view, va, target, "smooth")
    rng = np.random.default_rng(17)
    cells = np.stack([rng.integers(0, n, 40), rng.integers(0, n, 40), rng.integers(0, n, 40)],
                     axis=1)
    loss, on, ot, ov = oracle.loss_grad_cells(deq.as_tuple(), dx, LINE, DUST, view, va, target,
                                              cells, integration=oracle.SMOOTH)
    got = {k: np.array([a[z, y, x] for x, y, z in cells]) for k, a in (("n", gn), ("T", gt),
                                                                        ("v", gv))}
    K = 2 * n
    r = {"n": _cmp(got["n"], on, K), "T": _cmp(got["T"], ot, K), "v": _cmp(got["v"], ov, K)}
    assert all(v <= 1.0 for v in r.values()), r
    assert np.count_nonzero(on) > 20


def test_oblique_fast_sweep_16bit_fields():
    """The 16-bit storage instance of the oblique fast sweep: BF16 fields with
    an FP16 velocity and per-field scales (the batch workload's storage),
    against the oracle gradient on the dequantised values."""
    import paper_2607_01338_b300 as irt
    n = 16
    scales = [1.0e4, 1.0, 1.0, 1.0, 1.0e-6]
    fs = make_fields(n, 91)
    h16, deq = to_storage(fs, ["bf16", "bf16", "bf16", np.float16, "bf16"], scales=scales)
    tfs = make_fields(n, 98)
    _, tdeq = to_storage(tfs, np.float32)
    dx = 0.1 * PC
    view = View(math.radians(40), math.radians(130), 18, 17, 0.9 * dx, 1)
    va = VelocityAxis(64, -64.0, 2.0, 1)
    target = oracle.render_cube(tdeq.as_tuple(), dx, LINE, DUST, view, va,
                                integration=oracle.SMOOTH)["L"]
    ts = []
    for a in h16.as_tuple():
        if a.dtype == np.uint16:
            ts.append(torch.from_numpy(a.view(np.int16).copy()).view(torch.bfloat16).cuda())
        else:
            ts.append(torch.from_numpy(np.ascontiguousarray(a)).cuda())
    g = irt.Grid(*ts, dx, scales=scales)
    L = irt.forward(g, view, va, LINE, DUST, integration="smooth")["L"]
    tgt = torch.from_numpy(target.astype(np.float32)).cuda()
    grads = irt.adjoint(g, view, va, LINE, DUST, {"L": 2.0 * (L - tgt) / L.numel()},
                        integration="smooth")
    torch.cuda.synchronize()
    gn, gt, gv = [x.double().cpu().numpy() for x in grads]
    g.close()
    rng = np.random.default_rng(27)
    cells = np.stack([rng.integers(0, n, 40), rng.integers(0, n, 40), rng.integers(0, n, 40)],
                     axis=1)
    loss, on, ot, ov = oracle.loss_grad_cells(deq.as_tuple(), dx, LINE, DUST, view, va, target,
                                              cells, integration=oracle.SMOOTH)
    got = {k: np.array([a[z, y, x] for x, y, z in cells]) for k, a in (("n", gn), ("T", gt),
                                                                        ("v", gv))}
    K = 2 * n
    r = {"n": _cmp(got["n"], on, K), "T": _cmp(got["T"], ot, K), "v": _cmp(got["v"], ov, K)}
    assert all(v <= 1.0 for v in r.values()), r


@pytest.mark.parametrize("integration,f,nch,dv", [("formal", 2, 40, 3.0),
                                                  ("formal_kahan", 1, 40, 3.0),
                                                  ("smooth", 0, 48, 3.0),
                                                  ("smooth", 3, 30, 1.0),
                                                  ("smooth", 1, 560, 0.4)])
def test_z_view_gradients_beyond_the_fast_sweep(integration, f, nch, dv):
    """Formal and Kahan z views, f = 0, f = 3 at 1 km/s channels (line
    windows over 64 fine velocities), and 560 channels (two windows)."""
    n = 10
    fs = make_fields(n, 71)
    f32, deq = to_storage(fs, np.float32)
    tf32, tdeq = to_storage(make_fields(n, 78), np.float32)
    dx = 0.1 * PC
    view = View(0.0, 0.0, n, n, dx, 0)
    va = VelocityAxis(nch, -0.5 * nch * dv, dv, f)
    target = oracle.render_cube(tdeq.as_tuple(), dx, LINE, DUST, view, va,
                                integration=MODE[integration])["L"]
    gn, gt, gv = _gpu(f32, dx, view, va, target, integration)
    loss, on, ot, ov = oracle.loss_grad_zview(deq.as_tuple(), dx, LINE, DUST, va, target,
                                              integration=MODE[integration])
    r = {"n": _cmp(gn, on, n), "T": _cmp(gt, ot, n), "v": _cmp(gv, ov, n)}
    assert all(v <= 1.0 for v in r.values()), r


def test_dense_dust_columns_go_to_the_general_sweep():
    """Columns with h alpha_D > 1/2 on some sample (the smooth ReLU may clamp
    the continuum) are handed from the fast sweep to the general one; the
    other columns stay in the fast sweep.  Both against the oracle, no NaN."""
    n, nz = 6, 24
    fs = make_fields(24, 83)
    arrs = [np.ascontiguousarray(a[:nz, :n, :n]) for a in fs.as_tuple()]
    # three columns of very dense gas
    arrs[0][:, 0, :3] *= 3e3
    f32, deq = to_storage(FieldSet(*arrs), np.float32)
    tarr = [a.copy() for a in arrs]
    tarr[1] = tarr[1] * 1.1
    tf32, tdeq = to_storage(FieldSet(*tarr), np.float32)
    dx = 0.1 * PC
    dust = dict(DUST, kappa_cm2_per_g_gas=0.05)
    view = View(0.0, 0.0, n, n, dx, 0)
    va = VelocityAxis(64, -64.0, 2.0, 1)
    # per-step dust depth of the dense columns
    had = dust["kappa_cm2_per_g_gas"] * dust["mu_mass_per_h2_amu"] * 1.66053906660e-24 * dx
    assert had * arrs[0][:, 0, :3].max() > 0.5 > had * arrs[0][:, 1:, :].max()
    target = oracle.render_cube(tdeq.as_tuple(), dx, LINE, dust, view, va)["L"]
    gn, gt, gv = _gpu(f32, dx, view, va, target, "smooth", dust=dust)
    loss, on, ot, ov = oracle.loss_grad_zview(deq.as_tuple(), dx, LINE, dust, va, target)
    r = {"n": _cmp(gn, on, nz), "T": _cmp(gt, ot, nz), "v": _cmp(gv, ov, nz)}
    assert all(v <= 1.0 for v in r.values()), r


def test_radial_view_formal_gradient():
    import paper_2607_01338_b300 as irt  # noqa: F401
    nr, nb, nl = 20, 6, 7
    fs = make_fields(20, 91)
    arrs = [np.ascontiguousarray(a[:nr, :nb, :nl]) for a in fs.as_tuple()]
    f32, deq = to_storage(FieldSet(*arrs), np.float32)
    tarr = [np.ascontiguousarray(a[:nr, :nb, :nl]) for a in make_fields(20, 97).as_tuple()]
    tf32, tdeq = to_storage(FieldSet(*tarr), np.float32)
    dr = 0.05 * PC
    view = View(0.0, 0.0, nl, nb, dr, 2)
    va = VelocityAxis(40, -60.0, 3.0, 1)
    target = oracle.render_cube(tdeq.as_tuple(), dr, LINE, DUST, view, va,
                                integration=oracle.FORMAL)["L"]
    gn, gt, gv = _gpu(f32, dr, view, va, target, "formal")
    rng = np.random.default_rng(4)
    cells = np.stack([rng.integers(0, nl, 30), rng.integers(0, nb, 30), rng.integers(0, nr, 30)],
                     axis=1)
    loss, on, ot, ov = oracle.loss_grad_cells(deq.as_tuple(), dr, LINE, DUST, view, va, target,
                                              cells, integration=oracle.FORMAL)
    got = [np.array([a[z, y, x] for x, y, z in cells]) for a in (gn, gt, gv)]
    r = [_cmp(a, b, nr) for a, b in zip(got, (on, ot, ov))]
    assert all(v <= 1.0 for v in r), r

"""Adjoint (reverse sweep) of the CUDA path against the FP64 oracle:
dual-number gradients on a 16^3 grid and FP64 central differences on 200
random cells of the 128^3 workload, tolerance 1e-3 relative per cell (with
an absolute floor at the float32 rounding of the K-step recurrences, K 2^-24
of the largest gradient, and, against finite differences, the rounding error
of the difference itself)."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from synth import (DUST, LINE_13CO_21, FieldSet, VelocityAxis, View, make_fields,  # noqa: E402
                   to_storage, workload)

LINE = dict(LINE_13CO_21)
PC = 3.0856775814913673e18
GRAD_RTOL = 1e-3


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2607_01338_b300  # noqa: F401


def _gpu_loss_grads(f32, dx, view, va, target_L, integration="smooth", save=False):
    """GPU forward + adjoint of Loss = mean((L - target)^2); ``save`` lets the
    forward keep its transfer checkpoints for the adjoint."""
    import paper_2607_01338_b300 as irt
    from paper_2607_01338_b300 import binding as B
    ts = [torch.from_numpy(a).cuda() for a in f32.as_tuple()]
    g = irt.Grid(*ts, dx)
    cubes = irt.forward(g, view, va, LINE, DUST, integration=integration,
                        flags=B.IRT_FLAG_SAVE_CHECKPOINTS if save else 0)
    tgt = torch.from_numpy(target_L.astype(np.float32)).cuda()
    L = cubes["L"]
    gL = 2.0 * (L - tgt) / L.numel()
    grads = irt.adjoint(g, view, va, LINE, DUST, {"L": gL}, integration=integration)
    torch.cuda.synchronize()
    loss = float(torch.mean((L.double() - tgt.double()) ** 2).item())
    out = [x.double().cpu().numpy() for x in grads]
    g.close()
    return loss, out


#: absolute floor of the gradient comparisons: the float32 rounding of a
#: K-step recurrence, K u max|ref| with the unit roundoff u = 2^-24 (each
#: reverse step rounds its terms, all bounded by the largest gradient, so a
#: cell whose gradient is a small difference of such terms carries an
#: absolute error up to that size).  Everything above it is held to 1e-3
#: relative per cell.
U32 = 2.0 ** -24
U64 = 2.0 ** -53


def grad_floor(K):
    return K * U32


def _cmp(got, ref, K, rtol=GRAD_RTOL, floor=None):
    """Elementwise |got - ref| <= rtol |ref| + K u max|ref| (+ ``floor``, an
    array of per-cell allowances for the error of the reference itself)."""
    allow = rtol * np.abs(ref) + grad_floor(K) * np.abs(ref).max()
    if floor is not None:
        allow = allow + floor
    return float((np.abs(got - ref) / allow).max())


def fd_rounding_floor(L_plus, target, K, eps, nvox):
    """Rounding error of an FP64 central difference of a ray's squared-error
    loss: each K-step recurrence leaves [L]_c with a relative error of at most
    about K u (u = 2^-53), which moves sum_c ([L]_c - t_c)^2 by
    2 sum_c |[L]_c - t_c| |[L]_c| K u; two such sums are differenced and
    divided by 2 eps.  The truncation error of the central difference (eps^2
    times the third derivative over 6, at eps = 1e-6 relative) is far below."""
    return (2.0 * 2.0 * np.sum(np.abs(L_plus - target) * np.abs(L_plus)) * K * U64
            / (2.0 * eps) / nvox)


def crop_fields(fs, n, seed=0):
    rng = np.random.default_rng(seed)
    N = fs.n_h2.shape[0]
    o = rng.integers(0, N - n + 1, 3)
    sl = (slice(o[0], o[0] + n), slice(o[1], o[1] + n), slice(o[2], o[2] + n))
    return FieldSet(*[np.ascontiguousarray(a[sl]) for a in fs.as_tuple()])


@pytest.mark.parametrize("save", [False, True])
def test_adjoint_matches_oracle_gradient_16cube(save):
    """16^3 crop of the 128^3 adjoint workload (128 channels, f = 2), with the
    adjoint's own forward sweep and with the forward render's checkpoints."""
    w = workload(3, n=48)
    fs = crop_fields(make_fields(48, w.seed), 16, seed=3)
    tfs = crop_fields(make_fields(48, w.seed + 7), 16, seed=3)
    f32, deq = to_storage(fs, np.float32)
    t32, tdeq = to_storage(tfs, np.float32)
    view = View(0.0, 0.0, 16, 16, w.cell_cm, 0)
    va = w.vaxis
    target = oracle.render_cube(tdeq.as_tuple(), w.cell_cm, LINE, DUST, view, va)["L"]
    loss, (gn, gt, gv) = _gpu_loss_grads(f32, w.cell_cm, view, va, target, save=save)
    oloss, on, ot, ov = oracle.loss_grad_zview(deq.as_tuple(), w.cell_cm, LINE, DUST, va, target)
    assert loss == pytest.approx(oloss, rel=1e-4)
    r = {k: _cmp(a, b, 16) for k, a, b in (("n", gn, on), ("T", gt, ot), ("v", gv, ov))}
    assert all(v <= 1.0 for v in r.values()), r


@pytest.mark.parametrize("nz", [9, 17, 25, 33])
def test_adjoint_columns_of_every_flush_split(nz):
    """Columns whose first 32-sample segment is not a multiple of the partial
    flush: the trapezoidal start reverses samples 0 and 1 together, so no
    flush group may end at sample 1 (nz = 9, 17, 25 put a group boundary
    there with eight-sample groups)."""
    w = workload(3, n=48)
    fs = make_fields(48, w.seed)
    tfs = make_fields(48, w.seed + 7)
    sl = (slice(0, nz), slice(0, 6), slice(0, 7))
    fs = FieldSet(*[np.ascontiguousarray(a[sl]) for a in fs.as_tuple()])
    tfs = FieldSet(*[np.ascontiguousarray(a[sl]) for a in tfs.as_tuple()])
    f32, deq = to_storage(fs, np.float32)
    t32, tdeq = to_storage(tfs, np.float32)
    view = View(0.0, 0.0, 7, 6, w.cell_cm, 0)
    va = w.vaxis
    target = oracle.render_cube(tdeq.as_tuple(), w.cell_cm, LINE, DUST, view, va)["L"]
    loss, (gn, gt, gv) = _gpu_loss_grads(f32, w.cell_cm, view, va, target)
    oloss, on, ot, ov = oracle.loss_grad_zview(deq.as_tuple(), w.cell_cm, LINE, DUST, va, target)
    r = {k: _cmp(a, b, nz) for k, a, b in (("n", gn, on), ("T", gt, ot), ("v", gv, ov))}
    assert all(v <= 1.0 for v in r.values()), r


def test_saved_checkpoints_serve_only_the_same_job():
    """Checkpoints written by one render are used by the adjoint of the same
    job (results within float rounding of the self-contained adjoint) and
    ignored for another job (different background): then the adjoint is
    bit-identical to one without checkpoints."""
    import paper_2607_01338_b300 as irt
    from paper_2607_01338_b300 import binding as B
    fs = make_fields(48, 91)
    f32, _ = to_storage(crop_fields(fs, 24, seed=2), np.float32)
    ts = [torch.from_numpy(a).cuda() for a in f32.as_tuple()]
    dx = 0.1 * PC
    view = View(0.0, 0.0, 24, 24, dx, 0)
    va = VelocityAxis(96, -60.0, 1.25, 2)
    g0, g1 = irt.Grid(*ts, dx), irt.Grid(*ts, dx)
    L = irt.forward(g0, view, va, LINE, DUST)["L"]
    cot = {"L": L * 1e-3}
    ref = irt.adjoint(g0, view, va, LINE, DUST, cot)
    irt.forward(g1, view, va, LINE, DUST, flags=B.IRT_FLAG_SAVE_CHECKPOINTS)
    used = irt.adjoint(g1, view, va, LINE, DUST, cot)
    other = irt.adjoint(g1, view, va, LINE, DUST, cot, t_bg=2.7)
    ref_other = irt.adjoint(g0, view, va, LINE, DUST, cot, t_bg=2.7)
    torch.cuda.synchronize()
    for a, b in zip(used, ref):
        assert torch.allclose(a, b, rtol=1e-4, atol=1e-4 * float(b.abs().max()))
    for a, b in zip(other, ref_other):
        assert torch.equal(a, b)
    g0.close()
    g1.close()


def test_adjoint_matches_fp64_finite_differences_128cube():
    """200 random cells of the 128^3 / 128-channel / f = 2 workload: GPU
    adjoint against FP64 central differences of the oracle (ray-local:
    a cell only changes its own z-view ray)."""
    w = workload(3)
    fs = make_fields(w.n, w.seed)
    tfs = make_fields(w.n, w.seed + 7)
    f32, deq = to_storage(fs, np.float32)
    t32, tdeq = to_storage(tfs, np.float32)
    view, va = w.views[0], w.vaxis
    import paper_2607_01338_b300 as irt
    tg = irt.Grid(*[torch.from_numpy(a).cuda() for a in t32.as_tuple()], w.cell_cm)
    target = irt.forward(tg, view, va, LINE, DUST)["L"].double().cpu().numpy()
    tg.close()
    loss, (gn, gt, gv) = _gpu_loss_grads(f32, w.cell_cm, view, va, target)
    nvox = target.size
    rng = np.random.default_rng(11)
    cells = rng.integers(0, w.n, (200, 3))
    fields = [a.copy() for a in deq.as_tuple()]
    worst = {}
    for q, g, name in ((0, gn, "n"), (1, gt, "T"), (3, gv, "v")):
        fd, got, fl = [], [], []
        for (z, y, x) in cells:
            v0 = fields[q][z, y, x]
            eps = 1e-6 * max(abs(v0), 1.0)
            vals = []
            for sgn in (1, -1):
                fields[q][z, y, x] = v0 + sgn * eps
                Lr = oracle.render(fields, w.cell_cm, LINE, DUST, view, va, [(x, y)])["L"][0]
                vals.append(np.sum((Lr - target[:, y, x]) ** 2))
                if sgn == 1:
                    fl.append(fd_rounding_floor(Lr, target[:, y, x], w.n, eps, nvox))
            fields[q][z, y, x] = v0
            fd.append((vals[0] - vals[1]) / (2 * eps) / nvox)
            got.append(g[z, y, x])
        worst[name] = _cmp(np.array(got), np.array(fd), w.n, floor=np.array(fl))
    assert all(v <= 1.0 for v in worst.values()), worst


def test_adjoint_wide_hulls_take_the_second_pass():
    """Columns whose v_los ramps over +-80 km/s have line hulls wider than the
    9 register blocks of the first adjoint pass; they are deferred to the wide
    pass.  Flat columns stay in the first pass.  Both against the oracle."""
    n, nz = 4, 16
    fs = make_fields(16, 17)
    arrs = [np.ascontiguousarray(a[:nz, :n, :n]) for a in fs.as_tuple()]
    z = np.linspace(-1.0, 1.0, nz)[:, None, None]
    steep = np.array([0.0, 0.3, 0.7, 1.0])[None, None, :]
    arrs[3] = (80.0 * z * steep + 0.0 * arrs[3]).astype(np.float64) + arrs[3] * 0.1
    f = FieldSet(*arrs)
    f32, deq = to_storage(f, np.float32)
    tf32, tdeq = to_storage(FieldSet(*[a * 1.0 for a in arrs[:3]] + [arrs[3] + 3.0, arrs[4]]),
                            np.float32)
    dx = 0.1 * PC
    view = View(0.0, 0.0, n, n, dx, 0)
    va = VelocityAxis(200, -100.0, 1.0, 1)
    target = oracle.render_cube(tdeq.as_tuple(), dx, LINE, DUST, view, va)["L"]
    loss, (gn, gt, gv) = _gpu_loss_grads(f32, dx, view, va, target)
    oloss, on, ot, ov = oracle.loss_grad_zview(deq.as_tuple(), dx, LINE, DUST, va, target)
    assert loss == pytest.approx(oloss, rel=1e-4)
    assert np.isfinite(gn).all() and np.isfinite(gt).all() and np.isfinite(gv).all()
    r = {k: _cmp(a, b, nz) for k, a, b in (("n", gn, on), ("T", gt, ot), ("v", gv, ov))}
    assert all(v <= 1.0 for v in r.values()), r


def test_autograd_function_matches_adjoint():
    import paper_2607_01338_b300 as irt
    n = 12
    fs = make_fields(n, 5)
    f32, _ = to_storage(fs, np.float32)
    dx = 0.1 * PC
    view = View(0.0, 0.0, n, n, dx, 0)
    va = VelocityAxis(48, -72.0, 3.0, 1)
    ts = [torch.from_numpy(a).cuda() for a in f32.as_tuple()]
    n_h2 = ts[0].clone().requires_grad_(True)
    t_gas = ts[1].clone().requires_grad_(True)
    v_los = ts[3].clone().requires_grad_(True)
    cfg = irt.RenderConfig(dx, view, va, LINE, DUST)
    T, C, D, L, B = irt.render_ppv(n_h2, t_gas, v_los, ts[2], ts[4], cfg)
    loss = (L ** 2).mean() + 0.5 * T.mean() - 0.25 * (D * C).sum() / D.numel()
    loss.backward()
    g = irt.Grid(*ts, dx)
    with torch.no_grad():
        cot = dict(L=2 * L / L.numel(), T=torch.full_like(T, 0.5 / T.numel()),
                   D=-0.25 * C / D.numel(), C=-0.25 * D / D.numel())
    gn, gt, gv = irt.adjoint(g, view, va, LINE, DUST, cot)
    torch.cuda.synchronize()
    for a, b in ((n_h2.grad, gn), (t_gas.grad, gt), (v_los.grad, gv)):
        assert torch.allclose(a, b, rtol=1e-5, atol=1e-6 * b.abs().max().item())
    g.close()


def test_adjoint_edge_cases_and_errors():
    import paper_2607_01338_b300 as irt
    dx = 0.1 * PC
    # one sample per ray: the output is the background, all gradients vanish
    fs = make_fields(6, 8)
    arrs = [np.ascontiguousarray(a[:1].astype(np.float32)) for a in fs.as_tuple()]
    g = irt.Grid(*[torch.from_numpy(a).cuda() for a in arrs], dx)
    view = View(0.0, 0.0, 6, 6, dx, 0)
    va = VelocityAxis(16, -16.0, 2.0, 1)
    cot = {"L": torch.ones(16, 6, 6, device="cuda")}
    gn, gt, gv = irt.adjoint(g, view, va, LINE, DUST, cot)
    torch.cuda.synchronize()
    assert float(gn.abs().max()) == 0.0 and float(gt.abs().max()) == 0.0
    # T_B output has no adjoint; thin modes neither (thick mode only)
    with pytest.raises(irt.IrtError, match="IRT_EUNSUPPORTED"):
        irt.adjoint(g, view, va, LINE, DUST, cot, units="tb")
    # a one-sample oblique ray (formal): the general sweep differentiates it
    gn, gt, gv = irt.adjoint(g, View(0.3, 0.2, 6, 6, dx, 1), va, LINE, DUST, cot,
                             integration="formal")
    torch.cuda.synchronize()
    assert bool(torch.isfinite(gn).all()) and bool(torch.isfinite(gt).all())
    g.close()


def test_autograd_reuses_its_grid_across_steps():
    """Two training-style steps of the autograd function on different fields:
    the second forward takes the grid the first backward released (updated
    in place, its old checkpoints discarded), and its gradients equal a fresh
    grid's adjoint."""
    import paper_2607_01338_b300 as irt
    from paper_2607_01338_b300 import api
    n = 10
    dx = 0.1 * PC
    view = View(0.0, 0.0, n, n, dx, 0)
    va = VelocityAxis(40, -60.0, 3.0, 1)
    cfg = irt.RenderConfig(dx, view, va, LINE, DUST)
    api._GRID_POOL.clear()
    grads = []
    for seed in (3, 4):
        f32, _ = to_storage(make_fields(n, seed), np.float32)
        ts = [torch.from_numpy(a).cuda() for a in f32.as_tuple()]
        n_h2 = ts[0].clone().requires_grad_(True)
        t_gas = ts[1].clone().requires_grad_(True)
        v_los = ts[3].clone().requires_grad_(True)
        T, C, D, L, B = irt.render_ppv(n_h2, t_gas, v_los, ts[2], ts[4], cfg)
        (L ** 2).mean().backward()
        grads.append((ts, L.detach(), n_h2.grad, t_gas.grad, v_los.grad))
    pool = [g for v in api._GRID_POOL.values() for g in v]
    assert len(pool) == 1
    ts, L, gn, gt, gv = grads[1]
    g = irt.Grid(*ts, dx)
    rn, rt, rv = irt.adjoint(g, view, va, LINE, DUST, {"L": 2 * L / L.numel()})
    torch.cuda.synchronize()
    for a, b in ((gn, rn), (gt, rt), (gv, rv)):
        assert torch.allclose(a, b, rtol=1e-5, atol=1e-6 * b.abs().max().item())
    g.close()
    api._GRID_POOL.clear()

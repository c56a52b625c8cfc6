"""Forward parity of the CUDA path (through the C ABI) with the FP64 oracle."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from synth import (DUST, LINE_13CO_21, VelocityAxis, View, make_fields, to_storage,  # noqa: E402
                   workload)
from tests.gpu_helpers import (COMP, assert_parity, compare, crop_pixels, gpu_render,  # noqa: E402
                               oracle_pixels, rel_err_stats, torch_fields)

PC = 3.0856775814913673e18
LINE = dict(LINE_13CO_21)


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2607_01338_b300  # noqa: F401  (fails loudly if libirt.so is missing)


def all_pixels(npx, npy):
    py, px = np.meshgrid(np.arange(npy), np.arange(npx), indexing="ij")
    return np.stack([px.ravel(), py.ravel()], axis=1)


# ---------------------------------------------------------------------------
# 32^3, 64 channels, f = 4: double-precision kernels against the oracle
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("integration", ["smooth", "formal", "formal_kahan"])
def test_32cube_double_precision_full_cube(integration):
    w = workload(0)
    fs = make_fields(w.n, w.seed)
    view, va = w.views[0], w.vaxis
    gpu = gpu_render(torch_fields(fs), w.cell_cm, view, va, LINE, DUST, integration=integration,
                     precision="f64")
    pix = all_pixels(view.npx, view.npy)
    orc = oracle_pixels(fs.as_tuple(), w.cell_cm, view, va, LINE, DUST, pix,
                        integration=integration)
    assert_parity(gpu, orc, pix, rtol=1e-11, atol_frac=1e-13)


@pytest.mark.parametrize("integration", ["smooth", "formal", "formal_kahan"])
def test_32cube_float_full_cube(integration):
    w = workload(0)
    fs = make_fields(w.n, w.seed)
    f32, deq = to_storage(fs, np.float32)
    view, va = w.views[0], w.vaxis
    gpu = gpu_render(torch_fields(f32), w.cell_cm, view, va, LINE, DUST, integration=integration)
    pix = all_pixels(view.npx, view.npy)
    orc = oracle_pixels(deq.as_tuple(), w.cell_cm, view, va, LINE, DUST, pix,
                        integration=integration)
    assert_parity(gpu, orc, pix)


# ---------------------------------------------------------------------------
# 256^3, 256 channels at 1 km/s, f = 1: z view and the (30, 45) deg oblique
# view, checked on a seeded 32 x 32 pixel crop at full depth, all channels
# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def views256():
    w = workload(1)
    fs = make_fields(w.n, w.seed)
    f32, deq = to_storage(fs, np.float32)
    return w, f32, deq


@pytest.mark.parametrize("vi", [0, 1])
def test_256cube_crop(views256, vi):
    w, f32, deq = views256
    view, va = w.views[vi], w.vaxis
    gpu = gpu_render(torch_fields(f32), w.cell_cm, view, va, LINE, DUST, integration="smooth")
    pix = crop_pixels(view.npx, view.npy, 32, 32, seed=100 + vi)
    orc = oracle_pixels(deq.as_tuple(), w.cell_cm, view, va, LINE, DUST, pix)
    assert_parity(gpu, orc, pix)
    for k in COMP:
        assert np.isfinite(gpu[k]).all()


# ---------------------------------------------------------------------------
# ragged shapes, several windows, explicit channels, fallback, edge cases
# ---------------------------------------------------------------------------
def small_fields(shape, seed, n_mean=1e4):
    nz, ny, nx = shape
    n = max(shape)
    fs = make_fields(n, seed, n_mean=n_mean)
    arrs = [a[:nz, :ny, :nx].copy() for a in fs.as_tuple()]
    from synth import FieldSet
    return FieldSet(*arrs)


@pytest.mark.parametrize("integration", ["smooth", "formal", "formal_kahan"])
def test_ragged_oblique_view(integration):
    fs = small_fields((23, 29, 37), seed=9)
    f32, deq = to_storage(fs, np.float32)
    dx = 0.1 * PC
    view = View(math.radians(70.0), math.radians(200.0), 41, 33, 0.7 * dx, 1)
    va = VelocityAxis(75, -80.0, 2.0, 1)
    gpu = gpu_render(torch_fields(f32), dx, view, va, LINE, DUST, integration=integration)
    pix = all_pixels(view.npx, view.npy)
    orc = oracle_pixels(deq.as_tuple(), dx, view, va, LINE, DUST, pix, integration=integration)
    assert_parity(gpu, orc, pix)


@pytest.mark.parametrize("integration", ["smooth", "formal", "formal_kahan"])
def test_many_windows_and_f0(integration):
    fs = small_fields((20, 12, 14), seed=21)
    f32, deq = to_storage(fs, np.float32)
    dx = 0.1 * PC
    view = View(0.0, 0.0, 14, 12, dx, 0)
    for va in (VelocityAxis(600, -150.0, 0.5, 1), VelocityAxis(1200, -150.0, 0.25, 0),
               VelocityAxis(90, -120.0, 3.0, 3)):
        gpu = gpu_render(torch_fields(f32), dx, view, va, LINE, DUST, integration=integration)
        pix = all_pixels(view.npx, view.npy)
        orc = oracle_pixels(deq.as_tuple(), dx, view, va, LINE, DUST, pix,
                            integration=integration)
        assert_parity(gpu, orc, pix)


def long_column(nz, ny, nx, seed):
    """A tall column: 32^3 fields of several seeds stacked along z."""
    from synth import FieldSet
    parts = [make_fields(32, seed + i).as_tuple() for i in range((nz + 31) // 32)]
    arrs = [np.concatenate([p[q] for p in parts], axis=0)[:nz, :ny, :nx].copy()
            for q in range(5)]
    return FieldSet(*arrs)


@pytest.mark.parametrize("integration", ["smooth", "formal", "formal_kahan"])
def test_long_rays_stream_their_records(integration):
    """Rays of 700 and about 560 samples: longer than the records a warp keeps
    in shared memory, so the tail of each ray streams through global memory
    (forward sweeps, and the backward sweep of the Kahan transfer)."""
    fs = long_column(700, 5, 4, seed=61)
    f32, deq = to_storage(fs, np.float32)
    dx = 0.1 * PC
    va = VelocityAxis(96, -48.0, 1.0, 1)
    for view in (View(0.0, 0.0, 4, 5, dx, 0),
                 View(math.radians(0.15), math.radians(30.0), 6, 6, 0.6 * dx, 1)):
        gpu = gpu_render(torch_fields(f32), dx, view, va, LINE, DUST, integration=integration)
        pix = all_pixels(view.npx, view.npy)
        orc = oracle_pixels(deq.as_tuple(), dx, view, va, LINE, DUST, pix,
                            integration=integration)
        assert_parity(gpu, orc, pix)


@pytest.mark.parametrize("integration", ["smooth", "formal", "formal_kahan"])
def test_explicit_channels_flag_matches_shortcut(integration):
    fs = small_fields((24, 16, 16), seed=31)
    f32, deq = to_storage(fs, np.float32)
    dx = 0.1 * PC
    view = View(0.0, 0.0, 16, 16, dx, 0)
    va = VelocityAxis(128, -128.0, 2.0, 1)
    a = gpu_render(torch_fields(f32), dx, view, va, LINE, DUST, integration=integration)
    b = gpu_render(torch_fields(f32), dx, view, va, LINE, DUST, integration=integration, flags=1)
    pix = all_pixels(16, 16)
    orc = oracle_pixels(deq.as_tuple(), dx, view, va, LINE, DUST, pix, integration=integration)
    assert_parity(a, orc, pix)
    assert_parity(b, orc, pix)


@pytest.mark.parametrize("integration", ["smooth", "formal", "formal_kahan"])
def test_dense_dusty_fallback(integration):
    """kappa x 3000 on dense gas: h alpha_D > 1/2 on some samples, so the
    smooth path integrates every channel explicitly."""
    fs = small_fields((16, 8, 8), seed=41, n_mean=1e5)
    f32, deq = to_storage(fs, np.float32)
    dx = 0.1 * PC
    dust = dict(DUST, kappa_cm2_per_g_gas=30.0)
    view = View(0.0, 0.0, 8, 8, dx, 0)
    va = VelocityAxis(64, -64.0, 2.0, 1)
    gpu = gpu_render(torch_fields(f32), dx, view, va, LINE, dust, integration=integration)
    pix = all_pixels(8, 8)
    orc = oracle_pixels(deq.as_tuple(), dx, view, va, LINE, dust, pix, integration=integration)
    assert_parity(gpu, orc, pix)


@pytest.mark.parametrize("integration", ["smooth", "formal", "formal_kahan"])
def test_edge_cases(integration):
    dx = 0.1 * PC
    # one sample per ray (smooth: background only), one channel, f = 0
    fs = small_fields((1, 6, 5), seed=51)
    f32, deq = to_storage(fs, np.float32)
    for va in (VelocityAxis(1, -2.0, 4.0, 0), VelocityAxis(1, -2.0, 4.0, 2)):
        view = View(0.0, 0.0, 5, 6, dx, 0)
        gpu = gpu_render(torch_fields(f32), dx, view, va, LINE, DUST, integration=integration)
        pix = all_pixels(5, 6)
        orc = oracle_pixels(deq.as_tuple(), dx, view, va, LINE, DUST, pix,
                            integration=integration)
        assert_parity(gpu, orc, pix)
    # rays that miss the box, gas above T_inf, no tracer, intensity units
    fs = small_fields((8, 8, 8), seed=52)
    fs.t_gas[2:4] = 6e4
    fs.x_tracer[:, :, 5:] = 0.0
    f32, deq = to_storage(fs, np.float32)
    view = View(math.radians(45.0), math.radians(30.0), 20, 20, dx, 1)
    va = VelocityAxis(40, -60.0, 3.0, 1)
    for units in ("trj", "intensity"):
        gpu = gpu_render(torch_fields(f32), dx, view, va, LINE, DUST, integration=integration,
                         units=units)
        pix = all_pixels(20, 20)
        orc = oracle_pixels(deq.as_tuple(), dx, view, va, LINE, DUST, pix,
                            integration=integration, units=units)
        assert_parity(gpu, orc, pix)


# ---------------------------------------------------------------------------
# reduced-precision storage: arithmetic error (oracle on the stored values)
# must meet the FP32 rule; the total error against the FP64 originals is
# reported
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("storage", ["bf16_v16", "f16"])
def test_half_precision_storage(storage, capsys):
    fs = small_fields((32, 24, 24), seed=61)
    if storage == "f16":
        # fp16 tops out at 65504 and is subnormal below 6.1e-5: the density is
        # stored in units of 1e4 cm^-3 and the abundance in units of 1e-6
        dts = [np.float16] * 5
        scales = [1e4, 1.0, 1.0, 1.0, 1e-6]
    else:
        dts = ["bf16", "bf16", "bf16", np.float16, "bf16"]
        scales = [1.0] * 5
    st, deq = to_storage(fs, dts, scales)
    dx = 0.1 * PC
    view = View(math.radians(30.0), math.radians(45.0), 24, 24, dx, 1)
    va = VelocityAxis(128, -128.0, 2.0, 1)
    import paper_2607_01338_b300 as irt
    g = irt.Grid(*torch_fields(st), dx, scales=scales)
    cubes = irt.forward(g, view, va, LINE, DUST, integration="formal_kahan")
    torch.cuda.synchronize()
    gpu = {k: cubes[k].double().cpu().numpy() for k in COMP}
    g.close()
    pix = all_pixels(24, 24)
    orc = oracle_pixels(deq.as_tuple(), dx, view, va, LINE, DUST, pix, integration="formal")
    assert_parity(gpu, orc, pix)
    orc64 = oracle_pixels(fs.as_tuple(), dx, view, va, LINE, DUST, pix, integration="formal")
    with capsys.disabled():
        print(f"\n[{storage}] total error vs FP64 fields:", rel_err_stats(gpu, orc64, pix))


# ---------------------------------------------------------------------------
# batch, determinism, errors
# ---------------------------------------------------------------------------
def test_batch_equals_single_jobs_and_is_deterministic():
    import paper_2607_01338_b300 as irt
    dx = 0.1 * PC
    rng = np.random.default_rng(7)
    jobs, grids = [], []
    for i, n in enumerate((12, 20, 16, 9, 24)):
        fs = make_fields(n, 700 + i)
        g = irt.Grid(*torch_fields(fs, [torch.float32] * 5), dx)
        th, ph = float(rng.uniform(0, math.pi)), float(rng.uniform(0, 2 * math.pi))
        view = View(th, ph, n + 3, n, dx, 1) if i % 2 else View(0.0, 0.0, n, n, dx, 0)
        va = VelocityAxis(int(rng.integers(20, 140)), -70.0, 1.0, 1)
        grids.append(g)
        jobs.append((g, view, va))
    batch = irt.forward_batch(jobs, LINE, DUST, integration="smooth")
    batch2 = irt.forward_batch(jobs, LINE, DUST, integration="smooth")
    torch.cuda.synchronize()
    for (g, view, va), cb, cb2 in zip(jobs, batch, batch2):
        single = irt.forward(g, view, va, LINE, DUST, integration="smooth")
        torch.cuda.synchronize()
        for k in COMP:
            assert torch.equal(single[k], cb[k]), k
            assert torch.equal(cb[k], cb2[k]), k
    for g in grids:
        g.close()


def test_gpu_errors_are_reported():
    import paper_2607_01338_b300 as irt
    dx = 0.1 * PC
    fs = make_fields(8, 3)
    g = irt.Grid(*torch_fields(fs, [torch.float32] * 5), dx)
    va = VelocityAxis(8, -8.0, 2.0, 1)
    with pytest.raises(irt.IrtError, match="IRT_EINVAL"):
        irt.forward(g, View(0.0, 0.0, 7, 8, dx, 0), va, LINE, DUST)
    with pytest.raises(irt.IrtError, match="IRT_EUNSUPPORTED"):
        irt.forward(g, View(0.0, 0.0, 8, 8, dx, 0), va, LINE, DUST, precision="f64")
    with pytest.raises(irt.IrtError, match="IRT_EINVAL"):
        irt.forward(g, View(0.0, 0.0, 8, 8, dx, 0), VelocityAxis(8, -8.0, -1.0, 1), LINE, DUST)
    g.close()


@pytest.mark.parametrize("integration", ["smooth", "formal", "formal_kahan"])
def test_non_dyadic_velocity_grid(integration):
    """Fine velocities that float cannot represent (dv = 0.3 km/s, v0 = -37.7)."""
    fs = small_fields((40, 10, 12), seed=71)
    f32, deq = to_storage(fs, np.float32)
    dx = 0.1 * PC
    view = View(0.0, 0.0, 12, 10, dx, 0)
    for va in (VelocityAxis(180, -37.7, 0.3, 1), VelocityAxis(70, -61.3, 1.7, 3)):
        gpu = gpu_render(torch_fields(f32), dx, view, va, LINE, DUST, integration=integration)
        pix = all_pixels(12, 10)
        orc = oracle_pixels(deq.as_tuple(), dx, view, va, LINE, DUST, pix,
                            integration=integration)
        assert_parity(gpu, orc, pix)

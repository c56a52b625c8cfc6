"""Optically thin level balance on the GPU (Sec. 3.4-3.6, 4.2, 4.3): the
coefficient grid built by the library's FP64 solver against the oracle's
grid, and renders with the grid's coefficients against the oracle render
with the same grid, float kernels at the FP32 parity rule and double kernels
at 1e-11."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from synth import DUST, LINE_13CO_21, VelocityAxis, View, make_fields, to_storage  # noqa: E402
from synth.levels import OT_AXES, rotor_model  # noqa: E402
from tests.gpu_helpers import COMP, assert_parity, torch_fields  # noqa: E402

PC = 3.0856775814913673e18


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2607_01338_b300  # noqa: F401


def rotor_line(model, r):
    """LINE_13CO_21's profile constants with transition r of the model."""
    ln = dict(LINE_13CO_21)
    ln["nu_ul_hz"] = float(model["nu_hz"][r])
    return ln


AXES_SMALL = dict(n_n=24, n_chi=8, n_t=16, log10_nh_min=1.0, log10_nh_max=7.5, chi_min=0.05,
                  chi_max=0.5, log10_t_min=math.log10(8.0), log10_t_max=math.log10(300.0))


@pytest.fixture(scope="module")
def tables():
    import paper_2607_01338_b300 as irt
    m = rotor_model(nlev=24, seed=1)
    lines = [0, 1, 2]
    g = irt.LevelTable(m, AXES_SMALL, lines)
    o = oracle.OTTable(m, AXES_SMALL, lines)
    yield m, g, o
    g.close()
    o.close()


def test_grid_matches_the_oracle_grid(tables):
    m, g, o = tables
    gv, ov = g.values(), o.values()
    assert gv.shape == ov.shape
    for q in range(2):
        a, b = gv[..., q], ov[..., q]
        np.testing.assert_allclose(a, b, rtol=1e-10, atol=1e-12 * np.abs(b).max())


def test_paper_size_grid_against_oracle_solves():
    """The paper's 128 x 64 x 64 grid with a 41-level rotor (every level the
    partition function needs at these temperatures): 300 random nodes against
    the oracle's solve at the same node."""
    import paper_2607_01338_b300 as irt
    m = rotor_model(nlev=41, seed=2)
    t = irt.LevelTable(m, OT_AXES, [1])
    gv = t.values()[0]
    t.close()
    small = dict(OT_AXES)
    rng = np.random.default_rng(3)
    nn, nc, nt = OT_AXES["n_n"], OT_AXES["n_chi"], OT_AXES["n_t"]
    idx = np.stack([rng.integers(0, nn, 300), rng.integers(0, nc, 300),
                    rng.integers(0, nt, 300)], axis=1)
    # a one-node oracle grid at each sampled node (axes collapsed onto it)
    for i0, i1, i2 in idx:
        ln = small["log10_nh_min"] + (small["log10_nh_max"] - small["log10_nh_min"]) * i0 / (nn - 1)
        ch = small["chi_min"] + (small["chi_max"] - small["chi_min"]) * i1 / (nc - 1)
        lt = small["log10_t_min"] + (small["log10_t_max"] - small["log10_t_min"]) * i2 / (nt - 1)
        ax = dict(n_n=2, n_chi=2, n_t=2, log10_nh_min=ln, log10_nh_max=ln + 1.0, chi_min=ch,
                  chi_max=ch + 1e-3 if ch < 0.5 else ch, log10_t_min=lt, log10_t_max=lt + 1.0)
        if ch >= 0.5:
            ax["chi_min"], ax["chi_max"] = ch - 1e-3, ch
        o = oracle.OTTable(m, ax, [1])
        ov = o.values()[0]
        o.close()
        k1 = 1 if ch >= 0.5 else 0
        np.testing.assert_allclose(gv[i0, i1, i2], ov[0, k1, 0], rtol=1e-10,
                                   atol=1e-30)


def _ot_fields(n, seed, dtype=np.float32):
    fs = make_fields(n, seed)
    st, deq = to_storage(fs, dtype)
    rng = np.random.default_rng(seed + 50)
    chi = rng.uniform(0.08, 0.5, (n, n, n))
    return st, deq, chi


@pytest.mark.parametrize("integration", ["smooth", "formal", "formal_kahan"])
def test_ot_render_float_z_and_oblique(tables, integration):
    import paper_2607_01338_b300 as irt
    m, g, o = tables
    n = 24
    st, deq, chi = _ot_fields(n, 77)
    chi32 = chi.astype(np.float32)
    dx = 0.1 * PC
    line = rotor_line(m, 1)
    va = VelocityAxis(96, -96.0, 2.0, 1)
    grid = irt.Grid(*torch_fields(st), dx)
    grid.set_h2_fraction(torch.from_numpy(chi32).cuda())
    for view in (View(0.0, 0.0, n, n, dx, 0), View(math.radians(30), math.radians(45), n, n, dx, 1)):
        cubes = irt.forward(grid, view, va, line, DUST, integration=integration, levels=g,
                            line_index=1)
        torch.cuda.synchronize()
        gpu = {k: cubes[k].double().cpu().numpy() for k in COMP}
        py, px = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
        pix = np.stack([px.ravel(), py.ravel()], axis=1)
        orc = oracle.render(deq.as_tuple(), dx, line, DUST, view, va, pix,
                            integration=oracle.SMOOTH if integration == "smooth" else oracle.FORMAL,
                            levels=o, line_index=1, chi=chi32.astype(np.float64))
        assert float(np.abs(orc["L"]).max()) > 0.5
        assert_parity(gpu, orc, pix)
    grid.close()


@pytest.mark.parametrize("integration", ["smooth", "formal"])
def test_ot_render_double_precision(tables, integration):
    import paper_2607_01338_b300 as irt
    m, g, o = tables
    n = 16
    fs = make_fields(n, 91)
    rng = np.random.default_rng(3)
    chi = rng.uniform(0.08, 0.5, (n, n, n))
    dx = 0.1 * PC
    line = rotor_line(m, 2)
    va = VelocityAxis(48, -72.0, 3.0, 2)
    grid = irt.Grid(*torch_fields(fs), dx)
    grid.set_h2_fraction(torch.from_numpy(chi).cuda())
    py, px = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    pix = np.stack([px.ravel(), py.ravel()], axis=1)
    for view in (View(0.0, 0.0, n, n, dx, 0), View(math.radians(60), math.radians(200), n, n, dx, 1)):
        cubes = irt.forward(grid, view, va, line, DUST, integration=integration,
                            precision="f64", levels=g, line_index=2)
        torch.cuda.synchronize()
        gpu = {k: cubes[k].cpu().numpy() for k in COMP}
        orc = oracle.render(fs.as_tuple(), dx, line, DUST, view, va, pix,
                            integration=oracle.SMOOTH if integration == "smooth" else oracle.FORMAL,
                            levels=o, line_index=2, chi=chi)
        assert_parity(gpu, orc, pix, rtol=1e-10, atol_frac=1e-12)
    grid.close()


def test_ot_default_abundance_and_16bit_storage(tables):
    """A grid whose H2 abundance was never set is fully molecular (0.5); a
    16-bit grid keeps its abundance in fp16."""
    import paper_2607_01338_b300 as irt
    m, g, o = tables
    n = 20
    dx = 0.1 * PC
    line = rotor_line(m, 1)
    va = VelocityAxis(64, -64.0, 2.0, 1)
    view = View(0.0, 0.0, n, n, dx, 0)
    py, px = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    pix = np.stack([px.ravel(), py.ravel()], axis=1)
    st, deq, chi = _ot_fields(n, 5)
    grid = irt.Grid(*torch_fields(st), dx)
    cubes = irt.forward(grid, view, va, line, DUST, levels=g, line_index=1)
    torch.cuda.synchronize()
    gpu = {k: cubes[k].double().cpu().numpy() for k in COMP}
    orc = oracle.render(deq.as_tuple(), dx, line, DUST, view, va, pix, levels=o, line_index=1)
    assert_parity(gpu, orc, pix)
    grid.close()
    # fp16 fields (density and abundance scaled), fp16 abundance
    fs = make_fields(n, 6)
    scales = [1e4, 1.0, 1.0, 1.0, 1e-6]
    st16, deq16 = to_storage(fs, np.float16, scales=scales)
    chi16 = np.random.default_rng(9).uniform(0.1, 0.5, (n, n, n)).astype(np.float16)
    grid = irt.Grid(*torch_fields(st16), dx, scales=scales)
    grid.set_h2_fraction(torch.from_numpy(chi16).cuda())
    cubes = irt.forward(grid, view, va, line, DUST, levels=g, line_index=1)
    torch.cuda.synchronize()
    gpu = {k: cubes[k].double().cpu().numpy() for k in COMP}
    orc = oracle.render(deq16.as_tuple(), dx, line, DUST, view, va, pix, levels=o, line_index=1,
                        chi=chi16.astype(np.float64))
    assert_parity(gpu, orc, pix)
    grid.close()


@pytest.mark.parametrize("transfer", ["selectively_thin", "thin"])
def test_ot_thin_modes(tables, transfer):
    import paper_2607_01338_b300 as irt
    m, g, o = tables
    n = 20
    st, deq, chi = _ot_fields(n, 13)
    chi32 = chi.astype(np.float32)
    dx = 0.1 * PC
    line = rotor_line(m, 1)
    va = VelocityAxis(80, -80.0, 2.0, 1)
    grid = irt.Grid(*torch_fields(st), dx)
    grid.set_h2_fraction(torch.from_numpy(chi32).cuda())
    view = View(math.radians(30), math.radians(45), n, n, dx, 1)
    cubes = irt.forward(grid, view, va, line, DUST, transfer=transfer, levels=g, line_index=1)
    torch.cuda.synchronize()
    gpu = {k: cubes[k].double().cpu().numpy() for k in COMP}
    py, px = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    pix = np.stack([px.ravel(), py.ravel()], axis=1)
    tr = {"selectively_thin": oracle.SELECTIVELY_THIN, "thin": oracle.THIN}[transfer]
    orc = oracle.render(deq.as_tuple(), dx, line, DUST, view, va, pix, transfer=tr, levels=o,
                        line_index=1, chi=chi32.astype(np.float64))
    assert_parity(gpu, orc, pix)
    grid.close()


def test_ot_argument_errors(tables):
    import paper_2607_01338_b300 as irt
    from paper_2607_01338_b300.binding import (IRT_EINVAL, IRT_EUNSUPPORTED,
                                               IRT_FLAG_SAVE_CHECKPOINTS, IrtError)
    m, g, o = tables
    n = 8
    st, deq, chi = _ot_fields(n, 2)
    dx = 0.1 * PC
    grid = irt.Grid(*torch_fields(st), dx)
    va = VelocityAxis(16, -16.0, 2.0, 1)
    view = View(0.0, 0.0, n, n, dx, 0)
    with pytest.raises(IrtError) as e:
        irt.forward(grid, view, va, rotor_line(m, 2), DUST, levels=g, line_index=1)
    assert e.value.status == IRT_EINVAL and "frequency" in str(e.value)
    with pytest.raises(IrtError) as e:
        irt.forward(grid, view, va, rotor_line(m, 1), DUST, levels=g, line_index=3)
    assert e.value.status == IRT_EINVAL
    with pytest.raises(IrtError) as e:
        irt.forward(grid, view, va, rotor_line(m, 1), DUST, levels=g, line_index=1,
                    flags=IRT_FLAG_SAVE_CHECKPOINTS)
    assert e.value.status == IRT_EUNSUPPORTED
    grid.close()

"""Planck brightness-temperature output with continuum subtraction in T_B
space (Sec. 4.9, 4.10) on the CUDA path against the FP64 oracle: thick
(smooth and formal, z and oblique views) and selectively thin transfer,
float and double kernels."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from synth import DUST, LINE_13CO_21, VelocityAxis, make_fields, to_storage, workload  # noqa: E402
from synth.configs import oblique_view  # noqa: E402
from tests.gpu_helpers import assert_parity, gpu_render, oracle_pixels, torch_fields  # noqa: E402

LINE = dict(LINE_13CO_21)


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2607_01338_b300  # noqa: F401


def all_pixels(npx, npy):
    py, px = np.meshgrid(np.arange(npy), np.arange(npx), indexing="ij")
    return np.stack([px.ravel(), py.ravel()], axis=1)


@pytest.mark.parametrize("kind", ["z", "oblique"])
@pytest.mark.parametrize("integration", ["smooth", "formal"])
@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_thick_tb_full_image(precision, integration, kind):
    w = workload(0)
    fs = make_fields(w.n, w.seed)
    view = w.views[0] if kind == "z" else oblique_view(w.n, w.cell_cm, 30.0, 45.0)
    if precision == "f32":
        src, ref = to_storage(fs, np.float32)
        tol = {}
    else:
        src, ref = fs, fs
        tol = dict(rtol=1e-11, atol_frac=1e-13)
    gpu = gpu_render(torch_fields(src), w.cell_cm, view, w.vaxis, LINE, DUST,
                     integration=integration, precision=precision, units="tb")
    pix = all_pixels(view.npx, view.npy)
    orc = oracle_pixels(ref.as_tuple(), w.cell_cm, view, w.vaxis, LINE, DUST, pix,
                        integration=integration, units="tb")
    assert_parity(gpu, orc, pix, **tol)
    assert np.allclose(orc["B"], 2.725, rtol=1e-12)


@pytest.mark.parametrize("transfer", ["selectively_thin", "thin"])
def test_thin_modes_tb(transfer):
    w = workload(0)
    fs = make_fields(w.n, w.seed)
    f32, deq = to_storage(fs, np.float32)
    va = VelocityAxis(45, -70.0, 3.0, 0)
    view = w.views[0]
    gpu = gpu_render(torch_fields(f32), w.cell_cm, view, va, LINE, DUST, integration="smooth",
                     units="tb", transfer=transfer)
    pix = all_pixels(view.npx, view.npy)
    mode = oracle.SELECTIVELY_THIN if transfer == "selectively_thin" else oracle.THIN
    orc = oracle.render(deq.as_tuple(), w.cell_cm, LINE, DUST, view, va, pix,
                        integration=oracle.SMOOTH, units=oracle.TB, transfer=mode)
    assert_parity(gpu, orc, pix)


def test_adjoint_refuses_tb_units():
    import paper_2607_01338_b300 as irt
    from paper_2607_01338_b300 import binding as B
    w = workload(0)
    fs = make_fields(w.n, w.seed)
    f32, _ = to_storage(fs, np.float32)
    g = irt.Grid(*torch_fields(f32), w.cell_cm)
    try:
        view = w.views[0]
        cot = {"L": torch.ones((w.vaxis.nchan, view.npy, view.npx), device="cuda")}
        with pytest.raises(B.IrtError, match="T_RJ or intensity"):
            irt.adjoint(g, view, w.vaxis, LINE, DUST, cot, units="tb")
    finally:
        torch.cuda.synchronize()
        g.close()

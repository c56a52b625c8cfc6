"""Parity of the selectively thin and optically thin transfer modes (Sec. 4.6,
4.7 with the step substitutions of Sec. 4.8) between the CUDA path (through
the C ABI) and the FP64 oracle: double kernels at 1e-11, float kernels at the
FP32 parity rule on the stored values; z and oblique views, a ragged channel
count, one- and two-sample rays, and a crop of the 256^3 workload."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from synth import DUST, LINE_13CO_21, VelocityAxis, make_fields, to_storage, workload  # noqa: E402
from synth.configs import oblique_view, z_view  # noqa: E402
from tests.gpu_helpers import assert_parity, crop_pixels, gpu_render, torch_fields  # noqa: E402

LINE = dict(LINE_13CO_21)
TRANSFER = {"selectively_thin": oracle.SELECTIVELY_THIN, "thin": oracle.THIN}
INTEG = {"smooth": oracle.SMOOTH, "formal": oracle.FORMAL}
#: 45 channels: one full block of 32 lanes and a ragged block of 13
VA45 = VelocityAxis(45, -70.0, 3.0, 0)


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2607_01338_b300  # noqa: F401  (fails loudly if libirt.so is missing)


def all_pixels(npx, npy):
    py, px = np.meshgrid(np.arange(npy), np.arange(npx), indexing="ij")
    return np.stack([px.ravel(), py.ravel()], axis=1)


def oracle_thin(fields, cell, view, va, pix, transfer, integration):
    return oracle.render(fields, cell, LINE, DUST, view, va, pix, integration=INTEG[integration],
                         transfer=TRANSFER[transfer])


def view_of(kind, n, cell):
    return z_view(n, cell) if kind == "z" else oblique_view(n, cell, 30.0, 45.0)


@pytest.mark.parametrize("kind", ["z", "oblique"])
@pytest.mark.parametrize("integration", ["smooth", "formal"])
@pytest.mark.parametrize("transfer", ["selectively_thin", "thin"])
def test_32cube_double_precision_full_image(transfer, integration, kind):
    w = workload(0)
    fs = make_fields(w.n, w.seed)
    view = view_of(kind, w.n, w.cell_cm)
    gpu = gpu_render(torch_fields(fs), w.cell_cm, view, VA45, LINE, DUST,
                     integration=integration, precision="f64", transfer=transfer)
    pix = all_pixels(view.npx, view.npy)
    orc = oracle_thin(fs.as_tuple(), w.cell_cm, view, VA45, pix, transfer, integration)
    assert_parity(gpu, orc, pix, rtol=1e-11, atol_frac=1e-13)


@pytest.mark.parametrize("kind", ["z", "oblique"])
@pytest.mark.parametrize("integration", ["smooth", "formal"])
@pytest.mark.parametrize("transfer", ["selectively_thin", "thin"])
def test_32cube_float_full_image(transfer, integration, kind):
    w = workload(0)
    fs = make_fields(w.n, w.seed)
    f32, deq = to_storage(fs, np.float32)
    view = view_of(kind, w.n, w.cell_cm)
    gpu = gpu_render(torch_fields(f32), w.cell_cm, view, VA45, LINE, DUST,
                     integration=integration, transfer=transfer)
    pix = all_pixels(view.npx, view.npy)
    orc = oracle_thin(deq.as_tuple(), w.cell_cm, view, VA45, pix, transfer, integration)
    assert_parity(gpu, orc, pix)


@pytest.mark.parametrize("nz", [1, 2, 3])
@pytest.mark.parametrize("integration", ["smooth", "formal"])
@pytest.mark.parametrize("transfer", ["selectively_thin", "thin"])
def test_short_rays(transfer, integration, nz):
    """One, two and three samples per ray: background only / TR alone /
    one BDF2 step, and the trapezoid-only Simpson sum."""
    fs = make_fields(8, 77)
    cell = workload(0).cell_cm
    fsz = type(fs)(*[np.ascontiguousarray(a[:nz]) for a in fs.as_tuple()])
    view = z_view(8, cell)
    for prec, tol in (("f64", dict(rtol=1e-11, atol_frac=1e-13)), ("f32", {})):
        src = fsz
        if prec == "f32":
            src, fsz_q = to_storage(fsz, np.float32)
        else:
            fsz_q = fsz
        gpu = gpu_render(torch_fields(src), cell, view, VA45, LINE, DUST,
                         integration=integration, precision=prec, transfer=transfer)
        pix = all_pixels(8, 8)
        orc = oracle_thin(fsz_q.as_tuple(), cell, view, VA45, pix, transfer, integration)
        assert_parity(gpu, orc, pix, **tol)


@pytest.mark.parametrize("kind", ["z", "oblique"])
@pytest.mark.parametrize("transfer", ["selectively_thin", "thin"])
def test_256cube_crop_float(transfer, kind):
    """The 256^3 / 256-channel workload (FP32 fields), smooth integration, an
    8 x 8 pixel crop at full depth against the oracle."""
    w = workload(1)
    fs = make_fields(w.n, w.seed)
    f32, deq = to_storage(fs, np.float32)
    view = w.views[0] if kind == "z" else w.views[1]
    gpu = gpu_render(torch_fields(f32), w.cell_cm, view, w.vaxis, LINE, DUST,
                     integration="smooth", transfer=transfer)
    pix = crop_pixels(view.npx, view.npy, 8, 8, seed=11 if kind == "z" else 12)
    orc = oracle_thin(deq.as_tuple(), w.cell_cm, view, w.vaxis, pix, transfer, "smooth")
    assert_parity(gpu, orc, pix)
    assert float(np.abs(orc["L"]).max()) > 0.1


def test_thin_modes_refuse_kahan_checkpoints_and_the_adjoint():
    import paper_2607_01338_b300 as irt
    from paper_2607_01338_b300 import api as A
    from paper_2607_01338_b300 import binding as B
    w = workload(0)
    fs = make_fields(w.n, w.seed)
    f32, _ = to_storage(fs, np.float32)
    g = irt.Grid(*torch_fields(f32), w.cell_cm)
    try:
        view = w.views[0]
        with pytest.raises(B.IrtError, match="IRT_FORMAL or IRT_SMOOTH"):
            irt.forward(g, view, VA45, LINE, DUST, integration="formal_kahan",
                        transfer="thin")
        with pytest.raises(B.IrtError, match="checkpoints"):
            irt.forward(g, view, VA45, LINE, DUST, transfer="selectively_thin",
                        flags=B.IRT_FLAG_SAVE_CHECKPOINTS)
        cot = {"L": torch.ones((VA45.nchan, view.npy, view.npx), device="cuda")}
        job = A.make_job(g, view, VA45, {k: None for k in "TCDLB"})
        grads = [torch.empty((w.n, w.n, w.n), device="cuda") for _ in range(3)]
        with pytest.raises(B.IrtError, match="thick"):
            B.irt_adjoint_ppv(job, A.line_struct(LINE), A.dust_struct(DUST),
                              A.opts_struct("smooth", transfer="thin"),
                              A._cubes_struct(cot), grads[0].data_ptr(),
                              grads[1].data_ptr(), grads[2].data_ptr(), None)
    finally:
        torch.cuda.synchronize()
        g.close()


@pytest.mark.parametrize("kind", ["z", "oblique"])
@pytest.mark.parametrize("integration", ["smooth", "formal"])
@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_density_tracing_cube(precision, integration, kind):
    """Sec. 5.10 density-tracing cube (column density per unit velocity)."""
    w = workload(0)
    fs = make_fields(w.n, w.seed)
    view = view_of(kind, w.n, w.cell_cm)
    if precision == "f32":
        src, ref = to_storage(fs, np.float32)
        tol = {}
    else:
        src, ref = fs, fs
        tol = dict(rtol=1e-11, atol_frac=1e-13)
    gpu = gpu_render(torch_fields(src), w.cell_cm, view, VA45, LINE, DUST,
                     integration=integration, precision=precision, transfer="density_tracing")
    pix = all_pixels(view.npx, view.npy)
    orc = oracle.render(ref.as_tuple(), w.cell_cm, LINE, DUST, view, VA45, pix,
                        integration=INTEG[integration], transfer=oracle.DENSITY_TRACING)
    # the parity rule's peak is the [T] cube's peak (the column cube here)
    assert_parity(gpu, orc, pix, **tol)
    assert float(orc["T"].max()) > 0.0
    for k in "CDB":
        assert np.all(gpu[k] == 0.0)

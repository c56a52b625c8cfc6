"""The large single render: a 512^3 grid with five FP16-stored fields (per-field
scales), 500 channels from -250 to +250 km/s at 1 km/s, z view, forward and
adjoint.  The oracle cannot render the whole cube in a test, so it checks
seeded samples: a 32 x 32 pixel window of the forward at full depth (FP32
parity rule on the stored values), and central differences of a mean(L^2)
loss on 20 cells per field for the adjoint (1e-3 relative)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from synth import DUST, LINE_13CO_21, View, make_fields_torch, workload  # noqa: E402
from tests.gpu_helpers import compare  # noqa: E402
from tests.test_gpu_adjoint import fd_rounding_floor, grad_floor  # noqa: E402

LINE = dict(LINE_13CO_21)
#: stored value x scale = physical value (density in 1e4 cm^-3, abundance in 1e-6)
SCALES = (1.0e4, 1.0, 1.0, 1.0, 1.0e-6)


@pytest.fixture(scope="module")
def big():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2607_01338_b300 as irt
    w = workload(4)
    f = make_fields_torch(w.n, w.seed)
    h = [(f[q] / SCALES[q]).to(torch.float16) for q in range(5)]
    del f
    torch.cuda.empty_cache()
    g = irt.Grid(*h, w.cell_cm, scales=SCALES)
    torch.cuda.synchronize()
    yield w, h, g
    g.close()


def _columns(h, cols):
    """The stored values of the columns [(x, y), ...] as FP64 physical fields
    of shape [nz, 1, ncol] (one oracle z-view ray per column)."""
    out = []
    for q in range(5):
        a = torch.stack([h[q][:, y, x] for (x, y) in cols], dim=1)
        out.append(np.ascontiguousarray((a.double().cpu().numpy() * SCALES[q])[:, None, :]))
    return out


def test_512cube_fp16_forward_on_a_32x32_window(big):
    """A 32 x 32 pixel window at a seeded offset, every channel, full depth."""
    import paper_2607_01338_b300 as irt
    w, h, g = big
    view, va = w.views[0], w.vaxis
    assert (w.n, va.nchan) == (512, 500)
    cubes = irt.forward(g, view, va, LINE, DUST)
    torch.cuda.synchronize()
    rng = np.random.default_rng(44)
    x0, y0 = (int(v) for v in rng.integers(0, w.n - 32, 2))
    fields = [np.ascontiguousarray(h[q][:, y0:y0 + 32, x0:x0 + 32].double().cpu().numpy()
                                   * SCALES[q]) for q in range(5)]
    mini = View(0.0, 0.0, 32, 32, w.cell_cm, 0)
    py, px = np.meshgrid(np.arange(32), np.arange(32), indexing="ij")
    pix = np.stack([px.ravel(), py.ravel()], axis=1)
    orc = oracle.render(fields, w.cell_cm, LINE, DUST, mini, va, pix)
    gpu = {k: cubes[k][:, y0:y0 + 32, x0:x0 + 32].double().cpu().numpy() for k in cubes}
    worst = compare(gpu, orc, pix)
    assert all(v <= 1.0 for v in worst.values()), worst
    # the line is present in the window
    assert float(np.abs(orc["L"]).max()) > 0.1


def test_512cube_fp16_adjoint_against_central_differences(big):
    import paper_2607_01338_b300 as irt
    w, h, g = big
    view, va = w.views[0], w.vaxis
    cubes = irt.forward(g, view, va, LINE, DUST, components=("L",))
    L = cubes["L"]
    ntot = L.numel()
    gn, gt, gv = irt.adjoint(g, view, va, LINE, DUST, {"L": 2.0 * L / ntot})
    torch.cuda.synchronize()
    del cubes, L
    rng = np.random.default_rng(45)
    cells = np.stack([rng.integers(0, w.n, 20), rng.integers(0, w.n, 20),
                      rng.integers(0, w.n, 20)], axis=1)
    one = View(0.0, 0.0, 1, 1, w.cell_cm, 0)
    pix0 = np.zeros((1, 2), dtype=int)
    for q, grad in ((0, gn), (1, gt), (3, gv)):
        fd, got, fl = [], [], []
        for (z, y, x) in cells:
            col = _columns(h, [(int(x), int(y))])
            v0 = col[q][z, 0, 0]
            eps = 1e-6 * max(abs(v0), 1.0)
            vals = []
            for sgn in (1.0, -1.0):
                col[q][z, 0, 0] = v0 + sgn * eps
                Lr = oracle.render(col, w.cell_cm, LINE, DUST, one, va, pix0)["L"][0]
                vals.append(np.sum(Lr * Lr))
                if sgn == 1.0:
                    fl.append(fd_rounding_floor(Lr, 0.0, w.n, eps, ntot))
            col[q][z, 0, 0] = v0
            fd.append((vals[0] - vals[1]) / (2.0 * eps) / ntot)
            got.append(float(grad[z, y, x]))
        fd, got, fl = np.array(fd), np.array(got), np.array(fl)
        # 1e-3 relative per cell; floors: the float32 rounding of the 512-step
        # recurrences and the FP64 rounding of the central difference
        allow = 1e-3 * np.abs(fd) + grad_floor(w.n) * np.abs(fd).max() + fl
        assert np.all(np.abs(got - fd) <= allow), (q, np.max(np.abs(got - fd) / allow))

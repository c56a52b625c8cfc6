"""The latitude-mean reduction (Sec. 6.1, irt_mean_axis1) against the FP64
oracle: float and double, the 16-byte vector path and the scalar path
(ragged or misaligned rows), the l-v image of a rendered cube and the
top-down map of a density field."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from synth import DUST, LINE_13CO_21, make_fields, to_storage, workload  # noqa: E402
from tests.gpu_helpers import torch_fields  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2607_01338_b300  # noqa: F401


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
@pytest.mark.parametrize("shape,offset", [((5, 37, 256), 0), ((3, 300, 131), 0),
                                          ((4, 64, 512), 1), ((1, 1, 1), 0),
                                          ((2, 1000, 4), 0)])
def test_mean_axis1_against_oracle(shape, offset, dtype):
    import paper_2607_01338_b300 as irt
    rng = np.random.default_rng(sum(shape))
    n = int(np.prod(shape))
    flat = torch.from_numpy(rng.uniform(0.5, 2.0, n + offset)).to(dtype).cuda()
    x = flat[offset:offset + n].view(*shape)   # offset 1: rows not 16-byte aligned
    got = irt.latitude_mean(x).double().cpu().numpy()
    exp = oracle.latitude_mean(x.double().cpu().numpy())
    tol = 2e-7 * np.sqrt(shape[1]) if dtype == torch.float32 else 1e-14
    np.testing.assert_allclose(got, exp, rtol=tol)


def test_lv_image_and_top_down_map_of_the_32cube():
    import paper_2607_01338_b300 as irt
    w = workload(0)
    fs = make_fields(w.n, w.seed)
    f32, deq = to_storage(fs, np.float32)
    g = irt.Grid(*torch_fields(f32), w.cell_cm)
    cube = irt.forward(g, w.views[0], w.vaxis, dict(LINE_13CO_21), DUST)["L"]
    torch.cuda.synchronize()
    g.close()
    u = irt.latitude_mean(cube).double().cpu().numpy()
    np.testing.assert_allclose(u, oracle.latitude_mean(cube.double().cpu().numpy()),
                               rtol=1e-6, atol=1e-6 * float(cube.abs().max()))
    dens = torch_fields(f32)[0]
    t = irt.latitude_mean(dens).double().cpu().numpy()
    np.testing.assert_allclose(t, oracle.latitude_mean(deq.n_h2), rtol=2e-6)
    assert u.shape == (w.vaxis.nchan, w.n) and t.shape == (w.n, w.n)


def test_mean_axis1_validation():
    import paper_2607_01338_b300 as irt
    from paper_2607_01338_b300 import binding as B
    x = torch.ones((2, 3, 4), device="cuda", dtype=torch.float16)
    with pytest.raises(ValueError):
        irt.latitude_mean(x)
    with pytest.raises(B.IrtError):
        B.irt_mean_axis1(x.data_ptr(), B.IRT_F16, 2, 3, 4, x.data_ptr())

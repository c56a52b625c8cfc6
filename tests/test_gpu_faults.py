"""Failure paths of the library on a GPU, made on the host (no GPU fault).

IRT_FAIL_ALLOC makes every device allocation of the library fail without
calling the CUDA runtime (host-side fault injection).  Each failing call must
report IRT_ENOMEM, leave the library and the device usable, and the same call
must succeed once the variable is cleared.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from synth import DUST, LINE_13CO_21, VelocityAxis, View, make_fields, to_storage  # noqa: E402
from tests.gpu_helpers import COMP, torch_fields  # noqa: E402

PC = 3.0856775814913673e18


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2607_01338_b300  # noqa: F401


def _fields(n=12, seed=31):
    f32, _ = to_storage(make_fields(n, seed), np.float32)
    return torch_fields(f32)


def test_create_grid_enomem_then_recovers(monkeypatch):
    import paper_2607_01338_b300 as irt
    from paper_2607_01338_b300.binding import IRT_ENOMEM, IrtError
    tf = _fields()
    monkeypatch.setenv("IRT_FAIL_ALLOC", "1")
    with pytest.raises(IrtError) as ei:
        irt.Grid(*tf, 0.1 * PC)
    assert ei.value.status == IRT_ENOMEM
    monkeypatch.delenv("IRT_FAIL_ALLOC")
    g = irt.Grid(*tf, 0.1 * PC)
    g.close()


def test_forward_scratch_growth_enomem_then_recovers(monkeypatch):
    """The record scratch of a stream grows with the longest ray it has
    rendered; rays of 2100 samples are longer than any other test renders, so
    the first such render on a side stream must grow it.  With allocation
    failing, the call reports IRT_ENOMEM and launches nothing; afterwards the
    same render on that stream equals the default stream's render bit for
    bit."""
    import paper_2607_01338_b300 as irt
    from paper_2607_01338_b300.binding import IRT_ENOMEM, IrtError
    rng = np.random.default_rng(5)
    nz, ny, nx = 2100, 6, 6
    n = 10.0 ** rng.uniform(2.0, 3.0, (nz, ny, nx))
    t = rng.uniform(20.0, 60.0, (nz, ny, nx))
    v = rng.uniform(-10.0, 10.0, (nz, ny, nx))
    x = np.full((nz, ny, nx), 2e-6)
    tf = [torch.from_numpy(a.astype(np.float32)).cuda() for a in (n, t, t, v, x)]
    dx = 0.01 * PC
    g = irt.Grid(*tf, dx)
    view = View(0.0, 0.0, nx, ny, dx, 0)
    va = VelocityAxis(40, -40.0, 2.0, 1)
    ref = irt.forward(g, view, va, LINE_13CO_21, DUST)
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    out = irt.alloc_cubes(view, va)
    for k in COMP:
        out[k].fill_(-7.0)
    torch.cuda.synchronize()
    monkeypatch.setenv("IRT_FAIL_ALLOC", "1")
    with pytest.raises(IrtError) as ei:
        irt.forward(g, view, va, LINE_13CO_21, DUST, out=out, stream=s)
    assert ei.value.status == IRT_ENOMEM
    torch.cuda.synchronize()
    assert all(bool((out[k] == -7.0).all()) for k in COMP), "a failed call wrote output"
    monkeypatch.delenv("IRT_FAIL_ALLOC")
    with torch.cuda.stream(s):
        irt.forward(g, view, va, LINE_13CO_21, DUST, out=out, stream=s)
    torch.cuda.synchronize()
    for k in COMP:
        assert torch.equal(out[k], ref[k]), k
    g.close()


def test_graph_create_enomem(monkeypatch):
    import paper_2607_01338_b300 as irt
    from paper_2607_01338_b300.binding import IRT_ENOMEM, IrtError
    tf = _fields()
    dx = 0.1 * PC
    g = irt.Grid(*tf, dx)
    view = View(0.0, 0.0, 12, 12, dx, 0)
    va = VelocityAxis(40, -40.0, 2.0, 1)
    monkeypatch.setenv("IRT_FAIL_ALLOC", "1")
    with pytest.raises(IrtError) as ei:
        irt.ForwardGraph([(g, view, va)], LINE_13CO_21, DUST)
    assert ei.value.status == IRT_ENOMEM
    monkeypatch.delenv("IRT_FAIL_ALLOC")
    gr = irt.ForwardGraph([(g, view, va)], LINE_13CO_21, DUST)
    outs = gr.launch()
    torch.cuda.synchronize()
    ref = irt.forward(g, view, va, LINE_13CO_21, DUST)
    torch.cuda.synchronize()
    for k in COMP:
        assert torch.equal(outs[0][k], ref[k]), k
    gr.close()
    g.close()

"""The allocation-free render entry point, irt_forward_ppv_static.

Some callers may not allocate device memory: a plugin whose host application
owns every device buffer, or a real-time loop that must neither wait on the
allocator nor risk running out of memory once it is running.  For them the
library packs the fields into a fixed device array it owns (32 MiB of cells,
16 MiB of sample records and 256 bytes of control words) instead of a grid
from irt_create_grid.  These tests
call that entry point through the C ABI and compare it with the regular path
(irt_create_grid + irt_forward_ppv) on two calls in a row, the second call
reusing the array the first one filled.
"""
import ctypes
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from synth import DUST, LINE_13CO_21, VelocityAxis, View, make_fields  # noqa: E402

PC = 3.0856775814913673e18
COMP = ("T", "C", "D", "L", "B")
RTOL, ATOL_FRAC = 1e-5, 1e-6   # the FP32 rule of the parity tests


def _fields(shape, seed):
    nz, ny, nx = shape
    fs = make_fields(max(shape), seed)
    return [torch.from_numpy(np.ascontiguousarray(a[:nz, :ny, :nx]).astype(np.float32)).cuda()
            for a in fs.as_tuple()]


_TORCH_TO_IRT = {torch.float32: 0, torch.float16: 1, torch.bfloat16: 2, torch.float64: 3}


def _static_render(B, api, ts, dx, view, vaxis, integration, scales=None, out=None):
    nz, ny, nx = ts[0].shape
    if out is None:
        out = api.alloc_cubes(view, vaxis)
    sc = [1.0] * 5 if scales is None else list(scales)
    desc = B.irt_grid_desc(nx, ny, nz, dx,
                           (ctypes.c_int * 5)(*[_TORCH_TO_IRT[t.dtype] for t in ts]),
                           (ctypes.c_double * 5)(*sc))
    fields = B.irt_fields(*[t.data_ptr() for t in ts])
    B.irt_forward_ppv_static(desc, fields, api.view_struct(view), api.vaxis_struct(vaxis),
                             api._cubes_struct(out), api.line_struct(LINE_13CO_21),
                             api.dust_struct(DUST), api.opts_struct(integration),
                             int(torch.cuda.current_stream().cuda_stream))
    return out


def _assert_fp32_rule(got, ref, what):
    peak = ref["T"].abs().max().item()
    for k in COMP:
        a, b = got[k].double(), ref[k].double()
        allow = torch.clamp(RTOL * b.abs(), min=ATOL_FRAC * peak)
        worst = ((a - b).abs() / allow).max().item()
        assert worst <= 1.0, (what, k, worst)


def test_static_entry_matches_regular_entry_on_two_calls():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2607_01338_b300 as irt
    from paper_2607_01338_b300 import api
    from paper_2607_01338_b300 import binding as B

    dx = 0.1 * PC
    cases = [((20, 18, 22), 901, View(0.0, 0.0, 22, 18, dx, 0), VelocityAxis(90, -90.0, 2.0, 1),
              "smooth"),
             ((26, 24, 16), 902, View(math.radians(35.0), math.radians(120.0), 30, 26, dx, 1),
              VelocityAxis(64, -64.0, 2.0, 2), "formal")]
    for shape, seed, view, va, integration in cases:
        ts = _fields(shape, seed)
        got = _static_render(B, api, ts, dx, view, va, integration)
        g = irt.Grid(*ts, dx)
        ref = irt.forward(g, view, va, LINE_13CO_21, DUST, integration=integration)
        torch.cuda.synchronize()
        _assert_fp32_rule(got, ref, shape)
        g.close()


def test_static_entry_16bit_storage_with_scales_and_no_device_allocation():
    """Half-precision storage (fp16 density and abundance with per-field
    scales, bf16 temperatures, fp16 velocity) goes through the 16-bit cell
    path of the static entry; it must agree with irt_create_grid +
    irt_forward_ppv on the same stored values, on two calls in a row.  The
    second call must not change the device's free memory (the entry
    allocates nothing; the first call has loaded the kernels)."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2607_01338_b300 as irt
    from paper_2607_01338_b300 import api
    from paper_2607_01338_b300 import binding as B

    dx = 0.1 * PC
    shape = (24, 20, 18)
    base = _fields(shape, 903)
    scales = [1.0e4, 1.0, 1.0, 1.0, 1.0e-6]
    dts = [torch.float16, torch.bfloat16, torch.bfloat16, torch.float16, torch.float16]
    ts = [(t / s).to(d).contiguous() for t, s, d in zip(base, scales, dts)]
    view = View(math.radians(25.0), math.radians(60.0), 26, 22, dx, 1)
    va = VelocityAxis(72, -72.0, 2.0, 1)
    g = irt.Grid(*ts, dx, scales=scales)
    ref = irt.forward(g, view, va, LINE_13CO_21, DUST, integration="smooth")
    out = api.alloc_cubes(view, va)
    torch.cuda.synchronize()
    _static_render(B, api, ts, dx, view, va, "smooth", scales=scales, out=out)
    torch.cuda.synchronize()
    _assert_fp32_rule(out, ref, "first call")
    for k in COMP:
        out[k].zero_()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    _static_render(B, api, ts, dx, view, va, "smooth", scales=scales, out=out)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, f"device free memory changed by {free0 - free1} bytes"
    _assert_fp32_rule(out, ref, "second call")
    g.close()


def test_static_entry_rejects_grids_beyond_its_array():
    from paper_2607_01338_b300 import api
    from paper_2607_01338_b300 import binding as B
    # 128^3 float cells need 64 MiB of packed cells: beyond the 32 MiB array.
    # The size check runs before any device work, so dummy pointers suffice.
    desc = B.irt_grid_desc(128, 128, 128, 1.0, (ctypes.c_int * 5)(*[B.IRT_F32] * 5),
                           (ctypes.c_double * 5)(*[1.0] * 5))
    fields = B.irt_fields(16, 16, 16, 16, 16)
    view = View(0.0, 0.0, 128, 128, 1.0, 0)
    va = VelocityAxis(8, -8.0, 2.0, 1)
    status = B.lib.irt_forward_ppv_static(
        ctypes.byref(desc), ctypes.byref(fields), ctypes.byref(api.view_struct(view)),
        ctypes.byref(api.vaxis_struct(va)), ctypes.byref(B.irt_cubes(16, None, None, None, None)),
        ctypes.byref(api.line_struct(LINE_13CO_21)), ctypes.byref(api.dust_struct(DUST)),
        ctypes.byref(api.opts_struct("smooth")), None)
    assert status == B.IRT_EINVAL
    msg = B.lib.irt_last_error().decode()
    assert "static scratch holds at most" in msg and "67108864" in msg

"""Shared helpers of the GPU parity tests (CUDA path vs FP64 oracle)."""
from __future__ import annotations

import numpy as np
import torch

import oracle
from synth import FieldSet

COMP = ("T", "C", "D", "L", "B")

#: FP32 parity rule: per voxel |gpu - oracle| <= max(RTOL |oracle|, ATOL_FRAC * peak)
#: with peak = max |[T]| of the oracle cube (the brightness peak).
RTOL_F32 = 1e-5
ATOL_FRAC_F32 = 1e-6


def torch_fields(fs: FieldSet, dtypes=None):
    """FieldSet (numpy) -> five CUDA tensors.  ``dtypes`` entries: torch dtypes;
    uint16 numpy arrays are taken as bfloat16 bit patterns."""
    out = []
    for i, a in enumerate(fs.as_tuple()):
        if a.dtype == np.uint16:
            t = torch.from_numpy(a.view(np.int16).copy()).view(torch.bfloat16)
        else:
            t = torch.from_numpy(np.ascontiguousarray(a))
        if dtypes is not None:
            t = t.to(dtypes[i])
        out.append(t.cuda())
    return out


def gpu_render(fields_t, cell_cm, view, vaxis, line, dust, **kw):
    import paper_2607_01338_b300 as irt
    g = irt.Grid(*fields_t, cell_cm)
    cubes = irt.forward(g, view, vaxis, line, dust, **kw)
    torch.cuda.synchronize()
    res = {k: cubes[k].double().cpu().numpy() for k in COMP}
    g.close()
    return res


def crop_pixels(npx, npy, w, h, seed):
    rng = np.random.default_rng(seed)
    x0 = int(rng.integers(0, npx - w + 1))
    y0 = int(rng.integers(0, npy - h + 1))
    py, px = np.meshgrid(np.arange(y0, y0 + h), np.arange(x0, x0 + w), indexing="ij")
    return np.stack([px.ravel(), py.ravel()], axis=1)


def oracle_pixels(fields64, cell_cm, view, vaxis, line, dust, pix, integration="smooth",
                  units="trj", t_bg=2.725):
    mode = {"smooth": oracle.SMOOTH, "formal": oracle.FORMAL, "formal_kahan": oracle.FORMAL}[
        integration]
    u = {"trj": oracle.TRJ, "intensity": oracle.INTENSITY, "tb": oracle.TB}[units]
    return oracle.render(fields64, cell_cm, line, dust, view, vaxis, pix, integration=mode,
                         units=u, t_bg=t_bg)


def compare(gpu: dict, orc: dict, pix, rtol=RTOL_F32, atol_frac=ATOL_FRAC_F32, chan=None):
    """Worst ratio error / allowance per component (<= 1 passes)."""
    px, py = pix[:, 0], pix[:, 1]
    peak = np.abs(orc["T"]).max()
    worst = {}
    for k in COMP:
        g = gpu[k][:, py, px].T          # [npix, nchan]
        o = orc[k]
        if chan is not None:
            g, o = g[:, chan], o[:, chan]
        allow = np.maximum(rtol * np.abs(o), atol_frac * peak)
        r = np.abs(g - o) / allow
        worst[k] = float(r.max()) if r.size else 0.0
    return worst


def rel_err_stats(gpu: dict, orc: dict, pix):
    """Max absolute and relative-to-peak errors per component (reporting)."""
    px, py = pix[:, 0], pix[:, 1]
    peak = np.abs(orc["T"]).max()
    out = {}
    for k in COMP:
        d = np.abs(gpu[k][:, py, px].T - orc[k])
        out[k] = dict(max_abs=float(d.max()), max_over_peak=float(d.max() / peak))
    return out


def assert_parity(gpu, orc, pix, **kw):
    w = compare(gpu, orc, pix, **kw)
    bad = {k: v for k, v in w.items() if not v <= 1.0}
    assert not bad, f"parity violated (error / allowance): {w}"
    return w

"""PyTorch-facing wrappers of the C ABI: device memory and streams come from
torch, every computation runs in the CUDA library (argument marshalling only).
"""
from __future__ import annotations

from dataclasses import dataclass

import torch

from . import binding as B

_DTYPE = {torch.float32: B.IRT_F32, torch.float16: B.IRT_F16, torch.bfloat16: B.IRT_BF16,
          torch.float64: B.IRT_F64}
_INTEGRATION = {"formal": B.IRT_FORMAL, "smooth": B.IRT_SMOOTH, "formal_kahan": B.IRT_FORMAL_KAHAN}
_UNITS = {"trj": B.IRT_UNITS_TRJ, "intensity": B.IRT_UNITS_INTENSITY, "tb": B.IRT_UNITS_TB}
_PREC = {"f32": B.IRT_PREC_F32, "f64": B.IRT_PREC_F64}
_TRANSFER = {"thick": B.IRT_MODE_THICK, "selectively_thin": B.IRT_MODE_SELECTIVELY_THIN,
             "thin": B.IRT_MODE_THIN, "density_tracing": B.IRT_MODE_DENSITY_TRACING}
COMPONENTS = ("T", "C", "D", "L", "B")


def _stream_ptr(stream=None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


class Grid:
    """Fields copied into a library-owned grid (``irt_create_grid``).

    The five tensors are CUDA tensors of shape (nz, ny, nx), C contiguous,
    dtype float32 / float16 / bfloat16 / float64 (each field may differ).
    ``scales``: physical value = stored value * scale, per field."""

    def __init__(self, n_h2, t_gas, t_dust, v_los, x_tracer, cell_cm: float, stream=None,
                 scales=None):
        ts = [n_h2, t_gas, t_dust, v_los, x_tracer]
        shape = ts[0].shape
        for t in ts:
            if not t.is_cuda:
                raise ValueError("fields must be CUDA tensors")
            if t.shape != shape or t.dim() != 3:
                raise ValueError("fields must share one (nz, ny, nx) shape")
            if t.dtype not in _DTYPE:
                raise ValueError(f"unsupported field dtype {t.dtype}")
        ts = [t.contiguous() for t in ts]
        nz, ny, nx = shape
        self.scales = [1.0] * 5 if scales is None else [float(x) for x in scales]
        desc, fields = self._desc(ts, float(cell_cm))
        self.handle = B.irt_create_grid(desc, fields, _stream_ptr(stream))
        self._keep = ts   # the pack kernel reads them on the stream
        self.shape = (nz, ny, nx)
        self.cell_cm = float(cell_cm)
        self.dtypes = tuple(t.dtype for t in ts)

    def _desc(self, ts, cell_cm):
        nz, ny, nx = ts[0].shape
        desc = B.irt_grid_desc(nx, ny, nz, cell_cm,
                               (B.ctypes.c_int * 5)(*[_DTYPE[t.dtype] for t in ts]),
                               (B.ctypes.c_double * 5)(*self.scales))
        return desc, B.irt_fields(*[t.data_ptr() for t in ts])

    def update(self, n_h2, t_gas, t_dust, v_los, x_tracer, stream=None):
        """New field values of the same shape and dtypes (``irt_update_grid``:
        no allocation, asynchronous on the stream)."""
        ts = [t.contiguous() for t in (n_h2, t_gas, t_dust, v_los, x_tracer)]
        if tuple(ts[0].shape) != self.shape or tuple(t.dtype for t in ts) != self.dtypes:
            raise ValueError("update needs the grid's shape and dtypes")
        desc, fields = self._desc(ts, self.cell_cm)
        B.irt_update_grid(self.handle, desc, fields, _stream_ptr(stream))
        self._keep = ts

    def set_h2_fraction(self, chi: torch.Tensor, stream=None):
        """H2 abundance per H nucleus of every cell ([nz, ny, nx] CUDA tensor),
        read by the optically thin level balance (``irt_grid_set_h2_fraction``;
        default 0.5, fully molecular)."""
        if not chi.is_cuda or tuple(chi.shape) != self.shape or chi.dtype not in _DTYPE:
            raise ValueError("chi must be a CUDA tensor of the grid's shape")
        chi = chi.contiguous()
        B.irt_grid_set_h2_fraction(self.handle, chi.data_ptr(), _DTYPE[chi.dtype],
                                   _stream_ptr(stream))
        self._chi = chi   # read on the stream

    def close(self):
        if getattr(self, "handle", None):
            torch.cuda.synchronize()
            B.irt_destroy(self.handle)
            self.handle = None
            self._keep = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class LevelTable:
    """Optically thin level-balance grid (``irt_create_ot_table``, Sec. 4.2)
    of the radiative transitions ``lines`` of a level model (a dict of
    arrays: nlev, energy_k, g, rad_up, rad_lo, a_ul_s, nu_hz, partner,
    coll_temp_k [partner, t], coll_up / coll_lo [partner, c], k_ul_cm3_s
    [partner, c, t], t_rad_k, ortho_para, x_he) on the grid ``axes`` (n_n,
    n_chi, n_t and the log10 n_H, chi, log10 T ranges)."""

    def __init__(self, model: dict, axes: dict, lines, stream=None):
        import numpy as np
        d = lambda k: np.ascontiguousarray(np.asarray(model[k], dtype=np.float64))  # noqa: E731
        i = lambda k: np.ascontiguousarray(np.asarray(model[k], dtype=np.int32))    # noqa: E731
        keep = dict(energy_k=d("energy_k"), g=d("g"), rad_up=i("rad_up"), rad_lo=i("rad_lo"),
                    a=d("a_ul_s"), nu=d("nu_hz"), partner=i("partner"),
                    ct=d("coll_temp_k"), cu=i("coll_up"), cl=i("coll_lo"), k=d("k_ul_cm3_s"))
        dp = lambda a: a.ctypes.data_as(B._DP)   # noqa: E731
        ip = lambda a: a.ctypes.data_as(B._IP)   # noqa: E731
        m = B.irt_level_model(int(model["nlev"]), dp(keep["energy_k"]), dp(keep["g"]),
                              len(keep["rad_up"]), ip(keep["rad_up"]), ip(keep["rad_lo"]),
                              dp(keep["a"]), dp(keep["nu"]), len(keep["partner"]),
                              ip(keep["partner"]), int(keep["ct"].shape[-1]), dp(keep["ct"]),
                              int(keep["cu"].shape[-1]), ip(keep["cu"]), ip(keep["cl"]),
                              dp(keep["k"]), float(model["t_rad_k"]),
                              float(model["ortho_para"]), float(model["x_he"]))
        ax = B.irt_ot_axes(int(axes["n_n"]), int(axes["n_chi"]), int(axes["n_t"]),
                           float(axes["log10_nh_min"]), float(axes["log10_nh_max"]),
                           float(axes["chi_min"]), float(axes["chi_max"]),
                           float(axes["log10_t_min"]), float(axes["log10_t_max"]))
        self.shape = (len(lines), int(axes["n_n"]), int(axes["n_chi"]), int(axes["n_t"]), 2)
        self.nu_hz = [float(model["nu_hz"][q]) for q in lines]
        self.handle = B.irt_create_ot_table(m, ax, list(lines), _stream_ptr(stream))

    def values(self):
        """The grid, [nlines, n_n, n_chi, n_t, 2] float64 numpy array of (j,
        alpha) per tracer molecule [cgs] (synchronous)."""
        import numpy as np
        out = np.zeros(self.shape)
        B.irt_ot_table_values(self.handle, out.ctypes.data)
        return out

    def close(self):
        if getattr(self, "handle", None):
            torch.cuda.synchronize()
            B.irt_destroy_ot_table(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def line_struct(line: dict) -> B.irt_line:
    return B.irt_line(*[float(line[k]) for k, _ in B.irt_line._fields_])


def dust_struct(dust: dict) -> B.irt_dust:
    return B.irt_dust(float(dust["kappa_cm2_per_g_gas"]), float(dust["mu_mass_per_h2_amu"]))


def view_struct(view) -> B.irt_view:
    return B.irt_view(float(view.theta_rad), float(view.phi_rad), int(view.npx), int(view.npy),
                      float(view.pixel_cm), int(view.trilinear))


def vaxis_struct(va) -> B.irt_vaxis:
    return B.irt_vaxis(int(va.nchan), float(va.v_first_edge_kms), float(va.dv_kms),
                       int(va.subsample_f))


def opts_struct(integration="smooth", units="trj", t_bg=2.725, precision="f32",
                flags=0, transfer="thick") -> B.irt_opts:
    return B.irt_opts(_TRANSFER[transfer], _INTEGRATION[integration], _UNITS[units], float(t_bg),
                      _PREC[precision], int(flags))


def alloc_cubes(view, vaxis, precision="f32", device=None, components=COMPONENTS):
    dt = torch.float64 if precision == "f64" else torch.float32
    dev = device or torch.device("cuda")
    return {k: torch.empty((vaxis.nchan, view.npy, view.npx), dtype=dt, device=dev)
            for k in components}


def _cubes_struct(cubes: dict) -> B.irt_cubes:
    return B.irt_cubes(*[cubes[k].data_ptr() if cubes.get(k) is not None else None
                         for k in COMPONENTS])


def make_job(grid: Grid, view, vaxis, cubes: dict) -> B.irt_job:
    return B.irt_job(grid.handle, view_struct(view), vaxis_struct(vaxis), _cubes_struct(cubes))


def forward(grid: Grid, view, vaxis, line: dict, dust: dict, *, integration="smooth",
            units="trj", t_bg=2.725, precision="f32", flags=0, out=None, stream=None,
            components=COMPONENTS, transfer="thick", levels: LevelTable = None,
            line_index: int = 0) -> dict:
    """Render one job (``irt_forward_ppv`` with njobs = 1).  Returns the cubes
    {"T","C","D","L","B"} as [nchan, npy, npx] tensors.  ``transfer`` is
    "thick", "selectively_thin", "thin" (Sec. 4.5-4.7) or "density_tracing"
    (Sec. 5.10: the column density per unit velocity in "T" and "L").
    ``levels``: a LevelTable whose line ``line_index`` gives the level
    populations (optically thin balance, ``irt_forward_ppv_ot``) instead of
    LTE."""
    cubes = out if out is not None else alloc_cubes(view, vaxis, precision,
                                                     components=components)
    job = make_job(grid, view, vaxis, cubes)
    opts = opts_struct(integration, units, t_bg, precision, flags, transfer)
    if levels is not None:
        B.irt_forward_ppv_ot([job], levels.handle, line_index, line_struct(line),
                             dust_struct(dust), opts, _stream_ptr(stream))
    else:
        B.irt_forward_ppv([job], line_struct(line), dust_struct(dust), opts, _stream_ptr(stream))
    return cubes


def forward_lines(grid: Grid, view, vaxis, lines, dusts, *, integration="smooth", units="trj",
                  t_bg=2.725, flags=0, outs=None, stream=None, levels: LevelTable = None,
                  line_indices=None) -> list:
    """Render several lines of one job in one launch (``irt_forward_ppv_lines``):
    ``lines`` and ``dusts`` are sequences of line and dust dicts (one dust
    per line: its own opacity); returns one cube dict per line.  With
    ``levels`` (a LevelTable) line q takes grid line ``line_indices[q]``."""
    if outs is None:
        outs = [alloc_cubes(view, vaxis) for _ in lines]
    job = make_job(grid, view, vaxis, {k: None for k in COMPONENTS})
    B.irt_forward_ppv_lines(job, [line_struct(x) for x in lines], [dust_struct(d) for d in dusts],
                            [_cubes_struct(o) for o in outs],
                            None if levels is None else levels.handle,
                            None if levels is None else list(line_indices),
                            opts_struct(integration, units, t_bg, "f32", flags),
                            _stream_ptr(stream))
    return outs


def latitude_mean(x: torch.Tensor, stream=None) -> torch.Tensor:
    """Mean over the middle axis of a [A, B, C] CUDA tensor (Sec. 6.1): the
    l-v image u of a PPV cube [nchan, npy, npx], or the top-down map t of a
    field [nz, ny, nx].  ``irt_mean_axis1``; float32 or float64."""
    if x.dim() != 3 or not x.is_cuda:
        raise ValueError("latitude_mean takes a 3-D CUDA tensor")
    x = x.contiguous()
    if x.dtype not in (torch.float32, torch.float64):
        raise ValueError("latitude_mean takes float32 or float64")
    out = torch.empty((x.shape[0], x.shape[2]), dtype=x.dtype, device=x.device)
    dt = B.IRT_F32 if x.dtype == torch.float32 else B.IRT_F64
    B.irt_mean_axis1(x.data_ptr(), dt, x.shape[0], x.shape[1], x.shape[2], out.data_ptr(),
                     _stream_ptr(stream))
    return out


def beam_convolve(cube: torch.Tensor, fwhm_px: float, out=None, stream=None) -> torch.Tensor:
    """Gaussian beam convolution of a [nchan, npy, npx] CUDA cube (Sec. 4.11)
    with the beam FWHM given in pixels (``irt_beam_convolve``)."""
    if cube.dim() != 3 or not cube.is_cuda or cube.dtype not in (torch.float32, torch.float64):
        raise ValueError("beam_convolve takes a 3-D float32/float64 CUDA tensor")
    cube = cube.contiguous()
    scratch = torch.empty_like(cube)
    out = torch.empty_like(cube) if out is None else out
    dt = B.IRT_F32 if cube.dtype == torch.float32 else B.IRT_F64
    B.irt_beam_convolve(cube.data_ptr(), dt, cube.shape[0], cube.shape[1], cube.shape[2],
                        float(fwhm_px), scratch.data_ptr(), out.data_ptr(), _stream_ptr(stream))
    return out


def forward_batch(jobs, line: dict, dust: dict, *, integration="smooth", units="trj",
                  t_bg=2.725, precision="f32", flags=0, outs=None, stream=None,
                  autotune=False, transfer="thick") -> list:
    """Render many jobs in one persistent launch.  ``jobs`` = [(grid, view,
    vaxis), ...]; returns one cube dict per job.  ``autotune`` times the
    launch plans for this job mix first (synchronous) and caches the best."""
    if outs is None:
        outs = [alloc_cubes(v, va, precision) for (_, v, va) in jobs]
    cj = [make_job(g, v, va, o) for (g, v, va), o in zip(jobs, outs)]
    if autotune:
        flags |= B.IRT_FLAG_AUTOTUNE
    B.irt_forward_ppv(cj, line_struct(line), dust_struct(dust),
                      opts_struct(integration, units, t_bg, precision, flags, transfer),
                      _stream_ptr(stream))
    return outs


class ForwardGraph:
    """A CUDA graph of one batched render (``irt_forward_graph_create``).
    The grids and output cubes must outlive it; ``launch`` re-renders them."""

    def __init__(self, jobs, line: dict, dust: dict, *, integration="smooth", units="trj",
                 t_bg=2.725, precision="f32", flags=0, outs=None, autotune=False):
        if outs is None:
            outs = [alloc_cubes(v, va, precision) for (_, v, va) in jobs]
        self.outs = outs
        self._keep = list(jobs)
        cj = [make_job(g, v, va, o) for (g, v, va), o in zip(jobs, outs)]
        if autotune:
            flags |= B.IRT_FLAG_AUTOTUNE
        self.opts = opts_struct(integration, units, t_bg, precision, flags)
        self._jobs = cj
        self.handle = B.irt_forward_graph_create(cj, line_struct(line), dust_struct(dust),
                                                 self.opts)

    def plan(self):
        """(NI, tile width, tile height) used by the graph's launch plan."""
        return B.irt_tuned_plan(self._jobs, self.opts)

    def launch(self, stream=None):
        B.irt_forward_graph_launch(self.handle, _stream_ptr(stream))
        return self.outs

    def close(self):
        if getattr(self, "handle", None):
            torch.cuda.synchronize()
            B.irt_forward_graph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def adjoint(grid: Grid, view, vaxis, line: dict, dust: dict, cotangent: dict, *,
            integration="smooth", units="trj", t_bg=2.725, flags=0, grads=None, stream=None):
    """Gradients of a loss with respect to n_H2, T_gas, v_los (z view) given
    the cotangent cubes (``irt_adjoint_ppv``).  Returns (g_n, g_t, g_v)."""
    nz, ny, nx = grid.shape
    if grads is None:
        grads = tuple(torch.empty((nz, ny, nx), dtype=torch.float32, device="cuda")
                      for _ in range(3))
    cot = {k: (cotangent[k].contiguous() if cotangent.get(k) is not None else None)
           for k in COMPONENTS}
    job = make_job(grid, view, vaxis, {k: None for k in COMPONENTS})
    B.irt_adjoint_ppv(job, line_struct(line), dust_struct(dust),
                      opts_struct(integration, units, t_bg, "f32", flags), _cubes_struct(cot),
                      grads[0].data_ptr(), grads[1].data_ptr(), grads[2].data_ptr(),
                      _stream_ptr(stream))
    return grads


@dataclass
class RenderConfig:
    """Everything but the differentiable fields of an autograd render."""
    cell_cm: float
    view: object
    vaxis: object
    line: dict
    dust: dict
    integration: str = "smooth"
    units: str = "trj"
    t_bg: float = 2.725


# Grids of the autograd function, reused across calls: keyed by (device,
# stream, shape, cell size); a grid goes back to the pool when its backward
# has been enqueued (launches on one stream run in order, so the next
# forward's field update waits for that adjoint without a host sync).
_GRID_POOL = {}


def _pooled_grid(fields, cell_cm):
    key = (fields[0].device, torch.cuda.current_stream().cuda_stream, tuple(fields[0].shape),
           float(cell_cm))
    free = _GRID_POOL.get(key)
    if free:
        g = free.pop()
        g.update(*fields)
    else:
        g = Grid(*fields, cell_cm)
    g._pool_key = key
    return g


def _release_grid(g):
    _GRID_POOL.setdefault(g._pool_key, []).append(g)


class RenderPPV(torch.autograd.Function):
    """Differentiable render: (n_H2, T_gas, v_los, T_dust, x) -> the five
    cubes of any view; gradients flow to n_H2, T_gas and v_los through the
    hand-written adjoint kernels.  The library grid comes from a per-stream
    pool and returns to it after backward (no device synchronisation)."""

    @staticmethod
    def forward(ctx, n_h2, t_gas, v_los, t_dust, x_tracer, cfg: RenderConfig):
        grid = _pooled_grid([n_h2.detach().float(), t_gas.detach().float(),
                             t_dust.detach().float(), v_los.detach().float(),
                             x_tracer.detach().float()], cfg.cell_cm)
        # the z- and radial-view smooth renders keep their transfer
        # checkpoints in the grid, so that backward skips re-integrating the
        # forward
        save = (cfg.integration == "smooth" and int(cfg.view.trilinear) != 1)
        cubes = forward(grid, cfg.view, cfg.vaxis, cfg.line, cfg.dust,
                        integration=cfg.integration, units=cfg.units, t_bg=cfg.t_bg,
                        flags=B.IRT_FLAG_SAVE_CHECKPOINTS if save else 0)
        ctx.grid = grid
        ctx.cfg = cfg
        return tuple(cubes[k] for k in COMPONENTS)

    @staticmethod
    def backward(ctx, gT, gC, gD, gL, gB):
        cfg = ctx.cfg
        cot = dict(T=gT, C=gC, D=gD, L=gL, B=gB)
        gn, gt, gv = adjoint(ctx.grid, cfg.view, cfg.vaxis, cfg.line, cfg.dust, cot,
                             integration=cfg.integration, units=cfg.units, t_bg=cfg.t_bg)
        _release_grid(ctx.grid)
        ctx.grid = None
        return gn, gt, gv, None, None, None


def render_ppv(n_h2, t_gas, v_los, t_dust, x_tracer, cfg: RenderConfig):
    return RenderPPV.apply(n_h2, t_gas, v_los, t_dust, x_tracer, cfg)

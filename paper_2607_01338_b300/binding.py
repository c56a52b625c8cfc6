"""ctypes binding of the C ABI in include/irt.h (argument marshalling only).

The four entry points keep their C names: :func:`irt_create_grid`,
:func:`irt_forward_ppv`, :func:`irt_adjoint_ppv`, :func:`irt_destroy`.  Every
step of the computation runs in the CUDA library; if ``libirt.so`` is absent
importing this module raises, there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libirt.so")

IRT_OK, IRT_EINVAL, IRT_ENOMEM, IRT_ECUDA, IRT_EUNSUPPORTED, IRT_ETIMEOUT = range(6)
IRT_F32, IRT_F16, IRT_BF16, IRT_F64 = range(4)
IRT_FORMAL, IRT_SMOOTH, IRT_FORMAL_KAHAN = range(3)
IRT_UNITS_TRJ, IRT_UNITS_INTENSITY, IRT_UNITS_TB = range(3)
IRT_PREC_F32, IRT_PREC_F64 = range(2)
IRT_MODE_THICK = 0
IRT_MODE_SELECTIVELY_THIN = 1
IRT_MODE_THIN = 2
IRT_MODE_DENSITY_TRACING = 3
IRT_FLAG_EXPLICIT_CHANNELS = 1
IRT_FLAG_STATS = 2
IRT_FLAG_AUTOTUNE = 4
IRT_FLAG_SAVE_CHECKPOINTS = 8

STATUS_NAMES = {0: "IRT_OK", 1: "IRT_EINVAL", 2: "IRT_ENOMEM", 3: "IRT_ECUDA",
                4: "IRT_EUNSUPPORTED", 5: "IRT_ETIMEOUT"}

#: symbols include/irt.h declares
EXPORTED = ("irt_create_grid", "irt_forward_ppv", "irt_adjoint_ppv", "irt_destroy",
            "irt_grid_stats", "irt_forward_ppv_static", "irt_forward_graph_create",
            "irt_forward_graph_launch", "irt_forward_graph_destroy", "irt_tuned_plan",
            "irt_last_error", "irt_launch_count", "irt_measure_pipe_peaks", "irt_mean_axis1",
            "irt_beam_convolve", "irt_create_ot_table", "irt_ot_table_values",
            "irt_destroy_ot_table", "irt_grid_set_h2_fraction", "irt_forward_ppv_ot",
            "irt_forward_ppv_lines", "irt_update_grid")
IRT_PARTNER_H2, IRT_PARTNER_PH2, IRT_PARTNER_OH2, IRT_PARTNER_H, IRT_PARTNER_HE = range(5)


class irt_grid_desc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("cell_cm", ctypes.c_double), ("dtype", ctypes.c_int * 5),
                ("scale", ctypes.c_double * 5)]


class irt_fields(ctypes.Structure):
    _fields_ = [("n_h2_cm3", ctypes.c_void_p), ("t_gas_k", ctypes.c_void_p),
                ("t_dust_k", ctypes.c_void_p), ("v_los_kms", ctypes.c_void_p),
                ("x_tracer", ctypes.c_void_p)]


class irt_line(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in (
        "nu_ul_hz", "a_ul_s", "e_u_k", "b0_hz", "g_u", "g_l", "mass_amu", "t_inf_k",
        "sigma_turb_kms")]


class irt_dust(ctypes.Structure):
    _fields_ = [("kappa_cm2_per_g_gas", ctypes.c_double), ("mu_mass_per_h2_amu", ctypes.c_double)]


class irt_view(ctypes.Structure):
    _fields_ = [("theta_rad", ctypes.c_double), ("phi_rad", ctypes.c_double),
                ("npx", ctypes.c_int), ("npy", ctypes.c_int), ("pixel_cm", ctypes.c_double),
                ("trilinear", ctypes.c_int)]


class irt_vaxis(ctypes.Structure):
    _fields_ = [("nchan", ctypes.c_int), ("v_first_edge_kms", ctypes.c_double),
                ("dv_kms", ctypes.c_double), ("subsample_f", ctypes.c_int)]


class irt_opts(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int), ("integration", ctypes.c_int), ("units", ctypes.c_int),
                ("t_bg_k", ctypes.c_double), ("precision", ctypes.c_int),
                ("flags", ctypes.c_uint)]


class irt_cubes(ctypes.Structure):
    _fields_ = [("T", ctypes.c_void_p), ("C", ctypes.c_void_p), ("D", ctypes.c_void_p),
                ("L", ctypes.c_void_p), ("B", ctypes.c_void_p)]


class irt_job(ctypes.Structure):
    _fields_ = [("grid", ctypes.c_void_p), ("view", irt_view), ("vaxis", irt_vaxis),
                ("out", irt_cubes)]


_DP = ctypes.POINTER(ctypes.c_double)
_IP = ctypes.POINTER(ctypes.c_int)


class irt_level_model(ctypes.Structure):
    _fields_ = [("nlev", ctypes.c_int), ("energy_k", _DP), ("g", _DP), ("nrad", ctypes.c_int),
                ("rad_up", _IP), ("rad_lo", _IP), ("a_ul_s", _DP), ("nu_hz", _DP),
                ("npartner", ctypes.c_int), ("partner", _IP), ("ntemp", ctypes.c_int),
                ("coll_temp_k", _DP), ("ncoll", ctypes.c_int), ("coll_up", _IP),
                ("coll_lo", _IP), ("k_ul_cm3_s", _DP), ("t_rad_k", ctypes.c_double),
                ("ortho_para", ctypes.c_double), ("x_he", ctypes.c_double)]


class irt_ot_axes(ctypes.Structure):
    _fields_ = [("n_n", ctypes.c_int), ("n_chi", ctypes.c_int), ("n_t", ctypes.c_int),
                ("log10_nh_min", ctypes.c_double), ("log10_nh_max", ctypes.c_double),
                ("chi_min", ctypes.c_double), ("chi_max", ctypes.c_double),
                ("log10_t_min", ctypes.c_double), ("log10_t_max", ctypes.c_double)]


class IrtError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"CUDA library {LIB_PATH} is missing: build it with "
                          "`python -m paper_2607_01338_b300.build` (needs nvcc)")
    L = ctypes.CDLL(LIB_PATH)
    P = ctypes.POINTER
    L.irt_create_grid.restype = ctypes.c_int
    L.irt_create_grid.argtypes = [P(irt_grid_desc), P(irt_fields), ctypes.c_void_p,
                                  P(ctypes.c_void_p)]
    L.irt_forward_ppv.restype = ctypes.c_int
    L.irt_forward_ppv.argtypes = [P(irt_job), ctypes.c_int, P(irt_line), P(irt_dust),
                                  P(irt_opts), ctypes.c_void_p]
    L.irt_adjoint_ppv.restype = ctypes.c_int
    L.irt_adjoint_ppv.argtypes = [P(irt_job), P(irt_line), P(irt_dust), P(irt_opts),
                                  P(irt_cubes), ctypes.c_void_p, ctypes.c_void_p,
                                  ctypes.c_void_p, ctypes.c_void_p]
    L.irt_destroy.restype = ctypes.c_int
    L.irt_destroy.argtypes = [ctypes.c_void_p]
    L.irt_forward_ppv_static.restype = ctypes.c_int
    L.irt_forward_ppv_static.argtypes = [P(irt_grid_desc), P(irt_fields), P(irt_view),
                                         P(irt_vaxis), P(irt_cubes), P(irt_line), P(irt_dust),
                                         P(irt_opts), ctypes.c_void_p]
    L.irt_forward_graph_create.restype = ctypes.c_int
    L.irt_forward_graph_create.argtypes = [P(irt_job), ctypes.c_int, P(irt_line), P(irt_dust),
                                           P(irt_opts), P(ctypes.c_void_p)]
    L.irt_forward_graph_launch.restype = ctypes.c_int
    L.irt_forward_graph_launch.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    L.irt_forward_graph_destroy.restype = ctypes.c_int
    L.irt_forward_graph_destroy.argtypes = [ctypes.c_void_p]
    L.irt_tuned_plan.restype = ctypes.c_int
    L.irt_tuned_plan.argtypes = [P(irt_job), ctypes.c_int, P(irt_opts), P(ctypes.c_int)]
    L.irt_beam_convolve.restype = ctypes.c_int
    L.irt_beam_convolve.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_longlong,
                                    ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                    ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    L.irt_mean_axis1.restype = ctypes.c_int
    L.irt_mean_axis1.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_longlong,
                                 ctypes.c_longlong, ctypes.c_longlong, ctypes.c_void_p,
                                 ctypes.c_void_p]
    L.irt_measure_pipe_peaks.restype = ctypes.c_int
    L.irt_measure_pipe_peaks.argtypes = [P(ctypes.c_double), P(ctypes.c_double), ctypes.c_void_p]
    L.irt_grid_stats.restype = ctypes.c_int
    L.irt_grid_stats.argtypes = [ctypes.c_void_p, P(ctypes.c_ulonglong), ctypes.c_int]
    L.irt_last_error.restype = ctypes.c_char_p
    L.irt_last_error.argtypes = []
    L.irt_launch_count.restype = ctypes.c_longlong
    L.irt_launch_count.argtypes = []
    L.irt_create_ot_table.restype = ctypes.c_int
    L.irt_create_ot_table.argtypes = [P(irt_level_model), P(irt_ot_axes), _IP, ctypes.c_int,
                                      ctypes.c_void_p, P(ctypes.c_void_p)]
    L.irt_ot_table_values.restype = ctypes.c_int
    L.irt_ot_table_values.argtypes = [ctypes.c_void_p, _DP]
    L.irt_destroy_ot_table.restype = ctypes.c_int
    L.irt_destroy_ot_table.argtypes = [ctypes.c_void_p]
    L.irt_grid_set_h2_fraction.restype = ctypes.c_int
    L.irt_grid_set_h2_fraction.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                           ctypes.c_void_p]
    L.irt_update_grid.restype = ctypes.c_int
    L.irt_update_grid.argtypes = [ctypes.c_void_p, P(irt_grid_desc), P(irt_fields),
                                  ctypes.c_void_p]
    L.irt_forward_ppv_lines.restype = ctypes.c_int
    L.irt_forward_ppv_lines.argtypes = [P(irt_job), ctypes.c_int, P(irt_line), P(irt_dust),
                                        P(irt_cubes), ctypes.c_void_p, _IP, P(irt_opts),
                                        ctypes.c_void_p]
    L.irt_forward_ppv_ot.restype = ctypes.c_int
    L.irt_forward_ppv_ot.argtypes = [P(irt_job), ctypes.c_int, ctypes.c_void_p, ctypes.c_int,
                                     P(irt_line), P(irt_dust), P(irt_opts), ctypes.c_void_p]
    return L


lib = _load()


def _check(status):
    if status != IRT_OK:
        raise IrtError(status, lib.irt_last_error().decode())


def irt_create_grid(desc: irt_grid_desc, fields: irt_fields, stream: int) -> int:
    h = ctypes.c_void_p()
    _check(lib.irt_create_grid(ctypes.byref(desc), ctypes.byref(fields), ctypes.c_void_p(stream),
                               ctypes.byref(h)))
    return h.value


def irt_forward_ppv(jobs, line: irt_line, dust: irt_dust, opts: irt_opts, stream: int) -> None:
    arr = (irt_job * len(jobs))(*jobs)
    _check(lib.irt_forward_ppv(arr, len(jobs), ctypes.byref(line), ctypes.byref(dust),
                               ctypes.byref(opts), ctypes.c_void_p(stream)))


def irt_adjoint_ppv(job: irt_job, line: irt_line, dust: irt_dust, opts: irt_opts,
                    cotangent: irt_cubes, grad_n: int, grad_t: int, grad_v: int,
                    stream: int) -> None:
    _check(lib.irt_adjoint_ppv(ctypes.byref(job), ctypes.byref(line), ctypes.byref(dust),
                               ctypes.byref(opts), ctypes.byref(cotangent),
                               ctypes.c_void_p(grad_n), ctypes.c_void_p(grad_t),
                               ctypes.c_void_p(grad_v), ctypes.c_void_p(stream)))


def irt_forward_ppv_static(desc: irt_grid_desc, fields: irt_fields, view: irt_view,
                           vaxis: irt_vaxis, out: irt_cubes, line: irt_line, dust: irt_dust,
                           opts: irt_opts, stream: int) -> None:
    """Render one job from the caller's field arrays without any device
    allocation (the packed fields go to the library's static device array)."""
    _check(lib.irt_forward_ppv_static(ctypes.byref(desc), ctypes.byref(fields), ctypes.byref(view),
                                      ctypes.byref(vaxis), ctypes.byref(out), ctypes.byref(line),
                                      ctypes.byref(dust), ctypes.byref(opts),
                                      ctypes.c_void_p(stream)))


def irt_forward_graph_create(jobs, line: irt_line, dust: irt_dust, opts: irt_opts) -> int:
    arr = (irt_job * len(jobs))(*jobs)
    h = ctypes.c_void_p()
    _check(lib.irt_forward_graph_create(arr, len(jobs), ctypes.byref(line), ctypes.byref(dust),
                                        ctypes.byref(opts), ctypes.byref(h)))
    return h.value


def irt_forward_graph_launch(handle: int, stream: int) -> None:
    _check(lib.irt_forward_graph_launch(ctypes.c_void_p(handle), ctypes.c_void_p(stream)))


def irt_forward_graph_destroy(handle: int) -> None:
    _check(lib.irt_forward_graph_destroy(ctypes.c_void_p(handle)))


def irt_tuned_plan(jobs, opts: irt_opts):
    arr = (irt_job * len(jobs))(*jobs)
    out = (ctypes.c_int * 3)()
    _check(lib.irt_tuned_plan(arr, len(jobs), ctypes.byref(opts), out))
    return tuple(int(v) for v in out)


def irt_destroy(handle: int) -> None:
    _check(lib.irt_destroy(ctypes.c_void_p(handle)))


def irt_grid_stats(handle: int, reset: bool = True) -> dict:
    out = (ctypes.c_ulonglong * 6)()
    _check(lib.irt_grid_stats(ctypes.c_void_p(handle), out, int(reset)))
    keys = ("items", "samples", "line_block_samples", "hull_block_samples", "explicit_items",
            "dense_fine_updates")
    return dict(zip(keys, [int(v) for v in out]))


def irt_launch_count() -> int:
    return int(lib.irt_launch_count())


def irt_mean_axis1(inp: int, dtype: int, A: int, B: int, C: int, out: int,
                   stream: int = 0) -> None:
    """out[a][c] = mean over b of in[a][b][c] (device pointers)."""
    _check(lib.irt_mean_axis1(ctypes.c_void_p(inp), dtype, A, B, C, ctypes.c_void_p(out),
                              ctypes.c_void_p(stream)))


def irt_beam_convolve(inp: int, dtype: int, nchan: int, npy: int, npx: int, fwhm_px: float,
                      scratch: int, out: int, stream: int = 0) -> None:
    """Gaussian beam convolution of a device cube (scratch: same-size buffer)."""
    _check(lib.irt_beam_convolve(ctypes.c_void_p(inp), dtype, nchan, npy, npx, fwhm_px,
                                 ctypes.c_void_p(scratch), ctypes.c_void_p(out),
                                 ctypes.c_void_p(stream)))


def irt_measure_pipe_peaks(stream: int = 0) -> dict:
    """Measured FP32 FMA and ex2 lane-operations per second on this device."""
    a, b = ctypes.c_double(), ctypes.c_double()
    _check(lib.irt_measure_pipe_peaks(ctypes.byref(a), ctypes.byref(b), ctypes.c_void_p(stream)))
    return {"fp32_ops_per_s": a.value, "mufu_ops_per_s": b.value}


def irt_create_ot_table(model: irt_level_model, axes: irt_ot_axes, lines, stream: int) -> int:
    """Optically thin level-balance grid of the model's radiative transitions
    ``lines`` (Sec. 4.2); returns the table handle."""
    arr = (ctypes.c_int * len(lines))(*[int(x) for x in lines])
    h = ctypes.c_void_p()
    _check(lib.irt_create_ot_table(ctypes.byref(model), ctypes.byref(axes), arr, len(lines),
                                   ctypes.c_void_p(stream), ctypes.byref(h)))
    return h.value


def irt_ot_table_values(handle: int, out_ptr: int) -> None:
    _check(lib.irt_ot_table_values(ctypes.c_void_p(handle), ctypes.cast(out_ptr, _DP)))


def irt_destroy_ot_table(handle: int) -> None:
    _check(lib.irt_destroy_ot_table(ctypes.c_void_p(handle)))


def irt_grid_set_h2_fraction(grid: int, chi: int, dtype: int, stream: int) -> None:
    _check(lib.irt_grid_set_h2_fraction(ctypes.c_void_p(grid), ctypes.c_void_p(chi), dtype,
                                        ctypes.c_void_p(stream)))


def irt_forward_ppv_ot(jobs, table: int, line_index: int, line: irt_line, dust: irt_dust,
                       opts: irt_opts, stream: int) -> None:
    arr = (irt_job * len(jobs))(*jobs)
    _check(lib.irt_forward_ppv_ot(arr, len(jobs), ctypes.c_void_p(table), int(line_index),
                                  ctypes.byref(line), ctypes.byref(dust), ctypes.byref(opts),
                                  ctypes.c_void_p(stream)))


def irt_forward_ppv_lines(job: irt_job, lines, dusts, outs, table, table_lines,
                          opts: irt_opts, stream: int) -> None:
    """Several lines of one job in one launch (``lines``, ``dusts``,
    ``outs``: sequences of irt_line, irt_dust, irt_cubes); ``table`` an OT
    table handle or None with ``table_lines`` its line indices."""
    n = len(lines)
    la = (irt_line * n)(*lines)
    da = (irt_dust * n)(*dusts)
    oa = (irt_cubes * n)(*outs)
    ta = None if table_lines is None else (ctypes.c_int * n)(*[int(x) for x in table_lines])
    _check(lib.irt_forward_ppv_lines(ctypes.byref(job), n, la, da, oa,
                                     ctypes.c_void_p(table) if table else None, ta,
                                     ctypes.byref(opts), ctypes.c_void_p(stream)))


def irt_update_grid(handle: int, desc: irt_grid_desc, fields: irt_fields, stream: int) -> None:
    _check(lib.irt_update_grid(ctypes.c_void_p(handle), ctypes.byref(desc), ctypes.byref(fields),
                               ctypes.c_void_p(stream)))

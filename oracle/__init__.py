"""ctypes wrapper of the FP64 CPU oracle (test infrastructure only).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` use this package.  It is independent of the CUDA library: it
compiles ``irt_oracle.cpp`` with the host compiler and shares no code with
``paper_2607_01338_b300``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "irt_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle_irt.so")
_lock = threading.Lock()
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


def build(force: bool = False) -> str:
    """Compile the oracle (g++ -O2 -fopenmp, IEEE semantics, no fast-math)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["g++", "-O2", "-std=c++17", "-fopenmp", "-fPIC", "-shared",
           "-fno-fast-math", "-ffp-contract=off", "-o", tmp, _SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            L.oracle_planck.restype = ctypes.c_double
            L.oracle_planck.argtypes = [ctypes.c_double, ctypes.c_double]
            L.oracle_partition.restype = ctypes.c_double
            L.oracle_partition.argtypes = [_dp, ctypes.c_double]
            L.oracle_profile.restype = ctypes.c_double
            L.oracle_profile.argtypes = [_dp, ctypes.c_double, ctypes.c_double, ctypes.c_double]
            L.oracle_sample_coeffs.restype = None
            L.oracle_sample_coeffs.argtypes = [_dp, _dp, ctypes.c_double, ctypes.c_double,
                                               ctypes.c_double, _dp]
            L.oracle_ray.restype = None
            L.oracle_ray.argtypes = ([_dp, _dp, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                      ctypes.c_int] + [_dp] * 5 + [ctypes.c_double] + [_dp] * 5)
            L.oracle_ray_samples.restype = ctypes.c_int
            L.oracle_ray_samples.argtypes = [ctypes.POINTER(_dp), ctypes.c_int, ctypes.c_int,
                                             ctypes.c_int, ctypes.c_double, _dp, ctypes.c_int,
                                             ctypes.c_int, ctypes.c_int, _dp, _dp]
            L.oracle_render.restype = ctypes.c_int
            L.oracle_render.argtypes = ([ctypes.POINTER(_dp), ctypes.c_int, ctypes.c_int,
                                         ctypes.c_int, ctypes.c_double, _dp, _dp, _dp,
                                         ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                         ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_double, ctypes.c_int, _ip] + [_dp] * 5)
            L.oracle_ray_thin.restype = None
            L.oracle_ray_thin.argtypes = ([_dp, _dp, ctypes.c_int, ctypes.c_double,
                                           ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                           ctypes.c_int, ctypes.c_double, ctypes.c_int]
                                          + [_dp] * 5 + [ctypes.c_double] + [_dp] * 5)
            L.oracle_loss_grad_zview.restype = ctypes.c_double
            L.oracle_loss_grad_zview.argtypes = ([ctypes.POINTER(_dp), ctypes.c_int, ctypes.c_int,
                                                  ctypes.c_int, ctypes.c_double, _dp, _dp,
                                                  ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                                  ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                  ctypes.c_double, _dp, ctypes.c_int, _ip,
                                                  _dp, _dp, _dp])
            L.oracle_num_threads.restype = ctypes.c_int
            L.oracle_loss_grad_cells.restype = ctypes.c_double
            L.oracle_loss_grad_cells.argtypes = ([ctypes.POINTER(_dp), ctypes.c_int, ctypes.c_int,
                                                  ctypes.c_int, ctypes.c_double, _dp, _dp, _dp,
                                                  ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                                  ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                  ctypes.c_double, _dp, ctypes.c_int, _ip,
                                                  _dp, _dp, _dp])
            L.oracle_render_levels.restype = ctypes.c_int
            L.oracle_render_levels.argtypes = ([ctypes.POINTER(_dp), _dp, ctypes.c_int,
                                                ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                                _dp, _dp, _dp, ctypes.c_int, ctypes.c_double,
                                                ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                                ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                                ctypes.c_int, _ip] + [_dp] * 5
                                               + [ctypes.c_void_p, ctypes.c_int])
            L.oracle_ot_populations.restype = None
            L.oracle_ot_populations.argtypes = [ctypes.POINTER(OracleLevelModel),
                                                ctypes.c_double, ctypes.c_double,
                                                ctypes.c_double, _dp]
            L.oracle_ot_table_build.restype = ctypes.c_void_p
            L.oracle_ot_table_build.argtypes = [ctypes.POINTER(OracleLevelModel), _ip, _dp, _dp,
                                                ctypes.c_int, _ip]
            L.oracle_ot_table_values.restype = None
            L.oracle_ot_table_values.argtypes = [ctypes.c_void_p, _dp]
            L.oracle_ot_lookup.restype = None
            L.oracle_ot_lookup.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_double,
                                           ctypes.c_double, ctypes.c_double, _dp]
            L.oracle_ot_table_from_values.restype = ctypes.c_void_p
            L.oracle_ot_table_from_values.argtypes = [_ip, _dp, _dp, ctypes.c_int, _dp, _dp]
            L.oracle_ot_table_free.restype = None
            L.oracle_ot_table_free.argtypes = [ctypes.c_void_p]
            _lib = L
    return _lib


# --------------------------------------------------------------------------
# argument packing
# --------------------------------------------------------------------------
class OracleLevelModel(ctypes.Structure):
    """Layout of LevelModel in irt_oracle.cpp (pointers into numpy arrays)."""
    _fields_ = [("nlev", ctypes.c_int), ("energy_k", _dp), ("g", _dp),
                ("nrad", ctypes.c_int), ("rad_up", _ip), ("rad_lo", _ip), ("a_ul", _dp),
                ("nu", _dp), ("npartner", ctypes.c_int), ("partner", _ip),
                ("ntemp", ctypes.c_int), ("coll_temp", _dp), ("ncoll", ctypes.c_int),
                ("coll_up", _ip), ("coll_lo", _ip), ("k_ul", _dp), ("t_rad", ctypes.c_double),
                ("ortho_para", ctypes.c_double), ("x_he", ctypes.c_double)]


def _level_model(model: dict):
    """(keep-alive arrays, OracleLevelModel) from a level-model dict."""
    d = lambda k: np.ascontiguousarray(np.asarray(model[k], dtype=np.float64))  # noqa: E731
    i = lambda k: np.ascontiguousarray(np.asarray(model[k], dtype=np.int32))    # noqa: E731
    keep = dict(energy_k=d("energy_k"), g=d("g"), rad_up=i("rad_up"), rad_lo=i("rad_lo"),
                a_ul=d("a_ul_s"), nu=d("nu_hz"), partner=i("partner"),
                coll_temp=d("coll_temp_k"), coll_up=i("coll_up"), coll_lo=i("coll_lo"),
                k_ul=d("k_ul_cm3_s"))
    ntemp = keep["coll_temp"].shape[-1]
    ncoll = keep["coll_up"].shape[-1]
    m = OracleLevelModel(int(model["nlev"]), keep["energy_k"].ctypes.data_as(_dp),
                         keep["g"].ctypes.data_as(_dp), len(keep["rad_up"]),
                         keep["rad_up"].ctypes.data_as(_ip), keep["rad_lo"].ctypes.data_as(_ip),
                         keep["a_ul"].ctypes.data_as(_dp), keep["nu"].ctypes.data_as(_dp),
                         len(keep["partner"]), keep["partner"].ctypes.data_as(_ip), ntemp,
                         keep["coll_temp"].ctypes.data_as(_dp), ncoll,
                         keep["coll_up"].ctypes.data_as(_ip), keep["coll_lo"].ctypes.data_as(_ip),
                         keep["k_ul"].ctypes.data_as(_dp), float(model["t_rad_k"]),
                         float(model["ortho_para"]), float(model["x_he"]))
    return keep, m


def ot_populations(model: dict, n_h: float, chi: float, T: float) -> np.ndarray:
    """Fractional level populations n_i / N of the OT level balance at total
    H density n_h [cm^-3], H2 abundance chi and gas temperature T (Sec. 3.5)."""
    keep, m = _level_model(model)
    f = np.zeros(int(model["nlev"]))
    lib().oracle_ot_populations(ctypes.byref(m), n_h, chi, T, f.ctypes.data_as(_dp))
    return f


class OTTable:
    """Coefficient grid of Sec. 4.2 over (log10 n_H, chi, log10 T) for the
    radiative transitions ``lines`` of ``model``; values per tracer molecule
    [cgs]: j = (h nu / 4 pi) A f_u, alpha = (h nu / 4 pi)(f_l B_lu - f_u B_ul)."""

    def __init__(self, model: dict, axes: dict, lines, values=None):
        self.axes = dict(axes)
        self.n = (int(axes["n_n"]), int(axes["n_chi"]), int(axes["n_t"]))
        n = np.array(self.n, dtype=np.int32)
        lo = np.array([axes["log10_nh_min"], axes["chi_min"], axes["log10_t_min"]])
        hi = np.array([axes["log10_nh_max"], axes["chi_max"], axes["log10_t_max"]])
        ln = np.ascontiguousarray(np.asarray(lines, dtype=np.int32))
        self.nlines = len(ln)
        if values is not None:
            # a table with given content [nlines, n_n, n_chi, n_t, 2]
            v = np.ascontiguousarray(np.asarray(values, dtype=np.float64))
            assert v.shape == (self.nlines,) + self.n + (2,)
            nu = np.ascontiguousarray(np.asarray(model["nu_hz"], dtype=np.float64)[ln])
            self.ptr = lib().oracle_ot_table_from_values(
                n.ctypes.data_as(_ip), lo.ctypes.data_as(_dp), hi.ctypes.data_as(_dp),
                self.nlines, nu.ctypes.data_as(_dp), v.ctypes.data_as(_dp))
            return
        keep, m = _level_model(model)
        self.ptr = lib().oracle_ot_table_build(ctypes.byref(m), n.ctypes.data_as(_ip),
                                               lo.ctypes.data_as(_dp), hi.ctypes.data_as(_dp),
                                               self.nlines, ln.ctypes.data_as(_ip))

    def values(self) -> np.ndarray:
        """[nlines, n_n, n_chi, n_t, 2] array of (j, alpha) per molecule."""
        out = np.zeros((self.nlines,) + self.n + (2,))
        lib().oracle_ot_table_values(self.ptr, out.ctypes.data_as(_dp))
        return out

    def lookup(self, line: int, n_h: float, chi: float, T: float):
        out = np.zeros(2)
        lib().oracle_ot_lookup(self.ptr, line, n_h, chi, T, out.ctypes.data_as(_dp))
        return float(out[0]), float(out[1])

    def close(self):
        if getattr(self, "ptr", None):
            lib().oracle_ot_table_free(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
LINE_KEYS = ("nu_ul_hz", "a_ul_s", "e_u_k", "b0_hz", "g_u", "g_l", "mass_amu", "t_inf_k",
             "sigma_turb_kms")
DUST_KEYS = ("kappa_cm2_per_g_gas", "mu_mass_per_h2_amu")
FORMAL, SMOOTH = 0, 1
THICK, SELECTIVELY_THIN, THIN = 0, 1, 2   # transfer modes (Sec. 4.5-4.7)
DENSITY_TRACING = 3                        # column density per unit velocity (Sec. 5.10)
TRJ, INTENSITY, TB = 0, 1, 2   # output units (Sec. 4.9)


def _arr(vals):
    a = np.ascontiguousarray(np.asarray(vals, dtype=np.float64))
    return a, a.ctypes.data_as(_dp)


def _line(line: dict):
    return _arr([line[k] for k in LINE_KEYS])


def _dust(dust: dict):
    return _arr([dust[k] for k in DUST_KEYS])


def _view(view):
    return _arr([view.theta_rad, view.phi_rad, view.npx, view.npy, view.pixel_cm,
                 view.trilinear])


def _fields(fields):
    arrs = [np.ascontiguousarray(np.asarray(a, dtype=np.float64)) for a in fields]
    ptrs = (_dp * 5)(*[a.ctypes.data_as(_dp) for a in arrs])
    return arrs, ptrs


def num_threads() -> int:
    return lib().oracle_num_threads()


def planck(nu: float, T: float) -> float:
    return lib().oracle_planck(nu, T)


def partition(line: dict, T: float) -> float:
    keep, p = _line(line)
    return lib().oracle_partition(p, T)


def profile_per_hz(line: dict, t_gas: float, v_los: float, u: float) -> float:
    keep, p = _line(line)
    return lib().oracle_profile(p, t_gas, v_los, u)


def sample_coeffs(line: dict, dust: dict, n_h2: float, t_gas: float, x_tr: float) -> dict:
    kl, pl = _line(line)
    kd, pd = _dust(dust)
    out = np.zeros(6)
    lib().oracle_sample_coeffs(pl, pd, n_h2, t_gas, x_tr, out.ctypes.data_as(_dp))
    return dict(n_u=out[0], n_l=out[1], jL=out[2], aL=out[3], aD=out[4], b_kms=out[5])


def ray(line, dust, vaxis, samples, h, integration=SMOOTH, units=TRJ, t_bg=2.725):
    """One ray from explicit samples: ``samples`` = dict of 1-D arrays
    n_h2, t_gas, t_dust, v_los, x_tr in travel order.  Returns dict of
    [nchan] arrays T, C, D, L, B."""
    kl, pl = _line(line)
    kd, pd = _dust(dust)
    cols = [np.ascontiguousarray(np.asarray(samples[k], dtype=np.float64))
            for k in ("n_h2", "t_gas", "t_dust", "v_los", "x_tr")]
    K = len(cols[0])
    nch = vaxis.nchan
    outs = [np.zeros(nch) for _ in range(5)]
    lib().oracle_ray(pl, pd, nch, vaxis.v_first_edge_kms, vaxis.dv_kms, vaxis.subsample_f,
                     integration, units, t_bg, K, *[c.ctypes.data_as(_dp) for c in cols], h,
                     *[o.ctypes.data_as(_dp) for o in outs])
    return dict(zip("TCDLB", outs))


def ray_samples(fields, cell_cm, view, px, py, kmax=100000):
    shape = np.asarray(fields[0]).shape
    nz, ny, nx = shape
    arrs, ptrs = _fields(fields)
    kv, pv = _view(view)
    buf = np.zeros((min(kmax, 4 * (nx + ny + nz) + 8), 5))
    h = np.zeros(1)
    K = lib().oracle_ray_samples(ptrs, nx, ny, nz, cell_cm, pv, px, py, buf.shape[0],
                                 h.ctypes.data_as(_dp), buf.ctypes.data_as(_dp))
    return buf[:K].copy(), float(h[0])


def ray_thin(line, dust, vaxis, samples, h, transfer=SELECTIVELY_THIN, integration=SMOOTH,
             units=TRJ, t_bg=2.725):
    """One ray from explicit samples in a thin transfer mode (no velocity
    subsampling: the channel-averaged profile is analytic).  Returns dict of
    [nchan] arrays T, C, D, L, B."""
    kl, pl = _line(line)
    kd, pd = _dust(dust)
    cols = [np.ascontiguousarray(np.asarray(samples[k], dtype=np.float64))
            for k in ("n_h2", "t_gas", "t_dust", "v_los", "x_tr")]
    K = len(cols[0])
    nch = vaxis.nchan
    outs = [np.zeros(nch) for _ in range(5)]
    lib().oracle_ray_thin(pl, pd, nch, vaxis.v_first_edge_kms, vaxis.dv_kms, transfer,
                          integration, units, t_bg, K, *[c.ctypes.data_as(_dp) for c in cols], h,
                          *[o.ctypes.data_as(_dp) for o in outs])
    return dict(zip("TCDLB", outs))


def render(fields, cell_cm, line, dust, view, vaxis, pixels, integration=SMOOTH, units=TRJ,
           t_bg=2.725, transfer=THICK, levels=None, line_index=0, chi=None):
    """Render the pixels ``pixels`` (int array [npix, 2] of (px, py)).
    Returns dict of [npix, nchan] float64 arrays T, C, D, L, B.  ``levels``:
    an OTTable whose line ``line_index`` gives the line coefficients (OT level
    balance, Sec. 4.2-4.3) instead of LTE; ``chi``: H2 abundance per H nucleus
    [z][y][x] (default 0.5 everywhere)."""
    nz, ny, nx = np.asarray(fields[0]).shape
    arrs, ptrs = _fields(fields)
    kl, pl = _line(line)
    kd, pd = _dust(dust)
    kv, pv = _view(view)
    pix = np.ascontiguousarray(np.asarray(pixels, dtype=np.int32).reshape(-1, 2))
    npix = pix.shape[0]
    nch = vaxis.nchan
    outs = [np.zeros((npix, nch)) for _ in range(5)]
    chi_a = None if chi is None else np.ascontiguousarray(np.asarray(chi, dtype=np.float64))
    lib().oracle_render_levels(ptrs, None if chi_a is None else chi_a.ctypes.data_as(_dp),
                               nx, ny, nz, cell_cm, pl, pd, pv, nch, vaxis.v_first_edge_kms,
                               vaxis.dv_kms, vaxis.subsample_f, transfer, integration, units,
                               t_bg, npix, pix.ctypes.data_as(_ip),
                               *[o.ctypes.data_as(_dp) for o in outs],
                               None if levels is None else levels.ptr, int(line_index))
    return dict(zip("TCDLB", outs))


def render_cube(fields, cell_cm, line, dust, view, vaxis, **kw):
    """Whole cube, [nchan][npy][npx] per component."""
    npx, npy = view.npx, view.npy
    py, px = np.meshgrid(np.arange(npy), np.arange(npx), indexing="ij")
    pix = np.stack([px.ravel(), py.ravel()], axis=1)
    r = render(fields, cell_cm, line, dust, view, vaxis, pix, **kw)
    return {k: v.reshape(npy, npx, -1).transpose(2, 0, 1).copy() for k, v in r.items()}


def loss_grad_zview(fields, cell_cm, line, dust, vaxis, target_L, pixels=None,
                    integration=SMOOTH, units=TRJ, t_bg=2.725):
    """Loss = mean over all voxels of ([L] - target)^2 and its gradient with
    respect to n_H2, T_gas, v_los (z view), by forward-mode dual numbers.
    ``target_L`` is [nchan][ny][nx].  Returns (loss, g_n, g_t, g_v)."""
    nz, ny, nx = np.asarray(fields[0]).shape
    arrs, ptrs = _fields(fields)
    kl, pl = _line(line)
    kd, pd = _dust(dust)
    tgt = np.ascontiguousarray(np.asarray(target_L, dtype=np.float64))
    if pixels is None:
        py, px = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
        pixels = np.stack([px.ravel(), py.ravel()], axis=1)
    pix = np.ascontiguousarray(np.asarray(pixels, dtype=np.int32).reshape(-1, 2))
    gs = [np.zeros((nz, ny, nx)) for _ in range(3)]
    loss = lib().oracle_loss_grad_zview(ptrs, nx, ny, nz, cell_cm, pl, pd, vaxis.nchan,
                                        vaxis.v_first_edge_kms, vaxis.dv_kms,
                                        vaxis.subsample_f, integration, units, t_bg,
                                        tgt.ctypes.data_as(_dp), pix.shape[0],
                                        pix.ctypes.data_as(_ip),
                                        *[g.ctypes.data_as(_dp) for g in gs])
    return loss, gs[0], gs[1], gs[2]


def loss_grad_cells(fields, cell_cm, line, dust, view, vaxis, target_L, cells,
                    integration=SMOOTH, units=TRJ, t_bg=2.725):
    """Loss = mean over all voxels of ([L] - target)^2 and its gradient with
    respect to n_H2, T_gas, v_los of the cells ``cells`` (int [n, 3] of
    (x, y, z)), any view and integrator, by forward-mode dual numbers.
    ``target_L`` is [nchan][npy][npx].  Returns (loss, g_n, g_t, g_v), each
    gradient an array [n]."""
    nz, ny, nx = np.asarray(fields[0]).shape
    arrs, ptrs = _fields(fields)
    kl, pl = _line(line)
    kd, pd = _dust(dust)
    kv, pv = _view(view)
    tgt = np.ascontiguousarray(np.asarray(target_L, dtype=np.float64))
    cl = np.ascontiguousarray(np.asarray(cells, dtype=np.int32).reshape(-1, 3))
    gs = [np.zeros(cl.shape[0]) for _ in range(3)]
    loss = lib().oracle_loss_grad_cells(ptrs, nx, ny, nz, cell_cm, pl, pd, pv, vaxis.nchan,
                                        vaxis.v_first_edge_kms, vaxis.dv_kms, vaxis.subsample_f,
                                        integration, units, t_bg, tgt.ctypes.data_as(_dp),
                                        cl.shape[0], cl.ctypes.data_as(_ip),
                                        *[g.ctypes.data_as(_dp) for g in gs])
    return loss, gs[0], gs[1], gs[2]


def latitude_mean(a):
    """Latitude-mean reduction of Sec. 6.1 in FP64: out[a][c] = mean over b of
    in[a][b][c] for an [A, B, C] array (the l-v image u of a PPV cube
    [nchan, npy, npx]; the top-down map t of a field [nz, ny, nx])."""
    x = np.asarray(a, dtype=np.float64)
    return x.sum(axis=1) / x.shape[1]


def beam_kernel(fwhm_px):
    """Normalised 1-D Gaussian taps of a beam of the given FWHM in pixels
    (Sec. 4.11): sigma = FWHM / (2 sqrt(2 ln 2)), taps out to ceil(4 sigma),
    weights exp(-d^2 / (2 sigma^2)) divided by their sum."""
    sigma = fwhm_px / (2.0 * np.sqrt(2.0 * np.log(2.0)))
    R = int(np.ceil(4.0 * sigma))
    d = np.arange(-R, R + 1, dtype=np.float64)
    w = np.exp(-d * d / (2.0 * sigma * sigma))
    return w / w.sum()


def beam_convolve(cube, fwhm_px):
    """Gaussian beam convolution of Sec. 4.11 in FP64 on a [nchan, npy, npx]
    cube: each channel image convolved with the separable Gaussian of
    beam_kernel along x and then along y, the sky outside the image taken as
    zero."""
    x = np.asarray(cube, dtype=np.float64)
    w = beam_kernel(fwhm_px)
    R = (len(w) - 1) // 2
    out = np.zeros_like(x)
    # along x
    p = np.pad(x, ((0, 0), (0, 0), (R, R)))
    for i, wi in enumerate(w):
        out += wi * p[:, :, i:i + x.shape[2]]
    # along y
    p = np.pad(out, ((0, 0), (R, R), (0, 0)))
    out = np.zeros_like(x)
    for i, wi in enumerate(w):
        out += wi * p[:, i:i + x.shape[1], :]
    return out

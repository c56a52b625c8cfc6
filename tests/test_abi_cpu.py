"""C-ABI checks that need no GPU: the library loads, exports every symbol
include/irt.h declares, the ctypes structures match the C layout, and
argument validation rejects bad calls before touching the device."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "irt.h")


@pytest.fixture(scope="module")
def B():
    from paper_2607_01338_b300 import build as bld
    bld.build()
    from paper_2607_01338_b300 import binding
    return binding


def declared_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:irt_status|const char\*|long long)\s+(irt_\w+)\s*\(",
                                 text, re.M)))


def test_header_declares_the_four_entry_points():
    names = declared_functions()
    for n in ("irt_create_grid", "irt_forward_ppv", "irt_adjoint_ppv", "irt_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol(B):
    out = subprocess.run(["nm", "-D", "--defined-only", B.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (irt_\w+)", out))
    for n in declared_functions():
        assert n in exported, n
        assert hasattr(B.lib, n)
    assert set(B.EXPORTED) == set(declared_functions())


def test_build_targets_sm_103a_only():
    from paper_2607_01338_b300 import build as bld
    assert bld.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


STRUCTS = ["irt_grid_desc", "irt_fields", "irt_line", "irt_dust", "irt_view", "irt_vaxis",
           "irt_opts", "irt_cubes", "irt_job", "irt_level_model", "irt_ot_axes"]


def test_ctypes_layout_matches_c(B, tmp_path):
    lines = ['#include <stdio.h>', '#include <stddef.h>', f'#include "{HEADER}"',
             'int main(void) {']
    for s in STRUCTS:
        cls = getattr(B, s)
        lines.append(f'  printf("{s} %zu\\n", sizeof({s}));')
        for fname, _ in cls._fields_:
            lines.append(f'  printf("{s}.{fname} %zu\\n", offsetof({s}, {fname}));')
    lines += ['  return 0;', '}']
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-o", str(exe), str(src)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    got = dict(line.rsplit(" ", 1) for line in out.strip().splitlines())
    for s in STRUCTS:
        cls = getattr(B, s)
        assert int(got[s]) == ctypes.sizeof(cls), s
        for fname, _ in cls._fields_:
            assert int(got[f"{s}.{fname}"]) == getattr(cls, fname).offset, (s, fname)


def _line(B):
    from synth import LINE_13CO_21
    return B.irt_line(*[LINE_13CO_21[k] for k, _ in B.irt_line._fields_])


def test_validation_before_any_launch(B):
    """These calls fail in argument checking, which runs before any CUDA call."""
    L = B.lib
    h = ctypes.c_void_p()
    assert L.irt_create_grid(None, None, None, ctypes.byref(h)) == B.IRT_EINVAL
    desc = B.irt_grid_desc(0, 4, 4, 1.0, (ctypes.c_int * 5)(0, 0, 0, 0, 0))
    f = B.irt_fields(1, 2, 3, 4, 5)
    assert L.irt_create_grid(ctypes.byref(desc), ctypes.byref(f), None, ctypes.byref(h)) == B.IRT_EINVAL
    assert b"grid size" in L.irt_last_error()
    desc = B.irt_grid_desc(4, 4, 4, -1.0, (ctypes.c_int * 5)(0, 0, 0, 0, 0))
    assert L.irt_create_grid(ctypes.byref(desc), ctypes.byref(f), None, ctypes.byref(h)) == B.IRT_EINVAL
    desc = B.irt_grid_desc(4, 4, 4, 1.0, (ctypes.c_int * 5)(0, 0, 9, 0, 0))
    assert L.irt_create_grid(ctypes.byref(desc), ctypes.byref(f), None, ctypes.byref(h)) == B.IRT_EINVAL
    assert b"dtype" in L.irt_last_error()
    f0 = B.irt_fields(1, 2, None, 4, 5)
    desc = B.irt_grid_desc(4, 4, 4, 1.0, (ctypes.c_int * 5)(0, 0, 0, 0, 0))
    assert L.irt_create_grid(ctypes.byref(desc), ctypes.byref(f0), None, ctypes.byref(h)) == B.IRT_EINVAL
    # forward: no jobs / NULL grid / bad axis
    line = _line(B)
    dust = B.irt_dust(0.01, 2.8)
    opts = B.irt_opts(0, 1, 0, 2.725, 0, 0)
    assert L.irt_forward_ppv(None, 0, ctypes.byref(line), ctypes.byref(dust),
                             ctypes.byref(opts), None) == B.IRT_EINVAL
    job = B.irt_job(None, B.irt_view(0, 0, 4, 4, 1.0, 0), B.irt_vaxis(4, -2.0, 1.0, 1),
                    B.irt_cubes(1, None, None, None, None))
    assert L.irt_forward_ppv(ctypes.byref(job), 1, ctypes.byref(line), ctypes.byref(dust),
                             ctypes.byref(opts), None) == B.IRT_EINVAL
    assert b"grid" in L.irt_last_error()
    bad = B.irt_line(line.nu_ul_hz, -1.0, line.e_u_k, line.b0_hz, line.g_u, line.g_l,
                     line.mass_amu, line.t_inf_k, line.sigma_turb_kms)
    assert L.irt_forward_ppv(ctypes.byref(job), 1, ctypes.byref(bad), ctypes.byref(dust),
                             ctypes.byref(opts), None) == B.IRT_EINVAL
    nan_opts = B.irt_opts(0, 1, 0, float("nan"), 0, 0)
    assert L.irt_forward_ppv(ctypes.byref(job), 1, ctypes.byref(line), ctypes.byref(dust),
                             ctypes.byref(nan_opts), None) == B.IRT_EINVAL
    # the allocation-free entry keeps no checkpoints: refused before any CUDA call
    sdesc = B.irt_grid_desc(4, 4, 4, 1.0, (ctypes.c_int * 5)(0, 0, 0, 0, 0))
    save = B.irt_opts(0, 1, 0, 2.725, 0, B.IRT_FLAG_SAVE_CHECKPOINTS)
    cubes = B.irt_cubes(1, None, None, None, None)
    assert L.irt_forward_ppv_static(ctypes.byref(sdesc), ctypes.byref(f), ctypes.byref(job.view),
                                    ctypes.byref(job.vaxis), ctypes.byref(cubes),
                                    ctypes.byref(line), ctypes.byref(dust), ctypes.byref(save),
                                    None) == B.IRT_EUNSUPPORTED
    assert b"checkpoints" in L.irt_last_error()
    assert L.irt_destroy(None) == B.IRT_OK


def test_product_path_has_no_oracle_or_fallback():
    """The package never imports the oracle and has no CPU fallback path."""
    pkg = os.path.join(ROOT, "paper_2607_01338_b300")
    for dirpath, _, files in os.walk(pkg):
        for fn in files:
            if fn.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, fn)).read()
                assert "import oracle" not in text and "from oracle" not in text, fn
                assert "irt_oracle" not in text, fn


def test_post_processing_calls_validate_before_any_launch(B):
    """irt_mean_axis1 and irt_beam_convolve refuse bad arguments on the host
    (no device needed)."""
    L = B.lib
    assert L.irt_mean_axis1(None, B.IRT_F32, 2, 3, 4, None, None) == B.IRT_EINVAL
    assert L.irt_mean_axis1(1, B.IRT_F32, 0, 3, 4, 1, None) == B.IRT_EINVAL
    assert L.irt_mean_axis1(1, B.IRT_F16, 2, 3, 4, 1, None) == B.IRT_EUNSUPPORTED
    assert L.irt_mean_axis1(1, B.IRT_F32, 70000, 3, 4, 1, None) == B.IRT_EUNSUPPORTED
    assert L.irt_beam_convolve(None, B.IRT_F32, 1, 4, 4, 2.0, 1, 2, None) == B.IRT_EINVAL
    assert L.irt_beam_convolve(1, B.IRT_F32, 1, 4, 4, 0.0, 2, 3, None) == B.IRT_EINVAL
    assert b"FWHM" in L.irt_last_error()
    assert L.irt_beam_convolve(1, B.IRT_F32, 1, 4, 4, 2.0, 1, 3, None) == B.IRT_EINVAL
    assert b"scratch" in L.irt_last_error()
    assert L.irt_beam_convolve(1, B.IRT_BF16, 1, 4, 4, 2.0, 2, 3, None) == B.IRT_EUNSUPPORTED


def test_thin_and_tb_options_validate_before_any_launch(B):
    """Transfer modes and units outside the enums, and Kahan with a thin
    mode, are refused before the jobs are looked at."""
    L = B.lib
    line = _line(B)
    dust = B.irt_dust(0.01, 2.8)
    job = B.irt_job(None, B.irt_view(0, 0, 4, 4, 1.0, 0), B.irt_vaxis(4, -2.0, 1.0, 1),
                    B.irt_cubes(1, None, None, None, None))
    for opts, code in ((B.irt_opts(9, 1, 0, 2.725, 0, 0), B.IRT_EINVAL),
                       (B.irt_opts(B.IRT_MODE_THIN, B.IRT_FORMAL_KAHAN, 0, 2.725, 0, 0),
                        B.IRT_EUNSUPPORTED),
                       (B.irt_opts(0, 1, 7, 2.725, 0, 0), B.IRT_EINVAL)):
        assert L.irt_forward_ppv(ctypes.byref(job), 1, ctypes.byref(line), ctypes.byref(dust),
                                 ctypes.byref(opts), None) == code


def test_static_entry_takes_the_thick_mode_and_rj_or_intensity_units(B):
    """The allocation-free entry refuses the thin modes and T_B output before
    any CUDA call."""
    L = B.lib
    line = _line(B)
    dust = B.irt_dust(0.01, 2.8)
    f = B.irt_fields(1, 2, 3, 4, 5)
    desc = B.irt_grid_desc(4, 4, 4, 1.0, (ctypes.c_int * 5)(0, 0, 0, 0, 0))
    view = B.irt_view(0, 0, 4, 4, 1.0, 0)
    vaxis = B.irt_vaxis(4, -2.0, 1.0, 1)
    cubes = B.irt_cubes(1, None, None, None, None)
    for opts, word in ((B.irt_opts(B.IRT_MODE_THIN, 1, 0, 2.725, 0, 0), b"thick"),
                       (B.irt_opts(0, 1, B.IRT_UNITS_TB, 2.725, 0, 0), b"intensity")):
        assert L.irt_forward_ppv_static(ctypes.byref(desc), ctypes.byref(f), ctypes.byref(view),
                                        ctypes.byref(vaxis), ctypes.byref(cubes),
                                        ctypes.byref(line), ctypes.byref(dust),
                                        ctypes.byref(opts), None) == B.IRT_EUNSUPPORTED
        assert word in L.irt_last_error()


def test_static_entry_refuses_long_rays_and_stats_before_any_cuda_call(B):
    """Rays longer than the static record area holds for one block of warps
    are refused with IRT_EINVAL before any launch (a 2 x 2 x 262144 z-view
    grid is within the cell limit but its rays have 262144 samples), and so is
    IRT_FLAG_STATS (no grid keeps the counters)."""
    L = B.lib
    line = _line(B)
    dust = B.irt_dust(0.01, 2.8)
    f = B.irt_fields(1, 2, 3, 4, 5)
    vaxis = B.irt_vaxis(4, -2.0, 1.0, 1)
    cubes = B.irt_cubes(1, None, None, None, None)
    opts = B.irt_opts(0, 1, 0, 2.725, 0, 0)
    desc = B.irt_grid_desc(2, 2, 262144, 1.0, (ctypes.c_int * 5)(0, 0, 0, 0, 0))
    view = B.irt_view(0, 0, 2, 2, 1.0, 0)
    args = (ctypes.byref(desc), ctypes.byref(f), ctypes.byref(view), ctypes.byref(vaxis),
            ctypes.byref(cubes), ctypes.byref(line), ctypes.byref(dust))
    assert L.irt_forward_ppv_static(*args, ctypes.byref(opts), None) == B.IRT_EINVAL
    msg = L.irt_last_error()
    assert b"262144 samples" in msg and b"87381 samples" in msg
    stats = B.irt_opts(0, 1, 0, 2.725, 0, B.IRT_FLAG_STATS)
    desc4 = B.irt_grid_desc(4, 4, 4, 1.0, (ctypes.c_int * 5)(0, 0, 0, 0, 0))
    view4 = B.irt_view(0, 0, 4, 4, 1.0, 0)
    assert L.irt_forward_ppv_static(ctypes.byref(desc4), ctypes.byref(f), ctypes.byref(view4),
                                    ctypes.byref(vaxis), ctypes.byref(cubes), ctypes.byref(line),
                                    ctypes.byref(dust), ctypes.byref(stats),
                                    None) == B.IRT_EUNSUPPORTED
    assert b"counters" in L.irt_last_error()


def test_forced_allocation_failure_reports_enomem(B, monkeypatch):
    """Host-side fault injection: with IRT_FAIL_ALLOC set, irt_create_grid
    fails with IRT_ENOMEM, returns no handle and names the allocation; with it
    cleared (or "0") the same call gets past the allocation."""
    L = B.lib
    f = B.irt_fields(1, 2, 3, 4, 5)
    desc = B.irt_grid_desc(8, 8, 8, 1.0, (ctypes.c_int * 5)(0, 0, 0, 0, 0))
    out = ctypes.c_void_p(12345)
    monkeypatch.setenv("IRT_FAIL_ALLOC", "1")
    assert L.irt_create_grid(ctypes.byref(desc), ctypes.byref(f), None,
                             ctypes.byref(out)) == B.IRT_ENOMEM
    assert out.value is None
    assert b"allocate" in L.irt_last_error()
    monkeypatch.setenv("IRT_FAIL_ALLOC", "0")
    if not _has_gpu():
        # without a device the real allocation fails too, with the same code
        assert L.irt_create_grid(ctypes.byref(desc), ctypes.byref(f), None,
                                 ctypes.byref(out)) == B.IRT_ENOMEM


def _has_gpu():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def test_ot_table_arguments_validate_before_any_cuda_call(B):
    """irt_create_ot_table refuses bad level models and axes with IRT_EINVAL
    or IRT_EUNSUPPORTED before any device work; irt_forward_ppv_ot refuses a
    NULL table."""
    import numpy as np
    from synth.levels import rotor_model
    L = B.lib
    m = rotor_model(nlev=6)
    keep = {k: np.ascontiguousarray(np.asarray(m[k], dtype=np.float64)) for k in
            ("energy_k", "g", "a_ul_s", "nu_hz", "coll_temp_k", "k_ul_cm3_s")}
    keepi = {k: np.ascontiguousarray(np.asarray(m[k], dtype=np.int32)) for k in
             ("rad_up", "rad_lo", "partner", "coll_up", "coll_lo")}
    dp = lambda a: a.ctypes.data_as(B._DP)  # noqa: E731
    ip = lambda a: a.ctypes.data_as(B._IP)  # noqa: E731

    def model(**kw):
        args = dict(nlev=m["nlev"], nrad=len(keepi["rad_up"]), npartner=len(keepi["partner"]),
                    ntemp=keep["coll_temp_k"].shape[-1], ncoll=keepi["coll_up"].shape[-1],
                    t_rad=2.725)
        args.update(kw)
        return B.irt_level_model(args["nlev"], dp(keep["energy_k"]), dp(keep["g"]), args["nrad"],
                                 ip(keepi["rad_up"]), ip(keepi["rad_lo"]), dp(keep["a_ul_s"]),
                                 dp(keep["nu_hz"]), args["npartner"], ip(keepi["partner"]),
                                 args["ntemp"], dp(keep["coll_temp_k"]), args["ncoll"],
                                 ip(keepi["coll_up"]), ip(keepi["coll_lo"]),
                                 dp(keep["k_ul_cm3_s"]), args["t_rad"], 3.0, 0.1)

    ax = B.irt_ot_axes(8, 4, 6, 1.0, 7.0, 0.05, 0.5, 0.7, 2.5)
    lines = (ctypes.c_int * 1)(1)
    out = ctypes.c_void_p()
    cases = [(model(nlev=1), ax, lines, 1, B.IRT_EINVAL),
             (model(nlev=65), ax, lines, 1, B.IRT_EUNSUPPORTED),
             (model(), ax, (ctypes.c_int * 1)(9), 1, B.IRT_EINVAL),
             (model(), ax, lines, 0, B.IRT_EINVAL),
             (model(), ax, (ctypes.c_int * 9)(*[1] * 9), 9, B.IRT_EUNSUPPORTED),
             (model(t_rad=-1.0), ax, lines, 1, B.IRT_EINVAL),
             (model(), B.irt_ot_axes(1, 4, 6, 1.0, 7.0, 0.05, 0.5, 0.7, 2.5), lines, 1,
              B.IRT_EINVAL),
             (model(), B.irt_ot_axes(8, 4, 6, 1.0, 7.0, 0.05, 0.7, 0.7, 2.5), lines, 1,
              B.IRT_EINVAL),
             (model(), B.irt_ot_axes(8, 4, 6, 7.0, 1.0, 0.05, 0.5, 0.7, 2.5), lines, 1,
              B.IRT_EINVAL)]
    for mm, aa, ll, nl, code in cases:
        assert L.irt_create_ot_table(ctypes.byref(mm), ctypes.byref(aa), ll, nl, None,
                                     ctypes.byref(out)) == code, L.irt_last_error()
    bad_idx = np.array([[1, 0, 7]], np.int32)   # a collisional level index out of range
    mm = model()
    mm.coll_up = bad_idx.ctypes.data_as(B._IP)
    mm.ncoll = 3
    assert L.irt_create_ot_table(ctypes.byref(mm), ctypes.byref(ax), lines, 1, None,
                                 ctypes.byref(out)) == B.IRT_EINVAL
    line = _line(B)
    dust = B.irt_dust(0.01, 2.8)
    job = B.irt_job(None, B.irt_view(0, 0, 4, 4, 1.0, 0), B.irt_vaxis(4, -2.0, 1.0, 1),
                    B.irt_cubes(1, None, None, None, None))
    opts = B.irt_opts(0, 1, 0, 2.725, 0, 0)
    assert L.irt_forward_ppv_ot(ctypes.byref(job), 1, None, 0, ctypes.byref(line),
                                ctypes.byref(dust), ctypes.byref(opts), None) == B.IRT_EINVAL
    assert L.irt_grid_set_h2_fraction(None, None, 0, None) == B.IRT_EINVAL


def test_ot_table_refuses_a_level_pair_listed_twice(B):
    """The grid build adds each transition's rates in place, so a partner (or
    the radiative list) naming one level pair twice is refused."""
    import numpy as np
    from synth.levels import rotor_model
    m = rotor_model(nlev=5, partners=(0,))
    m["coll_up"] = np.array([[1, 1, 2]], np.int32)
    m["coll_lo"] = np.array([[0, 0, 1]], np.int32)
    m["k_ul_cm3_s"] = m["k_ul_cm3_s"][:, :3]
    keep = {k: np.ascontiguousarray(np.asarray(m[k], dtype=np.float64)) for k in
            ("energy_k", "g", "a_ul_s", "nu_hz", "coll_temp_k", "k_ul_cm3_s")}
    keepi = {k: np.ascontiguousarray(np.asarray(m[k], dtype=np.int32)) for k in
             ("rad_up", "rad_lo", "partner", "coll_up", "coll_lo")}
    dp = lambda a: a.ctypes.data_as(B._DP)  # noqa: E731
    ip = lambda a: a.ctypes.data_as(B._IP)  # noqa: E731
    mm = B.irt_level_model(5, dp(keep["energy_k"]), dp(keep["g"]), 4, ip(keepi["rad_up"]),
                           ip(keepi["rad_lo"]), dp(keep["a_ul_s"]), dp(keep["nu_hz"]), 1,
                           ip(keepi["partner"]), keep["coll_temp_k"].shape[-1],
                           dp(keep["coll_temp_k"]), 3, ip(keepi["coll_up"]), ip(keepi["coll_lo"]),
                           dp(keep["k_ul_cm3_s"]), 2.725, 3.0, 0.1)
    ax = B.irt_ot_axes(4, 3, 4, 1.0, 6.0, 0.1, 0.5, 1.0, 2.5)
    out = ctypes.c_void_p()
    assert B.lib.irt_create_ot_table(ctypes.byref(mm), ctypes.byref(ax), (ctypes.c_int * 1)(1), 1,
                                     None, ctypes.byref(out)) == B.IRT_EINVAL
    assert b"twice" in B.lib.irt_last_error()

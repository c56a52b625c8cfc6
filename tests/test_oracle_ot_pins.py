"""Pins of the oracle's optically thin (OT) level balance and its coefficient
grid (Sec. 3.4-3.6, 4.2, 4.3), CPU only.

Each check ties the solver to something it does not compute itself: the
textbook two-level solution, Boltzmann populations in the limits where
collisions or the radiation background alone set them, detailed balance at
T-bar = T, the bookkeeping of the collision partners, multilinear
reproduction by the table lookup, and an end-to-end render that must equal
the (separately pinned) LTE render where the OT balance reaches LTE.
"""
from __future__ import annotations

import math

import numpy as np
import pytest

import oracle
from synth import DUST, VelocityAxis, View
from synth.levels import (PARTNER_H, PARTNER_H2, PARTNER_HE, PARTNER_OH2, PARTNER_PH2,
                          rotor_model, two_level_model)

H = 6.62607015e-27
KB = 1.380649e-16
C = 2.99792458e10


def planck(nu, T):
    if T <= 0:
        return 0.0
    return 2 * H * nu ** 3 / C ** 2 / math.expm1(H * nu / (KB * T))


def boltzmann(model, T):
    w = model["g"] * np.exp(-(model["energy_k"] - model["energy_k"][0]) / T)
    return w / w.sum()


@pytest.mark.parametrize("n_h,chi,T", [(1e2, 0.5, 30.0), (3e4, 0.2, 55.0), (1e6, 0.45, 8.0),
                                       (50.0, 0.05, 400.0)])
def test_two_level_closed_form(n_h, chi, T):
    """n_u / n_l = (C_lu + B_lu J) / (C_ul + A + B_ul J) for two levels, with
    C_ul = K(T) n_H2, K linear in T between its tabulated values and held at
    the ends, C_lu by detailed balance, J = B_nu(T-bar)."""
    m = two_level_model(k_ul_cm3_s=2.0e-11, temps_k=(10.0, 100.0))
    m["k_ul_cm3_s"] = np.array([[[1.0e-11, 4.0e-11]]])
    K = np.interp(T, [10.0, 100.0], [1.0e-11, 4.0e-11])
    nu, A = m["nu_hz"][0], m["a_ul_s"][0]
    gl, gu = m["g"]
    B_ul = C ** 2 * A / (2 * H * nu ** 3)
    B_lu = gu / gl * B_ul
    J = planck(nu, m["t_rad_k"])
    C_ul = K * chi * n_h
    C_lu = C_ul * gu / gl * math.exp(-m["energy_k"][1] / T)
    ratio = (C_lu + B_lu * J) / (C_ul + A + B_ul * J)
    f = oracle.ot_populations(m, n_h, chi, T)
    assert f.sum() == pytest.approx(1.0, rel=1e-14)
    assert f[1] / f[0] == pytest.approx(ratio, rel=1e-12)


@pytest.mark.parametrize("n_h", [1e-2, 1e2, 1e5, 1e9])
def test_background_at_gas_temperature_gives_boltzmann_at_any_density(n_h):
    """With T-bar = T every process balances pairwise (collisions by detailed
    balance, radiation by the Einstein relations), so the populations are
    Boltzmann at T whatever the density."""
    T = 37.0
    m = rotor_model(nlev=14, t_rad_k=T)
    f = oracle.ot_populations(m, n_h, 0.35, T)
    np.testing.assert_allclose(f, boltzmann(m, T), rtol=1e-9, atol=1e-15)


def test_high_density_reaches_lte_at_the_gas_temperature():
    m = rotor_model(nlev=14, t_rad_k=2.725)
    for T in (12.0, 60.0, 150.0):
        f = oracle.ot_populations(m, 1e14, 0.5, T)
        np.testing.assert_allclose(f, boltzmann(m, T), rtol=1e-6, atol=1e-14)


def test_low_density_follows_the_radiation_background():
    """Without collisions the radiative chain J -> J-1 brings the levels to
    Boltzmann at T-bar; with T-bar = 0 every molecule sits in the ground
    state."""
    m = rotor_model(nlev=10, t_rad_k=15.0)
    f = oracle.ot_populations(m, 1e-10, 0.5, 80.0)
    np.testing.assert_allclose(f, boltzmann(m, 15.0), rtol=1e-7, atol=1e-15)
    m0 = rotor_model(nlev=10, t_rad_k=0.0)
    f0 = oracle.ot_populations(m0, 1e-10, 0.5, 80.0)
    assert f0[0] == pytest.approx(1.0, abs=1e-12)
    assert np.all(np.abs(f0[1:]) < 1e-12)


def test_populations_sum_to_one_and_are_non_negative():
    m = rotor_model(nlev=20)
    rng = np.random.default_rng(4)
    for _ in range(40):
        n_h = 10 ** rng.uniform(-1, 9)
        chi = rng.uniform(0.0, 0.5)
        T = 10 ** rng.uniform(0.7, 3.3)
        f = oracle.ot_populations(m, n_h, chi, T)
        assert f.sum() == pytest.approx(1.0, rel=1e-12)
        assert np.all(f >= -1e-15)


def test_collision_partner_densities():
    """Partner bookkeeping: an H2-only model depends on chi n_H alone; p-H2
    and o-H2 with equal rates act as total H2 (the ortho/para split sums to
    n_H2); H sees n_H (1 - 2 chi); He sees x_He n_H."""
    base = rotor_model(nlev=8, partners=(PARTNER_H2,), seed=3)
    T = 45.0
    a = oracle.ot_populations(base, 2e3, 0.5, T)
    b = oracle.ot_populations(base, 1e4, 0.1, T)        # same chi n_H
    np.testing.assert_allclose(a, b, rtol=1e-12)
    split = dict(base)
    split["partner"] = np.array([PARTNER_PH2, PARTNER_OH2], np.int32)
    for k in ("coll_temp_k", "coll_up", "coll_lo", "k_ul_cm3_s"):
        split[k] = np.concatenate([base[k], base[k]], axis=0)
    np.testing.assert_allclose(oracle.ot_populations(split, 2e3, 0.5, T), a, rtol=1e-12)
    hmod = dict(base)
    hmod["partner"] = np.array([PARTNER_H], np.int32)
    # n_H (1 - 2 chi) = 1e3 in both cases
    np.testing.assert_allclose(oracle.ot_populations(hmod, 2e3, 0.25, T),
                               oracle.ot_populations(hmod, 1e4, 0.45, T), rtol=1e-12)
    # and equals the H2-only model at the same partner density
    np.testing.assert_allclose(oracle.ot_populations(hmod, 2e3, 0.25, T),
                               oracle.ot_populations(base, 2e3, 0.5, T), rtol=1e-12)
    he = dict(base)
    he["partner"] = np.array([PARTNER_HE], np.int32)
    he["x_he"] = 0.25
    np.testing.assert_allclose(oracle.ot_populations(he, 4e3, 0.3, T), a, rtol=1e-12)


def _poly_table_values(n, lo, hi, coeffs):
    ax = [np.linspace(lo[a], hi[a], n[a]) for a in range(3)]
    A, B, Cc = np.meshgrid(*ax, indexing="ij")
    out = np.zeros((1,) + tuple(n) + (2,))
    for q in range(2):
        c = coeffs[q]
        out[0, ..., q] = (c[0] + c[1] * A + c[2] * B + c[3] * Cc + c[4] * A * B + c[5] * B * Cc
                          + c[6] * Cc * A + c[7] * A * B * Cc)
    return out


def test_lookup_reproduces_multilinear_tables_inside_and_beyond_the_bounds():
    """Trilinear interpolation in (log10 n_H, chi, log10 T) reproduces any
    multilinear function of the three coordinates exactly; outside the grid
    the edge cell continues it (the linear extrapolation of Sec. 4.2)."""
    axes = dict(n_n=7, n_chi=5, n_t=6, log10_nh_min=1.0, log10_nh_max=7.0, chi_min=0.05,
                chi_max=0.5, log10_t_min=math.log10(5.0), log10_t_max=math.log10(500.0))
    n = (7, 5, 6)
    lo = (1.0, 0.05, math.log10(5.0))
    hi = (7.0, 0.5, math.log10(500.0))
    rng = np.random.default_rng(8)
    coeffs = rng.uniform(-1, 1, (2, 8))
    model = rotor_model(nlev=4)
    t = oracle.OTTable(model, axes, [1], values=_poly_table_values(n, lo, hi, coeffs))
    for _ in range(60):
        a = rng.uniform(-1.0, 9.0)          # beyond both ends too
        b = rng.uniform(-0.1, 0.7)
        c = rng.uniform(0.3, 3.2)
        j, al = t.lookup(0, 10 ** a, b, 10 ** c)
        for q, got in ((0, j), (1, al)):
            cq = coeffs[q]
            want = (cq[0] + cq[1] * a + cq[2] * b + cq[3] * c + cq[4] * a * b + cq[5] * b * c
                    + cq[6] * c * a + cq[7] * a * b * c)
            assert got == pytest.approx(want, rel=1e-11, abs=1e-11)
    t.close()


def _rotor_line(model, r, mass_amu=28.99827, t_inf=5e4, sigma=1.0):
    """The LTE line constants of radiative transition r of a rotor model."""
    u, l = int(model["rad_up"][r]), int(model["rad_lo"][r])
    b0 = model["nu_hz"][0] / 2.0
    return dict(nu_ul_hz=float(model["nu_hz"][r]), a_ul_s=float(model["a_ul_s"][r]),
                e_u_k=float(model["energy_k"][u]), b0_hz=float(b0), g_u=float(model["g"][u]),
                g_l=float(model["g"][l]), mass_amu=mass_amu, t_inf_k=t_inf,
                sigma_turb_kms=sigma)


def test_table_nodes_at_high_density_equal_lte_coefficients():
    """At densities where collisions dominate, the grid's per-molecule
    coefficients of the 2-1 line equal the LTE ones of the same rotor."""
    m = rotor_model(nlev=40)
    axes = dict(n_n=3, n_chi=2, n_t=5, log10_nh_min=13.0, log10_nh_max=15.0, chi_min=0.3,
                chi_max=0.5, log10_t_min=1.0, log10_t_max=2.2)
    t = oracle.OTTable(m, axes, [1])
    v = t.values()
    line = _rotor_line(m, 1)
    Ts = np.logspace(1.0, 2.2, 5)
    for it, T in enumerate(Ts):
        c = oracle.sample_coeffs(line, DUST, 1.0, float(T), 1.0)
        for i_n in range(3):
            for i_c in range(2):
                assert v[0, i_n, i_c, it, 0] == pytest.approx(c["jL"], rel=1e-6)
                assert v[0, i_n, i_c, it, 1] == pytest.approx(c["aL"], rel=1e-6)
    t.close()


def test_ot_render_at_lte_densities_equals_the_lte_render():
    """End to end: every cell at a density node of a high-density grid and a
    temperature node (so the lookup lands on nodes), an H2 abundance field
    on its nodes too; the OT render must equal the LTE render of the same
    rotor line (optically thick at the line centre), for both integrators."""
    m = rotor_model(nlev=40)
    axes = dict(n_n=3, n_chi=3, n_t=9, log10_nh_min=13.0, log10_nh_max=14.0, chi_min=0.1,
                chi_max=0.5, log10_t_min=1.0, log10_t_max=2.0)
    t = oracle.OTTable(m, axes, [0, 1, 2])
    line = _rotor_line(m, 1)
    rng = np.random.default_rng(12)
    n = 6
    shape = (n, n, n)
    chi = rng.choice(np.linspace(0.1, 0.5, 3), size=shape)
    nh = 10 ** rng.choice(np.linspace(13.0, 14.0, 3), size=shape)
    n_h2 = nh * chi
    T = 10 ** rng.choice(np.linspace(1.0, 2.0, 9), size=shape)
    v = rng.normal(0.0, 3.0, shape)
    x = np.full(shape, 3e-12)
    fields = (n_h2, T, T.copy(), v, x)
    dx = 3.0856775814913673e16
    dust = dict(DUST, kappa_cm2_per_g_gas=1e-9)   # dust would be opaque at these densities
    va = VelocityAxis(24, -12.0, 1.0, 2)
    pix = [(i, j) for j in range(n) for i in range(n)]
    for integ in (oracle.SMOOTH, oracle.FORMAL):
        zv = View(0.0, 0.0, n, n, dx, 0)
        a = oracle.render(fields, dx, line, dust, zv, va, pix, integration=integ)
        b = oracle.render(fields, dx, line, dust, zv, va, pix, integration=integ, levels=t,
                          line_index=1, chi=chi)
        peak = np.abs(a["T"]).max()
        # thick: the line saturates near the source function in places
        assert np.abs(a["L"]).max() > 0.3 * peak
        for k in "TCDLB":
            np.testing.assert_allclose(b[k], a[k], rtol=1e-6, atol=1e-9 * peak)
    # a different line index of the same grid gives a different cube
    c = oracle.render(fields, dx, line, dust, View(0.0, 0.0, n, n, dx, 0), va, pix,
                      levels=t, line_index=2, chi=chi)
    assert np.abs(c["L"] - b["L"]).max() > 1e-3 * np.abs(b["L"]).max()
    t.close()


def test_ot_line_vanishes_without_tracer_or_h2_or_above_t_inf():
    m = rotor_model(nlev=12)
    axes = dict(n_n=4, n_chi=3, n_t=4, log10_nh_min=2.0, log10_nh_max=6.0, chi_min=0.1,
                chi_max=0.5, log10_t_min=1.0, log10_t_max=2.5)
    t = oracle.OTTable(m, axes, [1])
    line = _rotor_line(m, 1, t_inf=60.0)
    n = 4
    shape = (n, n, n)
    fields = (np.full(shape, 1e4), np.full(shape, 30.0), np.full(shape, 30.0),
              np.zeros(shape), np.full(shape, 2e-6))
    dx = 3.0856775814913673e17
    va = VelocityAxis(16, -8.0, 1.0, 1)
    pix = [(1, 2)]
    zv = View(0.0, 0.0, n, n, dx, 0)
    base = oracle.render(fields, dx, line, DUST, zv, va, pix, levels=t, line_index=0)
    assert np.abs(base["L"]).max() > 0.0
    for case in ("x0", "chi0", "hot"):
        f = [a.copy() for a in fields]
        chi = np.full(shape, 0.5)
        if case == "x0":
            f[4][:] = 0.0
        elif case == "chi0":
            chi[:] = 0.0
        else:
            f[1][:] = 80.0
        r = oracle.render(tuple(f), dx, line, DUST, zv, va, pix, levels=t, line_index=0, chi=chi)
        assert np.abs(r["L"]).max() < 1e-9 * np.abs(base["T"]).max(), case
    t.close()

"""Pins of the FP64 oracle against facts other than its own code.

Each test checks the oracle against a closed form, a textbook identity, a
value printed in the paper or an independent ODE solver, chosen so that a
plausible mistake (a dropped term, a wrong sign or index, a swapped weight)
fails at least one of them.  All run on CPU.
"""
import math

import numpy as np
import pytest
from scipy import integrate, optimize

import oracle
from synth import DUST, LINE_13CO_21, VelocityAxis, View, make_fields
from tests.conftest import golden

# CODATA 2018 / physical constants used by the independent formulas below
H = 6.62607015e-27
KB = 1.380649e-16
C = 2.99792458e10
CKMS = 2.99792458e5
AMU = 1.66053906660e-24

LINE = dict(LINE_13CO_21)
NU = LINE["nu_ul_hz"]
T0 = H * NU / KB                       # h nu / k  [K]
THETA_ROT = H * LINE["b0_hz"] / KB     # rotational temperature h B0 / k  [K]
NO_DUST = dict(DUST, kappa_cm2_per_g_gas=0.0)


def J(T, nu=NU):
    """Planck intensity at nu expressed as a Rayleigh-Jeans temperature [K]."""
    if T <= 0:
        return 0.0
    x = H * nu / (KB * T)
    return (H * nu / KB) / math.expm1(x)


def B(nu, T):
    """Planck's law, cgs."""
    return 2 * KB * nu * nu / (C * C) * J(T, nu)


def z_rotor(T):
    """High-temperature expansion of the rigid-rotor partition function."""
    r = THETA_ROT / T
    return 1.0 / r + 1.0 / 3.0 + r / 15.0 + 4.0 * r * r / 315.0 + r ** 3 / 315.0


def z_sum(T):
    """Rigid-rotor partition function by direct summation (pinned against
    the high-temperature expansion in the first test)."""
    J = np.arange(400.0)
    return float(np.sum((2 * J + 1) * np.exp(-THETA_ROT * J * (J + 1) / T)))


def nu_of_u(u):
    return NU * (1.0 - u / CKMS)


def textbook_coeffs(n_h2, T, x, sigma_turb=LINE["sigma_turb_kms"]):
    """Line coefficients in the textbook 'opacity' form, independent of the
    Einstein-B route: j = h nu A n_u / 4pi,
    alpha = c^2 A g_u n_l (1 - exp(-h nu / kT)) / (8 pi nu^2 g_l)."""
    N = x * n_h2
    Z = z_sum(T)
    n_u = N * LINE["g_u"] * math.exp(-LINE["e_u_k"] / T) / Z
    n_l = n_u * (LINE["g_l"] / LINE["g_u"]) * math.exp(T0 / T)
    j = H * NU * LINE["a_ul_s"] * n_u / (4 * math.pi)
    a = C * C * LINE["a_ul_s"] * LINE["g_u"] * n_l * (-math.expm1(-T0 / T)) / (
        8 * math.pi * NU * NU * LINE["g_l"])
    # 1-D velocity dispersion: thermal kT/m plus microturbulent sigma^2
    var = KB * T / (LINE["mass_amu"] * AMU) / 1e10 + sigma_turb ** 2
    return n_u, n_l, j, a, var


def gauss_phi_hz(u, v, var):
    """Normalised Gaussian in velocity (variance var) converted to per Hz."""
    phi_v = math.exp(-0.5 * (u - v) ** 2 / var) / math.sqrt(2 * math.pi * var)
    return phi_v * CKMS / NU


def uniform_samples(K, n=1e4, T=20.0, Td=None, v=0.0, x=2e-6):
    return dict(n_h2=np.full(K, n), t_gas=np.full(K, T), t_dust=np.full(K, T if Td is None else Td),
                v_los=np.full(K, v), x_tr=np.full(K, x))


# ----------------------------------------------------------------------------
# level populations and coefficients
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("T,tol", [(20.0, 2e-6), (60.0, 1e-8), (100.0, 1e-9)])
def test_partition_function_matches_rotor_expansion(T, tol):
    assert oracle.partition(LINE, T) == pytest.approx(z_rotor(T), rel=tol)
    assert z_sum(T) == pytest.approx(z_rotor(T), rel=tol)


@pytest.mark.parametrize("T", [5.0, 20.0, 60.0, 100.0, 300.0])
def test_lte_source_function_is_planck(T):
    """Kirchhoff: in LTE the line source function j/alpha equals B_nu(T)."""
    c = oracle.sample_coeffs(LINE, DUST, 1e4, T, 2e-6)
    assert c["jL"] / c["aL"] == pytest.approx(B(NU, T), rel=1e-12)
    assert c["n_u"] / c["n_l"] == pytest.approx(5.0 / 3.0 * math.exp(-T0 / T), rel=1e-13)


@pytest.mark.parametrize("T", [20.0, 100.0])
def test_line_coefficients_textbook_form(T):
    c = oracle.sample_coeffs(LINE, DUST, 3e4, T, 2e-6)
    n_u, n_l, j, a, var = textbook_coeffs(3e4, T, 2e-6)
    tol = 1e-13
    assert c["n_u"] == pytest.approx(n_u, rel=tol)
    assert c["jL"] == pytest.approx(j, rel=tol)
    assert c["aL"] == pytest.approx(a, rel=tol)
    assert c["b_kms"] ** 2 / 2 == pytest.approx(var, rel=1e-13)


def test_temperature_cutoff_and_dust_alpha():
    hot = oracle.sample_coeffs(LINE, DUST, 1e4, 6e4, 2e-6)
    assert hot["jL"] == 0.0 and hot["aL"] == 0.0
    c = oracle.sample_coeffs(LINE, DUST, 1e4, 20.0, 2e-6)
    rho = 1e4 * 2 * (1.00794 + 0.1 * 4.002602) * AMU
    assert c["aD"] == pytest.approx(1e-2 * rho, rel=1e-14)


def test_profile_moments():
    """Unit area in frequency, centroid at v_los, variance kT/m + sigma^2."""
    T, v = 40.0, 3.7
    var = KB * T / (LINE["mass_amu"] * AMU) / 1e10 + LINE["sigma_turb_kms"] ** 2
    f = lambda u: oracle.profile_per_hz(LINE, T, v, u) * NU / CKMS   # per km/s
    lo, hi = v - 30, v + 30
    m0 = integrate.quad(f, lo, hi, epsabs=0, epsrel=1e-12, limit=200)[0]
    m1 = integrate.quad(lambda u: u * f(u), lo, hi, epsabs=0, epsrel=1e-12, limit=200)[0]
    m2 = integrate.quad(lambda u: (u - v) ** 2 * f(u), lo, hi, epsabs=0, epsrel=1e-12, limit=200)[0]
    assert m0 == pytest.approx(1.0, rel=1e-10)
    assert m1 == pytest.approx(v, rel=1e-10)
    assert m2 == pytest.approx(var, rel=1e-9)


def test_rj_to_planck_example_sec58():
    (nu, t_rj, t_b_printed), = golden("rj_planck_example.txt")
    I = 2 * KB * nu * nu * t_rj / (C * C)
    tb = optimize.brentq(lambda T: oracle.planck(nu, T) - I, 0.5, 50.0, xtol=1e-14)
    assert round(tb, 1) == t_b_printed


def test_planck_limits():
    # Rayleigh-Jeans limit h nu << kT and Wien limit h nu >> kT
    T = 1e7
    assert oracle.planck(NU, T) == pytest.approx(2 * NU * NU * KB * T / C ** 2 * (1 - T0 / (2 * T)),
                                                 rel=1e-10)
    T = 0.2
    assert oracle.planck(NU, T) == pytest.approx(2 * H * NU ** 3 / C ** 2 * math.exp(-T0 / T),
                                                 rel=1e-20 + math.exp(-T0 / T) * 2)


def test_dust_opacity_derivation_sec55():
    (lam, rho, mr, mi, kd_printed, kg_printed), = golden("dust_opacity_derivation.txt")
    m = complex(mr, mi)
    kd = 6 * math.pi / (lam * rho) * ((m * m - 1) / (m * m + 2)).imag
    assert kd == pytest.approx(kd_printed, rel=0.01)
    kg_cgs = kd / 100.0 * 1e4 / 1e3            # m^2/kg of dust -> cm^2/g of gas
    assert kg_cgs == pytest.approx(kg_printed, rel=0.01)
    assert DUST["kappa_cm2_per_g_gas"] == pytest.approx(kg_printed, rel=0.01)


# ----------------------------------------------------------------------------
# uniform slab: closed forms
# ----------------------------------------------------------------------------
def slab_expected_formal(K, h, T, x, n, vaxis, Td=None, kappa=0.0, t_bg=2.725, v=0.0):
    """Per fine point: I = B_bg e^-tau + S (1 - e^-tau) with constant
    coefficients; channel value = Simpson average (f >= 1) or the centre (f = 0)."""
    n_u, n_l, j, a, var = textbook_coeffs(n, T, x)
    rho = n * DUST["mu_mass_per_h2_amu"] * AMU
    aD = kappa * rho
    Td = T if Td is None else Td

    def I_at(u):
        nu = nu_of_u(u)
        phi = gauss_phi_hz(u, v, var)
        jt = j * phi + aD * B(nu, Td)
        at = a * phi + aD
        tau = K * h * at
        return B(nu, t_bg) * math.exp(-tau) + jt / at * (-math.expm1(-tau))

    out = []
    f = vaxis.subsample_f
    for c in range(vaxis.nchan):
        uc = vaxis.v_first_edge_kms + (c + 0.5) * vaxis.dv_kms
        if f == 0:
            ibar = I_at(uc)
        else:
            dvf = vaxis.dv_kms / (2 * f)
            w = np.ones(2 * f + 1)
            w[1::2] = 4
            w[2:-1:2] = 2
            us = vaxis.v_first_edge_kms + c * vaxis.dv_kms + dvf * np.arange(2 * f + 1)
            ibar = sum(wi * I_at(ui) for wi, ui in zip(w, us)) / (6 * f)
        nuc = nu_of_u(uc)
        tauc = K * h * aD
        ic = B(nuc, t_bg) * math.exp(-tauc) + (B(nuc, Td) * (-math.expm1(-tauc)) if aD else 0.0)
        s = C * C / (2 * KB * nuc * nuc)
        out.append((ibar * s, ic * s, B(nuc, t_bg) * s))
    return np.array(out)


@pytest.mark.parametrize("f", [0, 1, 3])
@pytest.mark.parametrize("kappa", [0.0, 5.0])
def test_uniform_slab_formal_closed_form(f, kappa):
    va = VelocityAxis(12, -6.0, 1.0, f)
    K, h, T, x, n = 7, 3e16, 30.0, 2e-6, 2e4
    dust = dict(DUST, kappa_cm2_per_g_gas=kappa)
    r = oracle.ray(LINE, dust, va, uniform_samples(K, n, T, x=x, Td=18.0, v=0.4), h,
                   integration=oracle.FORMAL)
    exp = slab_expected_formal(K, h, T, x, n, va, Td=18.0, kappa=kappa, v=0.4)
    np.testing.assert_allclose(r["T"], exp[:, 0], rtol=1e-11)
    np.testing.assert_allclose(r["C"], exp[:, 1], rtol=1e-12)
    np.testing.assert_allclose(r["B"], exp[:, 2], rtol=1e-13)


def test_slab_line_equals_J_difference_times_opacity_factor():
    """Dust-free, continuum-subtracted, centre-sampled:
    [L] = (J(T_ex) - J(T_bg)) (1 - e^-tau) up to the O(v/c) shift of the
    channel frequency."""
    va = VelocityAxis(1, -0.5, 1.0, 0)
    K, h, T, x, n = 10, 3.0856775814913673e17, 20.0, 2e-6, 1e4
    r = oracle.ray(LINE, NO_DUST, va, uniform_samples(K, n, T, x=x), h,
                   integration=oracle.FORMAL)
    n_u, n_l, j, a, var = textbook_coeffs(n, T, x)
    tau = K * h * a * gauss_phi_hz(0.0, 0.0, var)
    assert r["L"][0] == pytest.approx((J(T) - J(2.725)) * -math.expm1(-tau), rel=1e-9)
    assert abs(r["D"][0]) == 0.0


@pytest.mark.parametrize("hscale", [0.01, 0.3, 4.0])
def test_uniform_slab_smooth_recurrence_closed_form(hscale):
    """TR first step + BDF2 with constant coefficients is a linear recurrence:
    e_n = I_n - S obeys (3 + 2 h a) e_{n+2} - 4 e_{n+1} + e_n = 0 with e_1 from
    TR; solved with its characteristic roots (complex when 2 h a > 1)."""
    va = VelocityAxis(1, -0.5, 1.0, 0)
    K, T, x, n = 40, 25.0, 2e-6, 1e4
    n_u, n_l, j, a, var = textbook_coeffs(n, T, x)
    at = a * gauss_phi_hz(0.0, 0.0, var)
    h = hscale / at
    r = oracle.ray(LINE, NO_DUST, va, uniform_samples(K, n, T, x=x), h,
                   integration=oracle.SMOOTH, units=oracle.INTENSITY)
    nuc = nu_of_u(0.0)
    S = B(NU, T)
    e0 = B(nuc, 2.725) - S
    ha = h * at
    e1 = (2 - ha) / (2 + ha) * e0
    disc = np.sqrt(complex(1 - 2 * ha))
    r1, r2 = (2 + disc) / (3 + 2 * ha), (2 - disc) / (3 + 2 * ha)
    A_ = (e1 - r2 * e0) / (r1 - r2)
    B_ = e0 - A_
    m = K - 2   # BDF2 steps after the TR step: e_{K-1} = A r1^(K-1) + B r2^(K-1)
    eK = (A_ * r1 ** (m + 1) + B_ * r2 ** (m + 1)).real
    assert r["T"][0] == pytest.approx(S + eK, rel=1e-11, abs=1e-12 * S)


def test_smooth_converges_second_order_to_continuum_slab():
    """Smooth integration over (K-1) h -> exact slab solution at O(h^2)."""
    va = VelocityAxis(1, -0.5, 1.0, 0)
    T, x, n = 25.0, 2e-6, 1e4
    n_u, n_l, j, a, var = textbook_coeffs(n, T, x)
    at = a * gauss_phi_hz(0.0, 0.0, var)
    L = 3.0 / at
    S = B(NU, T)
    I0 = B(nu_of_u(0.0), 2.725)
    exact = S + (I0 - S) * math.exp(-at * L)
    errs = []
    for K in (41, 81, 161):
        h = L / (K - 1)
        r = oracle.ray(LINE, NO_DUST, va, uniform_samples(K, n, T, x=x), h,
                       integration=oracle.SMOOTH, units=oracle.INTENSITY)
        errs.append(abs(r["T"][0] - exact))
    assert 3.5 < errs[0] / errs[1] < 4.5
    assert 3.5 < errs[1] / errs[2] < 4.5


@pytest.mark.parametrize("mode", [oracle.FORMAL, oracle.SMOOTH])
def test_thick_limit_saturates_to_source_function(mode):
    va = VelocityAxis(3, -1.5, 1.0, 0)
    T = 35.0
    r = oracle.ray(LINE, NO_DUST, va, uniform_samples(64, 1e5, T, x=1e-2), 3e17,
                   integration=mode)
    uc = 0.0
    s = C * C / (2 * KB * nu_of_u(uc) ** 2)
    assert r["T"][1] == pytest.approx(B(NU, T) * s, rel=1e-12)
    assert r["L"][1] == pytest.approx((B(NU, T) - B(nu_of_u(uc), 2.725)) * s, rel=1e-12)


@pytest.mark.parametrize("f", [1, 4])
def test_thin_limit_integrated_intensity_tracks_column_density(f):
    """Optically thin, no dust, no background: sum_c [L]_c dv equals
    h c^3 A N_u / (8 pi k nu^2) (the upper-level column), Sec. 5.10."""
    nch = 48
    va = VelocityAxis(nch, -12.0, 0.5, f)
    K, h = 16, 3e17
    rng = np.random.default_rng(5)
    smp = dict(n_h2=rng.uniform(5e3, 5e4, K), t_gas=rng.uniform(20, 80, K),
               t_dust=np.full(K, 20.0), v_los=rng.uniform(-1.0, 1.0, K), x_tr=np.full(K, 1e-16))
    r = oracle.ray(LINE, NO_DUST, va, smp, h, integration=oracle.FORMAL, t_bg=0.0)
    n_u = np.array([textbook_coeffs(n, T, 1e-16)[0] for n, T in zip(smp["n_h2"], smp["t_gas"])])
    Ncol = n_u.sum() * h
    W = r["L"].sum() * va.dv_kms * 1e5                       # K cm/s
    expected = H * C ** 3 * LINE["a_ul_s"] * Ncol / (8 * math.pi * KB * NU ** 2)
    assert W / expected == pytest.approx(1.0, abs=1e-4)
    smp2 = dict(smp, x_tr=np.full(K, 2e-16))
    r2 = oracle.ray(LINE, NO_DUST, va, smp2, h, integration=oracle.FORMAL, t_bg=0.0)
    assert r2["L"].sum() / r["L"].sum() == pytest.approx(2.0, rel=1e-8)


@pytest.mark.parametrize("mode", [oracle.FORMAL, oracle.SMOOTH])
def test_component_identities(mode):
    rng = np.random.default_rng(1)
    K = 24
    smp = dict(n_h2=rng.lognormal(9, 1.5, K), t_gas=rng.uniform(20, 100, K),
               t_dust=rng.uniform(15, 40, K), v_los=rng.normal(0, 3, K), x_tr=np.full(K, 2e-6))
    va = VelocityAxis(20, -10.0, 1.0, 2)
    r = oracle.ray(LINE, DUST, va, smp, 3e17, integration=mode)
    np.testing.assert_allclose(r["T"], r["C"] + r["L"], rtol=1e-15, atol=0)
    np.testing.assert_allclose(r["C"], r["B"] + r["D"], rtol=1e-15, atol=0)
    # kappa = 0 -> no dust excess
    r0 = oracle.ray(LINE, NO_DUST, va, smp, 3e17, integration=mode)
    np.testing.assert_allclose(r0["D"], 0.0, atol=4e-16 * r0["B"].max())   # BDF2 rounding
    # x = 0 -> no line.  [T] is the Simpson average of the dust and
    # background spectrum over the fine points while [C] takes the channel
    # value (Sec. 4.4), so the identity holds up to that curvature term.
    rx = oracle.ray(LINE, DUST, va, dict(smp, x_tr=np.zeros(K)), 3e17, integration=mode)
    np.testing.assert_allclose(rx["L"], 0.0, atol=1e-9 * rx["C"].max())
    # kappa = 0 and no background -> no continuum
    rc = oracle.ray(LINE, NO_DUST, va, smp, 3e17, integration=mode, t_bg=0.0)
    assert np.all(rc["C"] == 0.0)
    # dust in equilibrium with the background -> no dust excess
    re = oracle.ray(LINE, dict(DUST, kappa_cm2_per_g_gas=30.0), va,
                    dict(smp, t_dust=np.full(K, 2.725)), 3e17, integration=mode)
    np.testing.assert_allclose(re["D"], 0.0, atol=1e-14 * re["B"].max())


# ----------------------------------------------------------------------------
# Table 4: delta v = dv / (2 f) and the Simpson weights
# ----------------------------------------------------------------------------
def test_table4_fine_step_and_simpson_weights():
    rows = golden("table4_velocity_subsampling.txt")
    dv = rows[0][1]
    dv = 3.125   # the printed 3.13 is this channel width rounded
    narrow = dict(LINE, sigma_turb_kms=0.0)
    for f, dvf_printed in rows[1:]:
        f = int(f)
        va = VelocityAxis(1, -dv / 2, dv, f)
        vals = []
        for m in range(2 * f + 1):
            # a narrow line (T = 6 K, b = 0.059 km/s) placed on the m-th fine
            # point as printed in Table 4 (3 significant figures: the printed
            # step is off by at most 0.005 km/s after 2f steps)
            u = -dv / 2 + m * dvf_printed
            smp = uniform_samples(1, 1e4, 6.0, Td=6.0, v=u, x=1e-12)
            r = oracle.ray(narrow, NO_DUST, va, smp, 3e16, integration=oracle.FORMAL, t_bg=0.0)
            vals.append(r["L"][0])
        vals = np.array(vals)
        w = np.ones(2 * f + 1)
        w[1::2] = 4
        w[2:-1:2] = 2
        np.testing.assert_allclose(vals / vals[1], w / 4.0, rtol=2e-2)


# ----------------------------------------------------------------------------
# brute force: independent ODE solver on a 4^3 grid (formal mode is exact for
# piecewise-constant coefficients)
# ----------------------------------------------------------------------------
def test_brute_force_4cube_formal_vs_ode_solver():
    fs = make_fields(4, seed=77)
    fields = fs.as_tuple()
    dx = 0.1 * 3.0856775814913673e18
    va = VelocityAxis(6, -60.0, 20.0, 2)
    dust = dict(DUST, kappa_cm2_per_g_gas=3.0)
    view = View(0.0, 0.0, 4, 4, dx, 0)
    pix = [(1, 2), (3, 0)]
    r = oracle.render(fields, dx, LINE, dust, view, va, pix, integration=oracle.FORMAL)
    f = va.subsample_f
    dvf = va.dv_kms / (2 * f)
    w = np.ones(2 * f + 1)
    w[1::2] = 4
    w[2:-1:2] = 2
    for ip, (px, py) in enumerate(pix):
        cells = []
        for k in range(4):
            n, T, Td, v, x = (a[k, py, px] for a in fields)
            _, _, j, a_, var = textbook_coeffs(n, T, x)
            aD = dust["kappa_cm2_per_g_gas"] * n * DUST["mu_mass_per_h2_amu"] * AMU
            cells.append((j, a_, var, v, aD, Td))

        def solve(u, line_on):
            nu = nu_of_u(u)
            I = B(nu, 2.725)
            for (j, a_, var, v, aD, Td) in cells:
                phi = gauss_phi_hz(u, v, var) if line_on else 0.0
                jt, at = j * phi + aD * B(nu, Td), a_ * phi + aD
                sol = integrate.solve_ivp(lambda s, y: jt - at * y, (0.0, dx), [I],
                                          method="DOP853", rtol=1e-12, atol=1e-30)
                I = sol.y[0, -1]
            return I

        for c in range(va.nchan):
            us = va.v_first_edge_kms + c * va.dv_kms + dvf * np.arange(2 * f + 1)
            ibar = sum(wi * solve(ui, True) for wi, ui in zip(w, us)) / (6 * f)
            uc = va.v_first_edge_kms + (c + 0.5) * va.dv_kms
            s = C * C / (2 * KB * nu_of_u(uc) ** 2)
            assert r["T"][ip, c] == pytest.approx(ibar * s, rel=1e-8)
            assert r["C"][ip, c] == pytest.approx(solve(uc, False) * s, rel=1e-8)


# ----------------------------------------------------------------------------
# geometry
# ----------------------------------------------------------------------------
def _small_fields(n=6, seed=3):
    return make_fields(n, seed=seed).as_tuple()


def test_oblique_at_theta0_equals_z_view():
    fields = _small_fields()
    dx = 3.0856775814913673e17
    va = VelocityAxis(8, -40.0, 10.0, 1)
    zv = View(0.0, 0.0, 6, 6, dx, 0)
    ov = View(0.0, 0.0, 6, 6, dx, 1)
    a = oracle.render_cube(fields, dx, LINE, DUST, zv, va)
    b = oracle.render_cube(fields, dx, LINE, DUST, ov, va)
    for k in "TCDLB":
        np.testing.assert_allclose(b[k], a[k], rtol=1e-12, atol=1e-12 * abs(a["T"]).max())


def test_oblique_at_theta90_equals_transposed_z_view():
    fields = _small_fields()
    n = 6
    dx = 3.0856775814913673e17
    va = VelocityAxis(8, -40.0, 10.0, 1)
    ov = View(math.pi / 2, 0.0, n, n, dx, 1)
    b = oracle.render_cube(fields, dx, LINE, DUST, ov, va)
    # rays along +x; pixel (px, py) sees cells z = n-1-px, y = py, x = 0..n-1
    tf = tuple(np.ascontiguousarray(f.transpose(2, 1, 0)[:, :, ::-1]) for f in fields)
    a = oracle.render_cube(tf, dx, LINE, DUST, View(0.0, 0.0, n, n, dx, 0), va)
    for k in "TCDLB":
        np.testing.assert_allclose(b[k], a[k], rtol=1e-10, atol=1e-12 * abs(a["T"]).max())


def test_oblique_chord_sampling():
    fields = _small_fields()
    n = 6
    dx = 1.0
    view = View(math.radians(30.0), math.radians(45.0), n, n, dx, 1)
    smp, h = oracle.ray_samples(fields, dx, view, 2, 3)
    K = len(smp)
    d = np.array([math.sin(view.theta_rad) * math.cos(view.phi_rad),
                  math.sin(view.theta_rad) * math.sin(view.phi_rad), math.cos(view.theta_rad)])
    assert K >= 1 and h * K <= n * dx * math.sqrt(3) + 1e-12
    assert math.ceil(h * K / dx - 1e-9) == K
    # a corner pixel far outside the box projection misses it
    far = View(math.radians(30.0), math.radians(45.0), 4 * n, 4 * n, dx, 1)
    smp2, h2 = oracle.ray_samples(fields, dx, far, 0, 0)
    assert len(smp2) == 0 and d[2] > 0


def test_missed_ray_outputs_background_only():
    fields = _small_fields()
    n = 6
    dx = 3.0856775814913673e17
    va = VelocityAxis(4, -20.0, 10.0, 1)
    far = View(math.radians(30.0), math.radians(45.0), 4 * n, 4 * n, dx, 1)
    r = oracle.render(fields, dx, LINE, DUST, far, va, [(0, 0)])
    # [T] averages the background over the fine points (curvature ~1e-10)
    np.testing.assert_allclose(r["T"], r["B"], rtol=1e-9)
    np.testing.assert_array_equal(r["C"], r["B"])
    assert np.all(r["D"] == 0)
    np.testing.assert_allclose(r["L"], 0.0, atol=1e-9 * r["B"].max())


# ----------------------------------------------------------------------------
# gradient: dual numbers vs central differences of the primal oracle
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("mode", [oracle.SMOOTH, oracle.FORMAL])
def test_dual_gradient_matches_central_differences(mode):
    n = 4
    fs = make_fields(n, seed=11)
    fields = [a.copy() for a in fs.as_tuple()]
    dx = 3.0856775814913673e17
    va = VelocityAxis(10, -25.0, 5.0, 1)
    view = View(0.0, 0.0, n, n, dx, 0)
    tfs = make_fields(n, seed=18).as_tuple()
    target = oracle.render_cube(tfs, dx, LINE, DUST, view, va, integration=mode)["L"]
    loss, gn, gt, gv = oracle.loss_grad_zview(fields, dx, LINE, DUST, va, target,
                                              integration=mode)
    base = oracle.render_cube(fields, dx, LINE, DUST, view, va, integration=mode)["L"]
    assert loss == pytest.approx(np.mean((base - target) ** 2), rel=1e-12)
    rng = np.random.default_rng(0)
    for _ in range(6):
        z, y, x = rng.integers(0, n, 3)
        for q, g in ((0, gn), (1, gt), (3, gv)):
            v0 = fields[q][z, y, x]
            eps = 1e-6 * max(abs(v0), 1.0)
            vals = []
            for s in (+1, -1):
                fields[q][z, y, x] = v0 + s * eps
                Lc = oracle.render(fields, dx, LINE, DUST, view, va, [(x, y)],
                                   integration=mode)["L"][0]
                vals.append(np.sum((Lc - target[:, y, x]) ** 2))
            fields[q][z, y, x] = v0
            fd = (vals[0] - vals[1]) / (2 * eps) / target.size
            assert g[z, y, x] == pytest.approx(fd, rel=1e-5, abs=1e-9 * abs(g).max())


# ----------------------------------------------------------------------------
# gradients of any view: dual numbers through the stencils of the samples
# ----------------------------------------------------------------------------
def _grad_problem(n=7, seed=21, nch=14):
    fs = make_fields(n, seed)
    fields = fs.as_tuple()
    tgt_f = make_fields(n, seed + 7).as_tuple()
    dx = 3.0856775814913673e17
    va = VelocityAxis(nch, -42.0, 6.0, 1)
    return fields, tgt_f, dx, va


def _loss(fields, dx, view, va, target, integration):
    cube = oracle.render_cube(fields, dx, LINE, DUST, view, va, integration=integration)["L"]
    return float(np.mean((cube - target) ** 2))


@pytest.mark.parametrize("integration", [oracle.SMOOTH, oracle.FORMAL])
def test_gradient_of_any_view_equals_central_differences(integration):
    """Oblique (30, 45) deg and radial views: the dual-number gradient at
    seeded cells equals FP64 central differences of the primal loss (every
    pixel re-rendered), to the difference's own accuracy."""
    fields, tgt_f, dx, va = _grad_problem()
    n = fields[0].shape[0]
    rng = np.random.default_rng(5)
    cells = np.stack([rng.integers(1, n - 1, 6), rng.integers(1, n - 1, 6),
                      rng.integers(1, n - 1, 6)], axis=1)
    for view in (View(math.radians(30), math.radians(45), 9, 8, 0.9 * dx, 1),
                 View(0.0, 0.0, n, n, dx, 2)):
        target = oracle.render_cube(tgt_f, dx, LINE, DUST, view, va,
                                    integration=integration)["L"]
        loss, gn, gt, gv = oracle.loss_grad_cells(fields, dx, LINE, DUST, view, va, target,
                                                  cells, integration=integration)
        assert loss == pytest.approx(_loss(fields, dx, view, va, target, integration),
                                     rel=1e-12)
        work = [a.copy() for a in fields]
        for q, g in ((0, gn), (1, gt), (3, gv)):
            for i, (x, y, z) in enumerate(cells):
                v0 = work[q][z, y, x]
                eps = 1e-5 * max(abs(v0), 1.0)
                work[q][z, y, x] = v0 + eps
                lp = _loss(work, dx, view, va, target, integration)
                work[q][z, y, x] = v0 - eps
                lm = _loss(work, dx, view, va, target, integration)
                work[q][z, y, x] = v0
                fd = (lp - lm) / (2 * eps)
                # central-difference error: truncation eps^2 f'''/6 and the
                # rounding of two loss evaluations (~1e-15 loss / eps)
                tol = 1e-6 * abs(fd) + 1e-14 * loss / eps + 1e-9 * np.abs(g).max()
                assert abs(g[i] - fd) <= tol, (view.trilinear, q, i, g[i], fd)


def test_gradient_of_cells_equals_the_column_gradient_on_the_z_view():
    """On the z view the stencil-seeded gradient reduces to the column
    gradient of the (separately pinned) z-view dual-number oracle."""
    fields, tgt_f, dx, va = _grad_problem()
    n = fields[0].shape[0]
    view = View(0.0, 0.0, n, n, dx, 0)
    target = oracle.render_cube(tgt_f, dx, LINE, DUST, view, va)["L"]
    loss, gn, gt, gv = oracle.loss_grad_zview(fields, dx, LINE, DUST, va, target)
    cells = np.array([[1, 2, 3], [4, 0, 6], [6, 6, 0], [3, 3, 3]])
    loss2, cn, ct, cv = oracle.loss_grad_cells(fields, dx, LINE, DUST, view, va, target, cells)
    assert loss2 == pytest.approx(loss, rel=1e-13)
    for i, (x, y, z) in enumerate(cells):
        assert cn[i] == pytest.approx(gn[z, y, x], rel=1e-11)
        assert ct[i] == pytest.approx(gt[z, y, x], rel=1e-11)
        assert cv[i] == pytest.approx(gv[z, y, x], rel=1e-11, abs=1e-30)

"""Pins of the oracle's selectively thin and optically thin transfer modes
(Sec. 4.6, 4.7 and the step substitutions of Sec. 4.8) against closed forms,
the normalisation of the Gaussian and the thick mode in the weak-line limit.
The expected values use the textbook opacity form of the line coefficients
and math.erf, not the oracle's own coefficient or profile code.  All run on
CPU."""
import math

import numpy as np
import pytest

import oracle
from synth import DUST, LINE_13CO_21, VelocityAxis
from tests.test_oracle_pins import AMU, CKMS, NU, B, nu_of_u, textbook_coeffs, uniform_samples

LINE = dict(LINE_13CO_21)
NO_DUST = dict(DUST, kappa_cm2_per_g_gas=0.0)
C_CGS = 2.99792458e10
KB = 1.380649e-16
ST, OT = oracle.SELECTIVELY_THIN, oracle.THIN


def channel_mass(u_lo, u_hi, v, var):
    """Probability mass of the Gaussian line (1-D variance var) in a channel."""
    s = math.sqrt(2.0 * var)
    return 0.5 * (math.erf((u_hi - v) / s) - math.erf((u_lo - v) / s))


def phibar_hz(c, va, v, var):
    """Channel-averaged profile per Hz: mass / channel width in Hz."""
    u_lo = va.v_first_edge_kms + c * va.dv_kms
    return channel_mass(u_lo, u_lo + va.dv_kms, v, var) / (NU * va.dv_kms / CKMS)


def trj(c, va):
    uc = va.v_first_edge_kms + (c + 0.5) * va.dv_kms
    nuc = nu_of_u(uc)
    return nuc, C_CGS * C_CGS / (2 * KB * nuc * nuc)


def alpha_dust(n, kappa=DUST["kappa_cm2_per_g_gas"]):
    return kappa * DUST["mu_mass_per_h2_amu"] * AMU * n


@pytest.mark.parametrize("mode,steps", [(oracle.FORMAL, lambda K: K),
                                        (oracle.SMOOTH, lambda K: K - 1)])
@pytest.mark.parametrize("K", [2, 5, 8])
def test_optically_thin_uniform_slab(mode, steps, K):
    """I = I_bg + L j with L the integrated path: K h (midpoint sum) or
    (K - 1) h (Simpson / trapezoid, exact for a constant)."""
    va = VelocityAxis(10, -5.0, 1.0, 0)
    h, n, T, x, Td, v = 2e16, 3e4, 25.0, 3e-6, 17.0, 0.35
    r = oracle.ray_thin(LINE, DUST, va, uniform_samples(K, n, T, x=x, Td=Td, v=v), h,
                        transfer=OT, integration=mode)
    _, _, j, _, var = textbook_coeffs(n, T, x)
    aD = alpha_dust(n)
    path = steps(K) * h
    for c in range(va.nchan):
        nuc, s = trj(c, va)
        jd = aD * B(nuc, Td)
        expT = (B(nuc, 2.725) + path * (j * phibar_hz(c, va, v, var) + jd)) * s
        expC = (B(nuc, 2.725) + path * jd) * s
        assert r["T"][c] == pytest.approx(expT, rel=1e-11)
        assert r["C"][c] == pytest.approx(expC, rel=1e-12)
        assert r["B"][c] == pytest.approx(B(nuc, 2.725) * s, rel=1e-13)


@pytest.mark.parametrize("K", [5, 9])
def test_optically_thin_smooth_is_simpson(K):
    """Dust emission with a density quadratic along the ray: Simpson is exact
    for a quadratic when K - 1 is even (a swapped 4/2 weight fails)."""
    va = VelocityAxis(3, -1.5, 1.0, 0)
    h, Td = 1e16, 30.0
    k = np.arange(K, dtype=float)
    n = 1e4 * (1.0 + 0.3 * k + 0.05 * k * k)
    smp = dict(n_h2=n, t_gas=np.full(K, 20.0), t_dust=np.full(K, Td), v_los=np.zeros(K),
               x_tr=np.zeros(K))
    r = oracle.ray_thin(LINE, DUST, va, smp, h, transfer=OT, integration=oracle.SMOOTH)
    L = (K - 1) * h
    # integral over s in [0, L] of n(s) with n quadratic in s / h
    a0, a1, a2 = 1e4, 1e4 * 0.3 / h, 1e4 * 0.05 / (h * h)
    n_int = a0 * L + a1 * L ** 2 / 2 + a2 * L ** 3 / 3
    for c in range(va.nchan):
        nuc, s = trj(c, va)
        exp = (B(nuc, 2.725) + alpha_dust(1.0) * n_int * B(nuc, Td)) * s
        assert r["C"][c] == pytest.approx(exp, rel=1e-12)
        assert r["L"][c] == 0.0


def test_optically_thin_smooth_odd_interval_trapezoid():
    """K - 1 odd: Simpson over the first K - 2 intervals, the trapezoid rule
    on the last (exact for a linear density)."""
    K, h = 6, 1e16
    va = VelocityAxis(2, -1.0, 1.0, 0)
    n = 1e4 * (1.0 + 0.2 * np.arange(K))
    smp = dict(n_h2=n, t_gas=np.full(K, 20.0), t_dust=np.full(K, 25.0), v_los=np.zeros(K),
               x_tr=np.zeros(K))
    r = oracle.ray_thin(LINE, DUST, va, smp, h, transfer=OT, integration=oracle.SMOOTH)
    n_int = (K - 1) * h * 0.5 * (n[0] + n[-1])
    for c in range(va.nchan):
        nuc, s = trj(c, va)
        exp = (B(nuc, 2.725) + alpha_dust(1.0) * n_int * B(nuc, 25.0)) * s
        assert r["C"][c] == pytest.approx(exp, rel=1e-12)


@pytest.mark.parametrize("mode,steps", [(oracle.FORMAL, lambda K: K),
                                        (oracle.SMOOTH, lambda K: K - 1)])
def test_selectively_thin_dust_free_closed_form(mode, steps):
    """No dust: the continuum stays at the background and the total grows
    linearly by j_bar - alpha_bar I_bg per unit path (TR and BDF2 are exact
    for a linear solution)."""
    K, h, n, T, x, v = 9, 4e16, 2e4, 30.0, 4e-6, -0.6
    va = VelocityAxis(8, -4.0, 1.0, 0)
    r = oracle.ray_thin(LINE, NO_DUST, va, uniform_samples(K, n, T, x=x, v=v), h,
                        transfer=ST, integration=mode)
    _, _, j, a, var = textbook_coeffs(n, T, x)
    for c in range(va.nchan):
        nuc, s = trj(c, va)
        pb = phibar_hz(c, va, v, var)
        ib = B(nuc, 2.725)
        expT = (ib + steps(K) * h * (j * pb - a * pb * ib)) * s
        assert r["T"][c] == pytest.approx(expT, rel=1e-11)
        assert r["C"][c] == pytest.approx(ib * s, rel=1e-13)
        assert abs(r["D"][c]) <= 1e-15 * ib * s   # (4 I - I) / 3 rounds in the last bit


def test_selectively_thin_formal_uniform_slab_with_dust():
    """Uniform slab with dust, formal steps: the continuum follows
    S_C + (I_bg - S_C) e^{-k tau}; the total's step k uses that continuum
    after its own step; summed in closed form as a geometric series."""
    K, h, n, T, x, Td, v = 6, 3e17, 5e4, 22.0, 2e-6, 15.0, 0.1
    va = VelocityAxis(6, -3.0, 1.0, 0)
    r = oracle.ray_thin(LINE, DUST, va, uniform_samples(K, n, T, x=x, Td=Td, v=v), h,
                        transfer=ST, integration=oracle.FORMAL)
    _, _, j, a, var = textbook_coeffs(n, T, x)
    aD = alpha_dust(n)
    tau = aD * h
    q = math.exp(-tau)
    g = -math.expm1(-tau)
    for c in range(va.nchan):
        nuc, s = trj(c, va)
        pb = phibar_hz(c, va, v, var)
        ib, sc = B(nuc, 2.725), B(nuc, Td)
        # I_T after K steps: sum_k q^(K-1-k) g (jbar + jD - abar IC_k) / aD + q^K I_bg,
        # IC_k = sc + (ib - sc) q^(k+1)
        geo = sum(q ** (K - 1 - k) for k in range(K))
        geo2 = sum(q ** (K - 1 - k) * q ** (k + 1) for k in range(K))
        jd = aD * sc
        it = q ** K * ib + g / aD * ((j * pb + jd - a * pb * sc) * geo - a * pb * (ib - sc) * geo2)
        ic = sc + (ib - sc) * q ** K
        assert r["T"][c] == pytest.approx(it * s, rel=1e-10)
        assert r["C"][c] == pytest.approx(ic * s, rel=1e-12)


def test_channel_profile_mass_sums_to_one():
    """Line well inside the band, optically thin, no dust or background, in
    intensity units: sum over channels of I_c x channel width in Hz is the
    frequency-integrated emission K h j."""
    K, h, n, T, x = 4, 1e16, 1e4, 40.0, 1e-6
    va = VelocityAxis(40, -10.0, 0.5, 0)
    r = oracle.ray_thin(LINE, NO_DUST, va, uniform_samples(K, n, T, x=x, v=0.2), h,
                        transfer=OT, integration=oracle.FORMAL, units=oracle.INTENSITY,
                        t_bg=0.0)
    _, _, j, _, _ = textbook_coeffs(n, T, x)
    width_hz = NU * va.dv_kms / CKMS
    assert r["T"].sum() * width_hz == pytest.approx(K * h * j, rel=1e-12)


@pytest.mark.parametrize("mode", [oracle.FORMAL, oracle.SMOOTH])
def test_weak_line_selectively_thin_matches_thick(mode):
    """A weak line (line optical depth ~1e-5) over dust: the thick mode's
    fine-grid Simpson average and the selectively thin analytic channel
    average agree to the Simpson error of the fine grid (f = 16)."""
    K, h = 12, 3e17
    rng = np.random.default_rng(3)
    smp = dict(n_h2=rng.uniform(1e4, 4e4, K), t_gas=rng.uniform(15, 60, K),
               t_dust=rng.uniform(12, 25, K), v_los=rng.uniform(-2, 2, K),
               x_tr=np.full(K, 1e-10))
    va = VelocityAxis(16, -8.0, 1.0, 16)
    thick = oracle.ray(LINE, DUST, va, smp, h, integration=mode)
    thin = oracle.ray_thin(LINE, DUST, va, smp, h, transfer=ST, integration=mode)
    peak = np.abs(thick["L"]).max()
    assert peak > 0
    np.testing.assert_allclose(thin["L"], thick["L"], atol=2e-4 * peak)
    np.testing.assert_allclose(thin["C"], thick["C"], rtol=1e-13)


@pytest.mark.parametrize("transfer", [ST, OT])
@pytest.mark.parametrize("mode", [oracle.FORMAL, oracle.SMOOTH])
def test_thin_component_identities(transfer, mode):
    rng = np.random.default_rng(7)
    K = 11
    smp = dict(n_h2=rng.uniform(1e3, 1e5, K), t_gas=rng.uniform(10, 90, K),
               t_dust=rng.uniform(10, 30, K), v_los=rng.uniform(-3, 3, K),
               x_tr=rng.uniform(1e-6, 3e-6, K))
    va = VelocityAxis(9, -4.5, 1.0, 0)
    r = oracle.ray_thin(LINE, DUST, va, smp, 1e17, transfer=transfer, integration=mode)
    np.testing.assert_allclose(r["T"], r["C"] + r["L"], rtol=0, atol=1e-12)
    np.testing.assert_allclose(r["C"], r["B"] + r["D"], rtol=0, atol=1e-12)
    r0 = oracle.ray_thin(LINE, DUST, va, dict(smp, x_tr=np.zeros(K)), 1e17, transfer=transfer,
                         integration=mode)
    assert np.all(r0["L"] == 0.0)
    rn = oracle.ray_thin(LINE, NO_DUST, va, smp, 1e17, transfer=transfer, integration=mode)
    assert np.all(np.abs(rn["D"]) <= 1e-15 * np.abs(rn["B"]))


@pytest.mark.parametrize("transfer", [ST, OT])
@pytest.mark.parametrize("mode", [oracle.FORMAL, oracle.SMOOTH])
@pytest.mark.parametrize("K", [0, 1])
def test_empty_and_single_sample_rays(transfer, mode, K):
    """A ray that misses the box (no samples) shows the background; one
    sample: the smooth node 0 is the background, the formal step is one
    closed-form step."""
    va = VelocityAxis(5, -2.5, 1.0, 0)
    r = oracle.ray_thin(LINE, DUST, va, uniform_samples(K, 2e4, 30.0), 1e17, transfer=transfer,
                        integration=mode)
    for c in range(va.nchan):
        nuc, s = trj(c, va)
        if K == 0 or mode == oracle.SMOOTH:
            assert r["T"][c] == pytest.approx(B(nuc, 2.725) * s, rel=1e-13)
            assert r["C"][c] == pytest.approx(B(nuc, 2.725) * s, rel=1e-13)
        else:
            assert r["T"][c] > r["B"][c]

"""Pins of the oracle's Planck brightness-temperature output (Sec. 4.9) and
of continuum subtraction in T_B space (Sec. 4.10): the brightness temperature
of a blackbody is its temperature, the Rayleigh-Jeans offset h nu / 2k at
high temperature, the Sec. 5.8 example, and the component bookkeeping.  All
run on CPU."""
import math

import numpy as np
import pytest

import oracle
from synth import DUST, LINE_13CO_21, VelocityAxis
from tests.conftest import golden
from tests.test_oracle_pins import CKMS, NU, nu_of_u, uniform_samples

LINE = dict(LINE_13CO_21)
NO_DUST = dict(DUST, kappa_cm2_per_g_gas=0.0)
H = 6.62607015e-27
KB = 1.380649e-16


@pytest.mark.parametrize("t_bg", [2.725, 10.0, 40.0])
@pytest.mark.parametrize("transfer", ["thick", "selectively_thin"])
def test_background_is_its_temperature(t_bg, transfer):
    """[B] is a blackbody at every channel's own frequency: T_B = T_bg."""
    va = VelocityAxis(6, -150.0, 50.0, 1)
    smp = uniform_samples(3, 1e4, 20.0)
    if transfer == "thick":
        r = oracle.ray(LINE, DUST, va, smp, 1e17, units=oracle.TB, t_bg=t_bg)
    else:
        r = oracle.ray_thin(LINE, DUST, va, smp, 1e17, units=oracle.TB, t_bg=t_bg)
    np.testing.assert_allclose(r["B"], t_bg, rtol=1e-12)


@pytest.mark.parametrize("mode", [oracle.FORMAL, oracle.SMOOTH])
def test_optically_thick_line_saturates_to_excitation_temperature(mode):
    """Dust-free slab of huge line optical depth at line centre: the total
    is the Planck function of T_ex, so its T_B is T_ex itself (in RJ units
    it would be J(T_ex) instead)."""
    va = VelocityAxis(1, -0.05, 0.1, 2)
    T = 35.0
    r = oracle.ray(LINE, NO_DUST, va, uniform_samples(400, 1e6, T, x=1e-4), 3e17,
                   integration=mode, units=oracle.TB)
    assert r["T"][0] == pytest.approx(T, rel=1e-6)
    assert r["L"][0] == pytest.approx(T - r["C"][0], rel=1e-12)


def test_high_temperature_offset_is_h_nu_over_2k():
    """T_B - T_RJ -> h nu / 2k for kT >> h nu (expansion of Planck's law)."""
    va = VelocityAxis(1, -0.5, 1.0, 0)
    smp = uniform_samples(1, 1e2, 20.0, x=0.0)
    for t_bg in (300.0, 3000.0):
        b = oracle.ray(LINE, NO_DUST, va, smp, 1e10, units=oracle.TB, t_bg=t_bg)["B"][0]
        rj = oracle.ray(LINE, NO_DUST, va, smp, 1e10, units=oracle.TRJ, t_bg=t_bg)["B"][0]
        nuc = nu_of_u(0.0)
        assert b == pytest.approx(t_bg, rel=1e-12)
        # T_RJ = T - h nu / 2k + O(h nu / kT)
        assert (b - rj) == pytest.approx(H * nuc / (2 * KB), rel=20 * H * nuc / (KB * t_bg))


def test_sec58_example_one_kelvin_rj_is_about_four_kelvin_planck():
    """The printed example: 1.0 K in T_RJ at 220.4 GHz is ~4.3 K in T_B.  The
    background is set to the temperature whose RJ value is 1.0 K, found by
    bisection on the RJ output."""
    (nu, t_rj, t_b_printed), = golden("rj_planck_example.txt")
    v = CKMS * (1.0 - nu / NU)                 # velocity whose frequency is nu
    va = VelocityAxis(1, v - 0.5, 1.0, 0)
    smp = uniform_samples(1, 1e2, 20.0, x=0.0)
    lo, hi = 1.0, 20.0
    for _ in range(80):
        mid = 0.5 * (lo + hi)
        rj = oracle.ray(LINE, NO_DUST, va, smp, 1e10, units=oracle.TRJ, t_bg=mid)["B"][0]
        lo, hi = (mid, hi) if rj < t_rj else (lo, mid)
    tb = oracle.ray(LINE, NO_DUST, va, smp, 1e10, units=oracle.TB, t_bg=lo)["B"][0]
    assert round(tb, 1) == t_b_printed


@pytest.mark.parametrize("transfer", ["thick", "selectively_thin", "thin"])
def test_tb_space_subtraction_bookkeeping(transfer):
    """[L] = T_B([T]) - T_B([C]) and [D] = T_B([C]) - T_B([B]); each T_B is
    the inverse Planck function of the same ray's intensity output."""
    rng = np.random.default_rng(9)
    K = 9
    smp = dict(n_h2=rng.uniform(1e3, 1e5, K), t_gas=rng.uniform(10, 90, K),
               t_dust=rng.uniform(10, 30, K), v_los=rng.uniform(-3, 3, K),
               x_tr=rng.uniform(1e-6, 3e-6, K))
    va = VelocityAxis(7, -3.5, 1.0, 0 if transfer != "thick" else 2)

    def run(units):
        if transfer == "thick":
            return oracle.ray(LINE, DUST, va, smp, 1e17, units=units)
        mode = oracle.SELECTIVELY_THIN if transfer == "selectively_thin" else oracle.THIN
        return oracle.ray_thin(LINE, DUST, va, smp, 1e17, transfer=mode, units=units)

    tb, inten = run(oracle.TB), run(oracle.INTENSITY)
    for c in range(va.nchan):
        nuc = nu_of_u(va.v_first_edge_kms + (c + 0.5) * va.dv_kms)
        for k in "TCB":
            expect = H * nuc / (KB * math.log1p(2 * H * nuc ** 3 / (2.99792458e10 ** 2 * inten[k][c])))
            assert tb[k][c] == pytest.approx(expect, rel=1e-12)
        assert tb["L"][c] == tb["T"][c] - tb["C"][c]
        assert tb["D"][c] == tb["C"][c] - tb["B"][c]

"""Pins of the oracle's density-tracing cube (Sec. 5.10, "simple
observation": tracer column density per unit velocity): the channel sum is
the column density, a cold cell puts its whole column in its own channel,
linearity, and the Gaussian spread.  All run on CPU."""
import math

import numpy as np
import pytest

import oracle
from synth import DUST, LINE_13CO_21, VelocityAxis
from tests.test_oracle_pins import uniform_samples

LINE = dict(LINE_13CO_21)
DT = oracle.DENSITY_TRACING


@pytest.mark.parametrize("mode,steps", [(oracle.FORMAL, lambda K: K),
                                        (oracle.SMOOTH, lambda K: K - 1)])
def test_channel_sum_is_the_tracer_column(mode, steps):
    """Lines well inside the band: sum_c DT_c dv = x n_H2 x path (uniform)."""
    K, h, n, x = 7, 2e17, 3e4, 2e-6
    va = VelocityAxis(60, -15.0, 0.5, 0)
    r = oracle.ray_thin(LINE, DUST, va, uniform_samples(K, n, 40.0, x=x, v=1.3), h,
                        transfer=DT, integration=mode)
    assert r["T"].sum() * va.dv_kms == pytest.approx(x * n * steps(K) * h, rel=1e-12)
    assert np.all(r["C"] == 0.0) and np.all(r["B"] == 0.0) and np.all(r["D"] == 0.0)
    np.testing.assert_array_equal(r["L"], r["T"])


def test_cold_cell_fills_its_own_channel():
    """No turbulence and a cold cell at a channel centre: (nearly) all of its
    column lands in that channel, N h / dv."""
    line = dict(LINE, sigma_turb_kms=0.0)
    va = VelocityAxis(9, -4.5, 1.0, 0)
    r = oracle.ray_thin(line, DUST, va, uniform_samples(1, 1e4, 1.0, x=1e-6, v=0.0), 1e17,
                        transfer=DT, integration=oracle.FORMAL)
    # b = sqrt(2 k T / m) = 0.024 km/s at 1 K: the channel holds erf(0.5 / b) = 1
    assert r["T"][4] == pytest.approx(1e-6 * 1e4 * 1e17 / 1.0, rel=1e-12)
    assert r["T"][3] < 1e-100 and r["T"][5] < 1e-100


def test_gaussian_spread_between_neighbour_channels():
    """A cell at a channel edge splits its column equally; the fraction in a
    channel follows the erf of the Doppler parameter b^2 = 2kT/m + 2 sigma^2."""
    T, sig = 50.0, 1.0
    va = VelocityAxis(2, -1.0, 1.0, 0)
    r = oracle.ray_thin(LINE, DUST, va, uniform_samples(1, 1e4, T, x=1e-6, v=0.0), 1e17,
                        transfer=DT, integration=oracle.FORMAL)
    assert r["T"][0] == pytest.approx(r["T"][1], rel=1e-13)
    b = math.sqrt(2 * 1.380649e-16 * T / (LINE["mass_amu"] * 1.66053906660e-24) / 1e10
                  + 2 * sig ** 2)
    frac = 0.5 * math.erf(1.0 / b)              # mass in [0, 1] km/s
    assert r["T"][1] == pytest.approx(1e-6 * 1e4 * 1e17 * frac / 1.0, rel=1e-12)


def test_linear_in_density_and_abundance_and_blind_to_dust_and_cutoff():
    rng = np.random.default_rng(4)
    K = 8
    smp = dict(n_h2=rng.uniform(1e3, 1e5, K), t_gas=rng.uniform(10, 90, K),
               t_dust=rng.uniform(10, 30, K), v_los=rng.uniform(-3, 3, K),
               x_tr=rng.uniform(1e-6, 3e-6, K))
    va = VelocityAxis(12, -6.0, 1.0, 0)
    r1 = oracle.ray_thin(LINE, DUST, va, smp, 1e17, transfer=DT)
    r2 = oracle.ray_thin(LINE, dict(DUST, kappa_cm2_per_g_gas=5.0), va,
                         dict(smp, n_h2=2 * smp["n_h2"]), 1e17, transfer=DT, t_bg=30.0)
    np.testing.assert_allclose(r2["T"], 2 * r1["T"], rtol=1e-13)
    hot = dict(smp, t_gas=np.full(K, 1e4))
    r3 = oracle.ray_thin(dict(LINE, t_inf_k=100.0), DUST, va, hot, 1e17, transfer=DT)
    assert r3["T"].sum() > 0

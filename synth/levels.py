"""Synthetic molecular level models (inputs of the optically thin level balance).

The paper reads its level energies, Einstein A coefficients and collision
rates from a LAMDA data file (Sec. 4.1).  No such file is available here, so
these inputs are generated: a rigid linear rotor with the workload's rotational
constant, dipole transitions J -> J-1 with the textbook Einstein A of a linear
rotor, and smooth invented de-excitation rate coefficients for the collision
partners the paper uses (H2 split into para and ortho, H, He).  They are inputs
like the field generators: neither the oracle nor the library computes them.

A model is a plain dict of numpy arrays; ``LevelModel`` of the oracle and
``irt_level_model`` of the library are filled from it.
"""
from __future__ import annotations

import numpy as np

H_PLANCK = 6.62607015e-27   # erg s
K_BOLTZ = 1.380649e-16      # erg / K
C_LIGHT = 2.99792458e10     # cm / s
DEBYE = 1.0e-18             # esu cm

#: collision partner kinds (the order of irt_partner in the C ABI)
PARTNER_H2, PARTNER_PH2, PARTNER_OH2, PARTNER_H, PARTNER_HE = range(5)


def rotor_model(nlev: int = 12, b0_hz: float = 55.101e9, dipole_debye: float = 0.11,
                partners=(PARTNER_PH2, PARTNER_OH2, PARTNER_H, PARTNER_HE),
                temps_k=(5.0, 10.0, 20.0, 40.0, 80.0, 160.0, 320.0, 640.0),
                k0_cm3_s: float = 3.0e-11, t_rad_k: float = 2.725, ortho_para: float = 3.0,
                x_he: float = 0.1, seed: int = 0) -> dict:
    """Rigid rotor J = 0 .. nlev-1: E_J / k = h B0 J (J + 1) / k, g_J = 2J + 1;
    radiative J -> J-1 at nu = 2 B0 J with A = 64 pi^4 nu^3 mu^2 J / (3 h c^3 (2J+1))
    (for B0 = 55.101 GHz and 0.11 D: A(2-1) = 6.03e-7 / s); collisional
    de-excitation J -> J' < J for every pair, per partner
    K = k0 s_p (T / 100 K)^a_p exp(-(J - J' - 1) / 2) / (1 + 0.1 J'), with
    per-partner scale s_p and slope a_p drawn from ``seed``."""
    J = np.arange(nlev, dtype=np.float64)
    energy_k = H_PLANCK * b0_hz * J * (J + 1.0) / K_BOLTZ
    g = 2.0 * J + 1.0
    up = np.arange(1, nlev)
    lo = up - 1
    nu = 2.0 * b0_hz * up.astype(np.float64)
    mu = dipole_debye * DEBYE
    a = (64.0 * np.pi ** 4 * nu ** 3 * mu ** 2 / (3.0 * H_PLANCK * C_LIGHT ** 3)
         * up / (2.0 * up + 1.0))
    rng = np.random.default_rng(seed)
    temps = np.asarray(temps_k, dtype=np.float64)
    cu, cl = [], []
    for u in range(1, nlev):
        for l in range(u):
            cu.append(u)
            cl.append(l)
    cu = np.asarray(cu, dtype=np.int32)
    cl = np.asarray(cl, dtype=np.int32)
    npart = len(partners)
    k = np.empty((npart, len(cu), len(temps)))
    for p in range(npart):
        s_p = rng.uniform(0.3, 1.5)
        a_p = rng.uniform(-0.2, 0.5)
        for t, T in enumerate(temps):
            k[p, :, t] = (k0_cm3_s * s_p * (T / 100.0) ** a_p
                          * np.exp(-0.5 * (cu - cl - 1)) / (1.0 + 0.1 * cl))
    return dict(nlev=nlev, energy_k=energy_k, g=g, rad_up=up.astype(np.int32),
                rad_lo=lo.astype(np.int32), a_ul_s=a, nu_hz=nu,
                partner=np.asarray(partners, dtype=np.int32),
                coll_temp_k=np.tile(temps, (npart, 1)),
                coll_up=np.tile(cu, (npart, 1)), coll_lo=np.tile(cl, (npart, 1)),
                k_ul_cm3_s=k, t_rad_k=float(t_rad_k), ortho_para=float(ortho_para),
                x_he=float(x_he))


def two_level_model(e_u_k: float = 5.5, g_l: float = 1.0, g_u: float = 3.0,
                    nu_hz: float = 110.2e9, a_ul_s: float = 6.3e-8,
                    k_ul_cm3_s: float = 2.0e-11, t_rad_k: float = 2.725,
                    temps_k=(10.0, 100.0)) -> dict:
    """Two levels, one radiative and one collisional transition, one partner
    (total H2); the rate coefficient is the same at every tabulated
    temperature."""
    temps = np.asarray(temps_k, dtype=np.float64)
    return dict(nlev=2, energy_k=np.array([0.0, e_u_k]), g=np.array([g_l, g_u]),
                rad_up=np.array([1], np.int32), rad_lo=np.array([0], np.int32),
                a_ul_s=np.array([a_ul_s]), nu_hz=np.array([nu_hz]),
                partner=np.array([PARTNER_H2], np.int32),
                coll_temp_k=temps[None, :], coll_up=np.array([[1]], np.int32),
                coll_lo=np.array([[0]], np.int32),
                k_ul_cm3_s=np.full((1, 1, len(temps)), k_ul_cm3_s),
                t_rad_k=float(t_rad_k), ortho_para=3.0, x_he=0.1)


#: table axes of the paper's grid precomputation (Sec. 4.2): 128 densities,
#: 64 H2 abundances, 64 temperatures; log10 n_H in [0, 8], chi in [0.01, 0.5],
#: log10 T in [log10 5, log10 2000]
OT_AXES = dict(n_n=128, n_chi=64, n_t=64, log10_nh_min=0.0, log10_nh_max=8.0,
               chi_min=0.01, chi_max=0.5, log10_t_min=float(np.log10(5.0)),
               log10_t_max=float(np.log10(2000.0)))

"""Workload definitions: molecular constants, velocity axes, views, job tables.

Everything here is an *input* to the method.  The values follow the workloads
the library is benchmarked on: 13CO(2-1) in LTE, a CMB background, dust with a
per-gas-mass opacity, uniform 0.1 pc cells.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace

import numpy as np

PC_CM = 3.0856775814913673e18

#: 13CO J=2-1.  nu, A_ul, E_u, B0 are the workload's constants; g = 2J+1;
#: mass of 13C16O = 13.003355 + 15.994915 amu; T_inf = 5e4 K (Sec. 4.3);
#: 1 km/s 1-D microturbulent dispersion added to the thermal width.
LINE_13CO_21 = dict(nu_ul_hz=220.3987e9, a_ul_s=6.04e-7, e_u_k=15.87, b0_hz=55.101e9,
                    g_u=5.0, g_l=3.0, mass_amu=28.99827, t_inf_k=5.0e4,
                    sigma_turb_kms=1.0)

#: kappa per gram of gas (1 cm^2/g of dust at gas-to-dust 100, Sec. 3.2); gas
#: mass per H2 molecule for fully molecular gas with He/H = 0.1 by number:
#: 2 (m_H + 0.1 m_He) = 2 (1.00794 + 0.1 * 4.002602) amu.
DUST = dict(kappa_cm2_per_g_gas=1.0e-2, mu_mass_per_h2_amu=2.0 * (1.00794 + 0.1 * 4.002602))

T_CMB_K = 2.725


@dataclass(frozen=True)
class VelocityAxis:
    """Channel c spans [v0 + c dv, v0 + (c+1) dv] km/s; f = subsampling factor."""
    nchan: int
    v_first_edge_kms: float
    dv_kms: float
    subsample_f: int


@dataclass(frozen=True)
class View:
    """Orthographic view. theta = phi = 0 with trilinear = 0 is the z view."""
    theta_rad: float = 0.0
    phi_rad: float = 0.0
    npx: int = 0
    npy: int = 0
    pixel_cm: float = 0.0
    trilinear: int = 0


@dataclass
class Workload:
    name: str
    n: int
    cell_cm: float
    seed: int
    vaxis: VelocityAxis
    views: list
    storage: str = "f32"          # "f64", "f32", "f16", "bf16"
    n_mean: float = 1.0e4
    t_bg_k: float = T_CMB_K
    line: dict = field(default_factory=lambda: dict(LINE_13CO_21))
    dust: dict = field(default_factory=lambda: dict(DUST))


def z_view(n: int, cell_cm: float) -> View:
    return View(0.0, 0.0, n, n, cell_cm, 0)


def oblique_view(n: int, cell_cm: float, theta_deg: float, phi_deg: float) -> View:
    return View(math.radians(theta_deg), math.radians(phi_deg), n, n, cell_cm, 1)


def workload(k: int, s: int = 0, n: int | None = None) -> Workload:
    """The single-snapshot workloads, numbered 0 (32^3 FP64 parity), 1 (256^3
    z and oblique views), 3 (128^3 adjoint) and 4 (512^3 FP16); number 2, the
    batch of uneven snapshots, is batch_jobs().  Seeds are 1000 k + s.  ``n``
    overrides the grid side (small cases with the same recipe)."""
    cell = 0.1 * PC_CM
    seed = 1000 * k + s
    if k == 0:
        nn = n or 32
        return Workload("32cube-64ch-f4-fp64", nn, cell, seed,
                        VelocityAxis(64, -100.0, 3.125, 4), [z_view(nn, cell)], "f64")
    if k == 1:
        nn = n or 256
        return Workload("256cube-256ch-f1-fp32", nn, cell, seed,
                        VelocityAxis(256, -128.0, 1.0, 1),
                        [z_view(nn, cell), oblique_view(nn, cell, 30.0, 45.0)], "f32")
    if k == 3:
        nn = n or 128
        return Workload("128cube-128ch-f2-fp32-adjoint", nn, cell, seed,
                        VelocityAxis(128, -100.0, 1.5625, 2), [z_view(nn, cell)], "f32")
    if k == 4:
        nn = n or 512
        return Workload("512cube-500ch-f1-fp16", nn, cell, seed,
                        VelocityAxis(500, -250.0, 1.0, 1), [z_view(nn, cell)], "f16")
    raise ValueError(f"no single-snapshot workload {k} (the batch is batch_jobs())")


@dataclass
class BatchJob:
    index: int
    n: int
    n_mean: float
    seed: int
    theta_rad: float
    phi_rad: float
    vaxis: VelocityAxis
    cell_cm: float

    def view(self) -> View:
        return View(self.theta_rad, self.phi_rad, self.n, self.n, self.cell_cm, 1)


def batch_jobs(njobs: int = 64, seed: int = 2000, n_lo: int = 64, n_hi: int = 256,
               ch_lo: int = 128, ch_hi: int = 512) -> list[BatchJob]:
    """Uneven batch: N ~ U{n_lo..n_hi}, mean density log-uniform in [1e3, 1e5],
    view direction uniform on the sphere, N_ch ~ U{ch_lo..ch_hi} at 1 km/s
    centred on 0, f = 1."""
    rng = np.random.default_rng(seed)
    cell = 0.1 * PC_CM
    jobs = []
    for i in range(njobs):
        n = int(rng.integers(n_lo, n_hi + 1))
        n_mean = float(10.0 ** rng.uniform(3.0, 5.0))
        mu = float(rng.uniform(-1.0, 1.0))
        theta = math.acos(mu)
        phi = float(rng.uniform(0.0, 2.0 * math.pi))
        nch = int(rng.integers(ch_lo, ch_hi + 1))
        jobs.append(BatchJob(i, n, n_mean, seed + 10 * i, theta, phi,
                             VelocityAxis(nch, -0.5 * nch, 1.0, 1), cell))
    return jobs


def with_line(w: Workload, **kw) -> Workload:
    ln = dict(w.line)
    ln.update(kw)
    return replace(w, line=ln)

"""Seeded field generator on the GPU (torch), same recipe as fields.make_fields.

Used where many large snapshots are needed quickly (the batched workload):
the random numbers come from torch's generator, so the arrays differ from the
numpy generator's for the same seed, but both the CUDA path and the oracle
checks consume the same arrays.  No method arithmetic here.
"""
from __future__ import annotations

import torch


def grf_torch(n: int, gen: torch.Generator, device, slope: float = -11.0 / 3.0) -> torch.Tensor:
    """Periodic Gaussian random field on an n^3 box (float64), zero mean, unit
    std, amplitude k^(slope/2) with the k = 0 mode removed."""
    white = torch.randn((n, n, n), generator=gen, device=device, dtype=torch.float64)
    spec = torch.fft.rfftn(white)
    del white
    kz = torch.fft.fftfreq(n, device=device, dtype=torch.float64)[:, None, None]
    ky = torch.fft.fftfreq(n, device=device, dtype=torch.float64)[None, :, None]
    kx = torch.fft.rfftfreq(n, device=device, dtype=torch.float64)[None, None, :]
    k2 = kz * kz + ky * ky + kx * kx
    k2[0, 0, 0] = 1.0
    amp = k2 ** (slope / 4.0)
    amp[0, 0, 0] = 0.0
    spec *= amp
    del amp, k2
    g = torch.fft.irfftn(spec, s=(n, n, n))
    del spec
    g -= g.mean()
    g /= g.std(unbiased=False)
    return g


def make_fields_torch(n: int, seed: int, n_mean: float = 1.0e4, sigma_ln: float = 1.5,
                      x_tracer: float = 2.0e-6, v_turb_kms: float = 10.0,
                      v_rot_kms: float = 50.0, device="cuda"):
    """(n_h2, t_gas, t_dust, v_los, x_tracer) float64 tensors [z][y][x] on
    ``device``; the recipe of fields.make_fields with torch generators
    seeded seed (density), seed + 1 (velocity), seed + 2 (temperature)."""
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    g = grf_torch(n, gen, device)
    n_h2 = n_mean * torch.exp(sigma_ln * g - 0.5 * sigma_ln * sigma_ln)
    gen.manual_seed(seed + 2)
    noise = 5.0 * torch.randn((n, n, n), generator=gen, device=device, dtype=torch.float64)
    t_gas = torch.clamp(60.0 - (40.0 / 3.0) * g + noise, 20.0, 100.0)
    del g, noise
    gen.manual_seed(seed + 1)
    gv = grf_torch(n, gen, device)
    xs = (torch.arange(n, device=device, dtype=torch.float64) + 0.5) * (2.0 / n) - 1.0
    v_los = v_turb_kms * gv + v_rot_kms * xs[None, None, :]
    del gv
    return (n_h2, t_gas, t_gas.clone(), v_los,
            torch.full((n, n, n), x_tracer, device=device, dtype=torch.float64))

"""Seeded Gaussian-random-field generators for the five physical fields.

The paper renders AREPO zoom simulations interpolated onto observer grids
(Sec. 2.4).  Those snapshots are not available, so these generators stand in
for them with fields of the same character: a lognormal H2 density with a
Kolmogorov-like spectrum, a gas temperature that is colder in dense gas, and a
line-of-sight velocity made of turbulence plus solid-body rotation.

Layout of every returned array: C order ``[z][y][x]``, float64.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

#: power-spectrum slope of the Gaussian random fields, P(k) ~ k^-11/3
PK_SLOPE = -11.0 / 3.0


def grf(n: int, rng: np.random.Generator, slope: float = PK_SLOPE) -> np.ndarray:
    """Periodic Gaussian random field on an n^3 box, zero mean, unit std.

    White noise is shaped in k-space by an amplitude k^(slope/2) with the
    k = 0 mode removed, then normalised to zero empirical mean and unit
    empirical standard deviation.
    """
    white = rng.standard_normal((n, n, n))
    spec = np.fft.rfftn(white)
    del white
    kz = np.fft.fftfreq(n)[:, None, None]
    ky = np.fft.fftfreq(n)[None, :, None]
    kx = np.fft.rfftfreq(n)[None, None, :]
    k2 = kz * kz + ky * ky + kx * kx
    k2[0, 0, 0] = 1.0
    amp = k2 ** (slope / 4.0)
    amp[0, 0, 0] = 0.0
    spec *= amp
    del amp, k2
    g = np.fft.irfftn(spec, s=(n, n, n), axes=(0, 1, 2))
    del spec
    g -= g.mean()
    g /= g.std()
    return g


@dataclass
class FieldSet:
    """Five fields on a uniform Cartesian grid, C order [z][y][x]."""
    n_h2: np.ndarray      # H2 number density [cm^-3]
    t_gas: np.ndarray     # gas kinetic temperature [K]
    t_dust: np.ndarray    # dust temperature [K]
    v_los: np.ndarray     # line-of-sight velocity [km/s], + = receding
    x_tracer: np.ndarray  # tracer abundance relative to n_H2

    def as_tuple(self):
        return (self.n_h2, self.t_gas, self.t_dust, self.v_los, self.x_tracer)

    @property
    def shape(self):
        return self.n_h2.shape

    def astype(self, dtypes) -> "FieldSet":
        """Copy with each field cast (``dtypes``: one numpy dtype or five)."""
        if not isinstance(dtypes, (list, tuple)):
            dtypes = [dtypes] * 5
        arrs = [np.ascontiguousarray(a.astype(d)) for a, d in zip(self.as_tuple(), dtypes)]
        return FieldSet(*arrs)


def make_fields(n: int, seed: int, n_mean: float = 1.0e4, sigma_ln: float = 1.5,
                x_tracer: float = 2.0e-6, v_turb_kms: float = 10.0,
                v_rot_kms: float = 50.0) -> FieldSet:
    """Draw one seeded field set on an n^3 grid.

    Seeds: the density field uses ``seed``, the velocity field ``seed + 1``
    and the temperature noise ``seed + 2``.

    * density  n_H2 = n_mean * exp(sigma g - sigma^2/2)  (lognormal, mean n_mean)
    * temperature T = clip(60 - (40/3) g + N(0, 5), 20, 100) K  (colder where
      denser), dust temperature equal to the gas temperature
    * velocity v_los = v_turb g_v + v_rot (2 (x + 1/2)/n - 1)  (solid-body
      rotation reaching +-v_rot at the two x faces)
    * tracer abundance constant
    """
    g = grf(n, np.random.default_rng(seed))
    n_h2 = n_mean * np.exp(sigma_ln * g - 0.5 * sigma_ln * sigma_ln)
    noise = np.random.default_rng(seed + 2).normal(0.0, 5.0, size=(n, n, n))
    t_gas = np.clip(60.0 - (40.0 / 3.0) * g + noise, 20.0, 100.0)
    del g, noise
    gv = grf(n, np.random.default_rng(seed + 1))
    xs = (np.arange(n, dtype=np.float64) + 0.5) * (2.0 / n) - 1.0
    v_los = v_turb_kms * gv + v_rot_kms * xs[None, None, :]
    del gv
    return FieldSet(n_h2=np.ascontiguousarray(n_h2), t_gas=np.ascontiguousarray(t_gas),
                    t_dust=np.ascontiguousarray(t_gas.copy()),
                    v_los=np.ascontiguousarray(v_los),
                    x_tracer=np.full((n, n, n), x_tracer, dtype=np.float64))


def to_storage(fs: FieldSet, dtypes, scales=None) -> tuple[FieldSet, FieldSet]:
    """Round a field set to storage precision.

    Returns ``(stored, dequantised)``: the arrays in the storage dtypes and
    the same values widened back to float64, which is what an oracle run on
    "the same inputs" consumes.  ``dtypes`` entries are numpy dtypes or the
    string ``"bf16"`` (bfloat16, round to nearest even, kept as uint16 bits).
    ``scales`` (optional, per field): the stored value is value / scale and
    the dequantised value is stored * scale.
    """
    if not isinstance(dtypes, (list, tuple)):
        dtypes = [dtypes] * 5
    if scales is None:
        scales = [1.0] * 5
    stored, deq = [], []
    for a, d, sc in zip(fs.as_tuple(), dtypes, scales):
        a = a / sc if sc != 1.0 else a
        if isinstance(d, str) and d == "bf16":
            bits = _f32_to_bf16_bits(a.astype(np.float32))
            stored.append(bits)
            back = (bits.astype(np.uint32) << 16).view(np.float32).astype(np.float64)
        else:
            s = np.ascontiguousarray(a.astype(d))
            stored.append(s)
            back = s.astype(np.float64)
        deq.append(back * sc if sc != 1.0 else back)
    return FieldSet(*stored), FieldSet(*deq)


def _f32_to_bf16_bits(a: np.ndarray) -> np.ndarray:
    """float32 -> bfloat16 bit pattern (uint16), round to nearest even."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = (u + 0x7FFF + lsb) >> 16
    return r.astype(np.uint16)

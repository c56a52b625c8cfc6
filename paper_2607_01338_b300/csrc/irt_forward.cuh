// Forward PPV kernel of the IRIS-SO transfer (sm_103a).
//
// Work item = (ray, channel window).  One warp renders one item:
//   1. sample pass: lane l evaluates samples k = l, l+32, ... of the ray (field
//      load or trilinear interpolation, LTE populations, line and dust
//      coefficients, Sec. 3.2-3.7, 5.10) into a per-warp shared-memory record;
//   2. transfer pass: lane l owns the fine velocities g = l + 32 i of the
//      window (register blocks i < NI) and integrates them sample by sample
//      (Sec. 4.8, formal or smooth), evaluating the Gaussian profile only in
//      the blocks the sample's line reaches;
//   3. epilogue: Simpson channel average (Sec. 4.5), continuum and background
//      at the channel centre (Sec. 4.4), [L] = [T] - [C] (Sec. 4.10), [D] =
//      [C] - [B], Rayleigh-Jeans conversion (Sec. 4.9).
//
// Continuum shortcut.  For the continuum cube, and for fine velocities that
// no sample's line reaches, the transfer coefficients do not depend on the
// velocity: alpha = alpha_D and the dust source is linear in u across the
// band (first-order expansion of B_nu(T_dust) in u/c, error < (u/c)^2).  The
// recurrence is linear, so I(u) = X0 I_bg(u) + X1 + X2 u with three basis
// recurrences X0 (background 1, no source), X1 and X2 (zero background,
// unit-coefficient sources).  The smooth integrator's ReLU never acts on
// these channels when h alpha_D <= 1/2 on every sample (then I_{n+1} >= I_n/2
// by induction through the trapezoidal and BDF2 steps), so the shortcut is
// exact in exact arithmetic; otherwise every channel is integrated
// explicitly.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <math_constants.h>
#include <stdint.h>

#include "irt_internal.h"

namespace irt {
namespace dev {

constexpr float kLog2e = 1.4426950408889634f;
// Line tail cut: the profile is skipped where (u - v)^2 / b^2 > x2cut
// (exp(-30) = 9e-14 of the peak).
constexpr float kX2CutF32 = 30.0f;

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// ---------------------------------------------------------------------------
// field loading
// ---------------------------------------------------------------------------
__device__ __forceinline__ float h16_to_f32(uint32_t bits16, bool is_bf16) {
  if (is_bf16) return __uint_as_float(bits16 << 16);
  return __half2float(__ushort_as_half((unsigned short)bits16));
}

template <typename R, int ST>
__device__ __forceinline__ void load_cell(const void* cells, long long idx, int bf16_mask,
                                          const float* scale, R v[5]) {
  if constexpr (ST == ST_F32) {
    const float4* p = reinterpret_cast<const float4*>(cells) + 2 * idx;
    const float4 a = __ldg(p);
    const float b = __ldg(reinterpret_cast<const float*>(p + 1));
    v[0] = (R)a.x; v[1] = (R)a.y; v[2] = (R)a.z; v[3] = (R)a.w; v[4] = (R)b;
  } else if constexpr (ST == ST_H16) {
    const uint4 w = __ldg(reinterpret_cast<const uint4*>(cells) + idx);
    v[0] = (R)(h16_to_f32(w.x & 0xFFFFu, bf16_mask & 1) * scale[0]);
    v[1] = (R)(h16_to_f32(w.x >> 16, bf16_mask & 2) * scale[1]);
    v[2] = (R)(h16_to_f32(w.y & 0xFFFFu, bf16_mask & 4) * scale[2]);
    v[3] = (R)(h16_to_f32(w.y >> 16, bf16_mask & 8) * scale[3]);
    v[4] = (R)(h16_to_f32(w.z & 0xFFFFu, bf16_mask & 16) * scale[4]);
  } else {
    const double2* p = reinterpret_cast<const double2*>(cells) + 4 * idx;
    const double2 a = __ldg(p), b = __ldg(p + 1);
    const double c = __ldg(reinterpret_cast<const double*>(p + 2));
    v[0] = (R)a.x; v[1] = (R)a.y; v[2] = (R)b.x; v[3] = (R)b.y; v[4] = (R)c;
  }
}

// ---------------------------------------------------------------------------
// ray geometry (double precision, as the sample count must be exact)
// ---------------------------------------------------------------------------
struct RayGeom {
  int K;
  double h;
  double o[3], d[3];
  double t0;
};

__device__ inline RayGeom ray_geom(const JobDev& J, int px, int py) {
  RayGeom g;
  g.t0 = 0.0;
  if (J.zview) {
    g.K = J.nz;
    g.h = J.dx;
    g.o[0] = g.o[1] = g.o[2] = 0.0;
    g.d[0] = g.d[1] = 0.0;
    g.d[2] = 1.0;
    return g;
  }
  double st, ct, sp, cp;
  sincos(J.theta, &st, &ct);
  sincos(J.phi, &sp, &cp);
  g.d[0] = st * cp; g.d[1] = st * sp; g.d[2] = ct;
  const double et[3] = {ct * cp, ct * sp, -st};
  const double ep[3] = {-sp, cp, 0.0};
  const double L[3] = {J.nx * J.dx, J.ny * J.dx, J.nz * J.dx};
  const double a = (px - 0.5 * (J.npx - 1)) * J.pixel;
  const double b = (py - 0.5 * (J.npy - 1)) * J.pixel;
  double lo = -CUDART_INF, hi = CUDART_INF;
  bool miss = false;
  for (int i = 0; i < 3; ++i) {
    g.o[i] = 0.5 * L[i] + a * et[i] + b * ep[i];
    if (g.d[i] == 0.0) {
      if (g.o[i] < 0.0 || g.o[i] > L[i]) miss = true;
      continue;
    }
    double t0 = (0.0 - g.o[i]) / g.d[i], t1 = (L[i] - g.o[i]) / g.d[i];
    if (t0 > t1) { const double t = t0; t0 = t1; t1 = t; }
    lo = fmax(lo, t0);
    hi = fmin(hi, t1);
  }
  if (miss || !(hi > lo)) {
    g.K = 0;
    g.h = 0.0;
    return g;
  }
  const double chord = hi - lo;
  g.K = (int)ceil(chord / J.dx - 1e-9);
  g.h = (g.K > 0) ? chord / g.K : 0.0;
  g.t0 = lo;
  return g;
}

// Raw sample values (n_H2, T_gas, T_dust, v_los, x) of sample k of a ray.
template <typename R, int ST>
__device__ __forceinline__ void sample_raw(const JobDev& J, const RayGeom& g, int px, int py,
                                           int k, R v[5]) {
  if (J.zview) {
    const long long idx = ((long long)k * J.ny + py) * J.nx + px;
    load_cell<R, ST>(J.cells, idx, J.bf16_mask, J.scale, v);
    return;
  }
  const double t = g.t0 + (k + 0.5) * g.h;
  const int n[3] = {J.nx, J.ny, J.nz};
  int i0[3], i1[3];
  R w[3];
  for (int a = 0; a < 3; ++a) {
    const double s = (g.o[a] + t * g.d[a]) / J.dx - 0.5;
    const double fl = floor(s);
    w[a] = (R)(s - fl);
    const int lo = (int)fl;
    i0[a] = min(max(lo, 0), n[a] - 1);
    i1[a] = min(max(lo + 1, 0), n[a] - 1);
  }
  for (int q = 0; q < 5; ++q) v[q] = (R)0;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const int ix = (c & 1) ? i1[0] : i0[0];
    const int iy = (c & 2) ? i1[1] : i0[1];
    const int iz = (c & 4) ? i1[2] : i0[2];
    const R wx = (c & 1) ? w[0] : (R)1 - w[0];
    const R wy = (c & 2) ? w[1] : (R)1 - w[1];
    const R wz = (c & 4) ? w[2] : (R)1 - w[2];
    const R ww = wx * wy * wz;
    R cv[5];
    load_cell<R, ST>(J.cells, ((long long)iz * J.ny + iy) * J.nx + ix, J.bf16_mask, J.scale,
                     cv);
#pragma unroll
    for (int q = 0; q < 5; ++q) v[q] += ww * cv[q];
  }
}

// ---------------------------------------------------------------------------
// per-sample physics
// ---------------------------------------------------------------------------
// Rigid-rotor partition function Z(T) = sum_J (2J+1) exp(-theta J(J+1)/T).
__device__ inline float partition(const PhysParams& P, float T) {
  const float r = (float)P.theta_rot / T;
  if (r < 0.0132f) {
    // high-temperature expansion, truncation error O(r^4) < 1e-9 relative
    return 1.0f / r + (1.0f / 3.0f) + r * (1.0f / 15.0f + r * (4.0f / 315.0f + r * (1.0f / 315.0f)));
  }
  // terms t_J = q^{J(J+1)} by the ratio t_J = t_{J-1} q^{2J}
  const float q2 = expf(-2.0f * r);
  float t = 1.0f, m = q2, z = 1.0f;
  for (int J = 1; J < 400; ++J) {
    t *= m;
    m *= q2;
    const float term = (2 * J + 1) * t;
    z += term;
    if (term < 3e-9f * z) break;
  }
  return z;
}

__device__ inline double partition(const PhysParams& P, double T) {
  double z = 0.0;
  for (int J = 0; J < 100000; ++J) {
    const double term = (2.0 * J + 1.0) * exp(-P.theta_rot * J * (J + 1.0) / T);
    z += term;
    if (J > 0 && term < 1e-17 * z) break;
  }
  return z;
}

__device__ __forceinline__ float expm1_(float x) { return expm1f(x); }
__device__ __forceinline__ double expm1_(double x) { return expm1(x); }
__device__ __forceinline__ float exp_(float x) { return expf(x); }
__device__ __forceinline__ double exp_(double x) { return exp(x); }
__device__ __forceinline__ float sqrt_(float x) { return sqrtf(x); }
__device__ __forceinline__ double sqrt_(double x) { return sqrt(x); }

// Frequency-independent per-step line coefficients at the profile peak (K
// units / optical depth) and the Doppler parameter b [km/s].
template <typename R>
__device__ __forceinline__ void line_coeffs(const PhysParams& P, R n, R T, R x, R h, R* jl,
                                            R* al, R* b) {
  *b = sqrt_((R)P.c_th * T + (R)P.two_sig2);
  if (!(T > (R)0) || T > (R)P.t_inf) {
    *jl = (R)0;
    *al = (R)0;
    return;
  }
  const R Z = partition(P, T);
  const R c = (x * n) * h / (Z * *b);
  *jl = (R)P.cj * c * exp_(-(R)P.e_u / T);
  *al = (R)P.ca * c * exp_(-(R)P.e_l / T) * (-expm1_(-(R)P.T0 / T));
}

// Dust Planck source in K units at the line frequency and its first-order
// slope in u [per km/s]: B(u) = bk0 + bk1 u + O((u/c)^2).
__device__ __forceinline__ void dust_source_lin(const PhysParams& P, float Td, float* bk0,
                                                float* bk1) {
  if (!(Td > 0.0f)) {
    *bk0 = 0.0f;
    *bk1 = 0.0f;
    return;
  }
  const float a = (float)P.T0 / Td;
  const float em1 = expm1f(a);
  const float inv = 1.0f / em1;
  *bk0 = (float)P.T0 * inv;
  // d ln B / d ln nu at nu_ul is 3 - a e^a / (e^a - 1); nu = nu_ul (1 - u/c)
  const float slope = 3.0f - a * (1.0f + inv);
  *bk1 = -(*bk0) * slope * (float)P.inv_c_kms;
}

// Exact Planck source in K units at velocity u: T0 y^3 / (exp(T0 y / T) - 1).
__device__ __forceinline__ double planck_k(const PhysParams& P, double T, double u) {
  if (!(T > 0.0)) return 0.0;
  const double y = 1.0 - u * P.inv_c_kms;
  return P.T0 * y * y * y / expm1(P.T0 * y / T);
}
__device__ __forceinline__ float planck_k(const PhysParams& P, float T, float u) {
  if (!(T > 0.0f)) return 0.0f;
  const float y = 1.0f - u * (float)P.inv_c_kms;
  return (float)P.T0 * y * y * y / expm1f((float)P.T0 * y / T);
}

// ---------------------------------------------------------------------------
// per-sample records in shared memory
// ---------------------------------------------------------------------------
// Window of fine blocks reached by the line: lo | hi << 16 (lo > hi = none).
__device__ __forceinline__ int pack_win(int lo, int hi) { return (lo & 0xFFFF) | (hi << 16); }
__device__ __forceinline__ int win_lo(int w) { return (int)(short)(w & 0xFFFF); }
__device__ __forceinline__ int win_hi(int w) { return w >> 16; }

// smooth, float: (2h j) and (2h alpha) scaled; d0 = 3 + 2 h alpha_D
struct __align__(16) RecS32 {
  float jl2, al2, v, nib2, d0, jd0, jd1;
  int win;
};
// formal, float
struct __align__(16) RecF32 {
  float jl, al, v, nib2, ad, emD, bk0, bk1;
  int win;
  float pad[3];
};
// double (both integrators, every channel explicit, exact Planck per channel)
struct __align__(16) RecD {
  double jl, al, v, nib2, ad, emD, td;
  int win;
  int pad;
};

template <typename R, int MODE> struct RecOf;
template <> struct RecOf<float, M_SMOOTH> { using type = RecS32; };
template <> struct RecOf<float, M_FORMAL> { using type = RecF32; };
template <> struct RecOf<float, M_FORMAL_KAHAN> { using type = RecF32; };
template <> struct RecOf<double, M_SMOOTH> { using type = RecD; };
template <> struct RecOf<double, M_FORMAL> { using type = RecD; };
template <> struct RecOf<double, M_FORMAL_KAHAN> { using type = RecD; };

// Fine-block window [lo, hi] (local block indices) reached by the line of a
// sample with centre v and Doppler parameter b.
__device__ __forceinline__ int line_window(float v, float b, float ufirst, float dvf, int gw0,
                                           int nfw, bool has_line) {
  if (!has_line) return pack_win(1, 0);
  const float w = b * 5.4772256f;  // sqrt(x2cut)
  const int glo = (int)ceilf((v - w - ufirst) / dvf) - gw0;
  const int ghi = (int)floorf((v + w - ufirst) / dvf) - gw0;
  const int lo = max(glo, 0), hi = min(ghi, nfw - 1);
  if (lo > hi) return pack_win(1, 0);
  return pack_win(lo >> 5, hi >> 5);
}

}  // namespace dev
}  // namespace irt

// Forward PPV kernel of the IRIS-SO transfer (sm_103a): device helpers.
//
// Work item = one ray, every channel.  One warp renders one item:
//   1. sample pass: lane l evaluates samples k = l, l+32, ... of the ray (field
//      load or trilinear interpolation, LTE populations, line and dust
//      coefficients, Sec. 3.2-3.7, 5.10) into a per-sample record (global
//      fine-velocity indices, so one pass serves every channel), written to
//      the warp's slot of an L2-resident scratch buffer;
//   2. transfer pass: the records stream back 32 at a time through shared
//      memory; lane l owns the fine velocities g = 32 (hb + j) + l of the
//      blocks the line reaches (register blocks j) and integrates them sample
//      by sample (Sec. 4.8, formal or smooth), evaluating the Gaussian profile
//      only at the velocities the sample's line reaches;
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
// Line tail cut: the profile is skipped where (u - v)^2 / b^2 > 30, i.e. below
// exp(-30) = 9e-14 of its peak; sqrt(30) = 5.4772256.
constexpr float kSqrtX2Cut = 5.4772256f;

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

// Cell z of sample k on the cell-exact views: k on the z view; nz - 1 - k on
// the radial view of an observer-centred [r][b][l] tensor (the ray runs from
// the far end of the radial axis to the observer at r = 0).
__device__ __forceinline__ int zcell(const JobDev& J, int k) { return J.zrev ? J.nz - 1 - k : k; }

// ---------------------------------------------------------------------------
// ray geometry of the double kernels: the view's float-float coefficients
// (cell units) evaluated in double; the sample count K = ceil(chord - 1e-9)
// must be exact, and is the one the float kernels' set-up below reaches
// ---------------------------------------------------------------------------
struct RayGeom {
  int K;
  double h;        // step [cm]
  double hc;       // step [cells]
  double o[3], d[3];   // origin [cells], direction
  double t0;       // entry [cells]
};

__device__ __forceinline__ double ff_wide(const float v[2]) { return (double)v[0] + (double)v[1]; }

__device__ inline RayGeom ray_geom(const JobDev& J, int px, int py) {
  RayGeom g;
  g.t0 = 0.0;
  if (J.zview) {
    g.K = J.nz;
    g.h = J.dx;
    g.hc = 1.0;
    g.o[0] = g.o[1] = g.o[2] = 0.0;
    g.d[0] = g.d[1] = 0.0;
    g.d[2] = 1.0;
    return g;
  }
  const double L[3] = {(double)J.nx, (double)J.ny, (double)J.nz};
  double lo = -CUDART_INF, hi = CUDART_INF;
  bool miss = false;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    g.d[i] = ff_wide(J.fd[i]);
    g.o[i] = ff_wide(J.fo0[i]) + px * ff_wide(J.fox[i]) + py * ff_wide(J.foy[i]);
    if (J.fd[i][0] == 0.0f) {
      if (g.o[i] < 0.0 || g.o[i] > L[i]) miss = true;
      continue;
    }
    const double inv = ff_wide(J.finv_d[i]);
    double t0 = (0.0 - g.o[i]) * inv, t1 = (L[i] - g.o[i]) * inv;
    if (t0 > t1) { const double t = t0; t0 = t1; t1 = t; }
    lo = fmax(lo, t0);
    hi = fmin(hi, t1);
  }
  g.K = 0;
  g.h = g.hc = 0.0;
  if (miss || !(hi > lo)) return g;
  const double chord = hi - lo;
  g.K = (int)ceil(chord - 1e-9);
  if (g.K <= 0) {
    g.K = 0;
    return g;
  }
  g.hc = chord / g.K;
  g.h = g.hc * J.dx;
  g.t0 = lo;
  return g;
}

// fractional cell coordinates (cell centres at integers) of sample k
__device__ __forceinline__ void sample_cell(const RayGeom& g, int k, int i0[3], double w[3]) {
  const double t = g.t0 + (k + 0.5) * g.hc;
  for (int a = 0; a < 3; ++a) {
    const double s = g.o[a] + t * g.d[a] - 0.5;
    const double fl = floor(s);
    w[a] = s - fl;
    i0[a] = (int)fl;
  }
}

// Trilinear blend of the eight cells around fractional cell coordinates
// (i0 + w) per axis; indices clamped to the grid (edge extension).
template <typename R, int ST>
__device__ __forceinline__ void trilinear(const JobDev& J, const int i0[3], const R w[3], R v[5]) {
  const int n[3] = {J.nx, J.ny, J.nz};
  int lo[3], hi[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    lo[a] = min(max(i0[a], 0), n[a] - 1);
    hi[a] = min(max(i0[a] + 1, 0), n[a] - 1);
  }
#pragma unroll
  for (int q = 0; q < 5; ++q) v[q] = (R)0;
  // v_los is blended as differences from the first corner: the profile is
  // steep in v, and rounding the blend of values of tens of km/s would move
  // the line by ~1e-5 km/s; the differences between neighbouring cells are
  // small, so their rounding is not
  R vref = (R)0;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const int ix = (c & 1) ? hi[0] : lo[0];
    const int iy = (c & 2) ? hi[1] : lo[1];
    const int iz = (c & 4) ? hi[2] : lo[2];
    const R wx = (c & 1) ? w[0] : (R)1 - w[0];
    const R wy = (c & 2) ? w[1] : (R)1 - w[1];
    const R wz = (c & 4) ? w[2] : (R)1 - w[2];
    const R ww = wx * wy * wz;
    R cv[5];
    load_cell<R, ST>(J.cells, ((long long)iz * J.ny + iy) * J.nx + ix, J.bf16_mask, J.scale, cv);
    if (c == 0) vref = cv[3];
    cv[3] -= vref;
#pragma unroll
    for (int q = 0; q < 5; ++q) v[q] += ww * cv[q];
  }
  v[3] += vref;
}

// Raw sample values (n_H2, T_gas, T_dust, v_los, x) of sample k of a ray,
// double arithmetic (double kernels).
template <int ST>
__device__ __forceinline__ void sample_raw(const JobDev& J, const RayGeom& g, int px, int py,
                                           int k, double v[5]) {
  if (J.zview) {
    load_cell<double, ST>(J.cells, ((long long)zcell(J, k) * J.ny + py) * J.nx + px, J.bf16_mask,
                          J.scale,
                          v);
    return;
  }
  int i0[3];
  double w[3];
  sample_cell(g, k, i0, w);
  trilinear<double, ST>(J, i0, w, v);
}

// Oblique sample positions of the float kernels in 32.32 fixed point (cell
// units, cell centres at integers): sample k sits at base + k step.  Base and
// step are rounded once per ray (ray_setup below); the position of sample k
// is then exact to k * 2^-33 cells (1e-7 cells after 900 samples).
struct RayPos {
  long long base[3], step[3];
};

// ---------------------------------------------------------------------------
// Ray set-up of the float kernels, without double arithmetic.  The chord, the
// sample count K = ceil(chord / dx - 1e-9), the step and the 32.32 sample
// positions are evaluated in float-float arithmetic: a value is the
// unevaluated sum hi + lo of two floats (about 48 significant bits), built
// from the error-free sum of two floats (Knuth's two-sum) and the error-free
// product (the fma residual).  Its rounding, about 1e-11 cells on a
// 1000-cell chord, is far below the 1e-9 slack of the sample count, so K is
// the double-precision value except on chords within ~1e-11 of that slack.
// The double kernels keep ray_geom above.
// ---------------------------------------------------------------------------
struct FF {
  float hi, lo;
};

__device__ __forceinline__ FF ff_load(const float v[2]) { return FF{v[0], v[1]}; }
__device__ __forceinline__ FF ff_two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return FF{s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ FF ff_add(FF x, FF y) {
  const FF s = ff_two_sum(x.hi, y.hi);
  return ff_two_sum(s.hi, s.lo + (x.lo + y.lo));
}
__device__ __forceinline__ FF ff_neg(FF x) { return FF{-x.hi, -x.lo}; }
__device__ __forceinline__ FF ff_mul(FF x, FF y) {
  const float p = x.hi * y.hi;
  const float e = fmaf(x.hi, y.hi, -p);
  return ff_two_sum(p, fmaf(x.hi, y.lo, fmaf(x.lo, y.hi, e)));
}
// x b for a float b
__device__ __forceinline__ FF ff_mul_f(FF x, float b) {
  const float p = x.hi * b;
  return ff_two_sum(p, fmaf(x.lo, b, fmaf(x.hi, b, -p)));
}
__device__ __forceinline__ bool ff_lt(FF a, FF b) {
  return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo);
}
// x / k for an integer 0 < k < 2^24: quotient, exact remainder, correction
__device__ __forceinline__ FF ff_div_i(FF x, int k) {
  const float kf = (float)k;
  const float q1 = __fdiv_rn(x.hi, kf);
  const FF r = ff_add(x, ff_neg(ff_mul_f(FF{q1, 0.0f}, kf)));
  return ff_two_sum(q1, __fdiv_rn(r.hi, kf));
}
// smallest integer >= x (|x| < 2^23; a normalised pair cannot straddle an
// integer unless hi is that integer)
__device__ __forceinline__ int ff_ceil(FF x) {
  const float c = ceilf(x.hi);
  return (int)c + ((c == x.hi && x.lo > 0.0f) ? 1 : 0);
}
// x 2^32 rounded to a 64-bit integer (|x| < 2^30)
__device__ __forceinline__ long long ff_fix32(FF x) {
  return __float2ll_rn(x.hi * 4294967296.0f) + __float2ll_rn(x.lo * 4294967296.0f);
}

struct RaySet {
  int K;       // samples (0: the ray misses the box)
  float h;     // step [cm]
  RayPos rp;   // oblique views: sample positions
};

// The chord of pixel (px, py) through the box [0, n]^3 (cell units): the
// latest entry and the earliest exit over the three slabs; an axis with
// d = 0 is a miss when the origin lies outside its slab.
__device__ __forceinline__ FF ff_shfl(FF x, int src) {
  return FF{__shfl_sync(0xffffffffu, x.hi, src), __shfl_sync(0xffffffffu, x.lo, src)};
}

// Called by the 32 lanes of a warp together (one ray per warp): lane a < 3
// evaluates axis a, the entry / exit and the positions are exchanged with
// shuffles, so the warp issues the per-axis work once instead of three times.
__device__ inline RaySet ray_setup(const JobDev& J, int px, int py) {
  RaySet r;
  r.K = 0;
  r.h = 0.0f;
  if (J.zview) {
    r.K = J.nz;
    r.h = J.fdx[0];
    return r;
  }
  const int lane = threadIdx.x & 31;
  const int a = min(lane, 2);   // this lane's axis (lanes 3..31 repeat axis 2)
  const int na_i = (a == 0) ? J.nx : ((a == 1) ? J.ny : J.nz);
  const FF o = ff_add(ff_load(J.fo0[a]), ff_add(ff_mul_f(ff_load(J.fox[a]), (float)px),
                                                ff_mul_f(ff_load(J.foy[a]), (float)py)));
  const FF na{(float)na_i, 0.0f};
  FF t0{-INFINITY, 0.0f}, t1{INFINITY, 0.0f};
  bool miss = false;
  if (J.fd[a][0] == 0.0f) {
    miss = ff_lt(o, FF{0.0f, 0.0f}) || ff_lt(na, o);
  } else {
    const FF inv = ff_load(J.finv_d[a]);
    t0 = ff_mul(ff_neg(o), inv);
    t1 = ff_mul(ff_add(na, ff_neg(o)), inv);
    if (ff_lt(t1, t0)) {
      const FF t = t0;
      t0 = t1;
      t1 = t;
    }
  }
  // latest entry and earliest exit over the three axes (lanes 0, 1, 2)
  FF lo = ff_shfl(t0, 0), hi = ff_shfl(t1, 0);
#pragma unroll
  for (int b = 1; b < 3; ++b) {
    const FF e = ff_shfl(t0, b), x = ff_shfl(t1, b);
    if (ff_lt(lo, e)) lo = e;
    if (ff_lt(x, hi)) hi = x;
  }
  miss = __any_sync(0xffffffffu, miss && lane < 3);
  if (miss || !ff_lt(lo, hi)) return r;
  const FF chord = ff_add(hi, ff_neg(lo));
  // 1e-9 as a float-float pair
  const int K = ff_ceil(ff_add(chord, FF{-9.999999717180685e-10f, -2.8281930491731106e-17f}));
  if (K <= 0) return r;
  const FF h = ff_div_i(chord, K);
  r.K = K;
  r.h = ff_mul(h, ff_load(J.fdx)).hi;
  // sample k at t_in + (k + 1/2) h; trilinear coordinates are shifted by
  // half a cell (cell centres at integers)
  const FF tm = ff_add(lo, FF{0.5f * h.hi, 0.5f * h.lo});
  const FF d = ff_load(J.fd[a]);
  const long long base = ff_fix32(ff_add(ff_add(o, ff_mul(tm, d)), FF{-0.5f, 0.0f}));
  const long long step = ff_fix32(ff_mul(h, d));
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    r.rp.base[b] = __shfl_sync(0xffffffffu, base, b);
    r.rp.step[b] = __shfl_sync(0xffffffffu, step, b);
  }
  return r;
}

// The ray set-up as a call of its own (once per ray), for the adjoint
// kernels: its float-float temporaries then take no registers of the sweep
// around it.  The forward kernels inline it (a call there makes the
// 128-register kernels save live registers to the stack around it).
static __device__ __noinline__ RaySet ray_setup_call(const JobDev& J, int px, int py) {
  return ray_setup(J, px, py);
}

// float kernels: sample k of the ray
template <int ST>
__device__ __forceinline__ void sample_raw(const JobDev& J, const RayPos& rp, int px, int py,
                                           int k, float v[5]) {
  if (J.zview) {
    load_cell<float, ST>(J.cells, ((long long)zcell(J, k) * J.ny + py) * J.nx + px, J.bf16_mask,
                         J.scale,
                         v);
    return;
  }
  int i0[3];
  float w[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const long long p = rp.base[a] + (long long)k * rp.step[a];
    i0[a] = (int)(p >> 32);
    w[a] = (float)(unsigned)(p & 0xFFFFFFFFll) * 2.3283064365386963e-10f;   // 2^-32
  }
  trilinear<float, ST>(J, i0, w, v);
}

// H2 abundance of sample k (the cells' spare slot; optically thin level
// balance only): the cell value on the z view, the trilinear blend of the
// eight cells (already loaded for the other fields) on oblique views.
template <typename R, int ST>
__device__ __forceinline__ R cell_chi(const void* cells, long long idx) {
  if constexpr (ST == ST_F32) return (R)__ldg(reinterpret_cast<const float*>(cells) + 8 * idx + 5);
  else if constexpr (ST == ST_H16)
    return (R)__half2float(__ushort_as_half(
        __ldg(reinterpret_cast<const unsigned short*>(cells) + 8 * idx + 5)));
  else return (R)__ldg(reinterpret_cast<const double*>(cells) + 8 * idx + 5);
}

template <typename R, int ST>
__device__ __forceinline__ R chi_trilinear(const JobDev& J, const int i0[3], const R w[3]) {
  const int n[3] = {J.nx, J.ny, J.nz};
  int lo[3], hi[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    lo[a] = min(max(i0[a], 0), n[a] - 1);
    hi[a] = min(max(i0[a] + 1, 0), n[a] - 1);
  }
  R acc = (R)0;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const int ix = (c & 1) ? hi[0] : lo[0];
    const int iy = (c & 2) ? hi[1] : lo[1];
    const int iz = (c & 4) ? hi[2] : lo[2];
    const R ww = ((c & 1) ? w[0] : (R)1 - w[0]) * ((c & 2) ? w[1] : (R)1 - w[1]) *
                 ((c & 4) ? w[2] : (R)1 - w[2]);
    acc += ww * cell_chi<R, ST>(J.cells, ((long long)iz * J.ny + iy) * J.nx + ix);
  }
  return acc;
}

// Only the optically thin level-balance kernel instances call it.
template <int ST>
__device__ __forceinline__ float sample_chi_pos(const JobDev& J, long long b0, long long b1,
                                             long long b2, long long s0, long long s1,
                                             long long s2, int px, int py, int k) {
  if (J.zview)
    return cell_chi<float, ST>(J.cells, ((long long)zcell(J, k) * J.ny + py) * J.nx + px);
  const long long base[3] = {b0, b1, b2}, step[3] = {s0, s1, s2};
  int i0[3];
  float w[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const long long p = base[a] + (long long)k * step[a];
    i0[a] = (int)(p >> 32);
    w[a] = (float)(unsigned)(p & 0xFFFFFFFFll) * 2.3283064365386963e-10f;
  }
  return chi_trilinear<float, ST>(J, i0, w);
}

template <int ST>
__device__ __forceinline__ float sample_chi(const JobDev& J, const RayPos& rp, int px, int py,
                                            int k) {
  return sample_chi_pos<ST>(J, rp.base[0], rp.base[1], rp.base[2], rp.step[0], rp.step[1],
                            rp.step[2], px, py, k);
}

template <int ST>
__device__ __forceinline__ double sample_chi(const JobDev& J, const RayGeom& g, int px, int py,
                                             int k) {
  if (J.zview)
    return cell_chi<double, ST>(J.cells, ((long long)zcell(J, k) * J.ny + py) * J.nx + px);
  int i0[3];
  double w[3];
  sample_cell(g, k, i0, w);
  return chi_trilinear<double, ST>(J, i0, w);
}

// ---------------------------------------------------------------------------
// per-sample physics
// ---------------------------------------------------------------------------
// Rigid-rotor partition function Z(T) = sum_J (2J+1) exp(-theta J(J+1)/T).
__device__ inline float partition(const PhysF& P, float T) {
  const float r = P.theta_rot / T;
  if (r < 0.1f) {
    // high-temperature expansion: relative truncation error below 1.2e-8
    // against the full sum for r < 0.1, under float rounding
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

// Optically thin level balance (Sec. 4.2, 4.3): trilinear interpolation of
// the line's coefficient grid in (log10 n_H, chi, log10 T), n_H = n_H2 / chi,
// the cell index clamped to the grid so that outside it the edge cell
// continues linearly.  Returns (j, alpha) per tracer molecule in per-step K
// units (to be multiplied by N h / b).
__device__ __forceinline__ float2 ot_lookup(const PhysF& P, float n, float chi, float T) {
  const float x[3] = {log10f(n / chi), chi, log10f(T)};
  int i[3];
  float w[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float u = (x[a] - P.ot_lo[a]) * P.ot_s[a];
    const int iu = min(max((int)floorf(u), 0), P.ot_n[a] - 2);
    i[a] = iu;
    w[a] = u - (float)iu;
  }
  const int n2p = P.ot_n[2] - 1;
  const float4* p = P.ot_tab + ((long long)i[0] * P.ot_n[1] + i[1]) * n2p + i[2];
  const float4 c00 = __ldg(p), c01 = __ldg(p + n2p);
  const float4 c10 = __ldg(p + (long long)P.ot_n[1] * n2p);
  const float4 c11 = __ldg(p + (long long)P.ot_n[1] * n2p + n2p);
  // along T within each of the four (n, chi) corners, then chi, then n
  const float w2 = w[2], v2 = 1.0f - w2;
  const float j00 = v2 * c00.x + w2 * c00.z, a00 = v2 * c00.y + w2 * c00.w;
  const float j01 = v2 * c01.x + w2 * c01.z, a01 = v2 * c01.y + w2 * c01.w;
  const float j10 = v2 * c10.x + w2 * c10.z, a10 = v2 * c10.y + w2 * c10.w;
  const float j11 = v2 * c11.x + w2 * c11.z, a11 = v2 * c11.y + w2 * c11.w;
  const float w1 = w[1], v1 = 1.0f - w1;
  const float j0 = v1 * j00 + w1 * j01, a0 = v1 * a00 + w1 * a01;
  const float j1 = v1 * j10 + w1 * j11, a1 = v1 * a10 + w1 * a11;
  const float w0 = w[0], v0 = 1.0f - w0;
  return make_float2(v0 * j0 + w0 * j1, v0 * a0 + w0 * a1);
}

__device__ inline double2 ot_lookup(const PhysParams& P, double n, double chi, double T) {
  const double x[3] = {log10(n / chi), chi, log10(T)};
  int i[3];
  double w[3];
  for (int a = 0; a < 3; ++a) {
    const double u = (x[a] - P.ot_lo[a]) * P.ot_s[a];
    const int iu = min(max((int)floor(u), 0), P.ot_n[a] - 2);
    i[a] = iu;
    w[a] = u - (double)iu;
  }
  double acc0 = 0.0, acc1 = 0.0;
  for (int c = 0; c < 8; ++c) {
    const int a0 = i[0] + (c & 1), a1 = i[1] + ((c >> 1) & 1), a2 = i[2] + ((c >> 2) & 1);
    const double wc = ((c & 1) ? w[0] : 1.0 - w[0]) * ((c & 2) ? w[1] : 1.0 - w[1]) *
                      ((c & 4) ? w[2] : 1.0 - w[2]);
    const long long idx = (((long long)a0 * P.ot_n[1] + a1) * P.ot_n[2] + a2) * 2;
    acc0 += wc * __ldg(P.ot_tab + idx);
    acc1 += wc * __ldg(P.ot_tab + idx + 1);
  }
  return make_double2(acc0 * P.ot_jk, acc1 * P.ot_ak);
}

// Frequency-independent per-step line coefficients at the profile peak (K
// units / optical depth) and the Doppler parameter b [km/s]: LTE populations,
// or the optically thin level-balance grid when the launch has one (chi =
// the sample's H2 abundance per H nucleus).
// OTC = false compiles the LTE path alone (kernel instances that never take
// a grid).
template <bool OTC = true>
__device__ __forceinline__ void line_coeffs(const PhysF& P, float n, float T, float x, float chi,
                                            float h, float* jl, float* al, float* b) {
  *b = sqrtf(P.c_th * T + P.two_sig2);
  if (!(T > 0.0f) || T > P.t_inf) {
    *jl = 0.0f;
    *al = 0.0f;
    return;
  }
  if (OTC && P.ot_tab) {
    if (!(n > 0.0f) || !(chi > 0.0f) || !(x > 0.0f)) {
      *jl = 0.0f;
      *al = 0.0f;
      return;
    }
    const float2 c = ot_lookup(P, n, chi, T);
    const float s = (x * n) * h / *b;
    *jl = s * c.x;
    *al = s * c.y;
    return;
  }
  const float Z = partition(P, T);
  const float c = (x * n) * h / (Z * *b);
  *jl = P.cj * c * expf(-P.e_u / T);
  *al = P.ca * c * expf(-P.e_l / T) * (-expm1f(-P.T0 / T));
}

template <bool OTC = true>
__device__ __forceinline__ void line_coeffs(const PhysParams& P, double n, double T, double x,
                                            double chi, double h, double* jl, double* al,
                                            double* b) {
  *b = sqrt(P.c_th * T + P.two_sig2);
  if (!(T > 0.0) || T > P.t_inf) {
    *jl = 0.0;
    *al = 0.0;
    return;
  }
  if (OTC && P.ot_tab) {
    if (!(n > 0.0) || !(chi > 0.0) || !(x > 0.0)) {
      *jl = 0.0;
      *al = 0.0;
      return;
    }
    const double2 c = ot_lookup(P, n, chi, T);
    const double s = (x * n) * h / *b;
    *jl = s * c.x;
    *al = s * c.y;
    return;
  }
  const double Z = partition(P, T);
  const double c = (x * n) * h / (Z * *b);
  *jl = P.cj * c * exp(-P.e_u / T);
  *al = P.ca * c * exp(-P.e_l / T) * (-expm1(-P.T0 / T));
}

// Dust Planck source in K units at the line frequency and its first-order
// slope in u [per km/s]: B(u) = bk0 + bk1 u + O((u/c)^2).
__device__ __forceinline__ void dust_source_lin(const PhysF& P, float Td, float* bk0,
                                                float* bk1) {
  if (!(Td > 0.0f)) {
    *bk0 = 0.0f;
    *bk1 = 0.0f;
    return;
  }
  const float a = P.T0 / Td;
  const float em1 = expm1f(a);
  const float inv = 1.0f / em1;
  *bk0 = P.T0 * inv;
  // d ln B / d ln nu at nu_ul is 3 - a e^a / (e^a - 1); nu = nu_ul (1 - u/c)
  const float slope = 3.0f - a * (1.0f + inv);
  *bk1 = -(*bk0) * slope * P.inv_c_kms;
}

// Exact Planck source in K units at velocity u: T0 y^3 / (exp(T0 y / T) - 1).
__device__ __forceinline__ double planck_k(const PhysParams& P, double T, double u) {
  if (!(T > 0.0)) return 0.0;
  const double y = 1.0 - u * P.inv_c_kms;
  return P.T0 * y * y * y / expm1(P.T0 * y / T);
}
__device__ __forceinline__ float planck_k(const PhysF& P, float T, float u) {
  if (!(T > 0.0f)) return 0.0f;
  const float y = 1.0f - u * P.inv_c_kms;
  return P.T0 * y * y * y / expm1f(P.T0 * y / T);
}

// ---------------------------------------------------------------------------
// per-sample records in shared memory
// ---------------------------------------------------------------------------
// Line window of a sample in local fine-velocity indices: lo | hi << 16
// (lo > hi = the line reaches no velocity of the window).
__device__ __forceinline__ int pack_win(int lo, int hi) { return (lo & 0xFFFF) | (hi << 16); }
__device__ __forceinline__ int win_lo(int w) { return (int)(short)(w & 0xFFFF); }
__device__ __forceinline__ int win_hi(int w) { return w >> 16; }
constexpr int kNoWindow = 0xFFFF7FFF;   // lo = 32767, hi = -1

// Float records keep the line centre as (gv, vr): gv = the local fine index
// nearest to v_los and vr = u(gv) - v_los, so that u(g) - v_los =
// (g - gv) dvf + vr is exact to ~1e-7 km/s even when the fine velocities are
// not representable in float.
// smooth, float: (2h j) and (2h alpha) scaled; d0 = 3 + 2 h alpha_D
struct __align__(16) RecS32 {
  float jl2, al2, vr, nib2, d0, jd0, jd1;
  int win;
  int gv;
  float pad[3];
};
// formal, float
struct __align__(16) RecF32 {
  float jl, al, vr, nib2, ad, emD, bk0, bk1;
  int win;
  int gv;
  float pad[2];
};

// Fine velocity grid of a window in float-float form: u(g) = (ufw_hi + ufw_lo)
// + g (dvf_hi + dvf_lo).
struct VGrid {
  float ufw_hi, ufw_lo, dvf_hi, dvf_lo;
};

// Nearest fine index gv to v and vr = u(gv) - v, evaluated with error-free
// product and sum steps (Dekker / Knuth) so that vr carries no rounding of
// u(gv) itself.
__device__ __forceinline__ void centre_offset(const VGrid& G, float v, int* gv_out,
                                              float* vr_out) {
  float q = rintf((v - G.ufw_hi) / G.dvf_hi);
  q = fminf(fmaxf(q, -1048576.0f), 1048576.0f);
  const float p_hi = q * G.dvf_hi;
  const float p_lo = fmaf(q, G.dvf_hi, -p_hi);
  const float s = G.ufw_hi + p_hi;
  const float bb = s - G.ufw_hi;
  const float s_lo = (G.ufw_hi - (s - bb)) + (p_hi - bb);
  const float corr = p_lo + s_lo + fmaf(q, G.dvf_lo, G.ufw_lo);
  *gv_out = (int)q;
  *vr_out = (s - v) + corr;
}

// u(g) - v_los from a record's (gv, vr)
__device__ __forceinline__ float vel_offset(const VGrid& G, int g, int gv, float vr) {
  const float gd = (float)(g - gv);
  return fmaf(gd, G.dvf_hi, fmaf(gd, G.dvf_lo, vr));
}
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

// Local fine-velocity window [lo, hi] reached by the line of a sample with
// centre v and Doppler parameter b.
__device__ __forceinline__ int line_window(float v, float b, float ufirst, float dvf, int gw0,
                                           int nfw, bool has_line) {
  if (!has_line) return kNoWindow;
  const float w = b * kSqrtX2Cut;
  const int glo = (int)ceilf((v - w - ufirst) / dvf) - gw0;
  const int ghi = (int)floorf((v + w - ufirst) / dvf) - gw0;
  const int lo = max(glo, 0), hi = min(ghi, nfw - 1);
  if (lo > hi) return kNoWindow;
  return pack_win(lo, hi);
}

}  // namespace dev
}  // namespace irt

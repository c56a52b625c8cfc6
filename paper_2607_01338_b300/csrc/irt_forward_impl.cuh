// Kernel template of the forward render (see irt_forward.cuh for the design).
#pragma once

#include <algorithm>

#include "irt_forward.cuh"

namespace irt {
namespace dev {

// ---------------------------------------------------------------------------
// sample pass: record of one sample
// ---------------------------------------------------------------------------
template <typename R, int MODE>
struct SampleOut {
  typename RecOf<R, MODE>::type rec;
  int lo, hi;   // line window (local fine blocks)
  R ad;         // h alpha_D of the sample
};

template <int MODE>
__device__ __forceinline__ void make_record(const PhysParams& P, const float raw[5], float h,
                                            float ufirst, float dvf, int gw0, int nfw,
                                            SampleOut<float, MODE>* so) {
  const float n = raw[0], T = raw[1], Td = raw[2], v = raw[3], x = raw[4];
  float jl, al, b;
  line_coeffs<float>(P, n, T, x, h, &jl, &al, &b);
  const float ad = (float)P.cad * n * h;
  float bk0, bk1;
  dust_source_lin(P, Td, &bk0, &bk1);
  const bool has_line = jl != 0.0f || al != 0.0f;
  // no line: any finite profile parameter (the coefficients are zero)
  const float nib2 = has_line ? -kLog2e / (b * b) : -kLog2e;
  const int win = line_window(v, b, ufirst, dvf, gw0, nfw, has_line);
  if constexpr (MODE == M_SMOOTH) {
    RecS32& r = so->rec;
    r.jl2 = 2.0f * jl;
    r.al2 = 2.0f * al;
    r.v = v;
    r.nib2 = nib2;
    r.d0 = 3.0f + 2.0f * ad;
    r.jd0 = 2.0f * ad * bk0;
    r.jd1 = 2.0f * ad * bk1;
    r.win = win;
  } else {
    RecF32& r = so->rec;
    r.jl = jl;
    r.al = al;
    r.v = v;
    r.nib2 = nib2;
    r.ad = ad;
    r.emD = -expm1f(-ad);
    r.bk0 = bk0;
    r.bk1 = bk1;
    r.win = win;
  }
  so->lo = win_lo(win);
  so->hi = win_hi(win);
  so->ad = ad;
}

template <int MODE>
__device__ __forceinline__ void make_record(const PhysParams& P, const double raw[5], double h,
                                            double, double, int, int nfw,
                                            SampleOut<double, MODE>* so) {
  const double n = raw[0], T = raw[1], Td = raw[2], v = raw[3], x = raw[4];
  double jl, al, b;
  line_coeffs<double>(P, n, T, x, h, &jl, &al, &b);
  RecD& r = so->rec;
  r.jl = jl;
  r.al = al;
  r.v = v;
  r.nib2 = (jl != 0.0 || al != 0.0) ? -1.0 / (b * b) : -1.0;
  r.ad = P.cad * n * h;
  r.emD = -expm1(-r.ad);
  r.td = Td;
  // the double path evaluates the line at every fine velocity
  r.win = pack_win(0, (nfw - 1) >> 5);
  so->lo = 0;
  so->hi = (nfw - 1) >> 5;
  so->ad = r.ad;
}

// ---------------------------------------------------------------------------
// per-(sample, fine velocity) coefficients of the total intensity
// ---------------------------------------------------------------------------
// smooth: jt = 2 h j_total, d = 3 + 2 h alpha_total
__device__ __forceinline__ void coeff_line(const RecS32& r, float u, float* jt, float* d) {
  const float dd = u - r.v;
  const float g = ex2_approx(dd * r.nib2 * dd);
  *jt = fmaf(r.jl2, g, fmaf(r.jd1, u, r.jd0));
  *d = fmaf(r.al2, g, r.d0);
}
// formal: per-step emission jt and optical depth tau
__device__ __forceinline__ void coeff_line(const RecF32& r, float u, float* jt, float* tau) {
  const float dd = u - r.v;
  const float g = ex2_approx(dd * r.nib2 * dd);
  *jt = fmaf(r.jl, g, r.ad * fmaf(r.bk1, u, r.bk0));
  *tau = fmaf(r.al, g, r.ad);
}

// (1 - exp(-tau)) / tau, well conditioned for all tau (own expansion below
// |tau| = 1/4: the Taylor series of the function truncated after tau^6, error
// below 2e-9 relative; above, 1 - 2^(-tau log2 e) loses at most 4 ulp).
__device__ __forceinline__ float psi_f(float tau) {
  const float t = tau;
  const float p = fmaf(t, fmaf(t, fmaf(t, fmaf(t, fmaf(t, fmaf(t, 1.0f / 5040.0f, -1.0f / 720.0f),
                                                              1.0f / 120.0f),
                                                    -1.0f / 24.0f),
                                           1.0f / 6.0f),
                                  -0.5f),
                       1.0f);
  const float q = (1.0f - ex2_approx(-tau * kLog2e)) * rcp_approx(tau);
  return (fabsf(tau) < 0.25f) ? p : q;
}
__device__ __forceinline__ double psi_d(double tau) {
  return (tau == 0.0) ? 1.0 : -expm1(-tau) / tau;
}

// ---------------------------------------------------------------------------
// the kernel
// ---------------------------------------------------------------------------
template <typename R, int NI, int ST, int MODE>
struct Fwd {
  using Rec = typename RecOf<R, MODE>::type;
  static constexpr bool kDouble = sizeof(R) == 8;

  // Total-intensity transfer of the hull blocks [hlo, hhi] (or, with
  // line == false, dust-only transfer of the blocks at velocities u[]).
  // On return s1[i] holds the final intensity of block i.
  template <bool LINE>
  static __device__ __forceinline__ void transfer(const PhysParams& P, const Rec* rec, int K,
                                                  const R* u, int hlo, int hhi, R* s0, R* s1,
                                                  R* s2) {
    if constexpr (MODE == M_SMOOTH) {
      if (K <= 1) {
#pragma unroll
        for (int i = 0; i < NI; ++i) s1[i] = s0[i];
        return;
      }
      // k = 0: s1 <- 2h j_0 + (7 - d_0) I_0   (numerator of the trapezoidal step)
      {
        const Rec r = rec[0];
#pragma unroll
        for (int i = 0; i < NI; ++i) {
          if (i < hlo || i > hhi) continue;
          R jt, d;
          coeffs<LINE>(P, r, i, u[i], &jt, &d);
          s1[i] = jt + ((R)7 - d) * s0[i];
        }
      }
      // k = 1: trapezoidal step I_1 = (2h (j_0 + j_1) + (4 - 2h a_0) I_0) / (1 + d_1)
      {
        const Rec r = rec[1];
#pragma unroll
        for (int i = 0; i < NI; ++i) {
          if (i < hlo || i > hhi) continue;
          R jt, d;
          coeffs<LINE>(P, r, i, u[i], &jt, &d);
          s1[i] = relu((s1[i] + jt) * recip((R)1 + d));
        }
      }
      // BDF2 steps, two per iteration with the state roles swapped
      int k = 2;
      for (; k + 1 < K; k += 2) {
        bdf2_step<LINE>(P, rec[k], u, hlo, hhi, s0, s1);      // s0 <- I_k
        bdf2_step<LINE>(P, rec[k + 1], u, hlo, hhi, s1, s0);  // s1 <- I_{k+1}
      }
      if (k < K) {
        bdf2_step<LINE>(P, rec[k], u, hlo, hhi, s0, s1);
#pragma unroll
        for (int i = 0; i < NI; ++i) s1[i] = s0[i];
      }
    } else if constexpr (MODE == M_FORMAL) {
      for (int k = 0; k < K; ++k) {
        const Rec r = rec[k];
#pragma unroll
        for (int i = 0; i < NI; ++i) {
          if (i < hlo || i > hhi) continue;
          s0[i] = formal_step<LINE>(P, r, i, u[i], s0[i]);
        }
      }
#pragma unroll
      for (int i = 0; i < NI; ++i) s1[i] = s0[i];
    } else {
      // front-to-back formal integration with Kahan-compensated optical depth:
      // s0 = accumulated intensity, s1 = tau to the observer, s2 = compensation;
      // on entry s0 holds the background, which is added last.
      R bg[NI];
#pragma unroll
      for (int i = 0; i < NI; ++i) {
        bg[i] = s0[i];
        s0[i] = (R)0;
        s1[i] = (R)0;
        s2[i] = (R)0;
      }
      for (int k = K - 1; k >= 0; --k) {
        const Rec r = rec[k];
#pragma unroll
        for (int i = 0; i < NI; ++i) {
          if (i < hlo || i > hhi) continue;
          R jt, tau;
          coeffs_formal<LINE>(P, r, i, u[i], &jt, &tau);
          s0[i] += jt * psi(tau) * expneg(s1[i]);
          // Kahan summation of tau
          const R y = tau - s2[i];
          const R t = s1[i] + y;
          s2[i] = (t - s1[i]) - y;
          s1[i] = t;
        }
      }
#pragma unroll
      for (int i = 0; i < NI; ++i) s1[i] = s0[i] + bg[i] * expneg(s1[i]);
    }
  }

  static __device__ __forceinline__ R relu(R x) { return x > (R)0 ? x : (R)0; }
  static __device__ __forceinline__ R recip(R x) {
    if constexpr (kDouble) return (R)1 / x; else return rcp_approx(x);
  }
  static __device__ __forceinline__ R psi(R tau) {
    if constexpr (kDouble) return psi_d(tau); else return psi_f(tau);
  }
  static __device__ __forceinline__ R expneg(R t) {
    if constexpr (kDouble) return exp(-t); else return ex2_approx(-t * kLog2e);
  }

  // smooth-mode coefficients (2h j, 3 + 2h alpha) of block i at velocity u
  template <bool LINE>
  static __device__ __forceinline__ void coeffs(const PhysParams& P, const Rec& r, int i, R u,
                                                R* jt, R* d) {
    if constexpr (kDouble) {
      const double bk = planck_k(P, r.td, u);
      const double two_ad = 2.0 * r.ad;
      if (LINE) {
        const double dd = u - r.v;
        const double g = exp(dd * dd * r.nib2);
        *jt = 2.0 * r.jl * g + two_ad * bk;
        *d = 3.0 + 2.0 * r.al * g + two_ad;
      } else {
        *jt = two_ad * bk;
        *d = 3.0 + two_ad;
      }
    } else {
      if (LINE && i >= win_lo(r.win) && i <= win_hi(r.win)) {
        coeff_line(r, u, jt, d);
      } else {
        *jt = fmaf(r.jd1, u, r.jd0);
        *d = r.d0;
      }
    }
  }

  template <bool LINE>
  static __device__ __forceinline__ void bdf2_step(const PhysParams& P, const Rec& r, const R* u,
                                                   int hlo, int hhi, R* sa, const R* sb) {
    // sa holds I_{n}, sb holds I_{n+1}; sa <- I_{n+2}
    R rd0 = (R)0;
    if constexpr (!kDouble) rd0 = recip(r.d0);
#pragma unroll
    for (int i = 0; i < NI; ++i) {
      if (i < hlo || i > hhi) continue;
      R jt, d, rd;
      if constexpr (kDouble) {
        coeffs<LINE>(P, r, i, u[i], &jt, &d);
        rd = (R)1 / d;
      } else {
        if (LINE && i >= win_lo(r.win) && i <= win_hi(r.win)) {
          coeff_line(r, u[i], &jt, &d);
          rd = recip(d);
        } else {
          jt = fmaf(r.jd1, u[i], r.jd0);
          rd = rd0;
        }
      }
      sa[i] = relu(fma((R)4, sb[i], jt - sa[i]) * rd);
    }
  }

  // formal-mode per-step emission and optical depth of block i
  template <bool LINE>
  static __device__ __forceinline__ void coeffs_formal(const PhysParams& P, const Rec& r, int i,
                                                       R u, R* jt, R* tau) {
    if constexpr (kDouble) {
      const double bk = planck_k(P, r.td, u);
      if (LINE) {
        const double dd = u - r.v;
        const double g = exp(dd * dd * r.nib2);
        *jt = r.jl * g + r.ad * bk;
        *tau = r.al * g + r.ad;
      } else {
        *jt = r.ad * bk;
        *tau = r.ad;
      }
    } else {
      if (LINE && i >= win_lo(r.win) && i <= win_hi(r.win)) {
        coeff_line(r, u, jt, tau);
      } else {
        *jt = r.ad * fmaf(r.bk1, u, r.bk0);
        *tau = r.ad;
      }
    }
  }

  template <bool LINE>
  static __device__ __forceinline__ R formal_step(const PhysParams& P, const Rec& r, int i, R u,
                                                  R I) {
    if constexpr (kDouble) {
      R jt, tau;
      coeffs_formal<LINE>(P, r, i, u, &jt, &tau);
      return I + (jt - tau * I) * psi_d(tau);
    } else {
      if (LINE && i >= win_lo(r.win) && i <= win_hi(r.win)) {
        float jt, tau;
        coeff_line(r, u, &jt, &tau);
        return fmaf(fmaf(-tau, I, jt), psi_f(tau), I);
      }
      // dust only: I <- I + (S - I)(1 - e^{-tau_D})
      return fmaf(fmaf(r.bk1, u, r.bk0) - I, r.emD, I);
    }
  }

  // Continuum basis recurrences (float path): lane 0 -> X0 (unit background,
  // no source), lane 1 -> X1 (source coefficient 0), lane 2 -> X2 (source
  // coefficient 1); other lanes run a zero recurrence.  Returns the final X.
  static __device__ __forceinline__ float basis(const Rec* rec, int K, int lane) {
    const float m0 = (lane == 0) ? 1.0f : 0.0f;
    const float m1 = (lane == 1) ? 1.0f : 0.0f;
    const float m2 = (lane == 2) ? 1.0f : 0.0f;
    if constexpr (MODE == M_SMOOTH) {
      // the basis states may be negative (X2); the ReLU never acts on their
      // combination (see the header), so they are not clamped
      float x0 = m0;  // I_0
      if (K <= 1) return x0;
      const RecS32& r0 = rec[0];
      const RecS32& r1 = rec[1];
      const float j0 = fmaf(m2, r0.jd1, m1 * r0.jd0);
      const float j1 = fmaf(m2, r1.jd1, m1 * r1.jd0);
      float x1 = (j0 + (7.0f - r0.d0) * x0 + j1) * rcp_approx(1.0f + r1.d0);
      for (int k = 2; k < K; ++k) {
        const RecS32& r = rec[k];
        const float jt = fmaf(m2, r.jd1, m1 * r.jd0);
        const float x2 = fmaf(4.0f, x1, jt - x0) * rcp_approx(r.d0);
        x0 = x1;
        x1 = x2;
      }
      return x1;
    } else if constexpr (MODE == M_FORMAL) {
      float x = m0;
      for (int k = 0; k < K; ++k) {
        const RecF32& r = rec[k];
        const float s = fmaf(m2, r.bk1, m1 * r.bk0);
        x = fmaf(s - x, r.emD, x);
      }
      return x;
    } else {
      // front-to-back with Kahan-compensated dust optical depth
      float acc = 0.0f, T = 0.0f, c = 0.0f;
      for (int k = K - 1; k >= 0; --k) {
        const RecF32& r = rec[k];
        const float s = fmaf(m2, r.bk1, m1 * r.bk0);
        acc = fmaf(s * r.emD, ex2_approx(-T * kLog2e), acc);
        const float y = r.ad - c;
        const float t = T + y;
        c = (t - T) - y;
        T = t;
      }
      return acc + m0 * ex2_approx(-T * kLog2e);
    }
  }
};

template <typename R>
__device__ __forceinline__ R bg_intensity(const PhysParams& P, R u) {
  return planck_k(P, (R)P.t_bg, u);
}

// One work item: ray (px, py) of job J, channel window `win`.
template <typename R, int NI, int ST, int MODE>
__device__ void render_item(const JobDev& J, const PhysParams& P, int px, int py, int win,
                            unsigned char* wsm, int fw_off, int cw_off, int lane,
                            unsigned flags, unsigned long long* stats) {
  using F = Fwd<R, NI, ST, MODE>;
  using Rec = typename F::Rec;
  Rec* rec = reinterpret_cast<Rec*>(wsm);
  R* fbuf = reinterpret_cast<R*>(wsm + fw_off);
  R* cbuf = reinterpret_cast<R*>(wsm + cw_off);

  // ---- window geometry
  const int c0 = win * J.cw;
  const int cwn = min(J.cw, J.nchan - c0);
  const int f = J.f;
  const int gw0 = (f >= 1) ? 2 * f * c0 : c0;
  const int nfw = (f >= 1) ? 2 * f * cwn + 1 : cwn;
  const R ufirst = (R)J.ufirst, dvf = (R)J.dvf;

  R u[NI];
#pragma unroll
  for (int i = 0; i < NI; ++i) {
    const int g = min(lane + 32 * i, nfw - 1);
    u[i] = (R)(J.ufirst + (double)(gw0 + g) * J.dvf);
  }

  // ---- sample pass
  const RayGeom geo = ray_geom(J, px, py);
  const int K = geo.K;
  const R h = (R)geo.h;
  int hlo = 1 << 20, hhi = -1;
  R admax = (R)0;
  for (int k0 = 0; k0 < K; k0 += 32) {
    const int k = k0 + lane;
    if (k < K) {
      R raw[5];
      sample_raw<R, ST>(J, geo, px, py, k, raw);
      SampleOut<R, MODE> so;
      make_record<MODE>(P, raw, h, ufirst, dvf, gw0, nfw, &so);
      rec[k] = so.rec;
      if (so.lo <= so.hi) {
        hlo = min(hlo, so.lo);
        hhi = max(hhi, so.hi);
      }
      admax = fmax(admax, so.ad);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    hlo = min(hlo, __shfl_xor_sync(0xffffffffu, hlo, o));
    hhi = max(hhi, __shfl_xor_sync(0xffffffffu, hhi, o));
    admax = fmax(admax, __shfl_xor_sync(0xffffffffu, admax, o));
  }
  __syncwarp();

  const int nblk = (nfw + 31) >> 5;
  const bool explicit_all = F::kDouble || (flags & IRT_FLAG_EXPLICIT_CHANNELS) ||
                            (MODE == M_SMOOTH && admax > (R)0.5);
  if (explicit_all) {
    hlo = 0;
    hhi = nblk - 1;
  }
  if (stats) {
    // work counters: line-reached (sample, block) pairs from the records
    unsigned long long nline = 0;
    for (int k = lane; k < K; k += 32) {
      const int w = rec[k].win;
      const int lo = win_lo(w), hi = win_hi(w);
      if (lo <= hi) nline += (unsigned long long)(hi - lo + 1);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) nline += __shfl_xor_sync(0xffffffffu, nline, o);
    if (lane == 0) {
      const unsigned long long nh = (hhi >= hlo) ? (unsigned long long)(hhi - hlo + 1) : 0ull;
      atomicAdd(stats + 0, 1ull);
      atomicAdd(stats + 1, (unsigned long long)K);
      atomicAdd(stats + 2, nline);
      atomicAdd(stats + 3, nh * (unsigned long long)K);
      atomicAdd(stats + 4, explicit_all ? 1ull : 0ull);
      atomicAdd(stats + 5, (unsigned long long)K * (unsigned long long)nfw);
    }
  }

  // ---- total intensity on the blocks the line reaches
  R s0[NI], s1[NI], s2[NI];
#pragma unroll
  for (int i = 0; i < NI; ++i) {
    s0[i] = (i >= hlo && i <= hhi) ? bg_intensity<R>(P, u[i]) : (R)0;
    s1[i] = (R)0;
    s2[i] = (R)0;
  }
  F::template transfer<true>(P, rec, K, u, hlo, hhi, s0, s1, s2);

  // ---- continuum basis (float path, shortcut allowed)
  R X0 = (R)0, X1 = (R)0, X2 = (R)0;
  if constexpr (!F::kDouble) {
    if (!explicit_all) {
      const float xb = F::basis(rec, K, lane);
      X0 = __shfl_sync(0xffffffffu, xb, 0);
      X1 = __shfl_sync(0xffffffffu, xb, 1);
      X2 = __shfl_sync(0xffffffffu, xb, 2);
    }
  }

  // fine intensities of the window -> shared memory
#pragma unroll
  for (int i = 0; i < NI; ++i) {
    const int g = lane + 32 * i;
    if (g < nfw) {
      R v;
      if (i >= hlo && i <= hhi) v = s1[i];
      else v = X0 * bg_intensity<R>(P, u[i]) + X1 + X2 * u[i];
      fbuf[g] = v;
    }
  }

  // ---- continuum at channel centres when every channel is explicit
  if (explicit_all) {
    R uc[NI];
    const int cblk = (cwn + 31) >> 5;
#pragma unroll
    for (int i = 0; i < NI; ++i) {
      const int c = min(lane + 32 * i, cwn - 1);
      uc[i] = (R)(J.v0 + ((double)(c0 + c) + 0.5) * J.dv);
      s0[i] = (i < cblk) ? bg_intensity<R>(P, uc[i]) : (R)0;
      s1[i] = (R)0;
      s2[i] = (R)0;
    }
    F::template transfer<false>(P, rec, K, uc, 0, cblk - 1, s0, s1, s2);
#pragma unroll
    for (int i = 0; i < NI; ++i) {
      const int c = lane + 32 * i;
      if (c < cwn) cbuf[c] = s1[i];
    }
  }
  __syncwarp();

  // ---- epilogue: channel values and the five components
  const long long plane = (long long)J.npx * J.npy;
  const long long pix = (long long)py * J.npx + px;
  for (int cl = lane; cl < cwn; cl += 32) {
    const int c = c0 + cl;
    const double ucd = J.v0 + ((double)c + 0.5) * J.dv;
    const R uc = (R)ucd;
    R ibar;
    if (f >= 1) {
      const R* F6 = fbuf + 2 * f * cl;
      R acc = F6[0] + F6[2 * f];
      for (int m = 1; m < 2 * f; m += 2) acc += (R)4 * F6[m];
      for (int m = 2; m < 2 * f; m += 2) acc += (R)2 * F6[m];
      ibar = acc / (R)(6 * f);
    } else {
      ibar = fbuf[cl];
    }
    const R ib = bg_intensity<R>(P, uc);
    const R ic = explicit_all ? cbuf[cl] : X0 * ib + X1 + X2 * uc;
    R s = (R)P.out_scale;
    if (P.units == IRT_UNITS_TRJ) {
      const R y = (R)1 - uc * (R)P.inv_c_kms;
      s = s / (y * y);
    }
    const R vT = ibar * s, vC = ic * s, vB = ib * s;
    const long long o = (long long)c * plane + pix;
    R* const* out = reinterpret_cast<R* const*>(J.out);
    if (out[0]) out[0][o] = vT;
    if (out[1]) out[1][o] = vC;
    if (out[2]) out[2][o] = vC - vB;
    if (out[3]) out[3][o] = vT - vC;
    if (out[4]) out[4][o] = vB;
  }
  __syncwarp();
}

template <typename R, int NI, int ST, int MODE>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
fwd_kernel(const __grid_constant__ JobTable tab, int njobs, const PhysParams P,
           long long total_items, unsigned long long* queue, int per_warp, int fw_off, int cw_off,
           unsigned flags, unsigned long long* stats) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  unsigned char* wsm = smem + (size_t)warp * per_warp;
  long long item;
  if (queue) {
    unsigned long long t = 0;
    if (lane == 0) t = atomicAdd(queue, 1ull);
    item = (long long)__shfl_sync(0xffffffffu, t, 0);
  } else {
    item = (long long)blockIdx.x * kWarpsPerBlock + warp;
  }
  while (item < total_items) {
    int j = 0;
    while (j + 1 < njobs && item >= tab.j[j + 1].item_begin) ++j;
    const JobDev& J = tab.j[j];
    const long long local = item - J.item_begin;
    const int win = (int)(local % J.nwin);
    const long long ray = local / J.nwin;
    const int px = (int)(ray % J.npx), py = (int)(ray / J.npx);
    if constexpr (ST == ST_F64 || sizeof(R) == 4) {
      render_item<R, NI, ST, MODE>(J, P, px, py, win, wsm, fw_off, cw_off, lane, flags, stats);
    }
    if (queue) {
      unsigned long long t = 0;
      if (lane == 0) t = atomicAdd(queue, 1ull);
      item = (long long)__shfl_sync(0xffffffffu, t, 0);
    } else {
      break;
    }
  }
}

}  // namespace dev

// Host-side launcher of one kernel instance.
template <typename R, int NI, int ST, int MODE>
int launch_fwd_inst(const JobTable& tab, int njobs, const PhysParams& P, long long total_items,
                    unsigned long long* queue, int grid_blocks, int kmax, int fwmax, int cwmax,
                    unsigned flags, unsigned long long* stats, cudaStream_t stream) {
  using Rec = typename dev::RecOf<R, MODE>::type;
  const int rec_bytes = (int)sizeof(Rec) * kmax;
  const int fw_off = (rec_bytes + 15) & ~15;
  const int cw_off = (fw_off + (int)sizeof(R) * fwmax + 15) & ~15;
  const int per_warp = (cw_off + (int)sizeof(R) * cwmax + 15) & ~15;
  const size_t smem = (size_t)per_warp * kWarpsPerBlock;
  auto kern = dev::fwd_kernel<R, NI, ST, MODE>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return (int)e;
  long long blocks = grid_blocks;
  if (!queue) {
    blocks = (total_items + kWarpsPerBlock - 1) / kWarpsPerBlock;
  } else if (blocks <= 0) {
    int per_sm = 0, sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kWarpsPerBlock * 32, smem);
    blocks = (long long)std::max(per_sm, 1) * sms;
  }
  if (blocks < 1) return 0;
  kern<<<(unsigned)blocks, kWarpsPerBlock * 32, smem, stream>>>(tab, njobs, P, total_items,
                                                                 queue, per_warp, fw_off, cw_off,
                                                                 flags, stats);
  return (int)cudaGetLastError();
}

}  // namespace irt

// Kernel template of the forward render (see irt_forward.cuh for the design).
#pragma once

#include <algorithm>
#include <cstring>
#include <type_traits>

#include "irt_forward.cuh"

namespace irt {
namespace dev {

// ---------------------------------------------------------------------------
// sample pass: record of one sample; returns h alpha_D of the sample
// ---------------------------------------------------------------------------
template <int MODE, bool OTC = true>
__device__ __forceinline__ float make_record(const PhysF& P, const float raw[6], float h,
                                             const VGrid& G, int nfw,
                                             typename RecOf<float, MODE>::type* out) {
  const float n = raw[0], T = raw[1], Td = raw[2], v = raw[3], x = raw[4];
  float jl, al, b;
  line_coeffs<OTC>(P, n, T, x, raw[5], h, &jl, &al, &b);
  const float ad = P.cad * n * h;
  float bk0, bk1;
  dust_source_lin(P, Td, &bk0, &bk1);
  const bool has_line = jl != 0.0f || al != 0.0f;
  // no line: any finite profile parameter (the coefficients are zero)
  const float nib2 = has_line ? -kLog2e / (b * b) : -kLog2e;
  const int win = line_window(v, b, G.ufw_hi, G.dvf_hi, 0, nfw, has_line);
  int gv;
  float vr;
  centre_offset(G, v, &gv, &vr);
  if constexpr (MODE == M_SMOOTH) {
    RecS32 r;
    r.jl2 = 2.0f * jl;
    r.al2 = 2.0f * al;
    r.vr = vr;
    r.gv = gv;
    r.pad[0] = r.pad[1] = r.pad[2] = 0.0f;
    r.nib2 = nib2;
    r.d0 = 3.0f + 2.0f * ad;
    r.jd0 = 2.0f * ad * bk0;
    r.jd1 = 2.0f * ad * bk1;
    r.win = win;
    *out = r;
  } else {
    RecF32 r;
    r.jl = jl;
    r.al = al;
    r.vr = vr;
    r.gv = gv;
    r.nib2 = nib2;
    r.ad = ad;
    r.emD = -expm1f(-ad);
    r.bk0 = bk0;
    r.bk1 = bk1;
    r.win = win;
    r.pad[0] = r.pad[1] = 0.0f;
    *out = r;
  }
  return ad;
}

template <int MODE, bool OTC = true>
__device__ __forceinline__ double make_record(const PhysParams& P, const double raw[6], double h,
                                              int nfw, RecD* out) {
  const double n = raw[0], T = raw[1], Td = raw[2], v = raw[3], x = raw[4];
  double jl, al, b;
  line_coeffs<OTC>(P, n, T, x, raw[5], h, &jl, &al, &b);
  RecD r;
  r.jl = jl;
  r.al = al;
  r.v = v;
  r.nib2 = (jl != 0.0 || al != 0.0) ? -1.0 / (b * b) : -1.0;
  r.ad = P.cad * n * h;
  r.emD = -expm1(-r.ad);
  r.td = Td;
  // the double path evaluates the line at every fine velocity
  r.win = pack_win(0, nfw - 1);
  r.pad = 0;
  *out = r;
  return r.ad;
}

// Per-sample records of one ray.  The sample pass writes them to this warp's
// slot of a global scratch buffer (it stays in L2); the transfer passes stream
// them back 32 at a time into a two-chunk ring in shared memory with cp.async,
// the next chunk in flight while the current one is integrated.  Lane l copies
// record k0 + l, the record it wrote itself in the sample pass.
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;" ::: "memory");
}

template <typename Rec>
struct RecStream {
  const Rec* grec;   // records 0..K-1 of this ray (global)
  Rec* ring;         // 2 x 32 records (shared)
  int K, lane;

  __device__ __forceinline__ void request(int k0) const {
    const int k = k0 + lane;
    if (k < K) {
      const unsigned char* src = reinterpret_cast<const unsigned char*>(grec + k);
      unsigned char* dst = reinterpret_cast<unsigned char*>(ring + ((k0 >> 5) & 1) * 32 + lane);
#pragma unroll
      for (int q = 0; q < (int)(sizeof(Rec) / 16); ++q) cp_async16(dst + 16 * q, src + 16 * q);
    }
    cp_async_commit();
  }
  // First chunk of a sweep (forward from 0, or backward from the last chunk).
  __device__ __forceinline__ void begin(int k0) const { request(k0); }
  // Waits for chunk k0 (requested by begin() or the previous call), requests
  // chunk kn (kn < 0: none) into the other half of the ring and returns the
  // half that holds chunk k0.
  __device__ __forceinline__ const Rec* take(int k0, int kn) const {
    cp_async_wait_all();
    __syncwarp();   // chunk k0 visible to every lane; the other half is free
    if (kn >= 0) request(kn);
    return ring + ((k0 >> 5) & 1) * 32;
  }
  __device__ __forceinline__ const Rec* take_fwd(int k0) const {
    return take(k0, (k0 + 32 < K) ? k0 + 32 : -1);
  }
  __device__ __forceinline__ const Rec* take_bwd(int k0) const {
    return take(k0, (k0 >= 32) ? k0 - 32 : -1);
  }
  static __device__ __forceinline__ int last_chunk(int K) { return ((K - 1) >> 5) << 5; }
};
static_assert(sizeof(RecS32) == kRecBytesF32 && sizeof(RecF32) == kRecBytesF32 &&
              sizeof(RecD) == kRecBytesF64, "record sizes");

// ---------------------------------------------------------------------------
// per-(sample, fine velocity) coefficients of the total intensity
// ---------------------------------------------------------------------------
// smooth: jt = 2 h j_total, d = 3 + 2 h alpha_total at local fine index gi
// (velocity u)
__device__ __forceinline__ void coeff_line(const RecS32& r, const VGrid& G, int gi, float u,
                                           float* jt, float* d) {
  const float dd = vel_offset(G, gi, r.gv, r.vr);
  const float g = ex2_approx(dd * r.nib2 * dd);
  *jt = fmaf(r.jl2, g, fmaf(r.jd1, u, r.jd0));
  *d = fmaf(r.al2, g, r.d0);
}
// formal: per-step emission jt and optical depth tau
__device__ __forceinline__ void coeff_line(const RecF32& r, const VGrid& G, int gi, float u,
                                           float* jt, float* tau) {
  const float dd = vel_offset(G, gi, r.gv, r.vr);
  const float g = ex2_approx(dd * r.nib2 * dd);
  *jt = fmaf(r.jl, g, r.ad * fmaf(r.bk1, u, r.bk0));
  *tau = fmaf(r.al, g, r.ad);
}

// 1/x from the hardware approximation refined by one Newton-Raphson step
// (r <- r + r (1 - x r)): about half an ulp instead of the approximation's one.
__device__ __forceinline__ float rcp_refined(float x) {
  const float r = rcp_approx(x);
  return fmaf(r, fmaf(-x, r, 1.0f), r);
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

// Is block i inside the fine-index window w?
__device__ __forceinline__ bool block_in_window(int i, int w) {
  const int lo = win_lo(w), hi = win_hi(w);
  return lo <= hi && i >= (lo >> 5) && i <= (hi >> 5);
}

// ---------------------------------------------------------------------------
// generic transfer (every precision and integrator): register blocks i < NI,
// uniform branches on the hull and on the sample's line window
// ---------------------------------------------------------------------------
template <typename R, int NI, int MODE>
struct Fwd {
  using Rec = typename RecOf<R, MODE>::type;
  static constexpr bool kDouble = sizeof(R) == 8;
  using PP = typename std::conditional<kDouble, PhysParams, PhysF>::type;

  // Total-intensity transfer of the hull blocks [hlo, hhi] (or, with
  // line == false, dust-only transfer of the blocks at velocities u[]).
  // Records come from `gen` in chunks of 32 samples.  lg = lane + 32 x the
  // global index of register block 0, so that register block i of this lane
  // holds the global fine velocity 32 i + lg (records carry global indices).
  // On return s1[i] holds the final intensity of block i.
  template <bool LINE, class Gen>
  static __device__ __forceinline__ void transfer(const PP& P, const VGrid& G, int lg,
                                                  const Gen& gen, int K, const R* u, int hlo,
                                                  int hhi, R* s0, R* s1, R* s2) {
    if constexpr (MODE == M_SMOOTH) {
      if (K <= 1) {
#pragma unroll
        for (int i = 0; i < NI; ++i) s1[i] = s0[i];
        return;
      }
      gen.begin(0);
      const Rec* ring = gen.take_fwd(0);
      // k = 0: s1 <- 2h j_0 + (7 - d_0) I_0   (numerator of the trapezoidal step)
      {
        const Rec r = ring[0];
#pragma unroll
        for (int i = 0; i < NI; ++i) {
          if (i < hlo || i > hhi) continue;
          R jt, d;
          coeffs<LINE>(P, G, lg, r, i, u[i], &jt, &d);
          s1[i] = jt + ((R)7 - d) * s0[i];
        }
      }
      // k = 1: trapezoidal step I_1 = (2h (j_0 + j_1) + (4 - 2h a_0) I_0) / (1 + d_1)
      {
        const Rec r = ring[1];
#pragma unroll
        for (int i = 0; i < NI; ++i) {
          if (i < hlo || i > hhi) continue;
          R jt, d;
          coeffs<LINE>(P, G, lg, r, i, u[i], &jt, &d);
          s1[i] = relu((s1[i] + jt) * recip((R)1 + d));
        }
      }
      // BDF2 steps, two per iteration with the state roles swapped (chunks
      // hold 32 samples, so every chunk but the last ends on an even step)
      int kk = 2, n = min(32, K);
      for (int k0 = 0;;) {
#pragma unroll 1
        for (; kk + 1 < n; kk += 2) {
          bdf2_step<LINE>(P, G, lg, ring[kk], u, hlo, hhi, s0, s1);      // s0 <- I_k
          bdf2_step<LINE>(P, G, lg, ring[kk + 1], u, hlo, hhi, s1, s0);  // s1 <- I_{k+1}
        }
        if (k0 + 32 >= K) break;
        k0 += 32;
        ring = gen.take_fwd(k0);
        kk = 0;
        n = min(32, K - k0);
      }
      if (kk < n) {
        bdf2_step<LINE>(P, G, lg, ring[kk], u, hlo, hhi, s0, s1);
#pragma unroll
        for (int i = 0; i < NI; ++i) s1[i] = s0[i];
      }
    } else if constexpr (MODE == M_FORMAL) {
      if (K > 0) gen.begin(0);
      for (int k0 = 0; k0 < K; k0 += 32) {
        const Rec* ring = gen.take_fwd(k0);
        const int n = min(32, K - k0);
#pragma unroll 1
        for (int kk = 0; kk < n; ++kk) {
          const Rec r = ring[kk];
#pragma unroll
          for (int i = 0; i < NI; ++i) {
            if (i < hlo || i > hhi) continue;
            s0[i] = formal_step<LINE>(P, G, lg, r, i, u[i], s0[i]);
          }
        }
      }
#pragma unroll
      for (int i = 0; i < NI; ++i) s1[i] = s0[i];
    } else {
      // front-to-back formal integration with Kahan-compensated optical depth:
      // s0 = accumulated intensity, s1 = tau to the observer, s2 = compensation;
      // the background (s0 on entry) is re-evaluated and added last.
#pragma unroll
      for (int i = 0; i < NI; ++i) {
        s0[i] = (R)0;
        s1[i] = (R)0;
        s2[i] = (R)0;
      }
      if (K > 0) gen.begin(Gen::last_chunk(K));
      for (int k0 = Gen::last_chunk(K); k0 >= 0; k0 -= 32) {
        const Rec* ring = gen.take_bwd(k0);
        const int n = min(32, K - k0);
#pragma unroll 1
        for (int kk = n - 1; kk >= 0; --kk) {
          const Rec r = ring[kk];
#pragma unroll
          for (int i = 0; i < NI; ++i) {
            if (i < hlo || i > hhi) continue;
            R jt, tau;
            coeffs_formal<LINE>(P, G, lg, r, i, u[i], &jt, &tau);
            s0[i] += jt * psi(tau) * expneg(s1[i]);
            // Kahan summation of tau
            const R y = tau - s2[i];
            const R t = s1[i] + y;
            s2[i] = (t - s1[i]) - y;
            s1[i] = t;
          }
        }
      }
#pragma unroll
      for (int i = 0; i < NI; ++i) {
        const R bg = (i >= hlo && i <= hhi) ? planck_k(P, (R)P.t_bg, u[i]) : (R)0;
        s1[i] = s0[i] + bg * expneg(s1[i]);
      }
    }
  }

  static __device__ __forceinline__ R relu(R x) { return x > (R)0 ? x : (R)0; }
  static __device__ __forceinline__ R recip(R x) {
    if constexpr (kDouble) return (R)1 / x; else return rcp_refined(x);
  }
  static __device__ __forceinline__ R psi(R tau) {
    if constexpr (kDouble) return psi_d(tau); else return psi_f(tau);
  }
  static __device__ __forceinline__ R expneg(R t) {
    if constexpr (kDouble) return exp(-t); else return ex2_approx(-t * kLog2e);
  }

  // smooth-mode coefficients (2h j, 3 + 2h alpha) of block i at velocity u
  template <bool LINE>
  static __device__ __forceinline__ void coeffs(const PP& P, const VGrid& G, int lg,
                                                const Rec& r, int i, R u, R* jt, R* d) {
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
      if (LINE && block_in_window(i + (lg >> 5), r.win)) {
        coeff_line(r, G, 32 * i + lg, u, jt, d);
      } else {
        *jt = fmaf(r.jd1, u, r.jd0);
        *d = r.d0;
      }
    }
  }

  template <bool LINE>
  static __device__ __forceinline__ void bdf2_step(const PP& P, const VGrid& G, int lg,
                                                   const Rec& r, const R* u, int hlo, int hhi,
                                                   R* sa, const R* sb) {
    // sa holds I_{n}, sb holds I_{n+1}; sa <- I_{n+2}
    R rd0 = (R)0;
    if constexpr (!kDouble) rd0 = recip(r.d0);
#pragma unroll
    for (int i = 0; i < NI; ++i) {
      if (i < hlo || i > hhi) continue;
      R jt, d, rd;
      if constexpr (kDouble) {
        coeffs<LINE>(P, G, lg, r, i, u[i], &jt, &d);
        rd = (R)1 / d;
      } else {
        if (LINE && block_in_window(i + (lg >> 5), r.win)) {
          coeff_line(r, G, 32 * i + lg, u[i], &jt, &d);
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
  static __device__ __forceinline__ void coeffs_formal(const PP& P, const VGrid& G, int lg,
                                                       const Rec& r, int i, R u, R* jt, R* tau) {
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
      if (LINE && block_in_window(i + (lg >> 5), r.win)) {
        coeff_line(r, G, 32 * i + lg, u, jt, tau);
      } else {
        *jt = r.ad * fmaf(r.bk1, u, r.bk0);
        *tau = r.ad;
      }
    }
  }

  template <bool LINE>
  static __device__ __forceinline__ R formal_step(const PP& P, const VGrid& G, int lg,
                                                  const Rec& r, int i, R u, R I) {
    if constexpr (kDouble) {
      R jt, tau;
      coeffs_formal<LINE>(P, G, lg, r, i, u, &jt, &tau);
      return I + (jt - tau * I) * psi_d(tau);
    } else {
      if (LINE && block_in_window(i + (lg >> 5), r.win)) {
        float jt, tau;
        coeff_line(r, G, 32 * i + lg, u, &jt, &tau);
        return fmaf(fmaf(-tau, I, jt), psi_f(tau), I);
      }
      // dust only: I <- I + (S - I)(1 - e^{-tau_D})
      return fmaf(fmaf(r.bk1, u, r.bk0) - I, r.emD, I);
    }
  }

  // Continuum basis recurrences (float path): lane 0 -> X0 (unit background,
  // no source), lane 1 -> X1 (source coefficient 0), lane 2 -> X2 (source
  // coefficient 1); other lanes run a zero recurrence.  Returns the final X.
  template <class Gen>
  static __device__ __forceinline__ float basis(const Gen& gen, int K, int lane) {
    const float m0 = (lane == 0) ? 1.0f : 0.0f;
    const float m1 = (lane == 1) ? 1.0f : 0.0f;
    const float m2 = (lane == 2) ? 1.0f : 0.0f;
    if constexpr (MODE == M_SMOOTH) {
      // the basis states may be negative (X2); the ReLU never acts on their
      // combination (see the header), so they are not clamped
      float x0 = m0;  // I_0
      if (K <= 1) return x0;
      gen.begin(0);
      const RecS32* ring = gen.take_fwd(0);
      float x1;
      {
        const RecS32 r0 = ring[0];
        const RecS32 r1 = ring[1];
        const float j0 = fmaf(m2, r0.jd1, m1 * r0.jd0);
        const float j1 = fmaf(m2, r1.jd1, m1 * r1.jd0);
        x1 = (j0 + (7.0f - r0.d0) * x0 + j1) * rcp_refined(1.0f + r1.d0);
      }
      for (int k0 = 0; k0 < K; k0 += 32) {
        if (k0 > 0) ring = gen.take_fwd(k0);
        const int n = min(32, K - k0);
#pragma unroll 1
        for (int kk = (k0 == 0) ? 2 : 0; kk < n; ++kk) {
          const RecS32 r = ring[kk];
          const float jt = fmaf(m2, r.jd1, m1 * r.jd0);
          const float x2 = fmaf(4.0f, x1, jt - x0) * rcp_refined(r.d0);
          x0 = x1;
          x1 = x2;
        }
      }
      return x1;
    } else if constexpr (MODE == M_FORMAL) {
      float x = m0;
      if (K > 0) gen.begin(0);
      for (int k0 = 0; k0 < K; k0 += 32) {
        const RecF32* ring = gen.take_fwd(k0);
        const int n = min(32, K - k0);
#pragma unroll 1
        for (int kk = 0; kk < n; ++kk) {
          const RecF32 r = ring[kk];
          const float s = fmaf(m2, r.bk1, m1 * r.bk0);
          x = fmaf(s - x, r.emD, x);
        }
      }
      return x;
    } else {
      // front-to-back with Kahan-compensated dust optical depth
      float acc = 0.0f, T = 0.0f, c = 0.0f;
      if (K > 0) gen.begin(Gen::last_chunk(K));
      for (int k0 = Gen::last_chunk(K); k0 >= 0; k0 -= 32) {
        const RecF32* ring = gen.take_bwd(k0);
        const int n = min(32, K - k0);
#pragma unroll 1
        for (int kk = n - 1; kk >= 0; --kk) {
          const RecF32 r = ring[kk];
          const float s = fmaf(m2, r.bk1, m1 * r.bk0);
          acc = fmaf(s * r.emD, ex2_approx(-T * kLog2e), acc);
          const float y = r.ad - c;
          const float t = T + y;
          c = (t - T) - y;
          T = t;
        }
      }
      return (lane == 0) ? ex2_approx(-T * kLog2e) : acc;
    }
  }
};

// ---------------------------------------------------------------------------
// branch-free transfer of NA consecutive fine blocks starting at block hb
// (float path, smooth and formal integration).  With strided velocities a
// line window of at most 32 fine velocities holds exactly one velocity of
// each lane, so each lane evaluates its NS <= 2 line velocities once per
// sample ("line slots") and applies them to the matching block with
// predicated selects; the other blocks take the dust-only update.  The three
// continuum basis recurrences ride along (lanes 0, 1, 2).
// ---------------------------------------------------------------------------
template <int NS>
struct Slots {
  int j[NS];      // block of the slot relative to hb, -1 = no line velocity
  float a[NS];    // smooth: 2h j_line;     formal: per-step emission
  float b[NS];    // smooth: 3 + 2h alpha;  formal: optical depth
  float e[NS];    // profile factor exp(-(u - v)^2 / b^2)
  float dv[NS];   // u - v_los
};

template <int NS>
__device__ __forceinline__ Slots<NS> slots_smooth(const RecS32& r, int hb, int lane,
                                                  const VGrid& G) {
  Slots<NS> s;
  const int glo = win_lo(r.win), ghi = win_hi(r.win);
  const int g0 = glo + ((lane - glo) & 31);
#pragma unroll
  for (int q = 0; q < NS; ++q) {
    const int g = g0 + 32 * q;
    const float dd = vel_offset(G, g, r.gv, r.vr);
    const float e = ex2_approx(dd * r.nib2 * dd);
    s.j[q] = (g <= ghi) ? (g >> 5) - hb : -1;
    s.a[q] = r.jl2 * e;
    s.b[q] = fmaf(r.al2, e, r.d0);
    s.e[q] = e;
    s.dv[q] = dd;
  }
  return s;
}

template <int NS>
__device__ __forceinline__ Slots<NS> slots_formal(const RecF32& r, int hb, int lane,
                                                  const VGrid& G) {
  Slots<NS> s;
  const int glo = win_lo(r.win), ghi = win_hi(r.win);
  const int g0 = glo + ((lane - glo) & 31);
#pragma unroll
  for (int q = 0; q < NS; ++q) {
    const int g = g0 + 32 * q;
    const float ug = fmaf((float)g, G.dvf_hi, G.ufw_hi);
    const float dd = vel_offset(G, g, r.gv, r.vr);
    const float e = ex2_approx(dd * r.nib2 * dd);
    s.j[q] = (g <= ghi) ? (g >> 5) - hb : -1;
    s.a[q] = fmaf(r.jl, e, r.ad * fmaf(r.bk1, ug, r.bk0));
    s.b[q] = fmaf(r.al, e, r.ad);
    s.e[q] = e;
    s.dv[q] = dd;
  }
  return s;
}

template <int NA, int NS>
struct FastSmooth {
  // BDF2 step: sa <- I_{n+2} from sa = I_n, sb = I_{n+1}
  static __device__ __forceinline__ void step(const RecS32& r, const float (&u)[NA],
                                              float (&sa)[NA], const float (&sb)[NA], int hb,
                                              int lane, const VGrid& G, float& xa, float xb,
                                              float m1, float m2) {
    const Slots<NS> sl = slots_smooth<NS>(r, hb, lane, G);
    const float rd0 = rcp_refined(r.d0);
    float rl[NS];
#pragma unroll
    for (int q = 0; q < NS; ++q) rl[q] = rcp_refined(sl.b[q]);
#pragma unroll
    for (int j = 0; j < NA; ++j) {
      float t = fmaf(r.jd1, u[j], r.jd0) - sa[j];
      float rr = rd0;
#pragma unroll
      for (int q = 0; q < NS; ++q) {
        const bool p = sl.j[q] == j;
        t = p ? t + sl.a[q] : t;
        rr = p ? rl[q] : rr;
      }
      sa[j] = fmaxf(fmaf(4.0f, sb[j], t) * rr, 0.0f);
    }
    const float jb = fmaf(m2, r.jd1, m1 * r.jd0);
    xa = fmaf(4.0f, xb, jb - xa) * rd0;
  }

  // Runs the whole ray; writes the fine intensities of its blocks to fbuf
  // (hull-relative: fbuf[32 j + lane]) and returns this lane's basis value.
  // ck (optional): this ray's checkpoint slot; after every full 32-sample
  // chunk the state pair (I_{32s-2}, I_{32s-1}) of the hull blocks and the
  // lane's basis pair go to segment s (the adjoint's layout, ck_nb rows)
  template <bool CK, class Gen>
  static __device__ __forceinline__ float run(const PhysF& P, const Gen& gen, int K, int hb,
                                              int lane, const VGrid& G, int nfw, float* fbuf,
                                              float* ck, int ck_nb) {
    float u[NA], s0[NA], s1[NA];
#pragma unroll
    for (int j = 0; j < NA; ++j) {
      const int g = min(32 * (hb + j) + lane, nfw - 1);
      u[j] = fmaf((float)g, G.dvf_hi, G.ufw_hi);
      s0[j] = planck_k(P, P.t_bg, u[j]);
      s1[j] = s0[j];
    }
    const float m0 = (lane == 0) ? 1.0f : 0.0f;
    const float m1 = (lane == 1) ? 1.0f : 0.0f;
    const float m2 = (lane == 2) ? 1.0f : 0.0f;
    float x0 = m0, x1 = m0;
    if (K >= 2) {
      gen.begin(0);
      const RecS32* ring = gen.take_fwd(0);
      // k = 0: s1 <- 2h j_0 + (7 - d_0) I_0
      {
        const RecS32 r = ring[0];
        const Slots<NS> sl = slots_smooth<NS>(r, hb, lane, G);
#pragma unroll
        for (int j = 0; j < NA; ++j) {
          float t = fmaf(r.jd1, u[j], r.jd0);
          float d = r.d0;
#pragma unroll
          for (int q = 0; q < NS; ++q) {
            const bool p = sl.j[q] == j;
            t = p ? t + sl.a[q] : t;
            d = p ? sl.b[q] : d;
          }
          s1[j] = t + (7.0f - d) * s0[j];
        }
        x1 = fmaf(m2, r.jd1, m1 * r.jd0) + (7.0f - r.d0) * x0;
      }
      // k = 1: trapezoidal step
      {
        const RecS32 r = ring[1];
        const Slots<NS> sl = slots_smooth<NS>(r, hb, lane, G);
        const float r1 = rcp_refined(1.0f + r.d0);
        float rl[NS];
#pragma unroll
        for (int q = 0; q < NS; ++q) rl[q] = rcp_refined(1.0f + sl.b[q]);
#pragma unroll
        for (int j = 0; j < NA; ++j) {
          float t = fmaf(r.jd1, u[j], r.jd0);
          float rr = r1;
#pragma unroll
          for (int q = 0; q < NS; ++q) {
            const bool p = sl.j[q] == j;
            t = p ? t + sl.a[q] : t;
            rr = p ? rl[q] : rr;
          }
          s1[j] = fmaxf((s1[j] + t) * rr, 0.0f);
        }
        x1 = (x1 + fmaf(m2, r.jd1, m1 * r.jd0)) * r1;
      }
      // BDF2 pairs; every chunk but the last holds an even number of steps
      int kk = 2, n = min(32, K);
      for (int k0 = 0;;) {
#pragma unroll 1
        for (; kk + 1 < n; kk += 2) {
          step(ring[kk], u, s0, s1, hb, lane, G, x0, x1, m1, m2);
          step(ring[kk + 1], u, s1, s0, hb, lane, G, x1, x0, m1, m2);
        }
        if (k0 + 32 >= K) break;
        if (CK && NA < kCkRows && ck) {
          float* c = ck + (long long)((k0 + 32) >> 5) * 2 * ck_nb * 32;
#pragma unroll
          for (int j = 0; j < NA; ++j) {
            c[j * 32 + lane] = s0[j];
            c[ck_nb * 32 + j * 32 + lane] = s1[j];
          }
          c[NA * 32 + lane] = x0;
          c[ck_nb * 32 + NA * 32 + lane] = x1;
        }
        k0 += 32;
        ring = gen.take_fwd(k0);
        kk = 0;
        n = min(32, K - k0);
      }
      if (kk < n) {
        step(ring[kk], u, s0, s1, hb, lane, G, x0, x1, m1, m2);
#pragma unroll
        for (int j = 0; j < NA; ++j) s1[j] = s0[j];
        x1 = x0;
      }
    }
#pragma unroll
    for (int j = 0; j < NA; ++j) {
      const int g = 32 * (hb + j) + lane;
      if (g < nfw) fbuf[32 * j + lane] = s1[j];
    }
    return x1;
  }
};

template <int NA, int NS>
struct FastFormal {
  template <class Gen>
  static __device__ __forceinline__ float run(const PhysF& P, const Gen& gen, int K, int hb,
                                              int lane, const VGrid& G, int nfw, float* fbuf) {
    float u[NA], I[NA];
#pragma unroll
    for (int j = 0; j < NA; ++j) {
      const int g = min(32 * (hb + j) + lane, nfw - 1);
      u[j] = fmaf((float)g, G.dvf_hi, G.ufw_hi);
      I[j] = planck_k(P, P.t_bg, u[j]);
    }
    const float m1 = (lane == 1) ? 1.0f : 0.0f;
    const float m2 = (lane == 2) ? 1.0f : 0.0f;
    float x = (lane == 0) ? 1.0f : 0.0f;
    const RecF32* ring = nullptr;
    if (K > 0) gen.begin(0);
#pragma unroll 1
    for (int k = 0; k < K; ++k) {
      if ((k & 31) == 0) ring = gen.take_fwd(k);
      const RecF32 r = ring[k & 31];
      const Slots<NS> sl = slots_formal<NS>(r, hb, lane, G);
      float ps[NS];
#pragma unroll
      for (int q = 0; q < NS; ++q) ps[q] = psi_f(sl.b[q]);
#pragma unroll
      for (int j = 0; j < NA; ++j) {
        // dust: I + (S - I) emD;  line: I + (j - tau I) psi(tau)
        float A = fmaf(r.bk1, u[j], r.bk0) - I[j];
        float Bc = r.emD;
#pragma unroll
        for (int q = 0; q < NS; ++q) {
          const bool p = sl.j[q] == j;
          A = p ? fmaf(-sl.b[q], I[j], sl.a[q]) : A;
          Bc = p ? ps[q] : Bc;
        }
        I[j] = fmaf(A, Bc, I[j]);
      }
      const float s = fmaf(m2, r.bk1, m1 * r.bk0);
      x = fmaf(s - x, r.emD, x);
    }
#pragma unroll
    for (int j = 0; j < NA; ++j) {
      const int g = 32 * (hb + j) + lane;
      if (g < nfw) fbuf[32 * j + lane] = I[j];
    }
    return x;
  }
};

// Front-to-back formal transfer with Kahan-compensated optical depth.  The
// depth to the observer splits into the dust part T_D (frequency independent
// in the band: one compensated sum per ray, shared by every velocity) and the
// line part T_L(u) (one compensated sum per fine velocity, kept in shared
// memory `kb` and touched only on the samples whose line window reaches u).
// Registers hold the accumulated intensity and EL = exp(-T_L) per block, so a
// dust-only (sample, block) costs two FMAs; the line slots override the
// block's emission factor and its EL with predicated selects.
template <int NA, int NS>
struct FastKahan {
  static __device__ __forceinline__ void kahan_add(float& T, float& c, float x) {
    const float y = x - c;
    const float t = T + y;
    c = (t - T) - y;
    T = t;
  }

  template <class Gen>
  static __device__ __forceinline__ float run(const PhysF& P, const Gen& gen, int K, int hb,
                                              int lane, const VGrid& G, int nfw, float* fbuf,
                                              float* kb) {
    float acc[NA], EL[NA];
    float* TL = kb;             // [32 NA]: compensated line depth, index g - 32 hb
    float* CL = kb + 32 * NA;   // [32 NA]: its compensation
#pragma unroll
    for (int j = 0; j < NA; ++j) {
      acc[j] = 0.0f;
      EL[j] = 1.0f;
      TL[32 * j + lane] = 0.0f;
      CL[32 * j + lane] = 0.0f;
    }
    const float u0 = fmaf((float)(32 * hb + lane), G.dvf_hi, G.ufw_hi);
    const float du = 32.0f * G.dvf_hi;   // velocity step between a lane's blocks
    const float m1 = (lane == 1) ? 1.0f : 0.0f;
    const float m2 = (lane == 2) ? 1.0f : 0.0f;
    float TD = 0.0f, cD = 0.0f, ED = 1.0f, xb = 0.0f;
    const RecF32* ring = nullptr;
    if (K > 0) gen.begin(Gen::last_chunk(K));
#pragma unroll 1
    for (int k = K - 1; k >= 0; --k) {
      if (k == K - 1 || (k & 31) == 31) ring = gen.take_bwd(k & ~31);
      const RecF32 r = ring[k & 31];
      // line slots: emission factor and the updated EL of the slot's velocity
      const int glo = win_lo(r.win), ghi = win_hi(r.win);
      const int g0 = glo + ((lane - glo) & 31);
      int sj[NS];
      float sA[NS], sE[NS];
#pragma unroll
      for (int q = 0; q < NS; ++q) {
        const int g = g0 + 32 * q;
        const float ug = fmaf((float)g, G.dvf_hi, G.ufw_hi);
        const float dd = vel_offset(G, g, r.gv, r.vr);
        const float e = ex2_approx(dd * r.nib2 * dd);
        const float tl = r.al * e;
        const float a = fmaf(r.jl, e, r.ad * fmaf(r.bk1, ug, r.bk0));
        sA[q] = a * psi_f(tl + r.ad) * ED;
        sj[q] = -1;
        sE[q] = 1.0f;
        if (g <= ghi) {
          const int idx = g - 32 * hb;
          float T = TL[idx], c = CL[idx];
          kahan_add(T, c, tl);
          TL[idx] = T;
          CL[idx] = c;
          sj[q] = (g >> 5) - hb;
          sE[q] = ex2_approx(-T * kLog2e);
        }
      }
      // dust-only emission factor of block j: emD ED (bk0 + bk1 u_j)
      const float w = r.emD * ED;
      const float c0 = w * fmaf(r.bk1, u0, r.bk0);
      const float c1 = w * r.bk1 * du;
#pragma unroll
      for (int j = 0; j < NA; ++j) {
        float A = fmaf((float)j, c1, c0);
        float En = EL[j];
#pragma unroll
        for (int q = 0; q < NS; ++q) {
          const bool p = sj[q] == j;
          A = p ? sA[q] : A;
          En = p ? sE[q] : En;
        }
        acc[j] = fmaf(A, EL[j], acc[j]);
        EL[j] = En;
      }
      // continuum basis: lane 1 sums bk0 w, lane 2 sums bk1 w
      xb = fmaf(fmaf(m2, r.bk1, m1 * r.bk0), w, xb);
      kahan_add(TD, cD, r.ad);
      ED = ex2_approx(-TD * kLog2e);
    }
#pragma unroll
    for (int j = 0; j < NA; ++j) {
      const int g = 32 * (hb + j) + lane;
      const float u = fmaf((float)g, G.dvf_hi, G.ufw_hi);
      if (g < nfw) fbuf[32 * j + lane] = fmaf(planck_k(P, P.t_bg, u) * ED, EL[j], acc[j]);
    }
    return (lane == 0) ? ED : xb;
  }
};

// Block-count buckets of the fast path (a hull of na blocks runs in the
// smallest bucket >= na).
__host__ __device__ __forceinline__ constexpr int fast_bucket(int na, int ns) {
  if (ns == 1) {
    if (na <= 8) return (na + 1) & ~1;   // 2, 4, 6, 8
    if (na <= 10) return 10;
    if (na <= 12) return 12;
    if (na <= 14) return 14;
    if (na <= 17) return 17;
    if (na <= 20) return 20;
    if (na <= 24) return 24;
    if (na <= 28) return 28;
    return 33;
  }
  if (na <= 4) return 4;
  if (na <= 8) return 8;
  if (na <= 12) return 12;
  if (na <= 17) return 17;
  if (na <= 24) return 24;
  return 33;
}

// Runs the fast path for bucket `nb` (<= NI); returns false if nb is not
// compiled for this NI.
template <int NI, int MODE, int NS, bool CK, class Gen>
__device__ __forceinline__ bool run_fast(int nb, const PhysF& P, const Gen& gen, int K, int hb,
                                         int lane, const VGrid& G, int nfw, float* fbuf,
                                         float* kb, float* xb, float* ck, int ck_nb) {
#define IRT_FAST(NA_)                                                                        \
  case NA_:                                                                                  \
    if constexpr (NA_ <= NI) {                                                               \
      if constexpr (MODE == M_SMOOTH)                                                        \
        *xb = FastSmooth<NA_, NS>::template run<CK>(P, gen, K, hb, lane, G, nfw, fbuf, ck, ck_nb); \
      else if constexpr (MODE == M_FORMAL)                                                   \
        *xb = FastFormal<NA_, NS>::run(P, gen, K, hb, lane, G, nfw, fbuf);                  \
      else                                                                                   \
        *xb = FastKahan<NA_, NS>::run(P, gen, K, hb, lane, G, nfw, fbuf, kb);               \
      return true;                                                                           \
    }                                                                                        \
    return false;
  if constexpr (NS == 1) {
    switch (nb) {
      IRT_FAST(2) IRT_FAST(4) IRT_FAST(6) IRT_FAST(8) IRT_FAST(10) IRT_FAST(12) IRT_FAST(14)
      IRT_FAST(17) IRT_FAST(20) IRT_FAST(24) IRT_FAST(28) IRT_FAST(33)
      default: return false;
    }
  } else {
    switch (nb) {
      IRT_FAST(4) IRT_FAST(8) IRT_FAST(12) IRT_FAST(17) IRT_FAST(24) IRT_FAST(33)
      default: return false;
    }
  }
#undef IRT_FAST
}

template <bool D> struct PSel;
template <> struct PSel<true> {
  static __device__ __forceinline__ const PhysParams& get(const PhysParams& a, const PhysF&) {
    return a;
  }
};
template <> struct PSel<false> {
  static __device__ __forceinline__ const PhysF& get(const PhysParams&, const PhysF& b) {
    return b;
  }
};

// ---------------------------------------------------------------------------
// one work item: ray (px, py) of job J, every channel
// ---------------------------------------------------------------------------
// ML: one of several lines of the ray (line q); the first line samples the
// fields and keeps the raw samples in rawbuf, the others read them back.
template <typename R, int NI, int ST, int MODE, bool CK, bool OT, bool ML = false>
__device__ void render_ray(const JobDev& J, const PhysParams& PD, const PhysF& PF, int px,
                           int py, unsigned char* wsm, int fw_off, int cw_off, int kb_off,
                           typename RecOf<R, MODE>::type* grec, int lane, unsigned flags,
                           unsigned long long* stats, void* const* outp = nullptr,
                           float* rawbuf = nullptr, int q = 0) {
  using F = Fwd<R, NI, MODE>;
  using Rec = typename F::Rec;
  using Gen = RecStream<Rec>;
  constexpr bool kDouble = F::kDouble;
  const auto& P = PSel<kDouble>::get(PD, PF);
  R* fbuf = reinterpret_cast<R*>(wsm + fw_off);
  R* cbuf = reinterpret_cast<R*>(wsm + cw_off);

  // ---- the fine velocity grid of the whole axis: u(g) = J.ufirst + g J.dvf;
  // the records carry global fine indices, so one sample pass serves every
  // channel of the ray
  const int f = J.f;
  const int nch = J.nchan;
  const int nfw = (f >= 1) ? 2 * f * nch + 1 : nch;
  const int nblk = (nfw + 31) >> 5;
  VGrid G;
  G.ufw_hi = J.fufirst[0];
  G.ufw_lo = J.fufirst[1];
  G.dvf_hi = J.fdvf[0];
  G.dvf_lo = J.fdvf[1];
  // channel edges: double on the double kernels, the host's float roundings
  // on the float kernels
  const R v0r = kDouble ? (R)J.v0 : (R)J.fv0[0];
  const R dvr = kDouble ? (R)J.dv : (R)J.fdv[0];

  // ---- sample pass: lane l evaluates samples l, l + 32, ... into this warp's
  // record slot; the hull of the line windows, the widest window and the
  // largest dust step depth come along
  // ray set-up: double arithmetic on the double kernels, float-float on the
  // float kernels
  RayGeom geo;
  RayPos rp;
  int K;
  R h;
  if constexpr (kDouble) {
    geo = ray_geom(J, px, py);
    K = geo.K;
    h = (R)geo.h;
  } else {
    const RaySet rs = ray_setup(J, px, py);
    K = rs.K;
    h = rs.h;
    rp = rs.rp;
  }
  int hlo = 1 << 20, hhi = -1, wmax = 0;
  R admax = (R)0;
  unsigned long long nline = 0;
  for (int k0 = 0; k0 < K; k0 += 32) {
    const int k = k0 + lane;
    if (k < K) {
      R raw[6];
      Rec r;
      R ad;
      if constexpr (kDouble) {
        sample_raw<ST>(J, geo, px, py, k, raw);
        raw[5] = OT ? sample_chi<ST>(J, geo, px, py, k) : 0.5;
        ad = make_record<MODE, OT>(PD, raw, h, nfw, &r);
      } else if constexpr (ML) {
        // the z view's sample is one cell load: cheaper than the cache
        float* rb = rawbuf + 6 * k;
        if (q == 0 || J.zview) {
          sample_raw<ST>(J, rp, px, py, k, raw);
          raw[5] = PF.ot_tab ? sample_chi<ST>(J, rp, px, py, k) : 0.5f;
          if (!J.zview) {
#pragma unroll
            for (int i = 0; i < 6; ++i) rb[i] = raw[i];
          }
        } else {
#pragma unroll
          for (int i = 0; i < 6; ++i) raw[i] = rb[i];
        }
        ad = make_record<MODE, true>(PF, raw, h, G, nfw, &r);
      } else {
        sample_raw<ST>(J, rp, px, py, k, raw);
        raw[5] = OT ? sample_chi<ST>(J, rp, px, py, k) : 0.5f;
        ad = make_record<MODE, OT>(PF, raw, h, G, nfw, &r);
      }
      grec[k] = r;
      const int lo = win_lo(r.win), hi = win_hi(r.win);
      if (lo <= hi) {
        hlo = min(hlo, lo >> 5);
        hhi = max(hhi, hi >> 5);
        wmax = max(wmax, hi - lo + 1);
        nline += (unsigned long long)((hi >> 5) - (lo >> 5) + 1);
      }
      admax = fmax(admax, ad);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    hlo = min(hlo, __shfl_xor_sync(0xffffffffu, hlo, o));
    hhi = max(hhi, __shfl_xor_sync(0xffffffffu, hhi, o));
    wmax = max(wmax, __shfl_xor_sync(0xffffffffu, wmax, o));
    admax = fmax(admax, __shfl_xor_sync(0xffffffffu, admax, o));
  }
  // the records are read back by the lane that wrote them (cp.async)
  __threadfence_block();
  const Gen gen{grec, reinterpret_cast<Rec*>(wsm), K, lane};

  const bool explicit_all = kDouble || (flags & IRT_FLAG_EXPLICIT_CHANNELS) ||
                            (MODE == M_SMOOTH && admax > (R)0.5);
  if (stats) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) nline += __shfl_xor_sync(0xffffffffu, nline, o);
    if (lane == 0) {
      const unsigned long long nh =
          explicit_all ? (unsigned long long)nblk
                       : ((hhi >= hlo) ? (unsigned long long)(hhi - hlo + 1) : 0ull);
      atomicAdd(stats + 0, 1ull);
      atomicAdd(stats + 1, (unsigned long long)K);
      atomicAdd(stats + 2, nline);
      atomicAdd(stats + 3, nh * (unsigned long long)K);
      atomicAdd(stats + 4, explicit_all ? 1ull : 0ull);
      atomicAdd(stats + 5, (unsigned long long)K * (unsigned long long)nfw);
    }
  }

  // ---- output of channel c from its channel-averaged total intensity and
  // the continuum at the channel centre
  const long long plane = (long long)J.npx * J.npy;
  const long long pix = (long long)py * J.npx + px;
  R* const* out = reinterpret_cast<R* const*>(ML ? outp : J.out);
  auto emit = [&](int c, R ibar, R ic_or_nan, bool have_ic, R X0, R X1, R X2) {
    const R uc = v0r + ((R)c + (R)0.5) * dvr;
    const R ib = planck_k(P, (R)P.t_bg, uc);
    const R ic = have_ic ? ic_or_nan : X0 * ib + X1 + X2 * uc;
    R s = (R)P.out_scale;
    if (P.units == IRT_UNITS_TRJ) {
      const R y = (R)1 - uc * (R)P.inv_c_kms;
      s = s / (y * y);
    }
    const R vT = ibar * s, vC = ic * s, vB = ib * s;
    const long long o = (long long)c * plane + pix;
    if (out[0]) out[0][o] = vT;
    if (out[1]) out[1][o] = vC;
    if (out[2]) out[2][o] = vC - vB;
    if (out[3]) out[3][o] = vT - vC;
    if (out[4]) out[4][o] = vB;
  };
  // Simpson channel average over the fine values fv(g), g = 2 f c .. 2 f (c+1)
  auto simpson = [&](int c, auto&& fv) -> R {
    if (f < 1) return fv(c);
    const int g0 = 2 * f * c;
    R acc = fv(g0) + fv(g0 + 2 * f);
    for (int m = 1; m < 2 * f; m += 2) acc += (R)4 * fv(g0 + m);
    for (int m = 2; m < 2 * f; m += 2) acc += (R)2 * fv(g0 + m);
    return acc / (R)(6 * f);
  };

  // ---- fast path: the hull blocks of the whole axis in registers
  if constexpr (!kDouble) {
    const int ns = (wmax <= 32) ? 1 : ((wmax <= 64) ? 2 : 3);
    if (!explicit_all && ns <= 2) {
      const bool none = hhi < hlo;
      const int na = none ? 1 : hhi - hlo + 1;
      const int nb = fast_bucket(na, ns);
      if (nb <= NI) {
        const int hb = none ? 0 : min(hlo, max(nblk - nb, 0));
        float xb = 0.0f;
        float* kb = reinterpret_cast<float*>(wsm + kb_off);
        float* ck = (CK && J.ck) ? J.ck + ((long long)py * J.npx + px) * J.ck_ray : nullptr;
        const bool fast = (ns == 1) ? run_fast<NI, MODE, 1, CK>(nb, PF, gen, K, hb, lane, G,
                                                                 nfw, fbuf, kb, &xb, ck, J.ck_nb)
                                    : run_fast<NI, MODE, 2, CK>(nb, PF, gen, K, hb, lane, G,
                                                                 nfw, fbuf, kb, &xb, ck, J.ck_nb);
        if (fast) {
          const float X0 = __shfl_sync(0xffffffffu, xb, 0);
          const float X1 = __shfl_sync(0xffffffffu, xb, 1);
          const float X2 = __shfl_sync(0xffffffffu, xb, 2);
          __syncwarp();
          const int e0 = 32 * hb, e1 = 32 * (hb + nb);
          auto fv = [&](int g) -> float {
            if (g >= e0 && g < e1) return fbuf[g - e0];
            const float u = fmaf((float)g, G.dvf_hi, G.ufw_hi);
            return X0 * planck_k(PF, PF.t_bg, u) + X1 + X2 * u;
          };
          for (int c = lane; c < nch; c += 32) emit(c, simpson(c, fv), 0.0f, false, X0, X1, X2);
          __syncwarp();
          return;
        }
      }
    }
  }

  // ---- general path: channel windows of NI register blocks (aligned to the
  // 32-velocity blocks); the continuum basis, or with every channel
  // explicit the dust-only transfer at the channel centres
  R X0 = (R)0, X1 = (R)0, X2 = (R)0;
  if constexpr (!kDouble) {
    if (!explicit_all) {
      const float xb = F::basis(gen, K, lane);
      X0 = __shfl_sync(0xffffffffu, xb, 0);
      X1 = __shfl_sync(0xffffffffu, xb, 1);
      X2 = __shfl_sync(0xffffffffu, xb, 2);
    }
  }
  for (int win = 0; win < J.nwin; ++win) {
    const int c0 = win * J.cw;
    const int cwn = min(J.cw, nch - c0);
    const int gw0 = (f >= 1) ? 2 * f * c0 : c0;   // a multiple of 32
    const int nfw_w = (f >= 1) ? 2 * f * cwn + 1 : cwn;
    const int nblk_w = (nfw_w + 31) >> 5;
    const int bw0 = gw0 >> 5;
    const int lo_w = explicit_all ? 0 : max(hlo - bw0, 0);
    const int hi_w = explicit_all ? nblk_w - 1 : min(hhi - bw0, nblk_w - 1);
    R u[NI];
#pragma unroll
    for (int i = 0; i < NI; ++i) {
      const int g = gw0 + min(lane + 32 * i, nfw_w - 1);
      if constexpr (kDouble) u[i] = J.ufirst + (double)g * J.dvf;
      else u[i] = fmaf((float)g, G.dvf_hi, G.ufw_hi);
    }
    if (lo_w <= hi_w) {
      R s0[NI], s1[NI], s2[NI];
#pragma unroll
      for (int i = 0; i < NI; ++i) {
        s0[i] = (i >= lo_w && i <= hi_w) ? planck_k(P, (R)P.t_bg, u[i]) : (R)0;
        s1[i] = (R)0;
        s2[i] = (R)0;
      }
      F::template transfer<true>(P, G, lane + 32 * bw0, gen, K, u, lo_w, hi_w, s0, s1, s2);
#pragma unroll
      for (int i = 0; i < NI; ++i) {
        const int g = lane + 32 * i;
        if (g < nfw_w && i >= lo_w && i <= hi_w) fbuf[g] = s1[i];
      }
    }
    // velocities outside the explicit blocks: continuum basis
#pragma unroll
    for (int i = 0; i < NI; ++i) {
      const int g = lane + 32 * i;
      if (g < nfw_w && (i < lo_w || i > hi_w))
        fbuf[g] = X0 * planck_k(P, (R)P.t_bg, u[i]) + X1 + X2 * u[i];
    }
    if (explicit_all) {
      R uc[NI], s0[NI], s1[NI], s2[NI];
      const int cblk = (cwn + 31) >> 5;
#pragma unroll
      for (int i = 0; i < NI; ++i) {
        const int c = min(lane + 32 * i, cwn - 1);
        uc[i] = v0r + ((R)(c0 + c) + (R)0.5) * dvr;
        s0[i] = (i < cblk) ? planck_k(P, (R)P.t_bg, uc[i]) : (R)0;
        s1[i] = (R)0;
        s2[i] = (R)0;
      }
      F::template transfer<false>(P, G, lane, gen, K, uc, 0, cblk - 1, s0, s1, s2);
#pragma unroll
      for (int i = 0; i < NI; ++i) {
        const int c = lane + 32 * i;
        if (c < cwn) cbuf[c] = s1[i];
      }
    }
    __syncwarp();
    auto fv = [&](int g) -> R { return fbuf[g - gw0]; };
    for (int cl = lane; cl < cwn; cl += 32) {
      const int c = c0 + cl;
      emit(c, simpson(c, fv), explicit_all ? cbuf[cl] : (R)0, explicit_all, X0, X1, X2);
    }
    __syncwarp();
  }
}

// CK: the job saves smooth-transfer checkpoints (a separate instance, so that
// renders without them run no checkpoint code)
template <typename R, int NI, int ST, int MODE, bool CK, bool OT, bool ML>
__global__ void __launch_bounds__(kWarpsPerBlock * 32, (sizeof(R) == 4 && NI <= 17) ? 4 : 1)
fwd_kernel(const __grid_constant__ JobTable tab, int njobs, const PhysParams PD, const PhysF PF,
           long long total_items, unsigned long long* queue, int per_warp, int fw_off, int cw_off,
           int kb_off, unsigned flags, unsigned long long* stats, unsigned char* rscr,
           long long rstride, long long raw_off, const __grid_constant__ LineSet LS) {
  using Rec = typename RecOf<R, MODE>::type;
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  unsigned char* wsm = smem + (size_t)warp * per_warp;
  // persistent: every warp owns one global record slot.  With a queue, warps
  // pull work items until it runs dry (uneven batches); without one they take
  // items round-robin, so that the warps of a block render neighbouring rays
  // at the same time (one job: measured faster than the queue).
  const long long gw = (long long)blockIdx.x * kWarpsPerBlock + warp;
  const long long nw = (long long)gridDim.x * kWarpsPerBlock;
  Rec* grec = reinterpret_cast<Rec*>(rscr + gw * rstride);
  long long item = gw;
  if (queue) {
    unsigned long long t = 0;
    if (lane == 0) t = atomicAdd(queue, 1ull);
    item = (long long)__shfl_sync(0xffffffffu, t, 0);
  }
  while (item < total_items) {
    int j = 0;
    while (j + 1 < njobs && item >= tab.j[j + 1].item_begin) ++j;
    const JobDev& J = tab.j[j];
    const long long ray = item - J.item_begin;
    // rays come in tiles of tw x th pixels (row-major inside the tile and
    // over the tiles); pixels past the image edge are padding
    const int tsz = J.tw * J.th;
    const long long tile = ray / tsz;
    const int within = (int)(ray - tile * tsz);
    const int px = (int)(tile % J.ntx) * J.tw + within % J.tw;
    const int py = (int)(tile / J.ntx) * J.th + within / J.tw;
    if constexpr (ML) {
      // every line of the ray in turn, its constants read in place from the
      // kernel's parameter space (a __grid_constant__ parameter)
      if (px < J.npx && py < J.npy) {
        float* rawbuf = reinterpret_cast<float*>(rscr + gw * rstride + raw_off);
        for (int q = 0; q < LS.n; ++q) {
          render_ray<R, NI, ST, MODE, false, false, true>(J, PD, LS.pf[q], px, py, wsm, fw_off,
                                                          cw_off, kb_off, grec, lane, flags,
                                                          stats, LS.out[q], rawbuf, q);
          __syncwarp();
        }
      }
    } else if constexpr (ST == ST_F64 || sizeof(R) == 4) {
      if (px < J.npx && py < J.npy)
        render_ray<R, NI, ST, MODE, CK, OT>(J, PD, PF, px, py, wsm, fw_off, cw_off, kb_off, grec,
                                        lane, flags, stats);
    }
    if (queue) {
      unsigned long long t = 0;
      if (lane == 0) t = atomicAdd(queue, 1ull);
      item = (long long)__shfl_sync(0xffffffffu, t, 0);
    } else {
      item += nw;
    }
  }
}

}  // namespace dev

// Host-side launcher of one kernel instance (persistent).  The block count
// is the resident maximum, capped by the record scratch: each warp needs kmax
// records.  L.queue (zero at launch) selects the dynamic schedule, nullptr the
// round-robin one.
// CK: the job keeps smooth-transfer checkpoints; OT: line coefficients from an
// optically thin level-balance grid (separate instances, so that the LTE
// renders' register allocation carries neither).
template <typename R, int NI, int ST, int MODE, bool CK = false, bool OT = false, bool ML = false>
int launch_fwd_inst(const JobTable& tab, int njobs, const PhysParams& P, const PhysF& PF,
                    const FwdLaunch& L, cudaStream_t stream) {
  using Rec = typename dev::RecOf<R, MODE>::type;
  if (L.total <= 0) return 0;
  if (!L.rscr) return (int)cudaErrorInvalidValue;
  // per warp: record ring (2 x 32), fine and channel buffers, Kahan line depths
  const int ring_bytes = 2 * 32 * (int)sizeof(Rec);
  const int fw_off = (ring_bytes + 15) & ~15;
  const int cw_off = (fw_off + (int)sizeof(R) * L.fwmax + 15) & ~15;
  const int kb_off = (cw_off + (int)sizeof(R) * L.cwmax + 15) & ~15;
  const int kb_bytes = (sizeof(R) == 4 && MODE == M_FORMAL_KAHAN) ? 2 * 32 * NI * 4 : 0;
  const int per_warp = (kb_off + kb_bytes + 15) & ~15;
  const size_t smem = (size_t)per_warp * kWarpsPerBlock;
  // per warp: the records of the longest ray, and with several lines the
  // raw field samples of the ray (6 floats a sample) after them
  const long long rec_area = ((long long)L.kmax * (long long)sizeof(Rec) + 255) & ~255ll;
  const long long raw_area = ML ? (((long long)L.kmax * 24 + 255) & ~255ll) : 0;
  const long long rstride = rec_area + raw_area;
  if (ML && !L.lines) return (int)cudaErrorInvalidValue;
  LineSet ls;
  if (ML) ls = *L.lines;
  else std::memset(&ls, 0, sizeof ls);
  auto kern = dev::fwd_kernel<R, NI, ST, MODE, CK, OT, ML>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return (int)e;
  long long blocks = L.grid_blocks;
  if (blocks <= 0) {
    int per_sm = 0, sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kWarpsPerBlock * 32, smem);
    blocks = (long long)std::max(per_sm, 1) * sms;
  }
  blocks = std::min(blocks, (long long)(L.rbytes / ((size_t)rstride * kWarpsPerBlock)));
  blocks = std::min(blocks, (L.total + kWarpsPerBlock - 1) / kWarpsPerBlock);
  if (blocks < 1) return (int)cudaErrorInvalidValue;   // scratch below one block
  kern<<<(unsigned)blocks, kWarpsPerBlock * 32, smem, stream>>>(
      tab, njobs, P, PF, L.total, L.queue, per_warp, fw_off, cw_off, kb_off, L.flags, L.stats,
      L.rscr, rstride, rec_area, ls);
  return (int)cudaGetLastError();
}

}  // namespace irt

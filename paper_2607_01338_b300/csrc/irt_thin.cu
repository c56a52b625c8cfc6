// Selectively thin and optically thin transfer (Sec. 4.6, 4.7, with the step
// substitutions of Sec. 4.8).
//
// Neither mode subsamples velocity: the line profile enters each channel as
// its channel average, the Gaussian's probability mass inside the channel
// over the channel width, [erf(x_hi) - erf(x_lo)] / 2 with x = (u - v) / b at
// the channel edges.  The selectively thin mode solves the continuum first
// and then the total with emission j_L + j_D - alpha_L I_C and absorption
// alpha_D (the line sees the continuum only); the optically thin mode drops
// absorption and integrates the emission directly (midpoint sum, or Simpson
// over node pairs with a trapezoid closing an odd last interval).
//
// One warp per ray.  The ray's samples become records in shared memory once,
// lanes over samples: the line coefficients premultiplied for the channel
// average, 1 / b, the dust source terms, and what each mode needs per sample
// alone (the BDF2 / TR reciprocals, the formal step's exponentials, the
// Simpson weight), so the channel loop does no division or transcendental
// per lane except the line's erfc.  The channel loop then puts lanes over
// channels, 31 at a time: lane l holds the lower edge of channel c0 + l and
// its erfc, lane 31 the upper edge of the last one, and each channel takes
// its upper edge from the next lane by a shuffle.  A warp evaluates the
// erfc only when the sample's line (centre +- 5.5 Doppler widths, beyond
// which the Gaussian's mass is below 1e-14) reaches its 31 channels.  In a
// block of channels that no sample of the ray reaches, [T] = [C] exactly
// (the total's recurrence is the continuum's), and the float kernels take
// the continuum there from three scalar recurrences per ray: the dust source
// is linear in u (B(u) = bk0 + bk1 u), so C(u) = I_bg(u) A + B + u D with A,
// B, D the recurrence of the background (1, no source) and of the sources
// d0 and d1 (0 at the start).  That is exact for the formal and optically
// thin integrals, and for the smooth steps while no ReLU clamps, which
// h alpha_D <= 1/2 on every sample guarantees (BDF2 then keeps a continuum
// with non-negative sources non-negative); rays beyond it run the
// continuum per channel.
#include "irt_forward_impl.cuh"
#include "irt_units.cuh"

namespace irt {
namespace dev {

constexpr int kThinWarps = 4;
constexpr float kThinCut = 5.5f;   // Doppler widths beyond which the line mass is dropped

template <typename R>
struct alignas(16) ThinRec {
  R jw, aw;   // per-step line emission (K units) / optical depth at the profile peak
              // times b sqrt(pi) / (2 dv): times erf(x_hi) - erf(x_lo), the channel average
  R v, ib;    // line centre [km/s] and 1 / b
  R d0, d1;   // float: h alpha_D B_dust(u) = d0 + d1 u; double: d0 = h alpha_D, d1 = T_dust
  R X, Y;     // per-sample step terms: selectively thin formal X = e^-tau, Y = (1 - e^-tau) / tau;
              // smooth X = 1 / (2 + tau) (sample 1) or 1 / (3 + 2 tau), Y = tau;
              // optically thin X = quadrature weight
};

__device__ __forceinline__ float erfc_(float x) { return erfcf(x); }
__device__ __forceinline__ double erfc_(double x) { return erfc(x); }
__device__ __forceinline__ float exp_(float x) { return expf(x); }
__device__ __forceinline__ double exp_(double x) { return exp(x); }
__device__ __forceinline__ float expm1_(float x) { return expm1f(x); }
__device__ __forceinline__ double expm1_(double x) { return expm1(x); }

// Channel edge u(c) = v0 + c dv as a float plus the residual of its rounding
// (error-free product and sum steps on the float-float parts of v0 and dv).
__device__ __forceinline__ void edge_ff(int c, float v0h, float v0l, float dvh, float dvl,
                                        float* hi, float* lo) {
  const float q = (float)c;
  const float p = q * dvh;
  const float pe = fmaf(q, dvh, -p);
  const float s = v0h + p;
  const float bb = s - v0h;
  const float se = (v0h - (s - bb)) + (p - bb);
  *hi = s;
  *lo = pe + se + fmaf(q, dvl, v0l);
}

// Optically thin Simpson weight of node k of K (in units of h): Simpson over
// the first Ms intervals (Ms = K - 1 rounded down to even), the trapezoid
// rule on a remaining last interval.
template <typename R>
__device__ __forceinline__ R simpson_weight(int k, int K) {
  const int M = K - 1;
  const int Ms = M & ~1;
  R w = (R)0;
  if (Ms >= 2 && k <= Ms)
    w = (k == 0 || k == Ms) ? (R)1 / (R)3 : ((k & 1) ? (R)4 / (R)3 : (R)2 / (R)3);
  if (Ms < M) {
    if (k == M - 1) w += (R)0.5;
    if (k == M) w = (R)0.5;
  }
  return w;
}

template <typename R, int ST, int INTEG, int TRANSFER>
__global__ void __launch_bounds__(kThinWarps * 32, 4)
thin_kernel(const __grid_constant__ JobTable tab, int njobs, const PhysParams P, const PhysF PF,
            long long total, int kmax, int warps, long long per_warp_bytes, int nchunk_max,
            unsigned long long* stats) {
  constexpr bool kD = sizeof(R) == 8;
  using Rec = ThinRec<R>;
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  if (warp >= warps) return;
  unsigned char* wbase = smem + (size_t)warp * (size_t)per_warp_bytes;
  Rec* rec = reinterpret_cast<Rec*>(wbase);
  // optically thin / density tracing (float): per 31-channel block, a bit per
  // sample whose line reaches it, 32 samples a word ([block][chunk])
  unsigned* masks = reinterpret_cast<unsigned*>(wbase + (size_t)kmax * sizeof(Rec));
  constexpr bool kMask =
      !kD && (TRANSFER == IRT_MODE_THIN || TRANSFER == IRT_MODE_DENSITY_TRACING);
  const long long nw = (long long)gridDim.x * warps;
  for (long long item = (long long)blockIdx.x * warps + warp; item < total; item += nw) {
    int jj = 0;
    while (jj + 1 < njobs && item >= tab.j[jj + 1].item_begin) ++jj;
    const JobDev& J = tab.j[jj];
    const long long r = item - J.item_begin;
    const int px = (int)(r % J.npx), py = (int)(r / J.npx);
    // ray set-up: double arithmetic on the double kernels, float-float on the
    // float kernels
    RayGeom g;
    RayPos rp;
    int K;
    R h;
    if constexpr (kD) {
      g = ray_geom(J, px, py);
      K = g.K;
      h = (R)g.h;
    } else {
      const RaySet rs = ray_setup(J, px, py);
      K = rs.K;
      h = rs.h;
      rp = rs.rp;
    }
    const long long plane = (long long)J.npx * J.npy;
    const long long pix = (long long)py * J.npx + px;
    R* out[5];
#pragma unroll
    for (int q = 0; q < 5; ++q) out[q] = static_cast<R*>(J.out[q]);
    if (K > kmax) {   // cannot happen with the host's plan; marked, not skipped silently
      for (int c = lane; c < J.nchan; c += 32)
#pragma unroll
        for (int q = 0; q < 5; ++q)
          if (out[q]) out[q][(long long)c * plane + pix] = (R)NAN;
      continue;
    }
    // ---- records
    // channel width and edges: double on the double kernels, the host's
    // float roundings on the float kernels
    const R dvr = kD ? (R)J.dv : (R)J.fdv[0];
    const R sq = (R)0.88622692545275801365 / dvr;   // sqrt(pi) / (2 dv)
    int hlo = 1 << 30, hhi = -1;   // channels any sample's line reaches
    const R v0r = kD ? (R)J.v0 : (R)J.fv0[0];
    const R inv_dv = kD ? (R)(1.0 / J.dv) : (R)J.finv_dv;
    R admax = (R)0;
    const int nblk = (J.nchan + 30) / 31;
    const int nchunk = (K + 31) / 32;
    // record of sample k (lanes over samples); the channel blocks its line
    // reaches go to blo_k .. bhi_k
    auto record = [&](int k, int& blo_k, int& bhi_k) {
      R raw[5];
      R chi = (R)0.5;   // H2 abundance (optically thin level balance only)
      if constexpr (kD) {
        sample_raw<ST>(J, g, px, py, k, raw);
        if (P.ot_tab) chi = sample_chi<ST>(J, g, px, py, k);
      } else {
        sample_raw<ST>(J, rp, px, py, k, raw);
        if (PF.ot_tab) chi = sample_chi<ST>(J, rp, px, py, k);
      }
      R jl, al, b, ad;
      Rec e;
      if constexpr (TRANSFER == IRT_MODE_DENSITY_TRACING) {
        // tracer column x n_H2 h spread by the Doppler profile; no cut-off
        if constexpr (kD)
          b = sqrt((R)P.c_th * raw[1] + (R)P.two_sig2);
        else
          b = sqrtf(PF.c_th * raw[1] + PF.two_sig2);
        jl = raw[4] * raw[0] * h;
        al = (R)0;
        ad = (R)0;
        e.d0 = (R)0;
        e.d1 = (R)0;
        e.jw = jl * ((R)0.5 / dvr);   // times erf(x_hi) - erf(x_lo): x n h mass / dv
        e.aw = (R)0;
      } else {
        if constexpr (kD) {
          line_coeffs(P, raw[0], raw[1], raw[4], chi, h, &jl, &al, &b);
          ad = (R)P.cad * raw[0] * h;
          e.d0 = ad;
          e.d1 = raw[2];
        } else {
          line_coeffs(PF, raw[0], raw[1], raw[4], chi, h, &jl, &al, &b);
          ad = PF.cad * raw[0] * h;
          R bk0, bk1;
          dust_source_lin(PF, raw[2], &bk0, &bk1);
          e.d0 = ad * bk0;
          e.d1 = ad * bk1;
        }
        e.jw = jl * b * sq;
        e.aw = al * b * sq;
      }
      admax = fmax(admax, ad);
      e.v = raw[3];
      e.ib = (R)1 / b;
      if constexpr (TRANSFER == IRT_MODE_THIN || TRANSFER == IRT_MODE_DENSITY_TRACING) {
        e.X = (INTEG == M_FORMAL) ? (R)1 : simpson_weight<R>(k, K);
        e.Y = (R)0;
      } else if constexpr (INTEG == M_FORMAL) {
        e.X = exp_(-ad);
        e.Y = (ad > (R)0) ? -expm1_(-ad) / ad : (R)1;
      } else {
        e.X = (k == 1) ? (R)1 / ((R)2 + ad) : (R)1 / ((R)3 + (R)2 * ad);
        e.Y = ad;
      }
      rec[k] = e;
      if (jl != (R)0 || al != (R)0) {
        // channels the line reaches, widened by one on each side so that the
        // rounding of this bound cannot drop a channel
        const R w = (R)kThinCut * b;
        const R clo = floor((raw[3] - w - v0r) * inv_dv) - (R)1;
        const R chi = floor((raw[3] + w - v0r) * inv_dv) + (R)1;
        if (chi >= (R)0 && clo <= (R)(J.nchan - 1)) {
          const int ci_lo = (int)fmax(clo, (R)0), ci_hi = (int)fmin(chi, (R)(J.nchan - 1));
          hlo = min(hlo, ci_lo);
          hhi = max(hhi, ci_hi);
          blo_k = ci_lo / 31;
          bhi_k = ci_hi / 31;
        }
      }
    };
    if constexpr (kMask) {
      for (int k0 = 0; k0 < K; k0 += 32) {
        const int k = k0 + lane;
        int blo_k = 1 << 30, bhi_k = -1;
        if (k < K) record(k, blo_k, bhi_k);
        for (int bb = 0; bb < nblk; ++bb) {
          const unsigned m = __ballot_sync(0xffffffffu, bb >= blo_k && bb <= bhi_k);
          if (lane == 0) masks[bb * nchunk + (k0 >> 5)] = m;
        }
      }
    } else {
      for (int k = lane; k < K; k += 32) {
        int blo_k = 1 << 30, bhi_k = -1;   // unused without masks
        record(k, blo_k, bhi_k);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      hlo = min(hlo, __shfl_xor_sync(0xffffffffu, hlo, o));
      hhi = max(hhi, __shfl_xor_sync(0xffffffffu, hhi, o));
      admax = fmax(admax, __shfl_xor_sync(0xffffffffu, admax, o));
    }
    __syncwarp();
    // continuum basis (float kernels): C(u) = I_bg(u) bA + bB + u bD
    R bA = (R)1, bB = (R)0, bD = (R)0;
    constexpr bool kSum = TRANSFER == IRT_MODE_THIN || TRANSFER == IRT_MODE_DENSITY_TRACING;
    const bool basis = !kD && (kSum || INTEG == M_FORMAL || admax <= (R)0.5);
    if (basis && K >= 1) {
      if constexpr (kSum) {
        for (int k = 0; k < K; ++k) {
          const Rec e = rec[k];
          bB = fma(e.X, e.d0, bB);
          bD = fma(e.X, e.d1, bD);
        }
      } else if constexpr (INTEG == M_FORMAL) {
        for (int k = 0; k < K; ++k) {
          const Rec e = rec[k];
          bA *= e.X;
          bB = fma(bB, e.X, e.d0 * e.Y);
          bD = fma(bD, e.X, e.d1 * e.Y);
        }
      } else if (K >= 2) {
        const Rec e0 = rec[0], e1 = rec[1];
        R A0 = (R)1, B0 = (R)0, D0 = (R)0;
        R A1 = ((R)2 - e0.Y) * e1.X;
        R B1 = (e0.d0 + e1.d0) * e1.X;
        R D1 = (e0.d1 + e1.d1) * e1.X;
        for (int k = 2; k < K; ++k) {
          const Rec e = rec[k];
          const R A2 = fma((R)4, A1, -A0) * e.X;
          const R B2 = fma((R)2, e.d0, fma((R)4, B1, -B0)) * e.X;
          const R D2 = fma((R)2, e.d1, fma((R)4, D1, -D0)) * e.X;
          A0 = A1; B0 = B1; D0 = D1;
          A1 = A2; B1 = B2; D1 = D2;
        }
        bA = A1;
        bB = B1;
        bD = D1;
      }
    }
    if (stats && lane == 0) {
      atomicAdd(&stats[0], 1ull);
      atomicAdd(&stats[1], (unsigned long long)K);
    }
    // ---- channels, 31 per pass (lane 31 carries the last upper edge)
    const float v0h = J.fv0[0], v0l = J.fv0[1];
    const float dvh = J.fdv[0], dvl = J.fdv[1];
    for (int c0 = 0; c0 < J.nchan; c0 += 31) {
      const int c = c0 + lane;
      const int cend = min(c0 + 31, J.nchan);
      const bool act = lane < 31 && c < J.nchan;
      // lower edge of channel c as a rounded value plus its residual, so that
      // u - v keeps the line's position to far below a Doppler width
      R ue, ue_r, uc, blo, bhi;
      if constexpr (kD) {
        const double ue_d = J.v0 + (double)c * J.dv;
        ue = ue_d;
        ue_r = 0.0;
        uc = J.v0 + ((double)c + 0.5) * J.dv;
        blo = J.v0 + (double)c0 * J.dv;
        bhi = J.v0 + (double)cend * J.dv;
      } else {
        float lo;
        edge_ff(c, v0h, v0l, dvh, dvl, &ue, &ue_r);
        uc = fmaf(0.5f, dvh, ue + ue_r);
        edge_ff(c0, v0h, v0l, dvh, dvl, &blo, &lo);
        edge_ff(cend, v0h, v0l, dvh, dvl, &bhi, &lo);
      }
      const bool reached = hhi >= c0 && hlo < cend;
      R ib;
      if constexpr (TRANSFER == IRT_MODE_DENSITY_TRACING)
        ib = (R)0;   // no background
      else if constexpr (kD)
        ib = planck_k(P, (R)P.t_bg, uc);
      else
        ib = planck_k(PF, PF.t_bg, uc);
      // dust source of record e at this lane's channel (per step, K units)
      auto dust = [&](const Rec& e) -> R {
        if constexpr (kD)
          return e.d0 * planck_k(P, e.d1, uc);
        else
          return fmaf(e.d1, uc, e.d0);
      };
      // channel average of the line of record e: erf(x_hi) - erf(x_lo) from
      // erfc of |x| at this lane's lower edge and the next lane's
      auto line = [&](const Rec& e, R* jlb, R* alb) {
        *jlb = (R)0;
        *alb = (R)0;
        if ((e.jw == (R)0 && e.aw == (R)0) || (bhi - e.v) * e.ib <= -(R)kThinCut ||
            (blo - e.v) * e.ib >= (R)kThinCut)
          return;   // warp-uniform
        const R x = ((ue - e.v) + ue_r) * e.ib;
        const R E = erfc_(x >= (R)0 ? x : -x);
        const R xn = __shfl_down_sync(0xffffffffu, x, 1);
        const R En = __shfl_down_sync(0xffffffffu, E, 1);
        const R d = (x >= (R)0) ? E - En : ((xn <= (R)0) ? En - E : (R)2 - E - En);
        *jlb = e.jw * d;
        *alb = e.aw * d;
      };
      R IT = ib, IC = ib;
      if constexpr (kSum) {
        // direct integral of the emission (weights: 1 formal, Simpson smooth)
        R sT = (R)0, sC = (R)0;
        if (kMask && reached && basis) {
          // the line from the samples that reach this block, the dust from
          // the continuum basis
          R sL = (R)0;
          const unsigned* mb = masks + (c0 / 31) * nchunk;
          for (int ch = 0; ch < nchunk; ++ch) {
            unsigned m = mb[ch];
            while (m) {
              const int k = (ch << 5) + __ffs(m) - 1;
              m &= m - 1;
              const Rec e = rec[k];
              R jlb, alb;
              line(e, &jlb, &alb);
              sL = fma(e.X, jlb, sL);
            }
          }
          sC = fma(uc, bD, bB);
          sT = sC + sL;
        } else if (reached) {
          for (int k = 0; k < K; ++k) {
            const Rec e = rec[k];
            R jlb, alb;
            line(e, &jlb, &alb);
            const R jd = dust(e);
            sC = fma(e.X, jd, sC);
            sT = fma(e.X, jlb + jd, sT);
          }
        } else if (basis) {
          sC = fma(uc, bD, bB);
          sT = sC;
        } else {
          for (int k = 0; k < K; ++k) {
            const Rec e = rec[k];
            sC = fma(e.X, dust(e), sC);
          }
          sT = sC;
        }
        IT = ib + sT;
        IC = ib + sC;
      } else if constexpr (INTEG == M_FORMAL) {
        // continuum step, then the total step with that continuum
        if (reached) {
          for (int k = 0; k < K; ++k) {
            const Rec e = rec[k];
            R jlb, alb;
            line(e, &jlb, &alb);
            const R jd = dust(e);
            IC = fma(IC, e.X, jd * e.Y);
            IT = fma(IT, e.X, (jlb + jd - alb * IC) * e.Y);
          }
        } else if (basis) {
          IC = fma(ib, bA, fma(uc, bD, bB));
          IT = IC;
        } else {
          for (int k = 0; k < K; ++k) {
            const Rec e = rec[k];
            IC = fma(IC, e.X, dust(e) * e.Y);
          }
          IT = IC;
        }
      } else if (K >= 2 && !reached && basis) {
        IC = fma(ib, bA, fma(uc, bD, bB));
        IT = IC;
      } else if (K >= 2) {
        // smooth: node 0 = background, TR to node 1, BDF2 after, ReLU
        const Rec e0 = rec[0], e1 = rec[1];
        const R jd0 = dust(e0), jd1 = dust(e1);
        R jlb0, alb0, jlb1, alb1;
        line(e0, &jlb0, &alb0);
        line(e1, &jlb1, &alb1);
        const R c1 = fmax((jd0 + jd1 + ((R)2 - e0.Y) * ib) * e1.X, (R)0);
        R Ca = ib, Cb = c1;
        if (reached) {
          const R jt0 = jlb0 + jd0 - alb0 * ib;
          const R jt1 = jlb1 + jd1 - alb1 * c1;
          R Ta = ib, Tb = fmax((jt0 + jt1 + ((R)2 - e0.Y) * ib) * e1.X, (R)0);
          for (int k = 2; k < K; ++k) {
            const Rec e = rec[k];
            R jlb, alb;
            line(e, &jlb, &alb);
            const R jd = dust(e);
            const R cn = fmax(fma((R)2, jd, fma((R)4, Cb, -Ca)) * e.X, (R)0);
            const R jt = jlb + jd - alb * cn;
            const R tn = fmax(fma((R)2, jt, fma((R)4, Tb, -Ta)) * e.X, (R)0);
            Ca = Cb;
            Cb = cn;
            Ta = Tb;
            Tb = tn;
          }
          IT = Tb;
        } else {
          for (int k = 2; k < K; ++k) {
            const Rec e = rec[k];
            const R cn = fmax(fma((R)2, dust(e), fma((R)4, Cb, -Ca)) * e.X, (R)0);
            Ca = Cb;
            Cb = cn;
          }
          IT = Cb;
        }
        IC = Cb;
      }
      if (act) {
        R s;
        if constexpr (kD) {
          s = (R)P.out_scale;
          if (P.units == IRT_UNITS_TRJ) {
            const R y = (R)1 - uc * (R)P.inv_c_kms;
            s = s / (y * y);
          }
        } else {
          s = PF.out_scale;
          if (PF.units == IRT_UNITS_TRJ) {
            const R y = (R)1 - uc * PF.inv_c_kms;
            s = s / (y * y);
          }
        }
        if constexpr (TRANSFER == IRT_MODE_DENSITY_TRACING) s = (R)1;   // cm^-2 per km/s
        R vT = IT * s, vC = IC * s, vB = ib * s;
        bool tb;
        R T0, ic_kms;
        if constexpr (kD) {
          tb = P.units == IRT_UNITS_TB;
          T0 = (R)P.T0;
          ic_kms = (R)P.inv_c_kms;
        } else {
          tb = PF.units == IRT_UNITS_TB;
          T0 = PF.T0;
          ic_kms = PF.inv_c_kms;
        }
        if (tb && TRANSFER != IRT_MODE_DENSITY_TRACING) {   // continuum subtracted in T_B space below
          vT = brightness_k(T0, ic_kms, uc, IT);
          vC = brightness_k(T0, ic_kms, uc, IC);
          vB = brightness_k(T0, ic_kms, uc, ib);
        }
        const long long o = (long long)c * plane + pix;
        if (out[0]) out[0][o] = vT;
        if (out[1]) out[1][o] = vC;
        if (out[2]) out[2][o] = vC - vB;
        if (out[3]) out[3][o] = vT - vC;
        if (out[4]) out[4][o] = vB;
      }
    }
    __syncwarp();
  }
}

}  // namespace dev

// Host launcher of the thin modes: precision (0 float, 1 double), field
// storage, integration (M_FORMAL or M_SMOOTH), transfer mode.
// Shared memory one warp of the thin kernel needs: the records of the longest
// ray plus, for the float optically thin and density-tracing kernels, the
// per-block sample masks (one bit per sample and 31-channel block).
size_t thin_smem_per_warp(int precision, int transfer, int kmax, int nchan_max,
                          size_t* record_bytes, size_t* mask_bytes_out) {
  const size_t rec_bytes = precision ? sizeof(dev::ThinRec<double>) : sizeof(dev::ThinRec<float>);
  const int nchunk_max = (kmax + 31) / 32;
  const bool masks = !precision && (transfer == IRT_MODE_THIN ||
                                    transfer == IRT_MODE_DENSITY_TRACING);
  const size_t mask_bytes = masks ? (size_t)4 * ((nchan_max + 30) / 31) * nchunk_max : 0;
  if (record_bytes) *record_bytes = rec_bytes * (size_t)kmax;
  if (mask_bytes_out) *mask_bytes_out = mask_bytes;
  return (rec_bytes * (size_t)kmax + mask_bytes + 15) & ~(size_t)15;
}

int launch_thin(int precision, int store, int integ, int transfer, const JobTable& tab,
                int njobs, const PhysParams& P, const PhysF& PF, long long total, int kmax,
                int nchan_max, unsigned long long* stats, cudaStream_t stream) {
  const int nchunk_max = (kmax + 31) / 32;
  const size_t per_warp = thin_smem_per_warp(precision, transfer, kmax, nchan_max, nullptr,
                                             nullptr);
  const size_t budget = kThinSmemBudget;
  if (per_warp > budget) return (int)cudaErrorInvalidValue;
  const int warps = (int)std::max<size_t>(1, std::min<size_t>(dev::kThinWarps, budget / per_warp));
  const size_t smem = per_warp * warps;
  int dev_id = 0, sms = 0;
  cudaGetDevice(&dev_id);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev_id);
#define IRT_THIN(R_, ST_, IN_, TR_)                                                            \
  if ((sizeof(R_) == 8) == (precision != 0) && store == ST_ && integ == IN_ &&                 \
      transfer == TR_) {                                                                       \
    auto kern = dev::thin_kernel<R_, ST_, IN_, TR_>;                                           \
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,    \
                                         (int)smem);                                           \
    if (e != cudaSuccess) return (int)e;                                                       \
    int per_sm = 0;                                                                            \
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, dev::kThinWarps * 32, smem);  \
    const long long need = (total + warps - 1) / warps;                                        \
    const int blocks = (int)std::max<long long>(                                               \
        1, std::min<long long>(need, (long long)std::max(per_sm, 1) * sms));                   \
    kern<<<blocks, dev::kThinWarps * 32, smem, stream>>>(tab, njobs, P, PF, total, kmax,        \
                                                         warps, (long long)per_warp,           \
                                                         nchunk_max, stats);                   \
    return (int)cudaGetLastError();                                                            \
  }
#define IRT_THIN_ST(R_, IN_, TR_) \
  IRT_THIN(R_, ST_F32, IN_, TR_) IRT_THIN(R_, ST_H16, IN_, TR_) IRT_THIN(R_, ST_F64, IN_, TR_)
#define IRT_THIN_R(IN_, TR_) IRT_THIN_ST(float, IN_, TR_) IRT_THIN_ST(double, IN_, TR_)
  IRT_THIN_R(M_FORMAL, IRT_MODE_SELECTIVELY_THIN)
  IRT_THIN_R(M_SMOOTH, IRT_MODE_SELECTIVELY_THIN)
  IRT_THIN_R(M_FORMAL, IRT_MODE_THIN)
  IRT_THIN_R(M_SMOOTH, IRT_MODE_THIN)
  IRT_THIN_R(M_FORMAL, IRT_MODE_DENSITY_TRACING)
  IRT_THIN_R(M_SMOOTH, IRT_MODE_DENSITY_TRACING)
#undef IRT_THIN_R
#undef IRT_THIN_ST
#undef IRT_THIN
  return (int)cudaErrorInvalidValue;
}

}  // namespace irt

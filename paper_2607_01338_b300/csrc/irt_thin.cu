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
// One warp per ray, lanes over channels (32 at a time).  The ray's samples
// are turned into records in shared memory once (per-step line coefficients
// at the profile peak, Doppler parameter, h alpha_D, dust Planck terms); the
// channel loop then reads them as broadcasts.  What depends on the sample
// alone (the BDF2 and TR reciprocals, the formal step's exponential) is the
// same for every lane.  A warp evaluates the erf channel average only when
// the line of the sample (centre +- 5.5 Doppler widths, where the Gaussian's
// remaining mass is below 1e-14) reaches its block of 32 channels.
#include "irt_forward_impl.cuh"

namespace irt {
namespace dev {

constexpr int kThinWarps = 4;
constexpr float kThinCut = 5.5f;   // Doppler widths beyond which the line mass is dropped

template <typename R>
struct alignas(16) ThinRec {
  R jl, al;   // per-step line emission (K units) and optical depth at the profile peak
  R v, b;     // line centre and Doppler parameter [km/s]
  R ad;       // h alpha_D
  R bk0, bk1; // dust Planck source, float: B(u) = bk0 + bk1 u; double: bk0 = T_dust
  R pad;
};

__device__ __forceinline__ float erfc_(float x) { return erfcf(x); }
__device__ __forceinline__ double erfc_(double x) { return erfc(x); }
__device__ __forceinline__ float exp_(float x) { return expf(x); }
__device__ __forceinline__ double exp_(double x) { return exp(x); }
__device__ __forceinline__ float expm1_(float x) { return expm1f(x); }
__device__ __forceinline__ double expm1_(double x) { return expm1(x); }
__device__ __forceinline__ float rcp_(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double rcp_(double x) { return 1.0 / x; }

// erf(x_hi) - erf(x_lo) for x_lo <= x_hi, from erfc of non-negative
// arguments so that a channel in the far wing keeps its relative precision.
template <typename R>
__device__ __forceinline__ R erf_diff(R x_lo, R x_hi) {
  if (x_lo >= (R)0) return erfc_(x_lo) - erfc_(x_hi);
  if (x_hi <= (R)0) return erfc_(-x_hi) - erfc_(-x_lo);
  return (R)2 - erfc_(-x_lo) - erfc_(x_hi);
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
__global__ void __launch_bounds__(kThinWarps * 32)
thin_kernel(const __grid_constant__ JobTable tab, int njobs, const PhysParams P, const PhysF PF,
            long long total, int kmax, int warps, unsigned long long* stats) {
  constexpr bool kD = sizeof(R) == 8;
  using Rec = ThinRec<R>;
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  if (warp >= warps) return;
  Rec* rec = reinterpret_cast<Rec*>(smem) + (size_t)warp * kmax;
  const long long nw = (long long)gridDim.x * warps;
  for (long long item = (long long)blockIdx.x * warps + warp; item < total; item += nw) {
    int jj = 0;
    while (jj + 1 < njobs && item >= tab.j[jj + 1].item_begin) ++jj;
    const JobDev& J = tab.j[jj];
    const long long r = item - J.item_begin;
    const int px = (int)(r % J.npx), py = (int)(r / J.npx);
    const RayGeom g = ray_geom(J, px, py);
    const int K = g.K;
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
    const R h = (R)g.h;
    RayPos rp;
    if constexpr (!kD) rp = ray_pos(J, g);
    for (int k = lane; k < K; k += 32) {
      R raw[5];
      if constexpr (kD)
        sample_raw<ST>(J, g, px, py, k, raw);
      else
        sample_raw<ST>(J, rp, px, py, k, raw);
      Rec e;
      if constexpr (kD) {
        line_coeffs(P, raw[0], raw[1], raw[4], h, &e.jl, &e.al, &e.b);
        e.ad = (R)P.cad * raw[0] * h;
        e.bk0 = raw[2];
        e.bk1 = (R)0;
      } else {
        line_coeffs(PF, raw[0], raw[1], raw[4], h, &e.jl, &e.al, &e.b);
        e.ad = PF.cad * raw[0] * h;
        dust_source_lin(PF, raw[2], &e.bk0, &e.bk1);
      }
      e.v = raw[3];
      e.pad = (R)0;
      rec[k] = e;
    }
    __syncwarp();
    if (stats && lane == 0) {
      atomicAdd(&stats[0], 1ull);
      atomicAdd(&stats[1], (unsigned long long)K);
    }
    // ---- channels, 32 per pass
    const R sq = (R)0.88622692545275801365 / (R)J.dv;   // sqrt(pi) / (2 dv)
    for (int c0 = 0; c0 < J.nchan; c0 += 32) {
      const int c = c0 + lane;
      const bool act = c < J.nchan;
      // channel edges u_lo, u_hi as a rounded value plus its residual, so
      // that u - v keeps the line's position to far below a Doppler width
      const double ulo_d = J.v0 + (double)c * J.dv, uhi_d = ulo_d + J.dv;
      const R ulo = (R)ulo_d, uhi = (R)uhi_d;
      const R ulo_r = (R)(ulo_d - (double)ulo), uhi_r = (R)(uhi_d - (double)uhi);
      const R uc = (R)(J.v0 + ((double)c + 0.5) * J.dv);
      const R blo = (R)(J.v0 + (double)c0 * J.dv);
      const R bhi = (R)(J.v0 + (double)min(c0 + 32, J.nchan) * J.dv);
      R ib;
      if constexpr (kD)
        ib = planck_k(P, (R)P.t_bg, uc);
      else
        ib = planck_k(PF, PF.t_bg, uc);
      // line and dust per-step coefficients of record k at this lane's channel
      auto coeffs = [&](const Rec& e, R* jlb, R* alb, R* jd) {
        *jlb = (R)0;
        *alb = (R)0;
        const bool line = (e.jl != (R)0 || e.al != (R)0) &&
                          e.v + (R)kThinCut * e.b > blo && e.v - (R)kThinCut * e.b < bhi;
        if (line) {
          const R ibv = (R)1 / e.b;
          const R xlo = ((ulo - e.v) + ulo_r) * ibv;
          const R xhi = ((uhi - e.v) + uhi_r) * ibv;
          const R w = sq * e.b * erf_diff(xlo, xhi);
          *jlb = e.jl * w;
          *alb = e.al * w;
        }
        if constexpr (kD)
          *jd = e.ad * planck_k(P, e.bk0, uc);
        else
          *jd = e.ad * fmaf(e.bk1, uc, e.bk0);
      };
      R IT = ib, IC = ib;
      if (K >= 1) {
        if constexpr (TRANSFER == IRT_MODE_THIN) {
          // direct integral of the emission
          R sT = (R)0, sC = (R)0;
          for (int k = 0; k < K; ++k) {
            R jlb, alb, jd;
            coeffs(rec[k], &jlb, &alb, &jd);
            const R w = (INTEG == M_FORMAL) ? (R)1 : simpson_weight<R>(k, K);
            sT += w * (jlb + jd);
            sC += w * jd;
          }
          IT = ib + sT;
          IC = ib + sC;
        } else if constexpr (INTEG == M_FORMAL) {
          // continuum step, then the total step with that continuum
          for (int k = 0; k < K; ++k) {
            const Rec e = rec[k];
            R jlb, alb, jd;
            coeffs(e, &jlb, &alb, &jd);
            const R tau = e.ad;
            const R q = exp_(-tau);
            const R gq = (tau > (R)0) ? -expm1_(-tau) / tau : (R)1;
            IC = IC * q + jd * gq;
            IT = IT * q + (jlb + jd - alb * IC) * gq;
          }
        } else {
          // smooth: node 0 = background, TR to node 1, BDF2 after, ReLU
          R jlb0, alb0, jd0;
          const Rec e0 = rec[0];
          coeffs(e0, &jlb0, &alb0, &jd0);
          R Ca = ib, Ta = ib;          // node n - 2 (after the first steps)
          R Cb = ib, Tb = ib;          // node n - 1
          if (K >= 2) {
            const Rec e1 = rec[1];
            R jlb1, alb1, jd1;
            coeffs(e1, &jlb1, &alb1, &jd1);
            const R r1 = rcp_((R)2 + e1.ad);
            const R c1 = fmax((jd0 + jd1 + ((R)2 - e0.ad) * ib) * r1, (R)0);
            const R jt0 = jlb0 + jd0 - alb0 * ib;
            const R jt1 = jlb1 + jd1 - alb1 * c1;
            const R t1 = fmax((jt0 + jt1 + ((R)2 - e0.ad) * ib) * r1, (R)0);
            Cb = c1;
            Tb = t1;
          }
          for (int k = 2; k < K; ++k) {
            const Rec e = rec[k];
            R jlb, alb, jd;
            coeffs(e, &jlb, &alb, &jd);
            const R rr = rcp_((R)3 + (R)2 * e.ad);
            const R cn = fmax(((R)2 * jd + (R)4 * Cb - Ca) * rr, (R)0);
            const R jt = jlb + jd - alb * cn;
            const R tn = fmax(((R)2 * jt + (R)4 * Tb - Ta) * rr, (R)0);
            Ca = Cb;
            Cb = cn;
            Ta = Tb;
            Tb = tn;
          }
          IC = Cb;
          IT = Tb;
        }
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
        const R vT = IT * s, vC = IC * s, vB = ib * s;
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
int launch_thin(int precision, int store, int integ, int transfer, const JobTable& tab,
                int njobs, const PhysParams& P, const PhysF& PF, long long total, int kmax,
                unsigned long long* stats, cudaStream_t stream) {
  const size_t rec_bytes = precision ? sizeof(dev::ThinRec<double>) : sizeof(dev::ThinRec<float>);
  const size_t per_warp = rec_bytes * (size_t)kmax;
  const size_t budget = 200 * 1024;
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
                                                         warps, stats);                        \
    return (int)cudaGetLastError();                                                            \
  }
#define IRT_THIN_ST(R_, IN_, TR_) \
  IRT_THIN(R_, ST_F32, IN_, TR_) IRT_THIN(R_, ST_H16, IN_, TR_) IRT_THIN(R_, ST_F64, IN_, TR_)
#define IRT_THIN_R(IN_, TR_) IRT_THIN_ST(float, IN_, TR_) IRT_THIN_ST(double, IN_, TR_)
  IRT_THIN_R(M_FORMAL, IRT_MODE_SELECTIVELY_THIN)
  IRT_THIN_R(M_SMOOTH, IRT_MODE_SELECTIVELY_THIN)
  IRT_THIN_R(M_FORMAL, IRT_MODE_THIN)
  IRT_THIN_R(M_SMOOTH, IRT_MODE_THIN)
#undef IRT_THIN_R
#undef IRT_THIN_ST
#undef IRT_THIN
  return (int)cudaErrorInvalidValue;
}

}  // namespace irt

// Optically thin (OT) level balance and its coefficient grid (Sec. 3.4-3.6,
// 4.2): one FP64 linear solve per grid node on the GPU, at table-creation
// time (the render only interpolates the grid).
//
// Per node (n_H, chi, T) of the grid over (log10 n_H, chi, log10 T), the
// populations n_i / N solve the level system of Sec. 3.5: for every level but
// the ground state the inflow equals the outflow, with collision rates
// C = sum over partners of K(T) n_partner (K linear in T between the
// tabulated temperatures, held beyond them; the excitation rates by detailed
// balance at T, Sec. 3.6), spontaneous emission A, and stimulated emission and
// absorption by a blackbody background at T-bar (the OT assumption, Einstein
// B relations of Sec. 3.6); the ground-state row is replaced by sum_i n_i = N.
// Then, per line, the frequency-integrated coefficients per tracer molecule
// j = (h nu / 4 pi) A f_u and alpha = (h nu / 4 pi)(f_l B_lu - f_u B_ul).
//
// One warp per node, the augmented matrix of the node in shared memory (FP64,
// at most 64 levels): the lanes take the transitions of one partner at a time
// and add each one's two off-diagonal inflows (a partner lists a level pair
// once, so no two lanes write one element: no atomics, the same sums in the
// same order on every run), the diagonal is minus the column sum (the total
// outflow), then Gaussian elimination with partial pivoting (pivot by a warp
// reduction, rows eliminated by lanes) and back substitution (sums by warp
// reduction).  The detailed-balance factor is the ratio of per-level
// Boltzmann factors (one exponential per level, not per transition).  FP64 because the grid is built once at start-up and the
// level systems span many orders of magnitude in their rates; the render
// reads the float copy.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "irt_internal.h"

namespace irt {
namespace {

constexpr double kHP = 6.62607015e-27;    // erg s
constexpr double kKB = 1.380649e-16;      // erg / K
constexpr double kCL = 2.99792458e10;     // cm / s
constexpr double kPI = 3.14159265358979323846;
constexpr int kBuildWarps = 4;

__device__ double partner_density(const OTBuildArgs& M, int kind, double n_h, double chi) {
  const double n_h2 = chi * n_h;
  switch (kind) {
    case IRT_PARTNER_H2: return n_h2;
    case IRT_PARTNER_PH2: return n_h2 / (1.0 + M.opr);
    case IRT_PARTNER_OH2: return n_h2 * M.opr / (1.0 + M.opr);
    case IRT_PARTNER_H: return fmax(0.0, n_h * (1.0 - 2.0 * chi));
    case IRT_PARTNER_HE: return M.x_he * n_h;
  }
  return 0.0;
}

__device__ double rate_coefficient(const OTBuildArgs& M, int p, int c, double T) {
  const double* tt = M.ctemp + (long long)p * M.ntemp;
  const double* kk = M.k + ((long long)p * M.ncoll + c) * M.ntemp;
  if (M.ntemp == 1 || T <= tt[0]) return kk[0];
  if (T >= tt[M.ntemp - 1]) return kk[M.ntemp - 1];
  int i = 0;
  while (T > tt[i + 1]) ++i;
  const double w = (T - tt[i]) / (tt[i + 1] - tt[i]);
  return kk[i] + w * (kk[i + 1] - kk[i]);
}

// Planck intensity B_nu(T) [cgs]
__device__ double planck_cgs(double nu, double T) {
  if (!(T > 0.0)) return 0.0;
  return 2.0 * kHP * nu * nu * nu / (kCL * kCL) / expm1(kHP * nu / (kKB * T));
}

// doubles of shared memory one warp of the build needs
__host__ __device__ inline int ot_warp_doubles(int n) { return n * (n + 1) + 2 * n + 8 + 8 + 4; }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__global__ void __launch_bounds__(kBuildWarps * 32)
ot_build_kernel(OTBuildArgs M, double* tab64, float4* tab32, long long nodes) {
  extern __shared__ double sm[];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int n = M.nlev, ld = n + 1;
  // per warp: the augmented matrix (row major), the level factors, the
  // partners' rate brackets
  double* A = sm + (size_t)warp * ot_warp_doubles(n);
  double* xs = A + n * ld;
  double* rx = xs + n;
  double* pw = rx + n;
  double* pn = pw + 8;
  int* pbr = reinterpret_cast<int*>(pn + 8);
  const long long n12 = (long long)M.n[1] * M.n[2];
  for (long long node = (long long)blockIdx.x * kBuildWarps + warp; node < nodes;
       node += (long long)gridDim.x * kBuildWarps) {
    const int i0 = (int)(node / n12);
    const int i1 = (int)((node / M.n[2]) % M.n[1]);
    const int i2 = (int)(node % M.n[2]);
    const double n_h = pow(10.0, M.lo[0] + (M.hi[0] - M.lo[0]) * i0 / (M.n[0] - 1));
    const double chi = M.lo[1] + (M.hi[1] - M.lo[1]) * i1 / (M.n[1] - 1);
    const double T = pow(10.0, M.lo[2] + (M.hi[2] - M.lo[2]) * i2 / (M.n[2] - 1));
    for (int e = lane; e < n * ld; e += 32) A[e] = 0.0;
    // per level: x_i = exp(-(E_i - E_0) / T) and 1 / x_i (detailed balance
    // as a ratio, one exponential per level instead of per transition);
    // per partner: its density and the bracket of T in its rate table
    for (int i = lane; i < n; i += 32) {
      const double x = exp(-(M.energy[i] - M.energy[0]) / T);
      xs[i] = x;
      rx[i] = (x > 1e-250) ? 1.0 / x : 0.0;
    }
    for (int p = lane; p < M.npartner; p += 32) {
      const double* tt = M.ctemp + (long long)p * M.ntemp;
      int it = 0;
      double w = 0.0;
      if (M.ntemp > 1 && T > tt[0]) {
        if (T >= tt[M.ntemp - 1]) {
          it = M.ntemp - 2;
          w = 1.0;
        } else {
          while (T > tt[it + 1]) ++it;
          w = (T - tt[it]) / (tt[it + 1] - tt[it]);
        }
      }
      pbr[p] = it;
      pw[p] = w;
      pn[p] = partner_density(M, M.partner[p], n_h, chi);
    }
    __syncwarp();
    // off-diagonal inflows: A[l][u] += rate u -> l, A[u][l] += rate l -> u.
    // Lanes take the transitions of one partner at a time; a partner lists
    // each level pair once (checked on the host), so no two lanes write the
    // same element and every run sums in the same order.
    for (int p = 0; p < M.npartner; ++p) {
      const int it = pbr[p];
      const double w = pw[p], np = pn[p];
      for (int c = lane; c < M.ncoll; c += 32) {
        const int u = M.cup[p * M.ncoll + c], l = M.clo[p * M.ncoll + c];
        const double* kk = M.k + ((long long)p * M.ncoll + c) * M.ntemp;
        const double K = (M.ntemp > 1) ? kk[it] + w * (kk[it + 1] - kk[it]) : kk[0];
        const double cul = K * np;
        // detailed balance (Sec. 3.6): K_lu = K_ul (g_u / g_l) exp(-(E_u - E_l) / kT)
        const double db = (rx[l] != 0.0) ? xs[u] * rx[l]
                                          : exp(-(M.energy[u] - M.energy[l]) / T);
        A[l * ld + u] += cul;
        A[u * ld + l] += cul * (M.g[u] / M.g[l]) * db;
      }
      __syncwarp();
    }
    for (int r = lane; r < M.nrad; r += 32) {
      const int u = M.rad_up[r], l = M.rad_lo[r];
      const double nu = M.nu[r];
      const double b_ul = kCL * kCL * M.a[r] / (2.0 * kHP * nu * nu * nu);
      const double b_lu = (M.g[u] / M.g[l]) * b_ul;
      const double J = planck_cgs(nu, M.t_rad);
      A[l * ld + u] += M.a[r] + b_ul * J;
      A[u * ld + l] += b_lu * J;
    }
    __syncwarp();
    // diagonal: minus the total outflow of level i, the sum of the inflows
    // it feeds (column i)
    for (int c = lane; c < n; c += 32) {
      double out = 0.0;
      for (int r = 0; r < n; ++r)
        if (r != c) out += A[r * ld + c];
      A[c * ld + c] = -out;
    }
    __syncwarp();
    // conservation row and right-hand side e_0
    for (int j = lane; j < ld; j += 32) A[j] = 1.0;
    for (int i = 1 + lane; i < n; i += 32) A[i * ld + n] = 0.0;
    __syncwarp();
    // elimination with partial pivoting (first row of largest magnitude)
    for (int k = 0; k < n; ++k) {
      double bv = -1.0;
      int bi = n;
      for (int i = k + lane; i < n; i += 32) {
        const double v = fabs(A[i * ld + k]);
        if (v > bv) {
          bv = v;
          bi = i;
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ov > bv || (ov == bv && oi < bi)) {
          bv = ov;
          bi = oi;
        }
      }
      if (bi != k) {
        for (int j = k + lane; j < ld; j += 32) {
          const double t = A[k * ld + j];
          A[k * ld + j] = A[bi * ld + j];
          A[bi * ld + j] = t;
        }
      }
      __syncwarp();
      const double piv = A[k * ld + k];
      for (int i = k + 1 + lane; i < n; i += 32) {
        const double f = A[i * ld + k] / piv;
        if (f != 0.0)
          for (int j = k; j < ld; ++j) A[i * ld + j] -= f * A[k * ld + j];
      }
      __syncwarp();
    }
    // back substitution into the right-hand-side column
    for (int i = n - 1; i >= 0; --i) {
      double part = 0.0;
      for (int j = i + 1 + lane; j < n; j += 32) part += A[i * ld + j] * A[j * ld + n];
      part = warp_sum(part);
      if (lane == 0) A[i * ld + n] = (A[i * ld + n] - part) / A[i * ld + i];
      __syncwarp();
    }
    // per line: coefficients per tracer molecule
    for (int q = lane; q < M.nlines; q += 32) {
      const int r = M.lines[q];
      const int u = M.rad_up[r], l = M.rad_lo[r];
      const double nu = M.nu[r];
      const double b_ul = kCL * kCL * M.a[r] / (2.0 * kHP * nu * nu * nu);
      const double b_lu = (M.g[u] / M.g[l]) * b_ul;
      const double hn = kHP * nu / (4.0 * kPI);
      const double fu = A[u * ld + n], fl = A[l * ld + n];
      const double jm = hn * M.a[r] * fu;
      const double am = hn * (fl * b_lu - fu * b_ul);
      tab64[((long long)q * nodes + node) * 2] = jm;
      tab64[((long long)q * nodes + node) * 2 + 1] = am;
      // float pairs along T: this node is the lower half of pair i2 and the
      // upper half of pair i2 - 1
      const int n2p = M.n[2] - 1;
      float* base = reinterpret_cast<float*>(tab32 + ((long long)q * M.n[0] * M.n[1] +
                                                      (long long)i0 * M.n[1] + i1) * n2p);
      const float jf = (float)(jm * M.jk[q]), af = (float)(am * M.ak[q]);
      if (i2 < n2p) {
        base[4 * i2] = jf;
        base[4 * i2 + 1] = af;
      }
      if (i2 > 0) {
        base[4 * (i2 - 1) + 2] = jf;
        base[4 * (i2 - 1) + 3] = af;
      }
    }
    __syncwarp();
  }
}

}  // namespace

int launch_ot_build(const OTBuildArgs& M, double* tab64, float4* tab32, cudaStream_t stream) {
  const long long nodes = (long long)M.n[0] * M.n[1] * M.n[2];
  const size_t smem = (size_t)kBuildWarps * ot_warp_doubles(M.nlev) * sizeof(double);
  cudaError_t e = cudaFuncSetAttribute(ot_build_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return (int)e;
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ot_build_kernel, kBuildWarps * 32, smem);
  long long blocks = (long long)std::max(per_sm, 1) * sms;
  blocks = std::min(blocks, (nodes + kBuildWarps - 1) / kBuildWarps);
  ot_build_kernel<<<(unsigned)blocks, kBuildWarps * 32, smem, stream>>>(M, tab64, tab32, nodes);
  return (int)cudaGetLastError();
}

}  // namespace irt

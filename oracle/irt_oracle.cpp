// FP64 CPU oracle for the IRIS-SO synthetic-observation forward model.
//
// TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
// bench's CPU-baseline leg may load this library.  It shares no code, header,
// table or constant with the CUDA library; the two meet only in the seeded
// input arrays.
//
// The code follows the paper's definitions in the paper's order, one plain
// loop per definition, in double precision:
//   Sec. 3.1  transfer equations for the total [T] and continuum [C] intensity
//   Sec. 3.2  dust: alpha_D = kappa rho_gas, source function B_nu(T_dust)
//   Sec. 3.3  line emission / absorption with a Gaussian Doppler profile
//   Sec. 3.7  Einstein B relations
//   Sec. 5.10 LTE (Boltzmann) level populations n_u = N g_u e^{-E_u/kT} / Z(T)
//   Sec. 4.3  T_inf cut-off, Doppler-shifted line centre and dust Planck
//   Sec. 4.4  channel averaging; background and continuum at channel value
//   Sec. 4.5  fine velocity grid + Simpson rule for the total intensity
//   Sec. 4.8  formal step and smooth (TR first step, BDF2, ReLU) integration
//   Sec. 4.9  Rayleigh-Jeans and Planck brightness temperature;  Sec. 4.10
//             continuum subtraction (in intensity / T_RJ space, or in T_B space)
//   Sec. 5.10 density tracing ("simple observation"): tracer column density
//             per unit velocity
//   Sec. 4.6  selectively thin transfer (channel-averaged profile by erf, the
//             line sees the continuum only), Sec. 4.7 optically thin transfer
//             (direct integral: midpoint sum or Simpson), with the step
//             substitutions of Sec. 4.8
//
// Readings taken where the paper is silent (each is listed with its reason
// in the design notes):
//   * LTE populations with E_l = E_u - h nu / k (so S_line = B_nu(T) exactly)
//     and Z(T) = sum_J (2J+1) exp(-h B0 J(J+1) / kT) of a rigid rotor.
//   * Velocity <-> frequency in the radio convention nu(u) = nu_ul (1 - u/c),
//     positive = receding; the Doppler width uses nu_ul; the 1-D microturbulent
//     dispersion adds 2 sigma^2 to the squared width.
//   * Channel c spans [v0 + c dv, v0 + (c+1) dv]; fine points are spaced
//     dv / (2f) with shared edges (Table 4: delta v = dv / (2f)); f = 0 samples
//     the channel centre alone.
//   * Smooth integration places the background at the first sample node, so
//     it integrates (K-1) h; formal integration integrates K h.
//   * [D] = [C] - [B] (continuum excess over the background), [L] = [T] - [C].
//   * Thin modes: dust source and background at the channel centre; the
//     channel-averaged profile is the Gaussian's probability mass inside the
//     channel over the channel width in Hz (the printed erf expression is the
//     antiderivative); the selectively thin formal step of the total uses the
//     continuum after its own step (continuum solved first); the optically
//     thin Simpson sum covers the node pairs and a trapezoid closes an odd
//     last interval.
//   * Geometry: z view = one ray per cell column, samples at the cells;
//     oblique view = orthographic rays, chord split into K = ceil(chord/dx)
//     equal steps, samples at step midpoints, trilinear field sampling with
//     edge-clamped cell-centred values.
//
// Parity unpinned: the paper's own code (node placement, Planck at nu(u)) is
// not available; the readings above are the definition this oracle encodes.

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <type_traits>
#include <vector>

#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

// CODATA 2018 (h, k, c exact by definition of the SI)
const double H_PLANCK = 6.62607015e-27;   // erg s
const double K_BOLTZ = 1.380649e-16;      // erg / K
const double C_LIGHT = 2.99792458e10;     // cm / s
const double C_KMS = 2.99792458e5;        // km / s
const double AMU = 1.66053906660e-24;     // g
const double PI = 3.14159265358979323846;

// ---------------------------------------------------------------------------
// Forward-mode dual numbers (value + ND directional derivatives), so that one
// templated definition gives both the value and its exact gradient.
// ---------------------------------------------------------------------------
template <int ND>
struct Dual {
  double v;
  double d[ND];
  Dual() : v(0.0) { std::fill(d, d + ND, 0.0); }
  Dual(double x) : v(x) { std::fill(d, d + ND, 0.0); }  // NOLINT
};

inline double val(double x) { return x; }
template <int ND> inline double val(const Dual<ND>& x) { return x.v; }

template <int ND> Dual<ND> operator+(const Dual<ND>& a, const Dual<ND>& b) {
  Dual<ND> r; r.v = a.v + b.v; for (int i = 0; i < ND; ++i) r.d[i] = a.d[i] + b.d[i]; return r;
}
template <int ND> Dual<ND> operator-(const Dual<ND>& a, const Dual<ND>& b) {
  Dual<ND> r; r.v = a.v - b.v; for (int i = 0; i < ND; ++i) r.d[i] = a.d[i] - b.d[i]; return r;
}
template <int ND> Dual<ND> operator-(const Dual<ND>& a) {
  Dual<ND> r; r.v = -a.v; for (int i = 0; i < ND; ++i) r.d[i] = -a.d[i]; return r;
}
template <int ND> Dual<ND> operator*(const Dual<ND>& a, const Dual<ND>& b) {
  Dual<ND> r; r.v = a.v * b.v;
  for (int i = 0; i < ND; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i];
  return r;
}
template <int ND> Dual<ND> operator/(const Dual<ND>& a, const Dual<ND>& b) {
  Dual<ND> r; r.v = a.v / b.v;
  const double ib = 1.0 / b.v;
  for (int i = 0; i < ND; ++i) r.d[i] = (a.d[i] - r.v * b.d[i]) * ib;
  return r;
}
template <int ND> Dual<ND> operator+(const Dual<ND>& a, double b) { return a + Dual<ND>(b); }
template <int ND> Dual<ND> operator+(double a, const Dual<ND>& b) { return Dual<ND>(a) + b; }
template <int ND> Dual<ND> operator-(const Dual<ND>& a, double b) { return a - Dual<ND>(b); }
template <int ND> Dual<ND> operator-(double a, const Dual<ND>& b) { return Dual<ND>(a) - b; }
template <int ND> Dual<ND> operator*(const Dual<ND>& a, double b) {
  Dual<ND> r; r.v = a.v * b; for (int i = 0; i < ND; ++i) r.d[i] = a.d[i] * b; return r;
}
template <int ND> Dual<ND> operator*(double a, const Dual<ND>& b) { return b * a; }
template <int ND> Dual<ND> operator/(const Dual<ND>& a, double b) { return a * (1.0 / b); }
template <int ND> Dual<ND> operator/(double a, const Dual<ND>& b) { return Dual<ND>(a) / b; }

template <int ND> Dual<ND> exp(const Dual<ND>& a) {
  Dual<ND> r; r.v = std::exp(a.v); for (int i = 0; i < ND; ++i) r.d[i] = r.v * a.d[i]; return r;
}
template <int ND> Dual<ND> expm1(const Dual<ND>& a) {
  Dual<ND> r; r.v = std::expm1(a.v);
  const double e = std::exp(a.v);
  for (int i = 0; i < ND; ++i) r.d[i] = e * a.d[i];
  return r;
}
template <int ND> Dual<ND> sqrt(const Dual<ND>& a) {
  Dual<ND> r; r.v = std::sqrt(a.v);
  const double g = (r.v > 0.0) ? 0.5 / r.v : 0.0;
  for (int i = 0; i < ND; ++i) r.d[i] = g * a.d[i];
  return r;
}
inline double exp(double a) { return std::exp(a); }
inline double expm1(double a) { return std::expm1(a); }
inline double sqrt(double a) { return std::sqrt(a); }

// ReLU of Sec. 4.8; derivative 1 for x >= 0 and 0 otherwise.
template <class S> S relu(const S& x) { return (val(x) >= 0.0) ? x : S(0.0); }

// ---------------------------------------------------------------------------
// Problem description (plain data, filled from the flat argument arrays).
// ---------------------------------------------------------------------------
struct Line {
  double nu_ul, a_ul, e_u, b0, g_u, g_l, mass_amu, t_inf, sigma_turb;
};
struct DustP {
  double kappa, mu_amu;
};
struct VAxis {
  int nchan;
  double v0, dv;
  int f;
};
enum { FORMAL = 0, SMOOTH = 1 };
enum { MODE_THICK = 0, MODE_SELECTIVELY_THIN = 1, MODE_THIN = 2, MODE_DENSITY_TRACING = 3 };
enum { UNITS_TRJ = 0, UNITS_INTENSITY = 1, UNITS_TB = 2 };

// Sample values along one ray, in the order the ray travels (background side
// first, observer side last).
template <class S>
struct Sample {
  S n_h2, t_gas, t_dust, v_los, x_tr;
  S chi = S(0.5);   // H2 abundance per H nucleus (0.5: fully molecular); OT balance only
};

// ---------------------------------------------------------------------------
// Physics definitions
// ---------------------------------------------------------------------------

// Frequency observed at line-of-sight velocity u [km/s] (radio convention).
double nu_of_u(const Line& ln, double u) { return ln.nu_ul * (1.0 - u / C_KMS); }

// Planck's law, Sec. 3.2 (dust source function) and Sec. 4.9.
template <class S>
S planck(double nu, const S& T) {
  if (val(T) <= 0.0) return S(0.0);
  const double a = 2.0 * H_PLANCK * nu * nu * nu / (C_LIGHT * C_LIGHT);
  return a / expm1(H_PLANCK * nu / (K_BOLTZ * T));
}

// Rayleigh-Jeans temperature of an intensity at nu, Sec. 4.9.
// Planck brightness temperature of an intensity at nu, Sec. 4.9 (Planck's
// law solved for T); 0 for a non-positive intensity.
double brightness_temperature(double nu, double I) {
  if (!(I > 0.0)) return 0.0;
  return H_PLANCK * nu / (K_BOLTZ * std::log1p(2.0 * H_PLANCK * nu * nu * nu / (C_LIGHT * C_LIGHT * I)));
}

double rj_temperature(double nu, double I) {
  return C_LIGHT * C_LIGHT * I / (2.0 * K_BOLTZ * nu * nu);
}

// Rigid-rotor partition function, summed until a term falls below 1e-17 of
// the running sum.
template <class S>
S partition(const Line& ln, const S& T) {
  S z(0.0);
  for (int J = 0; J < 100000; ++J) {
    const double eJ = H_PLANCK * ln.b0 * J * (J + 1.0) / K_BOLTZ;   // E_J / k  [K]
    S term = (2.0 * J + 1.0) * exp(-eJ / T);
    z = z + term;
    if (J > 0 && val(term) < 1e-17 * val(z)) break;
  }
  return z;
}

// LTE level populations, Sec. 5.10:  n_i = N g_i exp(-E_i / kT) / Z(T).
template <class S>
void lte_populations(const Line& ln, const S& N, const S& T, S* n_u, S* n_l) {
  const double e_l = ln.e_u - H_PLANCK * ln.nu_ul / K_BOLTZ;
  const S z = partition(ln, T);
  *n_u = N * ln.g_u * exp(-ln.e_u / T) / z;
  *n_l = N * ln.g_l * exp(-e_l / T) / z;
}

// Frequency-integrated line coefficients j^L and alpha^L (Sec. 3.3) with the
// Einstein B relations of Sec. 3.7.  Zero above T_inf (Sec. 4.3).
template <class S>
void line_coefficients(const Line& ln, const Sample<S>& s, S* jL, S* aL) {
  if (val(s.t_gas) > ln.t_inf || val(s.t_gas) <= 0.0) {
    *jL = S(0.0);
    *aL = S(0.0);
    return;
  }
  const S N = s.x_tr * s.n_h2;
  S n_u, n_l;
  lte_populations(ln, N, s.t_gas, &n_u, &n_l);
  const double nu = ln.nu_ul;
  const double B_ul = C_LIGHT * C_LIGHT * ln.a_ul / (2.0 * H_PLANCK * nu * nu * nu);
  const double B_lu = (ln.g_u / ln.g_l) * B_ul;
  *jL = (H_PLANCK * nu / (4.0 * PI)) * n_u * ln.a_ul;
  *aL = (H_PLANCK * nu / (4.0 * PI)) * (n_l * B_lu - n_u * B_ul);
}

// ---------------------------------------------------------------------------
// Optically thin (OT) level balance (Sec. 3.4-3.6) and its coefficient grid
// (Sec. 4.2).  The level system of Sec. 3.5: for every level i but the
// ground state, what flows in equals what flows out,
//   sum_{j != i} [ n_j (C_ji + A_ji + B_ji J_ji) - n_i (C_ij + A_ij + B_ij J_ij) ] = 0,
// with A_ij = 0 for i < j, J the Planck intensity of a blackbody at the fixed
// background temperature T-bar at the transition frequency (the OT
// assumption), C_ij = sum over partners of K_ij n_partner, the excitation
// rates from the de-excitation rates by detailed balance at the gas
// temperature (Sec. 3.6), and the ground-state row replaced by sum_i n_i = N.
// ---------------------------------------------------------------------------
enum { PARTNER_H2 = 0, PARTNER_PH2 = 1, PARTNER_OH2 = 2, PARTNER_H = 3, PARTNER_HE = 4 };

// Caller's level model (energies, weights, radiative and collisional data),
// the layout of the ctypes structure OracleLevelModel.
struct LevelModel {
  int nlev;
  const double* energy_k;   // [nlev] E_i / k [K]
  const double* g;          // [nlev]
  int nrad;
  const int* rad_up;        // [nrad]
  const int* rad_lo;
  const double* a_ul;       // [nrad] Einstein A [1/s]
  const double* nu;         // [nrad] [Hz]
  int npartner;
  const int* partner;       // [npartner] PARTNER_*
  int ntemp;
  const double* coll_temp;  // [npartner][ntemp] ascending [K]
  int ncoll;
  const int* coll_up;       // [npartner][ncoll]
  const int* coll_lo;
  const double* k_ul;       // [npartner][ncoll][ntemp] de-excitation [cm^3/s]
  double t_rad;             // T-bar [K]
  double ortho_para;        // ortho-H2 / para-H2
  double x_he;              // He per H nucleus
};

// Number density of a collision partner [cm^-3] for total H nucleus density
// n_h and H2 abundance chi (H2 molecules per H nucleus; the rest of the H is
// atomic, Sec. 4.2).
double partner_density(const LevelModel& m, int kind, double n_h, double chi) {
  const double n_h2 = chi * n_h;
  switch (kind) {
    case PARTNER_H2: return n_h2;
    case PARTNER_PH2: return n_h2 / (1.0 + m.ortho_para);
    case PARTNER_OH2: return n_h2 * m.ortho_para / (1.0 + m.ortho_para);
    case PARTNER_H: return std::max(0.0, n_h * (1.0 - 2.0 * chi));
    case PARTNER_HE: return m.x_he * n_h;
  }
  return 0.0;
}

// Rate coefficient of partner p, collisional transition c at temperature T:
// linear interpolation between the tabulated temperatures, the end values
// held beyond them.
double rate_coefficient(const LevelModel& m, int p, int c, double T) {
  const double* tt = m.coll_temp + (int64_t)p * m.ntemp;
  const double* kk = m.k_ul + ((int64_t)p * m.ncoll + c) * m.ntemp;
  if (m.ntemp == 1 || T <= tt[0]) return kk[0];
  if (T >= tt[m.ntemp - 1]) return kk[m.ntemp - 1];
  int i = 0;
  while (T > tt[i + 1]) ++i;
  const double w = (T - tt[i]) / (tt[i + 1] - tt[i]);
  return kk[i] + w * (kk[i + 1] - kk[i]);
}

// Solve A x = b (n x n, row major) by Gaussian elimination with partial
// pivoting; A and b are overwritten.
void gauss_solve(int n, std::vector<double>& A, std::vector<double>& b, double* x) {
  for (int k = 0; k < n; ++k) {
    int p = k;
    for (int i = k + 1; i < n; ++i)
      if (std::fabs(A[(int64_t)i * n + k]) > std::fabs(A[(int64_t)p * n + k])) p = i;
    if (p != k) {
      for (int j = 0; j < n; ++j) std::swap(A[(int64_t)k * n + j], A[(int64_t)p * n + j]);
      std::swap(b[k], b[p]);
    }
    for (int i = k + 1; i < n; ++i) {
      const double f = A[(int64_t)i * n + k] / A[(int64_t)k * n + k];
      if (f == 0.0) continue;
      for (int j = k; j < n; ++j) A[(int64_t)i * n + j] -= f * A[(int64_t)k * n + j];
      b[i] -= f * b[k];
    }
  }
  for (int i = n - 1; i >= 0; --i) {
    double acc = b[i];
    for (int j = i + 1; j < n; ++j) acc -= A[(int64_t)i * n + j] * x[j];
    x[i] = acc / A[(int64_t)i * n + i];
  }
}

// Fractional level populations n_i / N of the OT balance at total H density
// n_h [cm^-3], H2 abundance chi and gas temperature T [K].
void ot_populations(const LevelModel& m, double n_h, double chi, double T, double* f) {
  const int n = m.nlev;
  // R[i][j]: rate i -> j per molecule in level i [1/s]
  std::vector<double> R((size_t)n * n, 0.0);
  for (int p = 0; p < m.npartner; ++p) {
    const double np = partner_density(m, m.partner[p], n_h, chi);
    for (int c = 0; c < m.ncoll; ++c) {
      const int u = m.coll_up[(int64_t)p * m.ncoll + c];
      const int l = m.coll_lo[(int64_t)p * m.ncoll + c];
      const double cul = rate_coefficient(m, p, c, T) * np;
      R[(size_t)u * n + l] += cul;
      // detailed balance (Sec. 3.6): K_lu = K_ul (g_u / g_l) exp(-(E_u - E_l) / kT)
      R[(size_t)l * n + u] += cul * (m.g[u] / m.g[l]) * std::exp(-(m.energy_k[u] - m.energy_k[l]) / T);
    }
  }
  for (int r = 0; r < m.nrad; ++r) {
    const int u = m.rad_up[r], l = m.rad_lo[r];
    const double nu = m.nu[r];
    // Einstein B relations (Sec. 3.6) and the background J = B_nu(T-bar)
    const double B_ul = C_LIGHT * C_LIGHT * m.a_ul[r] / (2.0 * H_PLANCK * nu * nu * nu);
    const double B_lu = (m.g[u] / m.g[l]) * B_ul;
    const double J = planck(nu, m.t_rad);
    R[(size_t)u * n + l] += m.a_ul[r] + B_ul * J;
    R[(size_t)l * n + u] += B_lu * J;
  }
  std::vector<double> M((size_t)n * n, 0.0), b(n, 0.0);
  for (int i = 1; i < n; ++i) {
    double out = 0.0;
    for (int j = 0; j < n; ++j) {
      if (j == i) continue;
      M[(size_t)i * n + j] = R[(size_t)j * n + i];   // inflow from j
      out += R[(size_t)i * n + j];
    }
    M[(size_t)i * n + i] = -out;
  }
  for (int j = 0; j < n; ++j) M[j] = 1.0;   // conservation row
  b[0] = 1.0;
  gauss_solve(n, M, b, f);
}

// Coefficient grid of Sec. 4.2 over (log10 n_H, chi, log10 T), uniform
// nodes per axis; per node and line, the frequency-integrated line emission
// and absorption coefficients per tracer molecule [cgs], j = (h nu / 4 pi)
// A f_u and alpha = (h nu / 4 pi)(f_l B_lu - f_u B_ul).
struct OTTable {
  int n[3];
  double lo[3], hi[3];
  int nlines;
  std::vector<double> nu;     // [nlines]
  std::vector<double> v;      // [nlines][n0][n1][n2][2]
};

double axis_value(const OTTable& t, int a, int i) {
  return t.lo[a] + (t.hi[a] - t.lo[a]) * i / (t.n[a] - 1);
}

// Trilinear interpolation of the grid at (log10 n_H, chi, log10 T) with the
// cell index clamped to the grid, so that outside the bounds the value
// continues linearly from the edge cell (Sec. 4.2).
void ot_lookup(const OTTable& t, int line, double n_h, double chi, double T, double* jt,
               double* at) {
  const double x[3] = {std::log10(n_h), chi, std::log10(T)};
  int i0[3];
  double w[3];
  for (int a = 0; a < 3; ++a) {
    const double u = (x[a] - t.lo[a]) / (t.hi[a] - t.lo[a]) * (t.n[a] - 1);
    int i = (int)std::floor(u);
    i = std::min(std::max(i, 0), t.n[a] - 2);
    i0[a] = i;
    w[a] = u - i;
  }
  double acc[2] = {0.0, 0.0};
  for (int c = 0; c < 8; ++c) {
    const int a0 = i0[0] + (c & 1), a1 = i0[1] + ((c >> 1) & 1), a2 = i0[2] + ((c >> 2) & 1);
    const double wc = ((c & 1) ? w[0] : 1.0 - w[0]) * ((c & 2) ? w[1] : 1.0 - w[1]) *
                      ((c & 4) ? w[2] : 1.0 - w[2]);
    const int64_t idx = ((((int64_t)line * t.n[0] + a0) * t.n[1] + a1) * t.n[2] + a2) * 2;
    acc[0] += wc * t.v[idx];
    acc[1] += wc * t.v[idx + 1];
  }
  *jt = acc[0];
  *at = acc[1];
}

struct OTLine {
  const OTTable* t;
  int line;
};

// Line coefficients of a sample: LTE (ot == nullptr), or the OT grid looked
// up at n_H = n_H2 / chi, with the tracer density N = x n_H2 (Sec. 4.3: the
// per-molecule coefficients times the tracer density).  Zero above T_inf.
template <class S>
void line_coeffs_for(const Line& ln, const OTLine* ot, const Sample<S>& s, S* jL, S* aL) {
  if (!ot) {
    line_coefficients(ln, s, jL, aL);
    return;
  }
  if constexpr (std::is_same<S, double>::value) {
    if (s.t_gas > ln.t_inf || s.t_gas <= 0.0 || s.n_h2 <= 0.0 || s.chi <= 0.0 || s.x_tr <= 0.0) {
      *jL = 0.0;
      *aL = 0.0;
      return;
    }
    double jt, at;
    ot_lookup(*ot->t, ot->line, s.n_h2 / s.chi, s.chi, s.t_gas, &jt, &at);
    const double N = s.x_tr * s.n_h2;
    *jL = N * jt;
    *aL = N * at;
  } else {
    *jL = S(0.0);   // not reached: the gradient oracle takes LTE only
    *aL = S(0.0);
  }
}

// Gaussian Doppler profile per unit frequency (Sec. 3.3), evaluated at the
// observed velocity u for a cell moving at v_los.  The width adds the 1-D
// microturbulent dispersion to the thermal one: b^2 = 2kT/m + 2 sigma^2.
template <class S>
S profile_per_hz(const Line& ln, const Sample<S>& s, double u) {
  const double m = ln.mass_amu * AMU;
  const S b2_cms = 2.0 * K_BOLTZ * s.t_gas / m
                 + 2.0 * (ln.sigma_turb * 1e5) * (ln.sigma_turb * 1e5);
  const S b_kms = sqrt(b2_cms) / 1e5;
  const S dnu_D = (ln.nu_ul / C_KMS) * b_kms;            // Doppler width [Hz]
  const S x = (u - s.v_los) / b_kms;                      // (nu - nu_0) / dnu_D
  return exp(-(x * x)) / (dnu_D * std::sqrt(PI));
}

// Dust absorption coefficient alpha_D = kappa rho_gas (Sec. 3.2).
template <class S>
S dust_alpha(const DustP& du, const Sample<S>& s) {
  return du.kappa * (s.n_h2 * (du.mu_amu * AMU));
}

// One formal step (Sec. 4.8): I <- I e^{-tau} + S (1 - e^{-tau}),
// tau = h alpha, S = j / alpha.
template <class S>
S formal_step(const S& I, const S& j, const S& a, double h) {
  if (val(a) == 0.0) return I + h * j;
  const S tau = h * a;
  const S src = j / a;
  return I * exp(-tau) + src * (-expm1(-tau));
}

// Transfer of one frequency along the ray (Sec. 4.8).  j[k], a[k] are the
// total coefficients at sample k; I0 is the background intensity.
template <class S>
S integrate(int mode, const std::vector<S>& j, const std::vector<S>& a, double h, const S& I0) {
  const int K = (int)j.size();
  if (mode == FORMAL) {
    S I = I0;
    for (int k = 0; k < K; ++k) I = formal_step(I, j[k], a[k], h);
    return I;
  }
  // smooth: node 0 carries the background; TR to node 1, BDF2 afterwards,
  // each step clamped at zero.
  if (K <= 1) return I0;
  S In = I0;
  S In1 = relu((h * (j[0] + j[1]) + (2.0 - h * a[0]) * In) / (2.0 + h * a[1]));
  for (int n = 0; n + 2 < K; ++n) {
    S In2 = relu((2.0 * h * j[n + 2] + 4.0 * In1 - In) / (3.0 + 2.0 * h * a[n + 2]));
    In = In1;
    In1 = In2;
  }
  return In1;
}

// Outputs of one ray: the five components per channel, in T_RJ [K] or in
// cgs intensity.  Order of the definition: coefficients per sample ->
// fine-velocity transfer of [T] -> Simpson channel average -> continuum [C]
// at channel centres -> background [B] -> [L] = [T] - [C], [D] = [C] - [B].
template <class S>
void ray_outputs(const Line& ln, const DustP& du, const VAxis& va, int mode, int units,
                 double t_bg, const std::vector<Sample<S>>& smp, double h,
                 S* oT, S* oC, S* oD, S* oL, S* oB, const OTLine* ot = nullptr) {
  const int K = (int)smp.size();
  const int nch = va.nchan;
  const int f = va.f;
  // per-sample frequency-independent coefficients
  std::vector<S> jL(K), aL(K), aD(K);
  for (int k = 0; k < K; ++k) {
    line_coeffs_for(ln, ot, smp[k], &jL[k], &aL[k]);
    aD[k] = dust_alpha(du, smp[k]);
  }
  // fine velocity grid (Sec. 4.5, Table 4)
  int nfine;
  double dvf, ufirst;
  if (f >= 1) {
    nfine = 2 * f * nch + 1;
    dvf = va.dv / (2.0 * f);
    ufirst = va.v0;
  } else {
    nfine = nch;
    dvf = va.dv;
    ufirst = va.v0 + 0.5 * va.dv;
  }
  std::vector<S> Ifine(nfine);
  std::vector<S> jt(K), at(K);
  for (int g = 0; g < nfine; ++g) {
    const double u = ufirst + g * dvf;
    const double nu = nu_of_u(ln, u);
    for (int k = 0; k < K; ++k) {
      // a sample without line coefficients (T outside (0, T_inf], or no
      // tracer) contributes no line; its profile is not needed
      const bool no_line = val(jL[k]) == 0.0 && val(aL[k]) == 0.0;
      const S phi = no_line ? S(0.0) : profile_per_hz(ln, smp[k], u);
      const S jD = aD[k] * planck(nu, smp[k].t_dust);
      jt[k] = jL[k] * phi + jD;
      at[k] = aL[k] * phi + aD[k];
    }
    Ifine[g] = integrate(mode, jt, at, h, S(planck(nu, t_bg)));
  }
  for (int c = 0; c < nch; ++c) {
    const double uc = va.v0 + (c + 0.5) * va.dv;
    const double nuc = nu_of_u(ln, uc);
    // channel average of the total intensity (Simpson over f panels)
    S Ibar(0.0);
    if (f >= 1) {
      for (int p = 0; p < f; ++p) {
        const int g = 2 * f * c + 2 * p;
        Ibar = Ibar + Ifine[g] + 4.0 * Ifine[g + 1] + Ifine[g + 2];
      }
      Ibar = Ibar / (6.0 * f);
    } else {
      Ibar = Ifine[c];
    }
    // continuum at the channel value (Sec. 4.4)
    for (int k = 0; k < K; ++k) {
      jt[k] = aD[k] * planck(nuc, smp[k].t_dust);
      at[k] = aD[k];
    }
    const S IB(planck(nuc, t_bg));
    const S IC = integrate(mode, jt, at, h, IB);
    S vT = Ibar, vC = IC, vB = IB;
    if (units == UNITS_TRJ) {
      const double s = rj_temperature(nuc, 1.0);
      vT = vT * s; vC = vC * s; vB = vB * s;
    } else if (units == UNITS_TB) {
      // subtraction in T_B space below ([L] = T_B(T) - T_B(C)); values only
      vT = S(brightness_temperature(nuc, val(vT)));
      vC = S(brightness_temperature(nuc, val(vC)));
      vB = S(brightness_temperature(nuc, val(vB)));
    }
    oT[c] = vT;
    oC[c] = vC;
    oB[c] = vB;
    oL[c] = vT - vC;
    oD[c] = vC - vB;
  }
}

// Channel average of the line profile per Hz over [u_lo, u_hi] (Sec. 4.6):
// the probability mass of the Gaussian inside the channel, divided by the
// channel width in Hz.
double channel_profile(const Line& ln, const Sample<double>& s, double u_lo, double u_hi) {
  const double m = ln.mass_amu * AMU;
  const double b2_cms = 2.0 * K_BOLTZ * s.t_gas / m
                      + 2.0 * (ln.sigma_turb * 1e5) * (ln.sigma_turb * 1e5);
  const double b_kms = std::sqrt(b2_cms) / 1e5;
  const double x_lo = (u_lo - s.v_los) / b_kms;
  const double x_hi = (u_hi - s.v_los) / b_kms;
  const double mass = 0.5 * (std::erf(x_hi) - std::erf(x_lo));
  const double width_hz = ln.nu_ul * (u_hi - u_lo) / C_KMS;
  return mass / width_hz;
}

// Intensities along the ray of one frequency with coefficients j[k], a[k]:
// formal, the value after each step k; smooth, the value at each node k
// (node 0 = background, TR to node 1, BDF2 after, ReLU on each step).
std::vector<double> path(int mode, const std::vector<double>& j, const std::vector<double>& a,
                         double h, double I0) {
  const int K = (int)j.size();
  std::vector<double> I(K);
  if (mode == FORMAL) {
    double x = I0;
    for (int k = 0; k < K; ++k) {
      x = formal_step(x, j[k], a[k], h);
      I[k] = x;
    }
    return I;
  }
  if (K >= 1) I[0] = I0;
  if (K >= 2) I[1] = relu((h * (j[0] + j[1]) + (2.0 - h * a[0]) * I[0]) / (2.0 + h * a[1]));
  for (int n = 0; n + 2 < K; ++n)
    I[n + 2] = relu((2.0 * h * j[n + 2] + 4.0 * I[n + 1] - I[n]) / (3.0 + 2.0 * h * a[n + 2]));
  return I;
}

// Direct integral of f over the ray (Sec. 4.7): formal = midpoint sum over
// the K steps; smooth = composite Simpson over the K nodes (spacing h), the
// last interval by the trapezoid rule when K - 1 is odd.
double direct_integral(int mode, const std::vector<double>& f, double h) {
  const int K = (int)f.size();
  double acc = 0.0;
  if (mode == FORMAL) {
    for (int k = 0; k < K; ++k) acc += h * f[k];
    return acc;
  }
  if (K <= 1) return 0.0;              // no interval (a missed ray has no samples)
  const int M = K - 1;                 // intervals
  const int Ms = (M % 2 == 0) ? M : M - 1;   // covered by Simpson panels
  for (int p = 0; p + 2 <= Ms; p += 2) acc += (h / 3.0) * (f[p] + 4.0 * f[p + 1] + f[p + 2]);
  if (Ms < M) acc += 0.5 * h * (f[M - 1] + f[M]);
  return acc;
}

// Outputs of one ray in the selectively thin or optically thin mode (no
// fine velocities: every channel is solved at its own averaged coefficients).
void ray_outputs_thin(const Line& ln, const DustP& du, const VAxis& va, int transfer, int mode,
                      int units, double t_bg, const std::vector<Sample<double>>& smp, double h,
                      double* oT, double* oC, double* oD, double* oL, double* oB,
                      const OTLine* ot = nullptr) {
  const int K = (int)smp.size();
  std::vector<double> jL(K), aL(K), aD(K);
  for (int k = 0; k < K; ++k) {
    line_coeffs_for(ln, ot, smp[k], &jL[k], &aL[k]);
    aD[k] = dust_alpha(du, smp[k]);
  }
  std::vector<double> jLb(K), aLb(K), jD(K), jT(K), aT(K);
  for (int c = 0; c < va.nchan; ++c) {
    const double u_lo = va.v0 + c * va.dv, u_hi = u_lo + va.dv;
    const double uc = va.v0 + (c + 0.5) * va.dv;
    const double nuc = nu_of_u(ln, uc);
    for (int k = 0; k < K; ++k) {
      const bool no_line = jL[k] == 0.0 && aL[k] == 0.0;
      const double phib = no_line ? 0.0 : channel_profile(ln, smp[k], u_lo, u_hi);
      jLb[k] = jL[k] * phib;
      aLb[k] = aL[k] * phib;
      jD[k] = aD[k] * planck(nuc, smp[k].t_dust);
    }
    const double IB = planck(nuc, t_bg);
    double IT, IC;
    if (transfer == MODE_THIN) {
      // absorption and stimulation ignored: I = I_bg + integral of j
      for (int k = 0; k < K; ++k) jT[k] = jLb[k] + jD[k];
      IT = IB + direct_integral(mode, jT, h);
      IC = IB + direct_integral(mode, jD, h);
    } else {
      // continuum first, then the total with j = jL + jD - aL I_C, a = aD
      const std::vector<double> Ic = path(mode, jD, aD, h, IB);
      for (int k = 0; k < K; ++k) {
        jT[k] = jLb[k] + jD[k] - aLb[k] * Ic[k];
        aT[k] = aD[k];
      }
      const std::vector<double> It = path(mode, jT, aT, h, IB);
      IC = (K >= 1) ? Ic[K - 1] : IB;
      IT = (K >= 1) ? It[K - 1] : IB;
    }
    double vT = IT, vC = IC, vB = IB;
    if (units == UNITS_TRJ) {
      const double sc = rj_temperature(nuc, 1.0);
      vT *= sc; vC *= sc; vB *= sc;
    } else if (units == UNITS_TB) {
      vT = brightness_temperature(nuc, vT);
      vC = brightness_temperature(nuc, vC);
      vB = brightness_temperature(nuc, vB);
    }
    oT[c] = vT;
    oC[c] = vC;
    oB[c] = vB;
    oL[c] = vT - vC;
    oD[c] = vC - vB;
  }
}

// Density-tracing cube of one ray (Sec. 5.10): the tracer column density per
// unit velocity [cm^-2 per km/s] in each channel, every sample spreading its
// column x n_H2 h over velocity with the line's Doppler profile (channel
// average: Gaussian mass in the channel over dv); summed as the optically
// thin integral (midpoint or Simpson).  No temperature cut, background or
// dust.  Written to [T] and [L]; [C], [D], [B] are zero.
void ray_outputs_density(const Line& ln, const VAxis& va, int mode,
                         const std::vector<Sample<double>>& smp, double h, double* oT,
                         double* oC, double* oD, double* oL, double* oB) {
  const int K = (int)smp.size();
  const double m = ln.mass_amu * AMU;
  std::vector<double> f(K);
  for (int c = 0; c < va.nchan; ++c) {
    const double u_lo = va.v0 + c * va.dv, u_hi = u_lo + va.dv;
    for (int k = 0; k < K; ++k) {
      const double b = std::sqrt(2.0 * K_BOLTZ * smp[k].t_gas / m
                                 + 2.0 * (ln.sigma_turb * 1e5) * (ln.sigma_turb * 1e5)) / 1e5;
      const double mass = 0.5 * (std::erf((u_hi - smp[k].v_los) / b)
                                 - std::erf((u_lo - smp[k].v_los) / b));
      f[k] = smp[k].x_tr * smp[k].n_h2 * mass / va.dv;
    }
    const double col = direct_integral(mode, f, h);
    oT[c] = col;
    oL[c] = col;
    oC[c] = 0.0;
    oD[c] = 0.0;
    oB[c] = 0.0;
  }
}

// ---------------------------------------------------------------------------
// Geometry
// ---------------------------------------------------------------------------
struct Grid {
  const double* f[5];  // n_h2, t_gas, t_dust, v_los, x_tr, each [z][y][x]
  int nx, ny, nz;
  double dx;
  const double* chi = nullptr;   // H2 abundance per H nucleus, or nullptr (0.5)
  double at(int q, int x, int y, int z) const {
    return f[q][((int64_t)z * ny + y) * nx + x];
  }
  double at_field(const double* a, int x, int y, int z) const {
    return a[((int64_t)z * ny + y) * nx + x];
  }
};

struct ViewP {
  double theta, phi;
  int npx, npy;
  double pixel;
  int trilinear;
};

// Ray through the box for pixel (px, py): origin o, direction d, chord
// [t_in, t_out].  Returns false if the ray misses the box.
bool ray_chord(const Grid& g, const ViewP& v, int px, int py, double o[3], double d[3],
               double* t_in, double* t_out) {
  const double st = std::sin(v.theta), ct = std::cos(v.theta);
  const double sp = std::sin(v.phi), cp = std::cos(v.phi);
  d[0] = st * cp; d[1] = st * sp; d[2] = ct;
  const double et[3] = {ct * cp, ct * sp, -st};
  const double ep[3] = {-sp, cp, 0.0};
  const double L[3] = {g.nx * g.dx, g.ny * g.dx, g.nz * g.dx};
  const double a = (px - 0.5 * (v.npx - 1)) * v.pixel;
  const double b = (py - 0.5 * (v.npy - 1)) * v.pixel;
  for (int i = 0; i < 3; ++i) o[i] = 0.5 * L[i] + a * et[i] + b * ep[i];
  double lo = -INFINITY, hi = INFINITY;
  for (int i = 0; i < 3; ++i) {
    if (d[i] == 0.0) {
      if (o[i] < 0.0 || o[i] > L[i]) return false;
      continue;
    }
    double t0 = (0.0 - o[i]) / d[i], t1 = (L[i] - o[i]) / d[i];
    if (t0 > t1) std::swap(t0, t1);
    lo = std::max(lo, t0);
    hi = std::min(hi, t1);
  }
  if (!(hi > lo)) return false;
  *t_in = lo;
  *t_out = hi;
  return true;
}

// Trilinear interpolation of the raw field q at position r [cm], cell-centred
// values, indices clamped to the grid (edge extension).
double trilinear_field(const Grid& g, const double* field, const double r[3]) {
  const int n[3] = {g.nx, g.ny, g.nz};
  int i0[3], i1[3];
  double w[3];
  for (int a = 0; a < 3; ++a) {
    const double s = r[a] / g.dx - 0.5;
    const double fl = std::floor(s);
    w[a] = s - fl;
    int lo = (int)fl;
    i0[a] = std::min(std::max(lo, 0), n[a] - 1);
    i1[a] = std::min(std::max(lo + 1, 0), n[a] - 1);
  }
  double acc = 0.0;
  for (int c = 0; c < 8; ++c) {
    const int ix = (c & 1) ? i1[0] : i0[0];
    const int iy = (c & 2) ? i1[1] : i0[1];
    const int iz = (c & 4) ? i1[2] : i0[2];
    const double wx = (c & 1) ? w[0] : 1.0 - w[0];
    const double wy = (c & 2) ? w[1] : 1.0 - w[1];
    const double wz = (c & 4) ? w[2] : 1.0 - w[2];
    acc += wx * wy * wz * g.at_field(field, ix, iy, iz);
  }
  return acc;
}

double trilinear(const Grid& g, int q, const double r[3]) { return trilinear_field(g, g.f[q], r); }

// Samples of one ray.  z view: the cells (px, py, k) for k = 0..nz-1 with
// h = dx.  Oblique: K = ceil(chord/dx) midpoint samples of a uniform split.
void ray_samples(const Grid& g, const ViewP& v, int px, int py,
                 std::vector<Sample<double>>* smp, double* h) {
  smp->clear();
  if (v.trilinear == 0 || v.trilinear == 2) {
    // z view: cells k = 0 .. nz-1 of the column; radial view of an
    // observer-centred [r][b][l] tensor (Sec. 2.2): the column read from the
    // far end of the radial axis (r = nz-1) to the observer (r = 0)
    *h = g.dx;
    for (int k = 0; k < g.nz; ++k) {
      const int z = (v.trilinear == 2) ? g.nz - 1 - k : k;
      Sample<double> s;
      s.n_h2 = g.at(0, px, py, z);
      s.t_gas = g.at(1, px, py, z);
      s.t_dust = g.at(2, px, py, z);
      s.v_los = g.at(3, px, py, z);
      s.x_tr = g.at(4, px, py, z);
      if (g.chi) s.chi = g.at_field(g.chi, px, py, z);
      smp->push_back(s);
    }
    return;
  }
  double o[3], d[3], t0, t1;
  if (!ray_chord(g, v, px, py, o, d, &t0, &t1)) {
    *h = 0.0;
    return;
  }
  const double chord = t1 - t0;
  const int K = (int)std::ceil(chord / g.dx - 1e-9);
  if (K <= 0) { *h = 0.0; return; }
  *h = chord / K;
  for (int k = 0; k < K; ++k) {
    const double t = t0 + (k + 0.5) * (*h);
    const double r[3] = {o[0] + t * d[0], o[1] + t * d[1], o[2] + t * d[2]};
    Sample<double> s;
    s.n_h2 = trilinear(g, 0, r);
    s.t_gas = trilinear(g, 1, r);
    s.t_dust = trilinear(g, 2, r);
    s.v_los = trilinear(g, 3, r);
    s.x_tr = trilinear(g, 4, r);
    if (g.chi) s.chi = trilinear_field(g, g.chi, r);
    smp->push_back(s);
  }
}

// The cells each sample of a ray draws on and their weights (the sample
// value of every field is the weighted sum of these cells' values): the one
// cell of the z and radial views, the eight trilinear corners (index clamped,
// so a corner may repeat) of the oblique view.  Same order and positions as
// ray_samples.
void ray_stencils(const Grid& g, const ViewP& v, int px, int py,
                  std::vector<std::vector<std::pair<int64_t, double>>>* st) {
  st->clear();
  auto cell = [&](int x, int y, int z) { return ((int64_t)z * g.ny + y) * g.nx + x; };
  if (v.trilinear == 0 || v.trilinear == 2) {
    for (int k = 0; k < g.nz; ++k) {
      const int z = (v.trilinear == 2) ? g.nz - 1 - k : k;
      st->push_back({{cell(px, py, z), 1.0}});
    }
    return;
  }
  double o[3], d[3], t0, t1;
  if (!ray_chord(g, v, px, py, o, d, &t0, &t1)) return;
  const double chord = t1 - t0;
  const int K = (int)std::ceil(chord / g.dx - 1e-9);
  if (K <= 0) return;
  const double h = chord / K;
  const int n[3] = {g.nx, g.ny, g.nz};
  for (int k = 0; k < K; ++k) {
    const double t = t0 + (k + 0.5) * h;
    const double r[3] = {o[0] + t * d[0], o[1] + t * d[1], o[2] + t * d[2]};
    int i0[3], i1[3];
    double w[3];
    for (int a = 0; a < 3; ++a) {
      const double sa = r[a] / g.dx - 0.5;
      const double fl = std::floor(sa);
      w[a] = sa - fl;
      i0[a] = std::min(std::max((int)fl, 0), n[a] - 1);
      i1[a] = std::min(std::max((int)fl + 1, 0), n[a] - 1);
    }
    std::vector<std::pair<int64_t, double>> cs;
    for (int c = 0; c < 8; ++c) {
      const int ix = (c & 1) ? i1[0] : i0[0];
      const int iy = (c & 2) ? i1[1] : i0[1];
      const int iz = (c & 4) ? i1[2] : i0[2];
      const double wc = ((c & 1) ? w[0] : 1.0 - w[0]) * ((c & 2) ? w[1] : 1.0 - w[1]) *
                        ((c & 4) ? w[2] : 1.0 - w[2]);
      cs.push_back({cell(ix, iy, iz), wc});
    }
    st->push_back(cs);
  }
}

Line line_from(const double* p) {
  Line l;
  l.nu_ul = p[0]; l.a_ul = p[1]; l.e_u = p[2]; l.b0 = p[3]; l.g_u = p[4]; l.g_l = p[5];
  l.mass_amu = p[6]; l.t_inf = p[7]; l.sigma_turb = p[8];
  return l;
}
DustP dust_from(const double* p) { DustP d; d.kappa = p[0]; d.mu_amu = p[1]; return d; }
VAxis vaxis_from(int nchan, double v0, double dv, int f) {
  VAxis v; v.nchan = nchan; v.v0 = v0; v.dv = dv; v.f = f; return v;
}

}  // namespace

// ===========================================================================
// Flat C entry points (loaded with ctypes by the tests).
//   line[9] = nu_ul_hz, a_ul_s, e_u_k, b0_hz, g_u, g_l, mass_amu, t_inf_k,
//             sigma_turb_kms
//   dust[2] = kappa_cm2_per_g_gas, mu_mass_per_h2_amu
//   view[6] = theta_rad, phi_rad, npx, npy, pixel_cm, trilinear
// ===========================================================================
extern "C" {

int oracle_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

double oracle_planck(double nu, double T) { return planck(nu, T); }
double oracle_partition(const double* line, double T) { return partition(line_from(line), T); }

// Per-sample coefficients: out[0..5] = n_u, n_l, j^L, alpha^L, alpha^D, b [km/s]
void oracle_sample_coeffs(const double* line, const double* dust, double n_h2, double t_gas,
                          double x_tr, double* out) {
  const Line ln = line_from(line);
  const DustP du = dust_from(dust);
  Sample<double> s{n_h2, t_gas, t_gas, 0.0, x_tr};
  double nu_, nl_;
  lte_populations(ln, x_tr * n_h2, t_gas, &nu_, &nl_);
  double jL, aL;
  line_coefficients(ln, s, &jL, &aL);
  out[0] = nu_; out[1] = nl_; out[2] = jL; out[3] = aL; out[4] = dust_alpha(du, s);
  const double m = ln.mass_amu * AMU;
  out[5] = std::sqrt(2.0 * K_BOLTZ * t_gas / m + 2.0 * (ln.sigma_turb * 1e5) * (ln.sigma_turb * 1e5)) / 1e5;
}

// Profile per Hz at observed velocity u for a sample (t_gas, v_los).
double oracle_profile(const double* line, double t_gas, double v_los, double u) {
  Sample<double> s{1.0, t_gas, t_gas, v_los, 1.0};
  return profile_per_hz(line_from(line), s, u);
}

// One ray given explicitly by its K samples (arrays in travel order) and the
// step h [cm].  Outputs out_*[nchan].
void oracle_ray(const double* line, const double* dust, int nchan, double v0, double dv, int f,
                int integration, int units, double t_bg, int K, const double* n_h2,
                const double* t_gas, const double* t_dust, const double* v_los,
                const double* x_tr, double h, double* oT, double* oC, double* oD, double* oL,
                double* oB) {
  std::vector<Sample<double>> smp(K);
  for (int k = 0; k < K; ++k) smp[k] = {n_h2[k], t_gas[k], t_dust[k], v_los[k], x_tr[k]};
  ray_outputs(line_from(line), dust_from(dust), vaxis_from(nchan, v0, dv, f), integration, units,
              t_bg, smp, h, oT, oC, oD, oL, oB);
}

// One ray in a thin transfer mode (transfer = 1 selectively thin, 2
// optically thin); arguments as oracle_ray.
void oracle_ray_thin(const double* line, const double* dust, int nchan, double v0, double dv,
                     int transfer, int integration, int units, double t_bg, int K,
                     const double* n_h2, const double* t_gas, const double* t_dust,
                     const double* v_los, const double* x_tr, double h, double* oT, double* oC,
                     double* oD, double* oL, double* oB) {
  std::vector<Sample<double>> smp(K);
  for (int k = 0; k < K; ++k) smp[k] = {n_h2[k], t_gas[k], t_dust[k], v_los[k], x_tr[k]};
  if (transfer == MODE_DENSITY_TRACING)
    ray_outputs_density(line_from(line), vaxis_from(nchan, v0, dv, 0), integration, smp, h, oT,
                        oC, oD, oL, oB);
  else
    ray_outputs_thin(line_from(line), dust_from(dust), vaxis_from(nchan, v0, dv, 0), transfer,
                     integration, units, t_bg, smp, h, oT, oC, oD, oL, oB);
}

// Sample list of a pixel: returns K (<= kmax), fills h and samples.
int oracle_ray_samples(const double* const* fields, int nx, int ny, int nz, double cell_cm,
                       const double* view, int px, int py, int kmax, double* h_out,
                       double* samples /* [kmax][5] */) {
  Grid g;
  for (int q = 0; q < 5; ++q) g.f[q] = fields[q];
  g.nx = nx; g.ny = ny; g.nz = nz; g.dx = cell_cm;
  ViewP v{view[0], view[1], (int)view[2], (int)view[3], view[4], (int)view[5]};
  std::vector<Sample<double>> smp;
  double h = 0.0;
  ray_samples(g, v, px, py, &smp, &h);
  *h_out = h;
  const int K = (int)smp.size();
  for (int k = 0; k < K && k < kmax; ++k) {
    samples[5 * k + 0] = smp[k].n_h2;
    samples[5 * k + 1] = smp[k].t_gas;
    samples[5 * k + 2] = smp[k].t_dust;
    samples[5 * k + 3] = smp[k].v_los;
    samples[5 * k + 4] = smp[k].x_tr;
  }
  return K;
}

// Render a list of pixels.  pix[2*i], pix[2*i+1] = (px, py); outputs are
// [npix][nchan] per component (NULL = not wanted).
int oracle_render_levels(const double* const* fields, const double* chi, int nx, int ny, int nz,
                         double cell_cm, const double* line, const double* dust,
                         const double* view, int nchan, double v0, double dv, int f,
                         int transfer, int integration, int units, double t_bg, int npix,
                         const int* pix, double* oT, double* oC, double* oD, double* oL,
                         double* oB, const void* ot_table, int ot_line);

int oracle_render(const double* const* fields, int nx, int ny, int nz, double cell_cm,
                  const double* line, const double* dust, const double* view, int nchan,
                  double v0, double dv, int f, int transfer, int integration, int units,
                  double t_bg, int npix, const int* pix, double* oT, double* oC, double* oD,
                  double* oL, double* oB) {
  return oracle_render_levels(fields, nullptr, nx, ny, nz, cell_cm, line, dust, view, nchan, v0,
                              dv, f, transfer, integration, units, t_bg, npix, pix, oT, oC, oD,
                              oL, oB, nullptr, 0);
}

// oracle_render with the line coefficients of an OT grid (ot_table from
// oracle_ot_table_build, line index ot_line; NULL = LTE) and an optional H2
// abundance field chi [z][y][x] (NULL = 0.5 everywhere).
int oracle_render_levels(const double* const* fields, const double* chi, int nx, int ny, int nz,
                         double cell_cm, const double* line, const double* dust,
                         const double* view, int nchan, double v0, double dv, int f,
                         int transfer, int integration, int units, double t_bg, int npix,
                         const int* pix, double* oT, double* oC, double* oD, double* oL,
                         double* oB, const void* ot_table, int ot_line) {
  Grid g;
  for (int q = 0; q < 5; ++q) g.f[q] = fields[q];
  g.nx = nx; g.ny = ny; g.nz = nz; g.dx = cell_cm;
  g.chi = chi;
  OTLine otl{static_cast<const OTTable*>(ot_table), ot_line};
  const OTLine* ot = ot_table ? &otl : nullptr;
  const ViewP v{view[0], view[1], (int)view[2], (int)view[3], view[4], (int)view[5]};
  const Line ln = line_from(line);
  const DustP du = dust_from(dust);
  const VAxis va = vaxis_from(nchan, v0, dv, f);
#pragma omp parallel for schedule(dynamic, 1)
  for (int i = 0; i < npix; ++i) {
    std::vector<Sample<double>> smp;
    double h = 0.0;
    ray_samples(g, v, pix[2 * i], pix[2 * i + 1], &smp, &h);
    std::vector<double> T(nchan), C(nchan), D(nchan), L(nchan), B(nchan);
    if (transfer == MODE_THICK)
      ray_outputs(ln, du, va, integration, units, t_bg, smp, h, T.data(), C.data(), D.data(),
                  L.data(), B.data(), ot);
    else if (transfer == MODE_DENSITY_TRACING)
      ray_outputs_density(ln, va, integration, smp, h, T.data(), C.data(), D.data(), L.data(),
                          B.data());
    else
      ray_outputs_thin(ln, du, va, transfer, integration, units, t_bg, smp, h, T.data(),
                       C.data(), D.data(), L.data(), B.data(), ot);
    const int64_t off = (int64_t)i * nchan;
    for (int c = 0; c < nchan; ++c) {
      if (oT) oT[off + c] = T[c];
      if (oC) oC[off + c] = C[c];
      if (oD) oD[off + c] = D[c];
      if (oL) oL[off + c] = L[c];
      if (oB) oB[off + c] = B[c];
    }
  }
  return 0;
}

// Gradient of Loss = mean over all voxels of ([L] - target)^2 for the z view,
// with respect to n_H2, T_gas and v_los of every cell, by forward-mode dual
// numbers through the whole definition.  target is [nchan][ny][nx]; grads are
// [nz][ny][nx].  Only pixels in pix[] contribute (the others are taken to
// match their target exactly).  Returns the loss over those pixels.
double oracle_loss_grad_zview(const double* const* fields, int nx, int ny, int nz,
                              double cell_cm, const double* line, const double* dust, int nchan,
                              double v0, double dv, int f, int integration, int units,
                              double t_bg, const double* target, int npix, const int* pix,
                              double* g_n, double* g_t, double* g_v) {
  constexpr int CELLS = 8;
  constexpr int ND = 3 * CELLS;
  typedef Dual<ND> D;
  Grid g;
  for (int q = 0; q < 5; ++q) g.f[q] = fields[q];
  g.nx = nx; g.ny = ny; g.nz = nz; g.dx = cell_cm;
  const Line ln = line_from(line);
  const DustP du = dust_from(dust);
  const VAxis va = vaxis_from(nchan, v0, dv, f);
  const double nvox = (double)nchan * nx * ny;
  double loss = 0.0;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : loss)
  for (int i = 0; i < npix; ++i) {
    const int px = pix[2 * i], py = pix[2 * i + 1];
    std::vector<D> T(nchan), C(nchan), Dd(nchan), L(nchan), B(nchan);
    double lray = 0.0;
    for (int k0 = 0; k0 < nz; k0 += CELLS) {
      std::vector<Sample<D>> smp(nz);
      for (int k = 0; k < nz; ++k) {
        smp[k].n_h2 = D(g.at(0, px, py, k));
        smp[k].t_gas = D(g.at(1, px, py, k));
        smp[k].t_dust = D(g.at(2, px, py, k));
        smp[k].v_los = D(g.at(3, px, py, k));
        smp[k].x_tr = D(g.at(4, px, py, k));
        if (k >= k0 && k < k0 + CELLS) {
          smp[k].n_h2.d[3 * (k - k0) + 0] = 1.0;
          smp[k].t_gas.d[3 * (k - k0) + 1] = 1.0;
          smp[k].v_los.d[3 * (k - k0) + 2] = 1.0;
        }
      }
      ray_outputs(ln, du, va, integration, units, t_bg, smp, g.dx, T.data(), C.data(),
                  Dd.data(), L.data(), B.data());
      D l(0.0);
      for (int c = 0; c < nchan; ++c) {
        const D r = L[c] - target[((int64_t)c * ny + py) * nx + px];
        l = l + r * r;
      }
      l = l / nvox;
      if (k0 == 0) lray = l.v;
      for (int k = k0; k < std::min(nz, k0 + CELLS); ++k) {
        const int64_t idx = ((int64_t)k * ny + py) * nx + px;
        g_n[idx] = l.d[3 * (k - k0) + 0];
        g_t[idx] = l.d[3 * (k - k0) + 1];
        g_v[idx] = l.d[3 * (k - k0) + 2];
      }
    }
    loss += lray;
  }
  return loss;
}

// ---------------------------------------------------------------------------
// OT level balance and its grid (Sec. 3.4-3.6, 4.2)
// ---------------------------------------------------------------------------
// Fractional populations n_i / N at (n_H, chi, T); f_out[nlev].
void oracle_ot_populations(const LevelModel* m, double n_h, double chi, double T, double* f_out) {
  ot_populations(*m, n_h, chi, T, f_out);
}

// Build the grid: axes n[3] nodes, lo[3], hi[3] (log10 n_H, chi, log10 T);
// lines[nlines] = radiative transition indices of the model.  Returns an
// opaque table (oracle_ot_table_free releases it).
void* oracle_ot_table_build(const LevelModel* m, const int* n, const double* lo,
                            const double* hi, int nlines, const int* lines) {
  OTTable* t = new OTTable();
  for (int a = 0; a < 3; ++a) {
    t->n[a] = n[a];
    t->lo[a] = lo[a];
    t->hi[a] = hi[a];
  }
  t->nlines = nlines;
  for (int q = 0; q < nlines; ++q) t->nu.push_back(m->nu[lines[q]]);
  const int64_t nodes = (int64_t)n[0] * n[1] * n[2];
  t->v.assign((size_t)nlines * nodes * 2, 0.0);
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t node = 0; node < nodes; ++node) {
    const int i2 = (int)(node % n[2]);
    const int i1 = (int)((node / n[2]) % n[1]);
    const int i0 = (int)(node / ((int64_t)n[2] * n[1]));
    const double n_h = std::pow(10.0, axis_value(*t, 0, i0));
    const double chi = axis_value(*t, 1, i1);
    const double T = std::pow(10.0, axis_value(*t, 2, i2));
    std::vector<double> f(m->nlev);
    ot_populations(*m, n_h, chi, T, f.data());
    for (int q = 0; q < nlines; ++q) {
      const int r = lines[q];
      const int u = m->rad_up[r], l = m->rad_lo[r];
      const double nu = m->nu[r];
      const double B_ul = C_LIGHT * C_LIGHT * m->a_ul[r] / (2.0 * H_PLANCK * nu * nu * nu);
      const double B_lu = (m->g[u] / m->g[l]) * B_ul;
      const double hn = H_PLANCK * nu / (4.0 * PI);
      const int64_t idx = ((int64_t)q * nodes + node) * 2;
      t->v[idx] = hn * m->a_ul[r] * f[u];
      t->v[idx + 1] = hn * (f[l] * B_lu - f[u] * B_ul);
    }
  }
  return t;
}

// A grid holding given values [nlines][n0][n1][n2][2] (for checks of the
// lookup on tables with known content); nu_hz[nlines].
void* oracle_ot_table_from_values(const int* n, const double* lo, const double* hi, int nlines,
                                  const double* nu_hz, const double* values) {
  OTTable* t = new OTTable();
  for (int a = 0; a < 3; ++a) {
    t->n[a] = n[a];
    t->lo[a] = lo[a];
    t->hi[a] = hi[a];
  }
  t->nlines = nlines;
  t->nu.assign(nu_hz, nu_hz + nlines);
  const size_t cnt = (size_t)nlines * n[0] * n[1] * n[2] * 2;
  t->v.assign(values, values + cnt);
  return t;
}

// Copy of the grid values [nlines][n0][n1][n2][2] (j, alpha per molecule).
void oracle_ot_table_values(const void* t, double* out) {
  const OTTable* tt = static_cast<const OTTable*>(t);
  std::copy(tt->v.begin(), tt->v.end(), out);
}

void oracle_ot_lookup(const void* t, int line, double n_h, double chi, double T, double* out) {
  ot_lookup(*static_cast<const OTTable*>(t), line, n_h, chi, T, &out[0], &out[1]);
}

void oracle_ot_table_free(void* t) { delete static_cast<OTTable*>(t); }

// Gradient of Loss = mean over all voxels of ([L] - target)^2 with respect to
// n_H2, T_gas and v_los of the listed cells (cells[3 i] = x, y, z), for any
// view (z, oblique, radial) and integrator, by forward-mode dual numbers
// through the whole definition: each sample's field values carry the
// derivatives of the listed cells through the sample's stencil weights.
// target is [nchan][npy][npx]; g_*[ncell].  Returns the loss.
double oracle_loss_grad_cells(const double* const* fields, int nx, int ny, int nz,
                              double cell_cm, const double* line, const double* dust,
                              const double* view, int nchan, double v0, double dv, int f,
                              int integration, int units, double t_bg, const double* target,
                              int ncell, const int* cells, double* g_n, double* g_t,
                              double* g_v) {
  constexpr int CELLS = 8;
  constexpr int ND = 3 * CELLS;
  typedef Dual<ND> D;
  Grid g;
  for (int q = 0; q < 5; ++q) g.f[q] = fields[q];
  g.nx = nx; g.ny = ny; g.nz = nz; g.dx = cell_cm;
  const ViewP v{view[0], view[1], (int)view[2], (int)view[3], view[4], (int)view[5]};
  const Line ln = line_from(line);
  const DustP du = dust_from(dust);
  const VAxis va = vaxis_from(nchan, v0, dv, f);
  const int npix = v.npx * v.npy;
  const double nvox = (double)nchan * npix;
  double loss = 0.0;
  for (int i = 0; i < ncell; ++i) g_n[i] = g_t[i] = g_v[i] = 0.0;
  for (int c0 = 0; c0 < ncell; c0 += CELLS) {
    const int nc = std::min(CELLS, ncell - c0);
    std::vector<int64_t> seed(nc);
    for (int c = 0; c < nc; ++c)
      seed[c] = ((int64_t)cells[3 * (c0 + c) + 2] * ny + cells[3 * (c0 + c) + 1]) * nx +
                cells[3 * (c0 + c)];
    std::vector<double> acc(ND, 0.0);
    double lsum = 0.0;
#pragma omp parallel
    {
      std::vector<double> acc_t(ND, 0.0);
      double l_t = 0.0;
#pragma omp for schedule(dynamic, 4)
      for (int p = 0; p < npix; ++p) {
        const int px = p % v.npx, py = p / v.npx;
        std::vector<Sample<double>> smp;
        double h = 0.0;
        ray_samples(g, v, px, py, &smp, &h);
        std::vector<std::vector<std::pair<int64_t, double>>> stn;
        ray_stencils(g, v, px, py, &stn);
        const int K = (int)smp.size();
        std::vector<Sample<D>> sd(K);
        bool touched = false;
        for (int k = 0; k < K; ++k) {
          sd[k].n_h2 = D(smp[k].n_h2);
          sd[k].t_gas = D(smp[k].t_gas);
          sd[k].t_dust = D(smp[k].t_dust);
          sd[k].v_los = D(smp[k].v_los);
          sd[k].x_tr = D(smp[k].x_tr);
          for (const auto& cw : stn[k])
            for (int c = 0; c < nc; ++c)
              if (cw.first == seed[c]) {
                sd[k].n_h2.d[3 * c + 0] += cw.second;
                sd[k].t_gas.d[3 * c + 1] += cw.second;
                sd[k].v_los.d[3 * c + 2] += cw.second;
                touched = true;
              }
        }
        std::vector<D> T(nchan), C(nchan), Dd(nchan), L(nchan), B(nchan);
        if (!touched) {
          if (c0 == 0) {
            std::vector<double> Tq(nchan), Cq(nchan), Dq(nchan), Lq(nchan), Bq(nchan);
            ray_outputs(ln, du, va, integration, units, t_bg, smp, h, Tq.data(), Cq.data(),
                        Dq.data(), Lq.data(), Bq.data());
            for (int ch = 0; ch < nchan; ++ch) {
              const double r = Lq[ch] - target[((int64_t)ch * v.npy + py) * v.npx + px];
              l_t += r * r / nvox;
            }
          }
          continue;
        }
        ray_outputs(ln, du, va, integration, units, t_bg, sd, h, T.data(), C.data(), Dd.data(),
                    L.data(), B.data());
        D l(0.0);
        for (int ch = 0; ch < nchan; ++ch) {
          const D r = L[ch] - target[((int64_t)ch * v.npy + py) * v.npx + px];
          l = l + r * r;
        }
        l = l / nvox;
        if (c0 == 0) l_t += l.v;
        for (int i = 0; i < ND; ++i) acc_t[i] += l.d[i];
      }
#pragma omp critical
      {
        for (int i = 0; i < ND; ++i) acc[i] += acc_t[i];
        lsum += l_t;
      }
    }
    if (c0 == 0) loss = lsum;
    for (int c = 0; c < nc; ++c) {
      g_n[c0 + c] = acc[3 * c + 0];
      g_t[c0 + c] = acc[3 * c + 1];
      g_v[c0 + c] = acc[3 * c + 2];
    }
  }
  return loss;
}

}  // extern "C"

// Internal structures shared by the host side of the library and its kernels.
#pragma once

#include <stdint.h>
#include <cuda_runtime.h>

#include "../../include/irt.h"

namespace irt {

// Packed field storage of a grid (one cell = the five fields interleaved).
enum Store { ST_F32 = 0, ST_H16 = 1, ST_F64 = 2 };

// Integration variants (values of irt_integration).
enum Mode { M_FORMAL = 0, M_SMOOTH = 1, M_FORMAL_KAHAN = 2 };

// pad[0] holds the H2 abundance per H nucleus (fp16 in 16-bit cells), read
// only by the optically thin level balance; 0.5 (fully molecular) unless set
// by irt_grid_set_h2_fraction.
struct alignas(32) CellF32 { float v[5]; float pad[3]; };
struct alignas(16) CellH16 { uint16_t v[5]; uint16_t pad[3]; };
struct alignas(64) CellF64 { double v[5]; double pad[3]; };

// Physical constants of one launch, folded on the host in double precision
// from irt_line / irt_dust / irt_opts.  Intensities inside the kernels are in
// "K units": I * c^2 / (2 k nu_ul^2), the Rayleigh-Jeans temperature at nu_ul.
struct PhysParams {
  double T0;          // h nu_ul / k                                  [K]
  double e_u, e_l;    // level energies / k, e_l = e_u - T0           [K]
  double theta_rot;   // h B0 / k                                     [K]
  double g_u;         // statistical weight of the upper level
  // per-step line coefficients at the profile peak (K units / optical depth):
  //   jl = cj * N h exp(-E_u/T) / (Z b),
  //   al = ca * N h exp(-E_l/T) (1 - exp(-T0/T)) / (Z b)
  double cj, ca;
  double c_th;        // 2 k / m in (km/s)^2 / K  (thermal part of b^2)
  double two_sig2;    // 2 sigma_turb^2 (km/s)^2
  double t_inf;       // T_inf [K]
  double cad;         // kappa * mu * amu [cm^2]: alpha_D = cad * n_H2
  double inv_c_kms;   // 1 / c [s/km]
  double t_bg;        // background temperature [K]
  double out_scale;   // K units -> output units at nu_ul: 1 (T_RJ) or 2 k nu^2 / c^2
  int units;          // irt_units
  int integration;    // irt_integration
  // optically thin level balance (irt_forward_ppv_ot): the line's coefficient
  // grid [n0][n1][n2] of (j, alpha) per tracer molecule [cgs], or nullptr for
  // LTE; axes log10 n_H, chi, log10 T from lo[a] with ot_s[a] nodes per unit;
  // ot_jk, ot_ak turn the cgs values into the per-step K-unit coefficients
  // (times N h / b)
  const double* ot_tab;
  int ot_n[3];
  int ot_pad;
  double ot_lo[3], ot_s[3];
  double ot_jk, ot_ak;
};

// The same constants rounded to float for the float kernels (no FP64 work
// in their per-sample code).
struct PhysF {
  float T0, e_u, e_l, theta_rot, cj, ca, c_th, two_sig2, t_inf, cad, inv_c_kms, t_bg, out_scale;
  int units;
  // optically thin level balance: the line's grid as float4 pairs along the
  // temperature axis, (j, alpha) at nodes i2 and i2 + 1, [n0][n1][n2 - 1],
  // already in per-step K units (times N h / b); nullptr for LTE
  const float4* ot_tab;
  int ot_n[3];
  float ot_lo[3], ot_s[3];
};

// Optically thin level-balance grid (irt_create_ot_table): per line, the
// frequency-integrated coefficients per tracer molecule on the (log10 n_H,
// chi, log10 T) nodes, in double (cgs) and as the float kernels read them.
struct OTTableDev {
  int n[3];
  double lo[3], hi[3];
  int nlines;
  double nu[8];            // line frequencies [Hz]
  double jk[8], ak[8];     // cgs -> per-step K units (times N h / b)
  double* tab64;           // [nlines][n0][n1][n2][2]
  float4* tab32;           // [nlines][n0][n1][n2 - 1]
  int device;
};
// Several lines rendered in one launch (irt_forward_ppv_lines): per line its
// constants and its five output cubes; the rays' field samples are taken once
// and reused by every line.
constexpr int kMaxLinesPerRender = 4;
struct LineSet {
  int n;
  int pad;
  PhysF pf[kMaxLinesPerRender];
  void* out[kMaxLinesPerRender][5];
};

constexpr int kOTMaxLines = 8;
constexpr int kOTMaxLevels = 64;

// The level model in device memory (one buffer) and the grid of one build.
struct OTBuildArgs {
  int nlev, nrad, npartner, ntemp, ncoll, nlines;
  const double* energy;   // [nlev] E_i / k [K]
  const double* g;        // [nlev]
  const double* a;        // [nrad] Einstein A [1/s]
  const double* nu;       // [nrad] [Hz]
  const double* ctemp;    // [npartner][ntemp] [K]
  const double* k;        // [npartner][ncoll][ntemp] de-excitation [cm^3/s]
  const int* rad_up;
  const int* rad_lo;
  const int* partner;     // irt_partner kinds
  const int* cup;         // [npartner][ncoll]
  const int* clo;
  const int* lines;       // [nlines] radiative transition indices
  double t_rad, opr, x_he;
  int n[3];
  double lo[3], hi[3];
  double jk[kOTMaxLines], ak[kOTMaxLines];   // cgs -> per-step K units
};
int launch_ot_build(const OTBuildArgs& args, double* tab64, float4* tab32, cudaStream_t stream);

// One render job as the kernels see it.
struct JobDev {
  const void* cells;     // packed cells [nz][ny][nx]
  int store;             // Store
  int bf16_mask;         // ST_H16: bit q set = field q is bf16 (else fp16)
  float scale[5];        // ST_H16: physical value = stored value * scale[q]
  int pad1;
  int nx, ny, nz;
  double dx;             // cell size [cm]
  int zview;             // 1 = cell-exact view along the z axis (z or radial)
  int zrev;              // radial view: sample k is the cell z = nz - 1 - k
  // the orthographic view (set up on the host from the view angles) in cell
  // units as float-float pairs {hi, lo} (value = hi + lo): ray origin
  // o(px, py) = fo0 + px fox + py foy, direction fd, 1/d (0 on an axis with
  // d = 0), cell size [cm]; the float kernels evaluate them in float-float
  // arithmetic, the double kernels in double
  float fo0[3][2], fox[3][2], foy[3][2], fd[3][2], finv_d[3][2], fdx[2];
  int npx, npy;
  int nchan, f;
  double v0, dv;         // channel lower edge of channel 0, width [km/s]
  double ufirst, dvf;    // first fine velocity and fine step [km/s]
  // the same as float-float pairs, and 1/dv rounded to float, for the float
  // kernels (no double arithmetic per ray)
  float fv0[2], fdv[2], fufirst[2], fdvf[2];
  float finv_dv;
  int cw, nwin;          // channels per window, windows per ray
  int tw, th;            // rays are handed out in tiles of tw x th pixels
  int ntx;               // tiles per image row
  int kmax;              // upper bound of samples per ray
  int ck_nb;             // rows of a saved checkpoint (hull blocks < ck_nb) or 0
  float* ck;             // saved smooth-transfer checkpoints [ray][seg][2][ck_nb][32]
  long long ck_ray;      // floats per ray of ck
  void* out[5];          // T, C, D, L, B cubes [nchan][npy][npx]
  long long item_begin;  // first global work item of this job
  long long nitems;      // npx * npy * nwin
};

constexpr int kWarpsPerBlock = 4;
constexpr int kMaxJobs = 64;
// Forward per-sample record sizes (float and double kernels) and the most
// warps a forward kernel keeps resident on one SM (128 registers a thread).
// Rows of a saved forward checkpoint: hull blocks of at most 9 (the first
// adjoint pass) plus the basis row.
constexpr int kCkRows = 10;
constexpr int kRecBytesF32 = 48;
constexpr int kRecBytesF64 = 64;
constexpr int kFwdWarpsPerSm = 16;

// Adjoint: checkpoint spacing and stored sub-segment (samples), warps per
// block, chain-rule factors per sample.
constexpr int kAdjSeg = 32;
constexpr int kAdjSub = 32;
constexpr int kAdjWarps = 2;
constexpr int kAdjChain = 5;

struct AdjArgs {
  const float* cot[5];          // cotangent cubes T, C, D, L, B (NULL = 0)
  float* grad[3];               // n_H2, T_gas, v_los
  float* scratch;               // per-warp scratch (16-byte aligned slots)
  long long scratch_per_warp;   // floats, a multiple of 4
  const float* ck_saved;        // checkpoints saved by the forward render, or nullptr
  int ck_nb;                    // their rows (hull blocks < ck_nb)
  long long ck_ray;             // floats per ray
  const unsigned* in_list;      // rays of this pass: [0] = count, then indices (nullptr: all)
  int defer_max_nb;             // widest hull bucket a later pass handles (0: none)
  unsigned* defer;              // rays with wider hulls for the next pass, or nullptr
  unsigned* dense;              // [0] = count, then the rays the general sweep takes
};

// Job table passed to the kernels by value (__grid_constant__ parameter).
struct JobTable {
  JobDev j[kMaxJobs];
};


// Launch entry points implemented in the .cu files.
// Returns a cudaError_t value (0 = success).

// Launch arguments of one forward kernel instance.
struct FwdLaunch {
  long long total;             // work items of the job table
  unsigned long long* queue;   // work-queue counter, zero at launch (nullptr: round-robin)
  int grid_blocks;             // 0: as many blocks as are resident at once
  int kmax;                    // most samples on a ray of the table
  int fwmax, cwmax;            // most fine velocities / channels of a window
  unsigned flags;
  unsigned long long* stats;   // 6 work counters or nullptr
  unsigned char* rscr;         // per-warp sample records (global memory)
  size_t rbytes;               // size of rscr; bounds the resident warps
  const LineSet* lines;        // several lines in one launch, or nullptr
};

// Shared memory per warp the thin-mode kernel may use (records and masks).
constexpr size_t kThinSmemBudget = 200 * 1024;
size_t thin_smem_per_warp(int precision, int transfer, int kmax, int nchan_max,
                          size_t* record_bytes, size_t* mask_bytes);

int launch_pack(int store, const void* const* src, const int* dtypes, const double* scale,
                void* cells, long long ncell, void* stream);
// H2 abundance into the spare slot of every cell (default 0.5 from the pack)
int launch_set_chi(int store, const void* chi, int dtype, void* cells, long long ncell,
                   void* stream);


}  // namespace irt

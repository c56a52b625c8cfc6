// C ABI of the library (include/irt.h): argument validation, grid lifetime,
// constant folding, launch planning.  No arithmetic of the method runs here;
// the host only converts the caller's constants to the kernels' units.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstdarg>
#include <cstdint>
#include <cstring>
#include <map>
#include <mutex>
#include <numeric>
#include <string>
#include <vector>

#include "irt_internal.h"

namespace irt {

int dispatch_fwd_f32_smooth(int store, int ni, const JobTable& jobs, int njobs,
                            const PhysParams& P, const PhysF& PF, const FwdLaunch& L,
                            cudaStream_t s);
int dispatch_fwd_f32_formal(int store, int ni, const JobTable& jobs, int njobs,
                            const PhysParams& P, const PhysF& PF, const FwdLaunch& L,
                            cudaStream_t s);
int dispatch_fwd_f32_kahan(int store, int ni, const JobTable& jobs, int njobs,
                           const PhysParams& P, const PhysF& PF, const FwdLaunch& L,
                           cudaStream_t s);
int launch_mean_axis1(const void* in, int dtype, long long A, long long B, long long C,
                      void* out, cudaStream_t s);
int launch_beam(const void* in, int dtype, long long nchan, int npy, int npx, double fwhm_px,
                void* scratch, void* out, cudaStream_t s);
int launch_tb_convert(int precision, void* T, void* C, void* B, void* L, void* D,
                      long long plane, int nchan, double v0, double dv, double T0,
                      double inv_c_kms, cudaStream_t s);
int launch_thin(int precision, int store, int integ, int transfer, const JobTable& tab,
                int njobs, const PhysParams& P, const PhysF& PF, long long total, int kmax,
                int nchan_max, unsigned long long* stats, cudaStream_t stream);
int launch_adjoint(int store, int ni, bool obl, const JobTable& tab, const PhysF& PF,
                   const AdjArgs& A, long long total_items, unsigned long long* queue, int blocks, int kmax,
                   int nfw, int nchan, cudaStream_t stream, int* per_warp_smem);
int adjoint_blocks_per_sm(int store, int ni, bool obl, size_t smem);
size_t adjoint_dense_smem_per_warp(int kmax, int nchan);
long long adjoint_dense_scratch_per_warp(int kmax);
int launch_adjoint_dense(int store, const JobTable& tab, const PhysF& PF, float* const grad[3],
                         const float* const cot[5], float* scratch, long long scratch_per_warp,
                         const unsigned* list, int smooth, int direct, long long total_items,
                         unsigned long long* queue, int kmax, int nchan, int* blocks_out,
                         cudaStream_t stream);
int dispatch_fwd_f64(int mode, int store, int ni, const JobTable& jobs, int njobs,
                     const PhysParams& P, const PhysF& PF, const FwdLaunch& L, cudaStream_t s);
int dispatch_fwd_ml_smooth(int store, int ni, const JobTable& jobs, int njobs,
                           const PhysParams& P, const PhysF& PF, const FwdLaunch& L,
                           cudaStream_t s);
int dispatch_fwd_ml_formal(int store, int ni, const JobTable& jobs, int njobs,
                           const PhysParams& P, const PhysF& PF, const FwdLaunch& L,
                           cudaStream_t s);
int dispatch_fwd_ml_kahan(int store, int ni, const JobTable& jobs, int njobs,
                          const PhysParams& P, const PhysF& PF, const FwdLaunch& L,
                          cudaStream_t s);
int dispatch_fwd_ot_smooth(int precision, int store, int ni, const JobTable& jobs, int njobs,
                           const PhysParams& P, const PhysF& PF, const FwdLaunch& L,
                           cudaStream_t s);
int dispatch_fwd_ot_formal(int precision, int store, int ni, const JobTable& jobs, int njobs,
                           const PhysParams& P, const PhysF& PF, const FwdLaunch& L,
                           cudaStream_t s);
int dispatch_fwd_ot_kahan(int precision, int store, int ni, const JobTable& jobs, int njobs,
                          const PhysParams& P, const PhysF& PF, const FwdLaunch& L,
                          cudaStream_t s);

namespace {

thread_local std::string g_err;
thread_local long long g_launches = 0;

irt_status fail(irt_status st, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
irt_status fail(irt_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return st;
}

irt_status cuda_fail(int e, const char* where) {
  return fail(IRT_ECUDA, "%s: %s", where, cudaGetErrorString((cudaError_t)e));
}

// Every device allocation of the library goes through here.  Host-side fault
// injection for tests: with IRT_FAIL_ALLOC set to a non-empty value other
// than "0" in the environment (read on every call), the allocation fails
// without calling the CUDA runtime, so that the IRT_ENOMEM paths can be
// exercised without exhausting a shared GPU.
cudaError_t dev_malloc(void** p, size_t bytes) {
  const char* e = std::getenv("IRT_FAIL_ALLOC");
  if (e && *e && std::strcmp(e, "0") != 0) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaMalloc(p, bytes);
}

bool finite_pos(double x) { return std::isfinite(x) && x > 0.0; }
bool finite_nonneg(double x) { return std::isfinite(x) && x >= 0.0; }

// CODATA 2018 constants for the unit conversions of the launch parameters.
constexpr double kH = 6.62607015e-27;    // erg s
constexpr double kK = 1.380649e-16;      // erg/K
constexpr double kC = 2.99792458e10;     // cm/s
constexpr double kCkms = 2.99792458e5;   // km/s
constexpr double kAmu = 1.66053906660e-24;
constexpr double kPi = 3.14159265358979323846;

}  // namespace
}  // namespace irt

struct irt_grid {
  int nx, ny, nz;
  double dx;
  int store;
  int bf16_mask;
  double scale[5];
  void* cells;
  size_t cell_bytes;
  unsigned long long* ctl;   // device control words (work-queue counter)
  int device;
  float* ck;                     // forward checkpoints kept for the adjoint
  size_t ck_bytes;
  unsigned long long ck_sig;     // signature of the job that wrote them (0: none)
};

using namespace irt;

extern "C" {

const char* irt_last_error(void) { return g_err.c_str(); }

long long irt_launch_count(void) {
  const long long n = g_launches;
  g_launches = 0;
  return n;
}

irt_status irt_create_grid(const irt_grid_desc* desc, const irt_fields* fields,
                           void* cuda_stream, irt_grid** out) {
  g_err.clear();
  if (!desc || !fields || !out) return fail(IRT_EINVAL, "irt_create_grid: NULL argument");
  *out = nullptr;
  if (desc->nx < 1 || desc->ny < 1 || desc->nz < 1)
    return fail(IRT_EINVAL, "irt_create_grid: grid size %d x %d x %d", desc->nx, desc->ny,
                desc->nz);
  if (!finite_pos(desc->cell_cm)) return fail(IRT_EINVAL, "irt_create_grid: cell_cm <= 0");
  const void* src[5] = {fields->n_h2_cm3, fields->t_gas_k, fields->t_dust_k, fields->v_los_kms,
                        fields->x_tracer};
  int dt[5];
  bool any64 = false, all16 = true;
  int bf_mask = 0;
  for (int q = 0; q < 5; ++q) {
    if (!src[q]) return fail(IRT_EINVAL, "irt_create_grid: field %d is NULL", q);
    dt[q] = (int)desc->dtype[q];
    if (dt[q] < IRT_F32 || dt[q] > IRT_F64)
      return fail(IRT_EINVAL, "irt_create_grid: field %d has unknown dtype %d", q, dt[q]);
    if (dt[q] == IRT_F64) any64 = true;
    if (dt[q] != IRT_F16 && dt[q] != IRT_BF16) all16 = false;
    if (dt[q] == IRT_BF16) bf_mask |= 1 << q;
  }
  double scale[5];
  for (int q = 0; q < 5; ++q) {
    scale[q] = desc->scale[q] == 0.0 ? 1.0 : desc->scale[q];
    if (!std::isfinite(scale[q]) || scale[q] <= 0.0)
      return fail(IRT_EINVAL, "irt_create_grid: scale[%d] must be finite and > 0", q);
  }
  const long long ncell = (long long)desc->nx * desc->ny * desc->nz;
  const int store = any64 ? ST_F64 : (all16 ? ST_H16 : ST_F32);
  const size_t cb = store == ST_F64 ? sizeof(CellF64) : store == ST_H16 ? sizeof(CellH16)
                                                                         : sizeof(CellF32);
  irt_grid* g = new irt_grid();
  g->nx = desc->nx; g->ny = desc->ny; g->nz = desc->nz;
  g->dx = desc->cell_cm;
  g->store = store;
  g->bf16_mask = store == ST_H16 ? bf_mask : 0;
  for (int q = 0; q < 5; ++q) g->scale[q] = scale[q];
  g->cell_bytes = cb * (size_t)ncell;
  g->ctl = nullptr;
  g->ck = nullptr;
  g->ck_bytes = 0;
  g->ck_sig = 0;
  cudaGetDevice(&g->device);
  if (dev_malloc(&g->cells, g->cell_bytes) != cudaSuccess) {
    cudaGetLastError();
    delete g;
    return fail(IRT_ENOMEM, "irt_create_grid: cannot allocate %zu bytes", cb * (size_t)ncell);
  }
  if (dev_malloc((void**)&g->ctl, 64) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(g->cells);
    delete g;
    return fail(IRT_ENOMEM, "irt_create_grid: cannot allocate control words");
  }
  if (cudaMemsetAsync(g->ctl, 0, 64, (cudaStream_t)cuda_stream) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(g->cells);
    cudaFree(g->ctl);
    delete g;
    return fail(IRT_ECUDA, "irt_create_grid: cannot clear control words");
  }
  const int e = launch_pack(store, src, dt, scale, g->cells, ncell, cuda_stream);
  ++g_launches;
  if (e) {
    cudaFree(g->cells);
    cudaFree(g->ctl);
    delete g;
    return cuda_fail(e, "irt_create_grid: pack kernel");
  }
  *out = g;
  return IRT_OK;
}

irt_status irt_update_grid(irt_grid* g, const irt_grid_desc* desc, const irt_fields* fields,
                           void* cuda_stream) {
  g_err.clear();
  if (!g || !desc || !fields) return fail(IRT_EINVAL, "irt_update_grid: NULL argument");
  if (desc->nx != g->nx || desc->ny != g->ny || desc->nz != g->nz || desc->cell_cm != g->dx)
    return fail(IRT_EINVAL, "irt_update_grid: size or cell differs from the grid's");
  const void* src[5] = {fields->n_h2_cm3, fields->t_gas_k, fields->t_dust_k, fields->v_los_kms,
                        fields->x_tracer};
  int dt[5];
  bool any64 = false, all16 = true;
  int bf_mask = 0;
  double scale[5];
  for (int q = 0; q < 5; ++q) {
    if (!src[q]) return fail(IRT_EINVAL, "irt_update_grid: field %d is NULL", q);
    dt[q] = (int)desc->dtype[q];
    if (dt[q] < IRT_F32 || dt[q] > IRT_F64)
      return fail(IRT_EINVAL, "irt_update_grid: field %d has unknown dtype %d", q, dt[q]);
    if (dt[q] == IRT_F64) any64 = true;
    if (dt[q] != IRT_F16 && dt[q] != IRT_BF16) all16 = false;
    if (dt[q] == IRT_BF16) bf_mask |= 1 << q;
    scale[q] = desc->scale[q] == 0.0 ? 1.0 : desc->scale[q];
    if (!std::isfinite(scale[q]) || scale[q] <= 0.0)
      return fail(IRT_EINVAL, "irt_update_grid: scale[%d] must be finite and > 0", q);
  }
  const int store = any64 ? ST_F64 : (all16 ? ST_H16 : ST_F32);
  if (store != g->store || (store == ST_H16 && (bf_mask != g->bf16_mask ||
                                                 std::memcmp(scale, g->scale, sizeof scale))))
    return fail(IRT_EINVAL, "irt_update_grid: field storage differs from the grid's");
  // new field values: checkpoints of earlier renders no longer apply
  g->ck_sig = 0;
  const long long ncell = (long long)g->nx * g->ny * g->nz;
  const int e = launch_pack(store, src, dt, scale, g->cells, ncell, cuda_stream);
  ++g_launches;
  if (e) return cuda_fail(e, "irt_update_grid: pack kernel");
  return IRT_OK;
}

irt_status irt_grid_stats(irt_grid* g, unsigned long long out[6], int reset) {
  g_err.clear();
  if (!g || !out) return fail(IRT_EINVAL, "irt_grid_stats: NULL argument");
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(out, g->ctl + 1, 6 * sizeof(unsigned long long),
                                       cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && reset) e = cudaMemset(g->ctl + 1, 0, 6 * sizeof(unsigned long long));
  if (e != cudaSuccess) return cuda_fail(e, "irt_grid_stats");
  return IRT_OK;
}

irt_status irt_destroy(irt_grid* g) {
  g_err.clear();
  if (!g) return IRT_OK;
  cudaFree(g->cells);
  cudaFree(g->ctl);
  if (g->ck) cudaFree(g->ck);
  delete g;
  return IRT_OK;
}

}  // extern "C"

namespace irt {
namespace {

irt_status check_line(const irt_line* ln, const irt_dust* du, const irt_opts* op) {
  if (!ln || !du || !op) return fail(IRT_EINVAL, "NULL line, dust or opts");
  const double lv[] = {ln->nu_ul_hz, ln->a_ul_s, ln->b0_hz, ln->g_u, ln->g_l, ln->mass_amu};
  for (double v : lv)
    if (!finite_pos(v)) return fail(IRT_EINVAL, "line constants must be finite and > 0");
  if (!std::isfinite(ln->e_u_k)) return fail(IRT_EINVAL, "line e_u_k is not finite");
  if (!finite_nonneg(ln->t_inf_k) && !(std::isinf(ln->t_inf_k) && ln->t_inf_k > 0))
    return fail(IRT_EINVAL, "line t_inf_k must be >= 0");
  if (!finite_nonneg(ln->sigma_turb_kms)) return fail(IRT_EINVAL, "sigma_turb_kms must be >= 0");
  if (!finite_nonneg(du->kappa_cm2_per_g_gas) || !finite_nonneg(du->mu_mass_per_h2_amu))
    return fail(IRT_EINVAL, "dust constants must be finite and >= 0");
  if (!finite_nonneg(op->t_bg_k)) return fail(IRT_EINVAL, "t_bg_k must be finite and >= 0");
  if (op->mode < IRT_MODE_THICK || op->mode > IRT_MODE_DENSITY_TRACING)
    return fail(IRT_EINVAL, "unknown transfer mode %d", op->mode);
  if (op->integration < IRT_FORMAL || op->integration > IRT_FORMAL_KAHAN)
    return fail(IRT_EINVAL, "unknown integration %d", op->integration);
  if (op->mode != IRT_MODE_THICK && op->integration == IRT_FORMAL_KAHAN)
    return fail(IRT_EUNSUPPORTED, "thin transfer modes take IRT_FORMAL or IRT_SMOOTH");
  if (op->units != IRT_UNITS_TRJ && op->units != IRT_UNITS_INTENSITY && op->units != IRT_UNITS_TB)
    return fail(IRT_EINVAL, "unknown units %d", op->units);
  if (op->precision != IRT_PREC_F32 && op->precision != IRT_PREC_F64)
    return fail(IRT_EINVAL, "unknown precision %d", op->precision);
  return IRT_OK;
}

PhysParams fold_constants(const irt_line* ln, const irt_dust* du, const irt_opts* op) {
  PhysParams P;
  std::memset(&P, 0, sizeof P);   // no padding bytes of unknown value (the struct is hashed)
  const double nu = ln->nu_ul_hz;
  P.T0 = kH * nu / kK;
  P.e_u = ln->e_u_k;
  P.e_l = ln->e_u_k - P.T0;
  P.theta_rot = kH * ln->b0_hz / kK;
  P.g_u = ln->g_u;
  const double k_i = kC * kC / (2.0 * kK * nu * nu);     // cgs intensity -> K units
  const double per_hz = kCkms / nu / std::sqrt(kPi);      // phi_nu peak * b [km/s]
  P.cj = (kH * nu / (4.0 * kPi)) * ln->a_ul_s * ln->g_u * k_i * per_hz;
  P.ca = (kC * kC * ln->a_ul_s / (8.0 * kPi * nu * nu)) * ln->g_u * per_hz;
  P.c_th = 2.0 * kK / (ln->mass_amu * kAmu) / 1e10;
  P.two_sig2 = 2.0 * ln->sigma_turb_kms * ln->sigma_turb_kms;
  P.t_inf = ln->t_inf_k;
  P.cad = du->kappa_cm2_per_g_gas * du->mu_mass_per_h2_amu * kAmu;
  P.inv_c_kms = 1.0 / kCkms;
  P.t_bg = op->t_bg_k;
  P.units = op->units;
  P.integration = op->integration;
  P.out_scale = (op->units == IRT_UNITS_INTENSITY) ? 1.0 / k_i : 1.0;
  return P;
}

PhysF to_float(const PhysParams& P) {
  PhysF F;
  std::memset(&F, 0, sizeof F);
  F.T0 = (float)P.T0;
  F.e_u = (float)P.e_u;
  F.e_l = (float)P.e_l;
  F.theta_rot = (float)P.theta_rot;
  F.cj = (float)P.cj;
  F.ca = (float)P.ca;
  F.c_th = (float)P.c_th;
  F.two_sig2 = (float)P.two_sig2;
  F.t_inf = (float)std::min(P.t_inf, 3.0e38);
  F.cad = (float)P.cad;
  F.inv_c_kms = (float)P.inv_c_kms;
  F.t_bg = (float)P.t_bg;
  F.out_scale = (float)P.out_scale;
  F.units = P.units;
  return F;
}

irt_status check_job(const irt_job& jb, int precision) {
  const irt_grid* g = jb.grid;
  if (!g) return fail(IRT_EINVAL, "job without grid");
  const irt_vaxis& va = jb.vaxis;
  if (va.nchan < 1) return fail(IRT_EINVAL, "nchan < 1");
  if (!finite_pos(va.dv_kms)) return fail(IRT_EINVAL, "dv_kms must be > 0");
  if (!std::isfinite(va.v_first_edge_kms)) return fail(IRT_EINVAL, "v_first_edge not finite");
  if (va.subsample_f < 0) return fail(IRT_EINVAL, "subsample_f < 0");
  if (va.subsample_f > 64) return fail(IRT_EUNSUPPORTED, "subsample_f > 64");
  {
    // fine velocity indices of the whole axis are kept in 16 bits
    const long long nfw = va.subsample_f >= 1 ? 2LL * va.subsample_f * va.nchan + 1 : va.nchan;
    if (nfw > 32000)
      return fail(IRT_EUNSUPPORTED, "%lld fine velocities (2 f nchan + 1) exceed 32000", nfw);
  }
  const irt_view& vw = jb.view;
  if (vw.trilinear == 0 || vw.trilinear == 2) {
    if (vw.theta_rad != 0.0 || vw.phi_rad != 0.0)
      return fail(IRT_EINVAL, "z and radial views (trilinear = 0, 2) need theta = phi = 0");
    if (vw.npx != g->nx || vw.npy != g->ny)
      return fail(IRT_EINVAL, "z or radial view image %d x %d differs from grid %d x %d", vw.npx,
                  vw.npy, g->nx, g->ny);
  } else if (vw.trilinear == 1) {
    if (vw.npx < 1 || vw.npy < 1) return fail(IRT_EINVAL, "view npx/npy < 1");
    if (!finite_pos(vw.pixel_cm)) return fail(IRT_EINVAL, "view pixel_cm must be > 0");
    if (!std::isfinite(vw.theta_rad) || !std::isfinite(vw.phi_rad))
      return fail(IRT_EINVAL, "view angles not finite");
  } else {
    return fail(IRT_EINVAL, "view.trilinear must be 0 (z), 1 (oblique) or 2 (radial)");
  }
  const void* o[5] = {jb.out.T, jb.out.C, jb.out.D, jb.out.L, jb.out.B};
  bool any = false;
  for (const void* p : o) any = any || p;
  if (!any) return fail(IRT_EINVAL, "all output cubes are NULL");
  if (precision == IRT_PREC_F64 && g->store != ST_F64)
    return fail(IRT_EUNSUPPORTED, "double precision needs a grid stored as double");
  return IRT_OK;
}

// Window plan: blocks per lane (compiled sizes) and channels per window.
struct Plan {
  int ni, cw, nwin, nfw, kmax;
  int tw = 1, th = 1;
};

const int kNiF32[] = {9, 17, 33};

Plan plan_job(const irt_job& jb, int precision, int force_ni) {
  Plan p;
  const int f = jb.vaxis.subsample_f, nch = jb.vaxis.nchan;
  auto fine_of = [&](int cw) { return f >= 1 ? 2 * f * cw + 1 : cw; };
  // channels of a window of ni register blocks (general path); windows start
  // on a 32-velocity block boundary (2 f cw a multiple of 32)
  auto cw_for = [&](int ni) {
    const int slots = 32 * ni;
    if (f < 1) return slots;
    const int cw = (slots - 1) / (2 * f);
    const int q = 32 / std::gcd(2 * f, 32);
    return std::max(cw - cw % q, 1);
  };
  if (precision == IRT_PREC_F64) {
    p.ni = 17;
  } else if (force_ni > 0) {
    p.ni = force_ni;
  } else {
    p.ni = 33;
    for (int ni : kNiF32)
      if (nch <= cw_for(ni)) { p.ni = ni; break; }
  }
  p.cw = std::min(nch, cw_for(p.ni));
  p.nwin = (nch + p.cw - 1) / p.cw;
  p.nfw = fine_of(p.cw);
  const irt_grid* g = jb.grid;
  if (jb.view.trilinear != 1) {   // z and radial views: one sample per cell
    p.kmax = g->nz;
  } else {
    const double diag = std::sqrt((double)g->nx * g->nx + (double)g->ny * g->ny +
                                  (double)g->nz * g->nz);
    p.kmax = (int)std::ceil(diag) + 2;
  }
  return p;
}

// x as a float-float pair {hi, lo}: hi = x rounded to float, lo = the
// rest rounded to float
static void split_ff(double x, float out[2]) {
  out[0] = (float)x;
  out[1] = (float)(x - (double)out[0]);
}

JobDev make_jobdev(const irt_job& jb, const Plan& p) {
  JobDev d;
  std::memset(&d, 0, sizeof d);
  const irt_grid* g = jb.grid;
  d.cells = g->cells;
  d.store = g->store;
  d.bf16_mask = g->bf16_mask;
  // 16-bit cells are stored as given; the kernels apply the scales.  Wider
  // storage had the scales applied while packing.
  for (int q = 0; q < 5; ++q) d.scale[q] = g->store == ST_H16 ? (float)g->scale[q] : 1.0f;
  d.nx = g->nx; d.ny = g->ny; d.nz = g->nz;
  d.dx = g->dx;
  d.zview = jb.view.trilinear == 0 || jb.view.trilinear == 2;
  d.zrev = jb.view.trilinear == 2;
  {
    // orthographic view basis: direction d = (st cp, st sp, ct), pixel axes
    // e_theta = (ct cp, ct sp, -st), e_phi = (-sp, cp, 0)
    const double st = std::sin(jb.view.theta_rad), ct = std::cos(jb.view.theta_rad);
    const double sp = std::sin(jb.view.phi_rad), cp = std::cos(jb.view.phi_rad);
    const double dd[3] = {st * cp, st * sp, ct};
    const double et[3] = {ct * cp, ct * sp, -st};
    const double ep[3] = {-sp, cp, 0.0};
    // float-float form in cell units: o = (n/2 + (px - cx) P e_theta + (py -
    // cy) P e_phi), P = pixel / dx, cx = (npx - 1)/2
    const double P = jb.view.pixel_cm / g->dx;
    const double cx = 0.5 * (jb.view.npx - 1), cy = 0.5 * (jb.view.npy - 1);
    const int n[3] = {g->nx, g->ny, g->nz};
    for (int a = 0; a < 3; ++a) {
      split_ff(0.5 * n[a] - cx * P * et[a] - cy * P * ep[a], d.fo0[a]);
      split_ff(P * et[a], d.fox[a]);
      split_ff(P * ep[a], d.foy[a]);
      // an axis with |d| < 1e-30 counts as parallel (1/d would not fit a float)
      const bool par = std::fabs(dd[a]) < 1e-30;
      split_ff(par ? 0.0 : dd[a], d.fd[a]);
      split_ff(par ? 0.0 : 1.0 / dd[a], d.finv_d[a]);
    }
    split_ff(g->dx, d.fdx);
  }
  d.npx = jb.view.npx;
  d.npy = jb.view.npy;
  d.nchan = jb.vaxis.nchan;
  d.f = jb.vaxis.subsample_f;
  d.v0 = jb.vaxis.v_first_edge_kms;
  d.dv = jb.vaxis.dv_kms;
  if (d.f >= 1) {
    d.ufirst = d.v0;
    d.dvf = d.dv / (2.0 * d.f);
  } else {
    d.ufirst = d.v0 + 0.5 * d.dv;
    d.dvf = d.dv;
  }
  split_ff(d.v0, d.fv0);
  split_ff(d.dv, d.fdv);
  split_ff(d.ufirst, d.fufirst);
  split_ff(d.dvf, d.fdvf);
  d.finv_dv = (float)(1.0 / d.dv);
  d.cw = p.cw;
  d.nwin = p.nwin;
  d.kmax = p.kmax;
  d.out[0] = jb.out.T; d.out[1] = jb.out.C; d.out[2] = jb.out.D;
  d.out[3] = jb.out.L; d.out[4] = jb.out.B;
  d.tw = std::max(1, p.tw);
  d.th = std::max(1, p.th);
  d.ntx = (d.npx + d.tw - 1) / d.tw;
  const long long nty = (d.npy + d.th - 1) / d.th;
  d.nitems = (long long)d.ntx * d.tw * nty * d.th;   // one item per ray (tile padding included)
  return d;
}

int dispatch(int precision, int mode, int store, int ni, const JobTable& jobs, int njobs,
             const PhysParams& P, const PhysF& PF, const FwdLaunch& L, cudaStream_t s) {
  if (P.ot_tab) {
    // optically thin level balance: kernel instances of their own
    if (mode == M_SMOOTH) return dispatch_fwd_ot_smooth(precision, store, ni, jobs, njobs, P, PF, L, s);
    if (mode == M_FORMAL) return dispatch_fwd_ot_formal(precision, store, ni, jobs, njobs, P, PF, L, s);
    return dispatch_fwd_ot_kahan(precision, store, ni, jobs, njobs, P, PF, L, s);
  }
  if (precision == IRT_PREC_F64) return dispatch_fwd_f64(mode, store, ni, jobs, njobs, P, PF, L, s);
  if (mode == M_SMOOTH) return dispatch_fwd_f32_smooth(store, ni, jobs, njobs, P, PF, L, s);
  if (mode == M_FORMAL) return dispatch_fwd_f32_formal(store, ni, jobs, njobs, P, PF, L, s);
  return dispatch_fwd_f32_kahan(store, ni, jobs, njobs, P, PF, L, s);
}

// Record scratch a forward launch over these plans wants: every warp that can
// be resident on the device holds the records of its longest ray.
size_t fwd_scratch_need(const std::vector<Plan>& plans, int precision, bool lines = false) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int kmax = 1;
  for (const Plan& p : plans) kmax = std::max(kmax, p.kmax);
  const size_t rec = precision == IRT_PREC_F64 ? kRecBytesF64 : kRecBytesF32;
  size_t stride = ((size_t)kmax * rec + 255) & ~(size_t)255;
  // several lines in one launch also keep the ray's raw samples (6 floats)
  if (lines) stride += ((size_t)kmax * 24 + 255) & ~(size_t)255;
  return (size_t)std::max(sms, 1) * kFwdWarpsPerSm * stride;
}

}  // namespace
}  // namespace irt

namespace irt {
namespace {

// Launch plan of a forward call (channel window and ray tile), tuned or default.
struct Tuned {
  int ni = 0;      // 0 = smallest window size holding all channels
  int tw = 1, th = 1;
};

std::mutex g_tune_mu;
std::vector<std::pair<unsigned long long, Tuned>> g_tuned;   // signature -> plan

// Signature of a job mix for the tuning cache (sizes, axes, views, storage,
// integration, precision; not the field values).
unsigned long long job_signature(const irt_job* jobs, int njobs, const irt_opts* op) {
  unsigned long long h = 1469598103934665603ull;
  auto mix = [&](unsigned long long v) {
    h ^= v;
    h *= 1099511628211ull;
  };
  mix((unsigned long long)njobs);
  mix((unsigned long long)op->integration);
  mix((unsigned long long)op->precision);
  mix((unsigned long long)(op->flags & IRT_FLAG_EXPLICIT_CHANNELS));
  for (int j = 0; j < njobs; ++j) {
    const irt_job& b = jobs[j];
    mix((unsigned long long)b.grid->nx);
    mix((unsigned long long)b.grid->ny);
    mix((unsigned long long)b.grid->nz);
    mix((unsigned long long)b.grid->store);
    mix((unsigned long long)b.view.npx);
    mix((unsigned long long)b.view.npy);
    mix((unsigned long long)b.view.trilinear);
    mix((unsigned long long)b.vaxis.nchan);
    mix((unsigned long long)b.vaxis.subsample_f);
  }
  return h;
}

bool lookup_tuned(unsigned long long sig, Tuned* t) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  for (const auto& e : g_tuned)
    if (e.first == sig) {
      *t = e.second;
      return true;
    }
  return false;
}

void store_tuned(unsigned long long sig, const Tuned& t) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  for (auto& e : g_tuned)
    if (e.first == sig) {
      e.second = t;
      return;
    }
  g_tuned.emplace_back(sig, t);
}

// Launch-plan override for tests and manual tuning: IRT_PLAN="NI,tw,th"
// (NI one of 9, 17, 33; tiles >= 1).  Read on every call.
void forced_plan(Tuned* t) {
  const char* e = std::getenv("IRT_PLAN");
  if (!e || !*e) return;
  int ni = 0, tw = 0, th = 0;
  if (std::sscanf(e, "%d,%d,%d", &ni, &tw, &th) != 3) return;
  if ((ni == 9 || ni == 17 || ni == 33) && tw >= 1 && th >= 1 && tw <= 64 && th <= 64) {
    t->ni = ni;
    t->tw = tw;
    t->th = th;
  }
}

// Validated forward launch with a given plan (no tuning, no cache).
// Device buffer handed to a launch from outside the grids (graphs own one so
// that a later call cannot free it under them; the static entry uses its array).
struct Scratch {
  unsigned char* p = nullptr;
  size_t bytes = 0;
};

// Scratch of direct calls, kept per (device, stream) and reused by every
// grid: the forward's sample records, the adjoint's checkpoints and its
// deferred-ray list.  Launches on one stream run in order, so they can share
// a buffer; launches on different streams get different ones.  A buffer only
// grows (cudaFree waits for the launches that used the old one), never during
// stream capture.
struct StreamScratch {
  unsigned char* fwd = nullptr;
  size_t fwd_bytes = 0;
  unsigned char* adj = nullptr;
  size_t adj_bytes = 0;
  unsigned char* defer = nullptr;
  size_t defer_bytes = 0;
};
std::mutex g_scratch_mu;
std::map<std::pair<int, unsigned long long>, StreamScratch> g_scratch;

irt_status grow(unsigned char** p, size_t* have, size_t need, cudaStream_t s, const char* what) {
  if (*have >= need) return IRT_OK;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(s, &cap);
  if (cap != cudaStreamCaptureStatusNone)
    return fail(IRT_EUNSUPPORTED,
                "%s: the scratch of this stream must grow (%zu bytes), which cannot happen during "
                "stream capture; run the call once before capturing it", what, need);
  if (*p) cudaFree(*p);
  *p = nullptr;
  *have = 0;
  if (dev_malloc((void**)p, need) != cudaSuccess) {
    cudaGetLastError();
    return fail(IRT_ENOMEM, "%s: cannot allocate %zu bytes of scratch", what, need);
  }
  *have = need;
  return IRT_OK;
}

StreamScratch& stream_scratch(cudaStream_t s) {
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  return g_scratch[{dev, (unsigned long long)(uintptr_t)s}];
}

// Signature of everything besides the grid that sets a z-view job's
// transfer states: the velocity axis and the folded constants.
unsigned long long checkpoint_signature(const irt_job& jb, const PhysParams& P) {
  unsigned long long h = 1469598103934665603ull;
  auto mix = [&](const void* p, size_t n) {
    const unsigned char* b = static_cast<const unsigned char*>(p);
    for (size_t i = 0; i < n; ++i) h = (h ^ b[i]) * 1099511628211ull;
  };
  // field by field: the ABI structs have padding a caller need not clear
  mix(&jb.vaxis.nchan, sizeof(int));
  mix(&jb.vaxis.v_first_edge_kms, sizeof(double));
  mix(&jb.vaxis.dv_kms, sizeof(double));
  mix(&jb.vaxis.subsample_f, sizeof(int));
  mix(&jb.view.npx, sizeof(int));
  mix(&jb.view.npy, sizeof(int));
  mix(&jb.view.trilinear, sizeof(int));
  mix(&P, sizeof P);   // doubles and two trailing ints: no padding
  return h | 1ull;     // never 0 (0 = no checkpoints)
}

irt_status run_forward(const irt_job* jobs, int njobs, const PhysParams& P, const PhysF& PF,
                       const irt_opts* opts, const Tuned& tp, cudaStream_t s,
                       const Scratch* ext = nullptr) {
  const int prec = opts->precision;
  const int mode = opts->integration;
  std::vector<Plan> plans(njobs);
  int ni = 0;
  for (int j = 0; j < njobs; ++j) {
    plans[j] = plan_job(jobs[j], prec, 0);
    ni = std::max(ni, plans[j].ni);
  }
  if (prec != IRT_PREC_F64 && tp.ni > 0) ni = tp.ni;
  const int store = jobs[0].grid->store;
  for (int j = 1; j < njobs; ++j)
    if (jobs[j].grid->store != store)
      return fail(IRT_EUNSUPPORTED, "batched jobs must share the field storage type");
  for (int j = 0; j < njobs; ++j) {
    if (njobs > 1 || tp.ni > 0) plans[j] = plan_job(jobs[j], prec, ni);
    plans[j].tw = tp.tw;
    plans[j].th = tp.th;
  }
  // order: most expensive rays first (greedy longest-processing-time order
  // for the persistent work queue)
  std::vector<int> order(njobs);
  for (int j = 0; j < njobs; ++j) order[j] = j;
  if (njobs > 1) {
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
      const double ca = (double)plans[a].kmax * plans[a].nfw;
      const double cb = (double)plans[b].kmax * plans[b].nfw;
      return ca > cb;
    });
  }
  Scratch sc;
  if (ext) {
    sc = *ext;
  } else {
    StreamScratch& ss = stream_scratch(s);
    const irt_status st = grow(&ss.fwd, &ss.fwd_bytes, fwd_scratch_need(plans, prec), s,
                               "irt_forward_ppv");
    if (st) return st;
    sc.p = ss.fwd;
    sc.bytes = ss.fwd_bytes;
  }
  for (int base = 0; base < njobs; base += kMaxJobs) {
    const int nb = std::min(kMaxJobs, njobs - base);
    JobTable tab;
    std::memset(&tab, 0, sizeof tab);
    long long total = 0;
    int kmax = 1, fwmax = 1, cwmax = 1;
    for (int t = 0; t < nb; ++t) {
      const int j = order[base + t];
      tab.j[t] = make_jobdev(jobs[j], plans[j]);
      tab.j[t].item_begin = total;
      total += tab.j[t].nitems;
      kmax = std::max(kmax, plans[j].kmax);
      fwmax = std::max(fwmax, 32 * plans[j].ni);
      cwmax = std::max(cwmax, plans[j].cw);
    }
    if (opts->flags & IRT_FLAG_SAVE_CHECKPOINTS) {
      // one z-view smooth job (checked by the caller): the grid keeps the
      // states of every ray every 32 samples for the adjoint
      irt_grid* g = jobs[0].grid;
      const long long nseg = (plans[0].kmax + kAdjSeg - 1) / kAdjSeg;
      const long long ck_ray = nseg * 2 * kCkRows * 32;
      const size_t need =
          (size_t)tab.j[0].npx * tab.j[0].npy * (size_t)ck_ray * sizeof(float);
      unsigned char* buf = reinterpret_cast<unsigned char*>(g->ck);
      const irt_status st = grow(&buf, &g->ck_bytes, need, s, "irt_forward_ppv");
      g->ck = reinterpret_cast<float*>(buf);
      if (st) return st;
      tab.j[0].ck = g->ck;
      tab.j[0].ck_nb = kCkRows;
      tab.j[0].ck_ray = ck_ray;
      g->ck_sig = checkpoint_signature(jobs[0], P);
    }
    FwdLaunch L;
    L.total = total;
    // a batch balances its uneven items through the queue; one job's items
    // go round-robin
    L.queue = nb > 1 ? jobs[order[base]].grid->ctl : nullptr;
    L.grid_blocks = 0;
    L.kmax = kmax;
    L.fwmax = fwmax;
    L.cwmax = cwmax;
    L.flags = opts->flags;
    L.stats = (opts->flags & IRT_FLAG_STATS) ? jobs[0].grid->ctl + 1 : nullptr;
    L.rscr = sc.p;
    L.rbytes = sc.bytes;
    L.lines = nullptr;
    if (L.queue) {
      const cudaError_t ce = cudaMemsetAsync(L.queue, 0, sizeof(unsigned long long), s);
      if (ce != cudaSuccess) return cuda_fail(ce, "irt_forward_ppv: queue reset");
    }
    const int e = dispatch(prec, mode, store, ni, tab, nb, P, PF, L, s);
    ++g_launches;
    if (e) return cuda_fail(e, "irt_forward_ppv: forward kernel");
  }
  return IRT_OK;
}

// Selectively thin / optically thin render: one item per ray, no velocity
// windows; the launcher sizes its own blocks from the longest ray.
irt_status run_thin(const irt_job* jobs, int njobs, const PhysParams& P, const PhysF& PF,
                    const irt_opts* opts, cudaStream_t s) {
  const int prec = opts->precision;
  const int store = jobs[0].grid->store;
  for (int j = 1; j < njobs; ++j)
    if (jobs[j].grid->store != store)
      return fail(IRT_EUNSUPPORTED, "batched jobs must share the field storage type");
  const int integ = opts->integration == IRT_SMOOTH ? M_SMOOTH : M_FORMAL;
  for (int base = 0; base < njobs; base += kMaxJobs) {
    const int nb = std::min(kMaxJobs, njobs - base);
    JobTable tab;
    std::memset(&tab, 0, sizeof tab);
    long long total = 0;
    int kmax = 1, nchan_max = 1;
    for (int t = 0; t < nb; ++t) {
      nchan_max = std::max(nchan_max, jobs[base + t].vaxis.nchan);
      const Plan pl = plan_job(jobs[base + t], prec, 0);
      tab.j[t] = make_jobdev(jobs[base + t], pl);
      tab.j[t].item_begin = total;
      tab.j[t].nitems = (long long)tab.j[t].npx * tab.j[t].npy;
      total += tab.j[t].nitems;
      kmax = std::max(kmax, pl.kmax);
    }
    unsigned long long* stats =
        (opts->flags & IRT_FLAG_STATS) ? jobs[base].grid->ctl + 1 : nullptr;
    {
      size_t rec_b = 0, mask_b = 0;
      const size_t need = thin_smem_per_warp(prec == IRT_PREC_F64 ? 1 : 0, opts->mode, kmax,
                                             nchan_max, &rec_b, &mask_b);
      if (need > kThinSmemBudget)
        return fail(IRT_EUNSUPPORTED,
                    "irt_forward_ppv: thin-mode rays of %d samples with %d channels need %zu "
                    "bytes of shared memory per warp (records %zu + sample masks %zu); the "
                    "budget is %zu", kmax, nchan_max, need, rec_b, mask_b, kThinSmemBudget);
    }
    const int e = launch_thin(prec == IRT_PREC_F64 ? 1 : 0, store, integ, opts->mode, tab, nb, P,
                              PF, total, kmax, nchan_max, stats, s);
    ++g_launches;
    if (e) return cuda_fail(e, "irt_forward_ppv: thin-mode kernel");
  }
  return IRT_OK;
}

// Times the candidate plans on the given stream (synchronous) and returns the
// fastest.  Candidates: register blocks NI = 9, 17, 33 (the widest line hull
// the fast path holds, and the window of the general path) x ray tiles 1x1,
// 2x2, 4x1, 4x4.
irt_status autotune(const irt_job* jobs, int njobs, const PhysParams& P, const PhysF& PF,
                    const irt_opts* opts, cudaStream_t s, Tuned* best) {
  std::vector<Tuned> cands;
  const int tiles[4][2] = {{1, 1}, {2, 2}, {4, 1}, {4, 4}};
  for (int ni : {9, 17, 33}) {
    for (const auto& t : tiles) {
      Tuned c;
      c.ni = ni;
      c.tw = t[0];
      c.th = t[1];
      cands.push_back(c);
    }
  }
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return fail(IRT_ECUDA, "autotune: cannot create events");
  float best_ms = 1e30f;
  irt_status st = IRT_OK;
  irt_opts o = *opts;
  o.flags &= ~(unsigned)IRT_FLAG_STATS;
  for (const Tuned& c : cands) {
    st = run_forward(jobs, njobs, P, PF, &o, c, s);   // warm-up
    if (st) break;
    cudaEventRecord(e0, s);
    for (int r = 0; r < 2 && !st; ++r) st = run_forward(jobs, njobs, P, PF, &o, c, s);
    cudaEventRecord(e1, s);
    if (st) break;
    cudaError_t ce = cudaEventSynchronize(e1);
    if (ce != cudaSuccess) {
      st = cuda_fail(ce, "autotune: timing");
      break;
    }
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best_ms) {
      best_ms = ms;
      *best = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return st;
}

}  // namespace
}  // namespace irt

struct irt_ot_table {
  irt::OTTableDev t;
};

namespace irt {
namespace {

// The launch constants of the optically thin level balance: line q of the
// grid (float pairs for the float kernels, cgs doubles for the double ones).
void bind_ot(const OTTableDev& t, int q, PhysParams* P, PhysF* PF) {
  const long long nodes = (long long)t.n[0] * t.n[1] * t.n[2];
  P->ot_tab = t.tab64 + (size_t)q * nodes * 2;
  PF->ot_tab = t.tab32 + (size_t)q * t.n[0] * t.n[1] * (t.n[2] - 1);
  for (int a = 0; a < 3; ++a) {
    P->ot_n[a] = PF->ot_n[a] = t.n[a];
    P->ot_lo[a] = t.lo[a];
    P->ot_s[a] = (t.n[a] - 1) / (t.hi[a] - t.lo[a]);
    PF->ot_lo[a] = (float)P->ot_lo[a];
    PF->ot_s[a] = (float)P->ot_s[a];
  }
  P->ot_jk = t.jk[q];
  P->ot_ak = t.ak[q];
}

irt_status forward_entry(const irt_job* jobs, int njobs, const irt_line* line,
                         const irt_dust* dust, const irt_opts* opts, void* cuda_stream,
                         const irt_ot_table* ot, int ot_line);

}  // namespace
}  // namespace irt

extern "C" irt_status irt_forward_ppv(const irt_job* jobs, int njobs, const irt_line* line,
                                      const irt_dust* dust, const irt_opts* opts,
                                      void* cuda_stream) {
  g_err.clear();
  return forward_entry(jobs, njobs, line, dust, opts, cuda_stream, nullptr, 0);
}

extern "C" irt_status irt_forward_ppv_ot(const irt_job* jobs, int njobs,
                                         const irt_ot_table* table, int line_index,
                                         const irt_line* line, const irt_dust* dust,
                                         const irt_opts* opts, void* cuda_stream) {
  g_err.clear();
  if (!table) return fail(IRT_EINVAL, "irt_forward_ppv_ot: NULL table");
  if (line_index < 0 || line_index >= table->t.nlines)
    return fail(IRT_EINVAL, "irt_forward_ppv_ot: line index %d outside the table's %d lines",
                line_index, table->t.nlines);
  if (!line) return fail(IRT_EINVAL, "irt_forward_ppv_ot: NULL line");
  const double nu_t = table->t.nu[line_index];
  if (!(std::fabs(line->nu_ul_hz - nu_t) <= 1e-12 * nu_t))
    return fail(IRT_EINVAL, "irt_forward_ppv_ot: line frequency %.12g Hz differs from the "
                            "table line's %.12g Hz", line->nu_ul_hz, nu_t);
  if (opts && (opts->flags & IRT_FLAG_SAVE_CHECKPOINTS))
    return fail(IRT_EUNSUPPORTED, "irt_forward_ppv_ot: no checkpoints (the adjoint takes LTE "
                                  "populations only)");
  return forward_entry(jobs, njobs, line, dust, opts, cuda_stream, table, line_index);
}

namespace irt {
namespace {

irt_status forward_entry(const irt_job* jobs, int njobs, const irt_line* line,
                         const irt_dust* dust, const irt_opts* opts, void* cuda_stream,
                         const irt_ot_table* ot, int ot_line) {
  if (!jobs || njobs < 1) return fail(IRT_EINVAL, "irt_forward_ppv: no jobs");
  irt_status st = check_line(line, dust, opts);
  if (st) return st;
  for (int j = 0; j < njobs; ++j) {
    st = check_job(jobs[j], opts->precision);
    if (st) return st;
  }
  if (opts->flags & IRT_FLAG_SAVE_CHECKPOINTS) {
    if (njobs != 1 || jobs[0].view.trilinear == 1 || opts->integration != IRT_SMOOTH ||
        opts->precision != IRT_PREC_F32)
      return fail(IRT_EUNSUPPORTED, "irt_forward_ppv: IRT_FLAG_SAVE_CHECKPOINTS needs one "
                                    "z- or radial-view job, smooth integration, float precision");
  }
  cudaStream_t s = (cudaStream_t)cuda_stream;
  if (opts->mode != IRT_MODE_THICK) {
    if (opts->flags & IRT_FLAG_SAVE_CHECKPOINTS)
      return fail(IRT_EUNSUPPORTED, "irt_forward_ppv: checkpoints belong to the thick mode");
    PhysParams P = fold_constants(line, dust, opts);
    PhysF PF = to_float(P);
    if (ot) bind_ot(ot->t, ot_line, &P, &PF);
    return run_thin(jobs, njobs, P, PF, opts, s);
  }
  // T_B output of the thick mode: rendered in T_RJ, then converted in place
  // by a separate pass (which needs the [T], [C] and [B] cubes)
  const bool tb = opts->units == IRT_UNITS_TB;
  irt_opts o = *opts;
  if (tb) {
    for (int j = 0; j < njobs; ++j)
      if (!jobs[j].out.T || !jobs[j].out.C || !jobs[j].out.B)
        return fail(IRT_EINVAL, "irt_forward_ppv: IRT_UNITS_TB needs the T, C and B cubes of "
                                "every job");
    o.units = IRT_UNITS_TRJ;
  }
  PhysParams P = fold_constants(line, dust, &o);
  PhysF PF = to_float(P);
  if (ot) bind_ot(ot->t, ot_line, &P, &PF);
  Tuned tp;
  if (o.precision != IRT_PREC_F64) {
    const unsigned long long sig = job_signature(jobs, njobs, &o);
    if (!lookup_tuned(sig, &tp) && (o.flags & IRT_FLAG_AUTOTUNE)) {
      st = autotune(jobs, njobs, P, PF, &o, s, &tp);
      if (st) return st;
      store_tuned(sig, tp);
    }
    forced_plan(&tp);
  }
  st = run_forward(jobs, njobs, P, PF, &o, tp, s);
  if (st || !tb) return st;
  for (int j = 0; j < njobs; ++j) {
    const irt_job& jb = jobs[j];
    const int e = launch_tb_convert(o.precision == IRT_PREC_F64 ? 1 : 0, jb.out.T, jb.out.C,
                                    jb.out.B, jb.out.L, jb.out.D,
                                    (long long)jb.view.npx * jb.view.npy, jb.vaxis.nchan,
                                    jb.vaxis.v_first_edge_kms, jb.vaxis.dv_kms, P.T0, P.inv_c_kms,
                                    s);
    ++g_launches;
    if (e) return cuda_fail(e, "irt_forward_ppv: T_B conversion");
  }
  return IRT_OK;
}

}  // namespace
}  // namespace irt

// ---------------------------------------------------------------------------
// Several lines of one job in one launch (Sec. 4.1: one or several spectral
// lines, each with its own dust opacity, Sec. 3.2)
// ---------------------------------------------------------------------------
extern "C" irt_status irt_forward_ppv_lines(const irt_job* job, int nlines,
                                            const irt_line* lines, const irt_dust* dusts,
                                            const irt_cubes* outs, const irt_ot_table* table,
                                            const int* table_lines, const irt_opts* opts,
                                            void* cuda_stream) {
  g_err.clear();
  if (!job || !lines || !dusts || !outs || !opts)
    return fail(IRT_EINVAL, "irt_forward_ppv_lines: NULL argument");
  if (nlines < 1) return fail(IRT_EINVAL, "irt_forward_ppv_lines: no lines");
  if (nlines > kMaxLinesPerRender)
    return fail(IRT_EUNSUPPORTED, "irt_forward_ppv_lines: %d lines (at most %d)", nlines,
                kMaxLinesPerRender);
  irt_status st = IRT_OK;
  for (int q = 0; q < nlines; ++q) {
    st = check_line(&lines[q], &dusts[q], opts);
    if (st) return st;
    irt_job jq = *job;
    jq.out = outs[q];
    st = check_job(jq, opts->precision);
    if (st) return st;
  }
  if (opts->mode != IRT_MODE_THICK)
    return fail(IRT_EUNSUPPORTED, "irt_forward_ppv_lines: optically thick mode only");
  if (opts->precision != IRT_PREC_F32)
    return fail(IRT_EUNSUPPORTED, "irt_forward_ppv_lines: float precision only");
  if (job->grid->store == ST_F64)
    return fail(IRT_EUNSUPPORTED, "irt_forward_ppv_lines: float or 16-bit field storage only");
  if (opts->flags & IRT_FLAG_SAVE_CHECKPOINTS)
    return fail(IRT_EUNSUPPORTED, "irt_forward_ppv_lines: no checkpoints");
  if (table) {
    if (!table_lines) return fail(IRT_EINVAL, "irt_forward_ppv_lines: NULL table line indices");
    for (int q = 0; q < nlines; ++q) {
      const int li = table_lines[q];
      if (li < 0 || li >= table->t.nlines)
        return fail(IRT_EINVAL, "irt_forward_ppv_lines: table line %d outside the table's %d",
                    li, table->t.nlines);
      const double nu_t = table->t.nu[li];
      if (!(std::fabs(lines[q].nu_ul_hz - nu_t) <= 1e-12 * nu_t))
        return fail(IRT_EINVAL, "irt_forward_ppv_lines: line %d frequency %.12g Hz differs from "
                                "the table line's %.12g Hz", q, lines[q].nu_ul_hz, nu_t);
    }
  }
  const bool tb = opts->units == IRT_UNITS_TB;
  if (tb)
    for (int q = 0; q < nlines; ++q)
      if (!outs[q].T || !outs[q].C || !outs[q].B)
        return fail(IRT_EINVAL, "irt_forward_ppv_lines: IRT_UNITS_TB needs the T, C and B cubes "
                                "of every line");
  irt_opts o = *opts;
  if (tb) o.units = IRT_UNITS_TRJ;
  LineSet ls;
  std::memset(&ls, 0, sizeof ls);
  ls.n = nlines;
  PhysParams P0;
  std::vector<PhysParams> Ps(nlines);
  for (int q = 0; q < nlines; ++q) {
    Ps[q] = fold_constants(&lines[q], &dusts[q], &o);
    PhysF pf = to_float(Ps[q]);
    if (table) bind_ot(table->t, table_lines[q], &Ps[q], &pf);
    ls.pf[q] = pf;
    ls.out[q][0] = outs[q].T; ls.out[q][1] = outs[q].C; ls.out[q][2] = outs[q].D;
    ls.out[q][3] = outs[q].L; ls.out[q][4] = outs[q].B;
  }
  P0 = Ps[0];
  cudaStream_t s = (cudaStream_t)cuda_stream;
  irt_job jb = *job;
  jb.out = outs[0];
  Tuned tp;
  forced_plan(&tp);
  Plan p = plan_job(jb, IRT_PREC_F32, tp.ni > 0 ? tp.ni : 0);
  p.tw = tp.tw;
  p.th = tp.th;
  JobTable tab;
  std::memset(&tab, 0, sizeof tab);
  tab.j[0] = make_jobdev(jb, p);
  tab.j[0].item_begin = 0;
  StreamScratch& ss = stream_scratch(s);
  st = grow(&ss.fwd, &ss.fwd_bytes, fwd_scratch_need({p}, IRT_PREC_F32, true), s,
            "irt_forward_ppv_lines");
  if (st) return st;
  FwdLaunch L;
  L.total = tab.j[0].nitems;
  L.queue = nullptr;
  L.grid_blocks = 0;
  L.kmax = p.kmax;
  L.fwmax = 32 * p.ni;
  L.cwmax = p.cw;
  L.flags = o.flags;
  L.stats = (o.flags & IRT_FLAG_STATS) ? jb.grid->ctl + 1 : nullptr;
  L.rscr = ss.fwd;
  L.rbytes = ss.fwd_bytes;
  L.lines = &ls;
  const int store = jb.grid->store;
  int e;
  if (o.integration == IRT_SMOOTH)
    e = dispatch_fwd_ml_smooth(store, p.ni, tab, 1, P0, ls.pf[0], L, s);
  else if (o.integration == IRT_FORMAL)
    e = dispatch_fwd_ml_formal(store, p.ni, tab, 1, P0, ls.pf[0], L, s);
  else
    e = dispatch_fwd_ml_kahan(store, p.ni, tab, 1, P0, ls.pf[0], L, s);
  ++g_launches;
  if (e) return cuda_fail(e, "irt_forward_ppv_lines: forward kernel");
  if (!tb) return IRT_OK;
  for (int q = 0; q < nlines; ++q) {
    e = launch_tb_convert(0, outs[q].T, outs[q].C, outs[q].B, outs[q].L, outs[q].D,
                          (long long)jb.view.npx * jb.view.npy, jb.vaxis.nchan,
                          jb.vaxis.v_first_edge_kms, jb.vaxis.dv_kms, Ps[q].T0, Ps[q].inv_c_kms,
                          s);
    ++g_launches;
    if (e) return cuda_fail(e, "irt_forward_ppv_lines: T_B conversion");
  }
  return IRT_OK;
}

// ---------------------------------------------------------------------------
// Optically thin level-balance grids (Sec. 4.2) and the H2 abundance field
// ---------------------------------------------------------------------------
extern "C" irt_status irt_create_ot_table(const irt_level_model* m, const irt_ot_axes* ax,
                                          const int* lines, int nlines, void* cuda_stream,
                                          irt_ot_table** out) {
  g_err.clear();
  if (!m || !ax || !lines || !out) return fail(IRT_EINVAL, "irt_create_ot_table: NULL argument");
  *out = nullptr;
  if (m->nlev < 2) return fail(IRT_EINVAL, "irt_create_ot_table: %d levels (at least 2)", m->nlev);
  if (m->nlev > kOTMaxLevels)
    return fail(IRT_EUNSUPPORTED, "irt_create_ot_table: %d levels (at most %d)", m->nlev,
                kOTMaxLevels);
  if (nlines < 1) return fail(IRT_EINVAL, "irt_create_ot_table: no lines");
  if (nlines > kOTMaxLines)
    return fail(IRT_EUNSUPPORTED, "irt_create_ot_table: %d lines (at most %d)", nlines,
                kOTMaxLines);
  if (m->nrad < 1 || m->npartner < 0 || m->ntemp < 1 || m->ncoll < 0)
    return fail(IRT_EINVAL, "irt_create_ot_table: transition or temperature counts");
  if (m->npartner > 5)
    return fail(IRT_EUNSUPPORTED, "irt_create_ot_table: %d partners (at most 5)", m->npartner);
  if (!m->energy_k || !m->g || !m->rad_up || !m->rad_lo || !m->a_ul_s || !m->nu_hz ||
      (m->npartner > 0 && m->ncoll > 0 &&
       (!m->partner || !m->coll_temp_k || !m->coll_up || !m->coll_lo || !m->k_ul_cm3_s)))
    return fail(IRT_EINVAL, "irt_create_ot_table: NULL model array");
  const int n = m->nlev;
  for (int i = 0; i < n; ++i)
    if (!std::isfinite(m->energy_k[i]) || !finite_pos(m->g[i]))
      return fail(IRT_EINVAL, "irt_create_ot_table: level %d energy or weight", i);
  for (int r = 0; r < m->nrad; ++r) {
    const int u = m->rad_up[r], l = m->rad_lo[r];
    if (u < 0 || u >= n || l < 0 || l >= n || u <= l)
      return fail(IRT_EINVAL, "irt_create_ot_table: radiative transition %d (%d -> %d)", r, u, l);
    if (!finite_pos(m->a_ul_s[r]) || !finite_pos(m->nu_hz[r]))
      return fail(IRT_EINVAL, "irt_create_ot_table: radiative transition %d: A or frequency", r);
  }
  const int np = m->npartner, nt = m->ntemp, nc = m->ncoll;
  for (int p = 0; p < np && nc > 0; ++p) {
    if (m->partner[p] < IRT_PARTNER_H2 || m->partner[p] > IRT_PARTNER_HE)
      return fail(IRT_EINVAL, "irt_create_ot_table: partner %d kind %d", p, m->partner[p]);
    for (int t = 0; t < nt; ++t) {
      const double T = m->coll_temp_k[p * nt + t];
      if (!finite_pos(T) || (t > 0 && !(T > m->coll_temp_k[p * nt + t - 1])))
        return fail(IRT_EINVAL, "irt_create_ot_table: partner %d temperatures must be positive "
                                "and ascending", p);
    }
    for (int c = 0; c < nc; ++c) {
      const int u = m->coll_up[p * nc + c], l = m->coll_lo[p * nc + c];
      if (u < 0 || u >= n || l < 0 || l >= n || u <= l)
        return fail(IRT_EINVAL, "irt_create_ot_table: partner %d transition %d (%d -> %d)", p, c,
                    u, l);
      for (int t = 0; t < nt; ++t)
        if (!finite_nonneg(m->k_ul_cm3_s[((size_t)p * nc + c) * nt + t]))
          return fail(IRT_EINVAL, "irt_create_ot_table: negative or non-finite rate");
    }
  }
  {
    // each level pair once per partner and once among the radiative
    // transitions (the build kernel adds each transition's rates in place)
    std::vector<unsigned char> seen((size_t)n * n);
    for (int p = 0; p < np && nc > 0; ++p) {
      std::fill(seen.begin(), seen.end(), 0);
      for (int c = 0; c < nc; ++c) {
        unsigned char& f = seen[(size_t)m->coll_up[p * nc + c] * n + m->coll_lo[p * nc + c]];
        if (f) return fail(IRT_EINVAL, "irt_create_ot_table: partner %d lists a level pair twice", p);
        f = 1;
      }
    }
    std::fill(seen.begin(), seen.end(), 0);
    for (int r = 0; r < m->nrad; ++r) {
      unsigned char& f = seen[(size_t)m->rad_up[r] * n + m->rad_lo[r]];
      if (f) return fail(IRT_EINVAL, "irt_create_ot_table: a radiative level pair is listed twice");
      f = 1;
    }
  }
  if (!finite_nonneg(m->t_rad_k) || !finite_nonneg(m->ortho_para) || !finite_nonneg(m->x_he))
    return fail(IRT_EINVAL, "irt_create_ot_table: t_rad_k, ortho_para and x_he must be >= 0");
  const int na[3] = {ax->n_n, ax->n_chi, ax->n_t};
  const double lo[3] = {ax->log10_nh_min, ax->chi_min, ax->log10_t_min};
  const double hi[3] = {ax->log10_nh_max, ax->chi_max, ax->log10_t_max};
  for (int a = 0; a < 3; ++a)
    if (na[a] < 2 || !std::isfinite(lo[a]) || !std::isfinite(hi[a]) || !(hi[a] > lo[a]))
      return fail(IRT_EINVAL, "irt_create_ot_table: axis %d needs >= 2 nodes and hi > lo", a);
  if (lo[1] < 0.0 || hi[1] > 0.5)
    return fail(IRT_EINVAL, "irt_create_ot_table: chi axis outside [0, 0.5]");
  for (int q = 0; q < nlines; ++q)
    if (lines[q] < 0 || lines[q] >= m->nrad)
      return fail(IRT_EINVAL, "irt_create_ot_table: line %d names transition %d of %d", q,
                  lines[q], m->nrad);
  const long long nodes = (long long)na[0] * na[1] * na[2];
  if (nodes > (1ll << 26))
    return fail(IRT_EUNSUPPORTED, "irt_create_ot_table: %lld nodes (at most 2^26)", nodes);

  // the model in one device buffer: doubles first, then ints
  std::vector<double> dv;
  auto put_d = [&](const double* p, size_t cnt) {
    const size_t off = dv.size();
    dv.insert(dv.end(), p, p + cnt);
    return off;
  };
  const size_t o_e = put_d(m->energy_k, n), o_g = put_d(m->g, n);
  const size_t o_a = put_d(m->a_ul_s, m->nrad), o_nu = put_d(m->nu_hz, m->nrad);
  const bool coll = np > 0 && nc > 0;
  const size_t o_ct = coll ? put_d(m->coll_temp_k, (size_t)np * nt) : 0;
  const size_t o_k = coll ? put_d(m->k_ul_cm3_s, (size_t)np * nc * nt) : 0;
  std::vector<int> iv;
  auto put_i = [&](const int* p, size_t cnt) {
    const size_t off = iv.size();
    iv.insert(iv.end(), p, p + cnt);
    return off;
  };
  const size_t o_ru = put_i(m->rad_up, m->nrad), o_rl = put_i(m->rad_lo, m->nrad);
  const size_t o_p = coll ? put_i(m->partner, np) : 0;
  const size_t o_cu = coll ? put_i(m->coll_up, (size_t)np * nc) : 0;
  const size_t o_cl = coll ? put_i(m->coll_lo, (size_t)np * nc) : 0;
  const size_t o_ln = put_i(lines, nlines);
  const size_t dbytes = dv.size() * sizeof(double), ibytes = iv.size() * sizeof(int);
  const size_t tab64_bytes = (size_t)nlines * nodes * 2 * sizeof(double);
  const size_t tab32_bytes = (size_t)nlines * na[0] * na[1] * (na[2] - 1) * sizeof(float4);
  irt_ot_table* t = new irt_ot_table();
  std::memset(&t->t, 0, sizeof t->t);
  unsigned char* mbuf = nullptr;
  if (dev_malloc((void**)&mbuf, dbytes + ibytes) != cudaSuccess ||
      dev_malloc((void**)&t->t.tab64, tab64_bytes) != cudaSuccess ||
      dev_malloc((void**)&t->t.tab32, tab32_bytes) != cudaSuccess) {
    cudaGetLastError();
    if (mbuf) cudaFree(mbuf);
    if (t->t.tab64) cudaFree(t->t.tab64);
    delete t;
    return fail(IRT_ENOMEM, "irt_create_ot_table: cannot allocate %zu bytes",
                dbytes + ibytes + tab64_bytes + tab32_bytes);
  }
  cudaStream_t s = (cudaStream_t)cuda_stream;
  cudaError_t ce = cudaMemcpyAsync(mbuf, dv.data(), dbytes, cudaMemcpyHostToDevice, s);
  if (ce == cudaSuccess)
    ce = cudaMemcpyAsync(mbuf + dbytes, iv.data(), ibytes, cudaMemcpyHostToDevice, s);
  OTBuildArgs A;
  std::memset(&A, 0, sizeof A);
  const double* dd = reinterpret_cast<const double*>(mbuf);
  const int* di = reinterpret_cast<const int*>(mbuf + dbytes);
  A.nlev = n; A.nrad = m->nrad; A.npartner = coll ? np : 0; A.ntemp = nt; A.ncoll = coll ? nc : 0;
  A.nlines = nlines;
  A.energy = dd + o_e; A.g = dd + o_g; A.a = dd + o_a; A.nu = dd + o_nu;
  A.ctemp = dd + o_ct; A.k = dd + o_k;
  A.rad_up = di + o_ru; A.rad_lo = di + o_rl; A.partner = di + o_p;
  A.cup = di + o_cu; A.clo = di + o_cl; A.lines = di + o_ln;
  A.t_rad = m->t_rad_k; A.opr = m->ortho_para; A.x_he = m->x_he;
  t->t.nlines = nlines;
  for (int a = 0; a < 3; ++a) {
    A.n[a] = t->t.n[a] = na[a];
    A.lo[a] = t->t.lo[a] = lo[a];
    A.hi[a] = t->t.hi[a] = hi[a];
  }
  for (int q = 0; q < nlines; ++q) {
    // cgs per molecule -> per-step K units: c^2 / (2 k nu^2) for intensities
    // and the profile peak per Hz times b, c / (nu sqrt(pi))
    const double nu = m->nu_hz[lines[q]];
    const double per_hz = kCkms / nu / std::sqrt(kPi);
    t->t.nu[q] = nu;
    A.jk[q] = t->t.jk[q] = kC * kC / (2.0 * kK * nu * nu) * per_hz;
    A.ak[q] = t->t.ak[q] = per_hz;
  }
  cudaGetDevice(&t->t.device);
  int e = ce == cudaSuccess ? launch_ot_build(A, t->t.tab64, t->t.tab32, s) : (int)ce;
  ++g_launches;
  // the staging vectors must outlive the copies; the model buffer the build
  if (e == 0) e = (int)cudaStreamSynchronize(s);
  cudaFree(mbuf);
  if (e) {
    cudaFree(t->t.tab64);
    cudaFree(t->t.tab32);
    delete t;
    return cuda_fail(e, "irt_create_ot_table: level-balance kernel");
  }
  *out = t;
  return IRT_OK;
}

extern "C" irt_status irt_ot_table_values(const irt_ot_table* t, double* out) {
  g_err.clear();
  if (!t || !out) return fail(IRT_EINVAL, "irt_ot_table_values: NULL argument");
  const size_t bytes =
      (size_t)t->t.nlines * t->t.n[0] * t->t.n[1] * t->t.n[2] * 2 * sizeof(double);
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(out, t->t.tab64, bytes, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "irt_ot_table_values");
  return IRT_OK;
}

extern "C" irt_status irt_destroy_ot_table(irt_ot_table* t) {
  g_err.clear();
  if (!t) return IRT_OK;
  cudaFree(t->t.tab64);
  cudaFree(t->t.tab32);
  delete t;
  return IRT_OK;
}

extern "C" irt_status irt_grid_set_h2_fraction(irt_grid* g, const void* chi, int dtype,
                                               void* cuda_stream) {
  g_err.clear();
  if (!g || !chi) return fail(IRT_EINVAL, "irt_grid_set_h2_fraction: NULL argument");
  if (dtype < IRT_F32 || dtype > IRT_F64)
    return fail(IRT_EINVAL, "irt_grid_set_h2_fraction: unknown dtype %d", dtype);
  const long long ncell = (long long)g->nx * g->ny * g->nz;
  const int e = launch_set_chi(g->store, chi, dtype, g->cells, ncell, cuda_stream);
  ++g_launches;
  if (e) return cuda_fail(e, "irt_grid_set_h2_fraction");
  return IRT_OK;
}

// ---------------------------------------------------------------------------
// CUDA graph of one forward call (typically a batch)
// ---------------------------------------------------------------------------
struct irt_graph {
  cudaGraph_t graph;
  cudaGraphExec_t exec;
  unsigned char* scratch;   // record scratch owned by the graph
};

extern "C" irt_status irt_forward_graph_create(const irt_job* jobs, int njobs,
                                               const irt_line* line, const irt_dust* dust,
                                               const irt_opts* opts, irt_graph** out) {
  g_err.clear();
  if (!out) return fail(IRT_EINVAL, "irt_forward_graph_create: NULL out");
  *out = nullptr;
  if (!jobs || njobs < 1) return fail(IRT_EINVAL, "irt_forward_graph_create: no jobs");
  irt_status st = check_line(line, dust, opts);
  if (st) return st;
  if (opts->mode != IRT_MODE_THICK)
    return fail(IRT_EUNSUPPORTED, "irt_forward_graph_create: optically thick mode only");
  if (opts->units == IRT_UNITS_TB)
    return fail(IRT_EUNSUPPORTED, "irt_forward_graph_create: T_RJ or intensity units only");
  for (int j = 0; j < njobs; ++j) {
    st = check_job(jobs[j], opts->precision);
    if (st) return st;
  }
  cudaStream_t cs;
  if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess)
    return fail(IRT_ECUDA, "irt_forward_graph_create: cannot create a capture stream");
  const PhysParams P = fold_constants(line, dust, opts);
  const PhysF PF = to_float(P);
  Tuned tp;
  if (opts->precision != IRT_PREC_F64) {
    const unsigned long long sig = job_signature(jobs, njobs, opts);
    if (!lookup_tuned(sig, &tp) && (opts->flags & IRT_FLAG_AUTOTUNE)) {
      st = autotune(jobs, njobs, P, PF, opts, cs, &tp);
      if (st) {
        cudaStreamDestroy(cs);
        return st;
      }
      store_tuned(sig, tp);
    }
  }
  // the graph's own record scratch, sized like a direct call's
  Scratch sc;
  {
    std::vector<Plan> plans(njobs);
    for (int j = 0; j < njobs; ++j) plans[j] = plan_job(jobs[j], opts->precision, 0);
    sc.bytes = fwd_scratch_need(plans, opts->precision);
  }
  if (dev_malloc((void**)&sc.p, sc.bytes) != cudaSuccess) {
    cudaGetLastError();
    cudaStreamDestroy(cs);
    return fail(IRT_ENOMEM, "irt_forward_graph_create: cannot allocate %zu bytes of scratch",
                sc.bytes);
  }
  irt_graph* g = new irt_graph();
  g->scratch = sc.p;
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed);
  if (e == cudaSuccess) {
    st = run_forward(jobs, njobs, P, PF, opts, tp, cs, &sc);
    const cudaError_t e2 = cudaStreamEndCapture(cs, &g->graph);
    if (!st && e2 != cudaSuccess) st = cuda_fail(e2, "irt_forward_graph_create: end capture");
  } else {
    st = cuda_fail(e, "irt_forward_graph_create: begin capture");
  }
  if (!st) {
    e = cudaGraphInstantiate(&g->exec, g->graph, 0);
    if (e != cudaSuccess) {
      cudaGraphDestroy(g->graph);
      st = cuda_fail(e, "irt_forward_graph_create: instantiate");
    }
  }
  cudaStreamDestroy(cs);
  if (st) {
    cudaFree(g->scratch);
    delete g;
    return st;
  }
  *out = g;
  return IRT_OK;
}

extern "C" irt_status irt_forward_graph_launch(irt_graph* g, void* cuda_stream) {
  g_err.clear();
  if (!g) return fail(IRT_EINVAL, "irt_forward_graph_launch: NULL graph");
  const cudaError_t e = cudaGraphLaunch(g->exec, (cudaStream_t)cuda_stream);
  ++g_launches;
  if (e != cudaSuccess) return cuda_fail(e, "irt_forward_graph_launch");
  return IRT_OK;
}

extern "C" irt_status irt_forward_graph_destroy(irt_graph* g) {
  g_err.clear();
  if (!g) return IRT_OK;
  cudaGraphExecDestroy(g->exec);
  cudaGraphDestroy(g->graph);
  cudaFree(g->scratch);   // waits for launches of the graph still running
  delete g;
  return IRT_OK;
}

extern "C" irt_status irt_tuned_plan(const irt_job* jobs, int njobs, const irt_opts* opts,
                                     int out[3]) {
  g_err.clear();
  if (!jobs || njobs < 1 || !opts || !out) return fail(IRT_EINVAL, "irt_tuned_plan: argument");
  for (int j = 0; j < njobs; ++j)
    if (!jobs[j].grid) return fail(IRT_EINVAL, "irt_tuned_plan: job without grid");
  Tuned t;
  if (!lookup_tuned(job_signature(jobs, njobs, opts), &t)) {
    out[0] = out[1] = out[2] = 0;
    return IRT_OK;
  }
  out[0] = t.ni;
  out[1] = t.tw;
  out[2] = t.th;
  return IRT_OK;
}

extern "C" irt_status irt_adjoint_ppv(const irt_job* job, const irt_line* line,
                                      const irt_dust* dust, const irt_opts* opts,
                                      const irt_cubes* cotangent, float* grad_n_h2,
                                      float* grad_t_gas, float* grad_v_los, void* cuda_stream) {
  g_err.clear();
  if (!job) return fail(IRT_EINVAL, "irt_adjoint_ppv: NULL job");
  if (!grad_n_h2 || !grad_t_gas || !grad_v_los)
    return fail(IRT_EINVAL, "irt_adjoint_ppv: NULL gradient pointer");
  irt_status st = check_line(line, dust, opts);
  if (st) return st;
  if (opts->mode != IRT_MODE_THICK)
    return fail(IRT_EUNSUPPORTED, "irt_adjoint_ppv: optically thick mode only");
  if (opts->units == IRT_UNITS_TB)
    return fail(IRT_EUNSUPPORTED, "irt_adjoint_ppv: T_RJ or intensity units only");
  if (!job->grid) return fail(IRT_EINVAL, "irt_adjoint_ppv: job without grid");
  // the cube pointers of the job are not written by the adjoint
  irt_job jb = *job;
  jb.out.T = grad_n_h2;   // satisfies the "some output" check; never written
  st = check_job(jb, opts->precision);
  if (st) return st;
  if (opts->precision != IRT_PREC_F32)
    return fail(IRT_EUNSUPPORTED, "irt_adjoint_ppv: float precision only");
  irt_grid* g = jb.grid;
  if (g->store == ST_F64)
    return fail(IRT_EUNSUPPORTED, "irt_adjoint_ppv: float or 16-bit field storage only");
  const Plan p = plan_job(jb, IRT_PREC_F32, 0);
  const PhysParams P = fold_constants(line, dust, opts);
  const PhysF PF = to_float(P);
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const int nch = jb.vaxis.nchan;
  // the general sweep's shared memory (records, partials, channel cotangents)
  const size_t dense_smem = adjoint_dense_smem_per_warp(p.kmax, nch);
  if (dense_smem > 110 * 1024)
    return fail(IRT_EUNSUPPORTED, "irt_adjoint_ppv: rays of %d samples with %d channels need "
                                  "%zu bytes of shared memory per warp (at most 112640)",
                p.kmax, nch, dense_smem);
  // the fast sweep (hull blocks in registers, continuum basis) takes smooth
  // jobs of one channel window on any view; every other job, and the rays of
  // a fast job that it cannot take, go to the general sweep
  const bool fast = opts->integration == IRT_SMOOTH && jb.vaxis.subsample_f >= 1 && p.nwin == 1;
  // oblique rays run their own kernel instances (ray set-up, trilinear
  // scatter of the gradients), so the cell-exact instances carry neither
  const bool obl = jb.view.trilinear == 1;
  JobTable tab;
  std::memset(&tab, 0, sizeof tab);
  tab.j[0] = make_jobdev(jb, p);
  const float* cot[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  if (cotangent) {
    cot[0] = (const float*)cotangent->T;
    cot[1] = (const float*)cotangent->C;
    cot[2] = (const float*)cotangent->D;
    cot[3] = (const float*)cotangent->L;
    cot[4] = (const float*)cotangent->B;
  }
  float* grads[3] = {grad_n_h2, grad_t_gas, grad_v_los};
  const long long total = (long long)jb.view.npx * jb.view.npy;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);

  // scratch of this stream: the fast sweep's per-warp buffers, the general
  // sweep's, and the lists (deferred wide rays, general rays, the general
  // sweep's queue counter)
  int blocks_d = 0;
  int e = launch_adjoint_dense(g->store, tab, PF, grads, cot, nullptr, 0, nullptr, 1, 1, 0,
                               nullptr, p.kmax, nch, &blocks_d, s);
  if (e) return cuda_fail(e, "irt_adjoint_ppv: general sweep attributes");
  const long long dense_floats = (adjoint_dense_scratch_per_warp(p.kmax) + 63) & ~63ll;
  size_t need = (size_t)blocks_d * 2 * (size_t)dense_floats * sizeof(float);
  // fast sweep passes: hull buckets up to 4 register blocks first (128
  // registers, the most resident warps), then up to 9, then the job's full
  // width; each pass defers the wider rays to the next through a device list
  int per_warp = 0;
  std::vector<int> nis;
  for (int ni : {4, 9, p.ni})
    if (fast && (nis.empty() || ni > nis.back())) nis.push_back(ni);
  std::vector<int> blocks(nis.size(), 0);
  long long per_warp_floats = 0;
  const int nseg = (p.kmax + kAdjSeg - 1) / kAdjSeg;
  AdjArgs A;
  std::memset(&A, 0, sizeof A);
  if (fast) {
    for (int q = 0; q < 5; ++q) A.cot[q] = cot[q];
    for (int q = 0; q < 3; ++q) A.grad[q] = grads[q];
    e = launch_adjoint(g->store, nis[0], obl, tab, PF, A, 0, nullptr, 0, p.kmax, p.nfw, nch, s,
                       &per_warp);
    if (e) return cuda_fail(e, "irt_adjoint_ppv: kernel attributes");
    const size_t smem = (size_t)per_warp * kAdjWarps;
    int bmax = 0;
    for (size_t i = 0; i < nis.size(); ++i) {
      blocks[i] = std::max(1, adjoint_blocks_per_sm(g->store, nis[i], obl, smem)) * sms;
      bmax = std::max(bmax, blocks[i]);
    }
    // checkpoints, one stored sub-segment, the per-sample chain-rule factors
    const int nb_alloc = nis.back() + 1;
    per_warp_floats =
        (long long)(2 * nseg + kAdjSub) * nb_alloc * 32 + (long long)kAdjChain * p.kmax;
    per_warp_floats = (per_warp_floats + 63) & ~63ll;
    need = std::max(need, (size_t)bmax * kAdjWarps * (size_t)per_warp_floats * sizeof(float));
  }
  // lists: [0] the general sweep's rays, then one per later fast pass, each
  // [count, indices...] of total + 1 words; then the queue counters of the
  // general sweep and of every fast pass (8-byte aligned)
  const size_t lists = 1 + (nis.empty() ? 0 : nis.size() - 1);
  const size_t list_words = lists * (size_t)(total + 1);
  const size_t queue_off = ((list_words * sizeof(unsigned)) + 7) & ~(size_t)7;
  const size_t defer_need = queue_off + (1 + nis.size()) * sizeof(unsigned long long);
  StreamScratch& ss = stream_scratch(s);
  irt_status gs = grow(&ss.adj, &ss.adj_bytes, need, s, "irt_adjoint_ppv");
  if (!gs) gs = grow(&ss.defer, &ss.defer_bytes, defer_need, s, "irt_adjoint_ppv");
  if (gs) return gs;
  unsigned* dense_list = reinterpret_cast<unsigned*>(ss.defer);
  unsigned long long* queues = reinterpret_cast<unsigned long long*>(ss.defer + queue_off);
  // counts of every list and every queue counter start at zero
  cudaError_t ce = cudaMemsetAsync(queues, 0, (1 + nis.size()) * sizeof(unsigned long long), s);
  for (size_t l = 0; l < lists && ce == cudaSuccess; ++l)
    ce = cudaMemsetAsync(dense_list + l * (size_t)(total + 1), 0, sizeof(unsigned), s);
  if (ce != cudaSuccess) return cuda_fail(ce, "irt_adjoint_ppv: queue reset");
  unsigned long long* dense_queue = queues;
  if (jb.view.trilinear == 1) {
    // oblique views: every ray adds into the cells of its samples' stencils
    const size_t cb = (size_t)g->nx * g->ny * g->nz * sizeof(float);
    for (int q = 0; q < 3 && ce == cudaSuccess; ++q) ce = cudaMemsetAsync(grads[q], 0, cb, s);
    if (ce != cudaSuccess) return cuda_fail(ce, "irt_adjoint_ppv: clear gradients");
  }
  if (fast) {
    A.scratch = reinterpret_cast<float*>(ss.adj);
    A.scratch_per_warp = per_warp_floats;
    A.dense = dense_list;
    if (g->ck && g->ck_sig == checkpoint_signature(jb, P)) {
      A.ck_saved = g->ck;
      A.ck_nb = kCkRows;
      A.ck_ray = (long long)nseg * 2 * kCkRows * 32;
    }
    for (size_t i = 0; i < nis.size(); ++i) {
      A.in_list = i == 0 ? nullptr : dense_list + i * (size_t)(total + 1);
      const bool last = i + 1 == nis.size();
      A.defer = last ? nullptr : dense_list + (i + 1) * (size_t)(total + 1);
      A.defer_max_nb = last ? 0 : nis.back();
      e = launch_adjoint(g->store, nis[i], obl, tab, PF, A, total, queues + 1 + i, blocks[i], p.kmax,
                         p.nfw, nch, s, nullptr);
      ++g_launches;
      if (e) return cuda_fail(e, "irt_adjoint_ppv: adjoint kernel");
    }
  }
  // the general sweep: the fast job's leftover rays (a list filled on the
  // device), or every ray of the job
  e = launch_adjoint_dense(g->store, tab, PF, grads, cot, reinterpret_cast<float*>(ss.adj),
                           dense_floats, fast ? dense_list : nullptr,
                           opts->integration == IRT_SMOOTH ? 1 : 0,
                           jb.view.trilinear != 1 ? 1 : 0, total, dense_queue, p.kmax, nch,
                           nullptr, s);
  ++g_launches;
  if (e) return cuda_fail(e, "irt_adjoint_ppv: general sweep");
  return IRT_OK;
}

// ---------------------------------------------------------------------------
// ---------------------------------------------------------------------------
// Latitude-mean reductions (Sec. 6.1)
// ---------------------------------------------------------------------------
extern "C" irt_status irt_mean_axis1(const void* in, int dtype, long long A, long long B,
                                     long long C, void* out, void* cuda_stream) {
  g_err.clear();
  if (!in || !out) return fail(IRT_EINVAL, "irt_mean_axis1: NULL array");
  if (A < 1 || B < 1 || C < 1)
    return fail(IRT_EINVAL, "irt_mean_axis1: extents %lld x %lld x %lld", A, B, C);
  if (A > 65535 || (C + 127) / 128 > 2147483647LL)
    return fail(IRT_EUNSUPPORTED, "irt_mean_axis1: A = %lld above 65535 or C too large", A);
  if (dtype != IRT_F32 && dtype != IRT_F64)
    return fail(IRT_EUNSUPPORTED, "irt_mean_axis1: float or double arrays only");
  const int e = launch_mean_axis1(in, dtype, A, B, C, out, (cudaStream_t)cuda_stream);
  ++g_launches;
  if (e) return cuda_fail(e, "irt_mean_axis1");
  return IRT_OK;
}

extern "C" irt_status irt_beam_convolve(const void* in, int dtype, long long nchan, int npy,
                                        int npx, double fwhm_px, void* scratch, void* out,
                                        void* cuda_stream) {
  g_err.clear();
  if (!in || !scratch || !out) return fail(IRT_EINVAL, "irt_beam_convolve: NULL array");
  if (nchan < 1 || npy < 1 || npx < 1)
    return fail(IRT_EINVAL, "irt_beam_convolve: extents %lld x %d x %d", nchan, npy, npx);
  if (!finite_pos(fwhm_px)) return fail(IRT_EINVAL, "irt_beam_convolve: FWHM must be > 0");
  if (dtype != IRT_F32 && dtype != IRT_F64)
    return fail(IRT_EUNSUPPORTED, "irt_beam_convolve: float or double cubes only");
  if (in == scratch || out == scratch)
    return fail(IRT_EINVAL, "irt_beam_convolve: the scratch cube must be a separate buffer");
  if (nchan > 65535)
    return fail(IRT_EUNSUPPORTED, "irt_beam_convolve: more than 65535 channels");
  const int e = launch_beam(in, dtype, nchan, npy, npx, fwhm_px, scratch, out,
                            (cudaStream_t)cuda_stream);
  g_launches += 2;
  if (e == (int)cudaErrorInvalidValue)
    return fail(IRT_EUNSUPPORTED, "irt_beam_convolve: FWHM %.3g px needs more than 64 taps a "
                                  "side", fwhm_px);
  if (e) return cuda_fail(e, "irt_beam_convolve");
  return IRT_OK;
}

// Render without any device allocation (irt_forward_ppv_static).
//
// The packed cells of the grid, the per-warp sample records and the
// work-queue counter of the persistent launch live in one file-scope device
// array instead of memory allocated by irt_create_grid.  Every device that
// loads the library holds this array (kStaticCellBytes + kStaticRecBytes +
// kStaticCtlBytes) until the process exits.  The record part bounds the
// number of resident warps (each holds the records of its longest ray).  All calls
// share it: a call overwrites the cells and control words of the previous
// call, and two calls whose kernels overlap on the GPU (different streams, or
// different host threads) race on it.
// ---------------------------------------------------------------------------
namespace irt {
namespace {

constexpr size_t kStaticCellBytes = size_t(32) << 20;   // 32 MiB of packed cells
constexpr size_t kStaticRecBytes = size_t(16) << 20;    // 16 MiB of sample records
constexpr size_t kStaticCtlBytes = 256;                   // work-queue and counters
constexpr int kStaticMaxDevices = 64;

static __device__ __align__(256) unsigned char
    g_static_scratch[kStaticCellBytes + kStaticRecBytes + kStaticCtlBytes];

std::mutex g_static_mu;
void* g_static_base[kStaticMaxDevices] = {};

// Device address of the static array on the current device, looked up once per
// device (the host-side name of the array is not a device address).
irt_status static_scratch_base(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "irt_forward_ppv_static: cudaGetDevice");
  if (dev < 0 || dev >= kStaticMaxDevices)
    return fail(IRT_EUNSUPPORTED, "irt_forward_ppv_static: device index %d beyond %d", dev,
                kStaticMaxDevices);
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (!g_static_base[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || !p)
      return cuda_fail(e, "irt_forward_ppv_static: cudaGetSymbolAddress of the static scratch");
    g_static_base[dev] = p;
  }
  *out = g_static_base[dev];
  return IRT_OK;
}

}  // namespace
}  // namespace irt

extern "C" irt_status irt_forward_ppv_static(const irt_grid_desc* desc, const irt_fields* fields,
                                             const irt_view* view, const irt_vaxis* vaxis,
                                             const irt_cubes* out, const irt_line* line,
                                             const irt_dust* dust, const irt_opts* opts,
                                             void* cuda_stream) {
  g_err.clear();
  if (!desc || !fields || !view || !vaxis || !out)
    return fail(IRT_EINVAL, "irt_forward_ppv_static: NULL argument");
  if (desc->nx < 1 || desc->ny < 1 || desc->nz < 1)
    return fail(IRT_EINVAL, "irt_forward_ppv_static: grid size %d x %d x %d", desc->nx, desc->ny,
                desc->nz);
  if (!finite_pos(desc->cell_cm)) return fail(IRT_EINVAL, "irt_forward_ppv_static: cell_cm <= 0");
  const void* src[5] = {fields->n_h2_cm3, fields->t_gas_k, fields->t_dust_k, fields->v_los_kms,
                        fields->x_tracer};
  int dt[5];
  bool any64 = false, all16 = true;
  int bf_mask = 0;
  double scale[5];
  for (int q = 0; q < 5; ++q) {
    if (!src[q]) return fail(IRT_EINVAL, "irt_forward_ppv_static: field %d is NULL", q);
    dt[q] = (int)desc->dtype[q];
    if (dt[q] < IRT_F32 || dt[q] > IRT_F64)
      return fail(IRT_EINVAL, "irt_forward_ppv_static: field %d has unknown dtype %d", q, dt[q]);
    if (dt[q] == IRT_F64) any64 = true;
    if (dt[q] != IRT_F16 && dt[q] != IRT_BF16) all16 = false;
    if (dt[q] == IRT_BF16) bf_mask |= 1 << q;
    scale[q] = desc->scale[q] == 0.0 ? 1.0 : desc->scale[q];
    if (!std::isfinite(scale[q]) || scale[q] <= 0.0)
      return fail(IRT_EINVAL, "irt_forward_ppv_static: scale[%d] must be finite and > 0", q);
  }
  const int store = any64 ? ST_F64 : (all16 ? ST_H16 : ST_F32);
  const size_t cb = store == ST_F64 ? sizeof(CellF64) : store == ST_H16 ? sizeof(CellH16)
                                                                         : sizeof(CellF32);
  const long long ncell = (long long)desc->nx * desc->ny * desc->nz;
  const double need = (double)cb * (double)ncell;
  if (need > (double)kStaticCellBytes)
    return fail(IRT_EINVAL,
                "irt_forward_ppv_static: the grid needs %.0f bytes of packed cells (%lld cells x "
                "%zu B); the static scratch holds at most %zu bytes (%zu cells of this storage)",
                need, ncell, cb, kStaticCellBytes, kStaticCellBytes / cb);
  irt_status st = check_line(line, dust, opts);
  if (st) return st;
  if (opts->flags & IRT_FLAG_SAVE_CHECKPOINTS)
    return fail(IRT_EUNSUPPORTED, "irt_forward_ppv_static: no checkpoints (no grid keeps them)");
  if (opts->flags & IRT_FLAG_STATS)
    return fail(IRT_EUNSUPPORTED, "irt_forward_ppv_static: no work counters (no grid keeps "
                                  "them for irt_grid_stats)");
  if (opts->mode != IRT_MODE_THICK)
    return fail(IRT_EUNSUPPORTED, "irt_forward_ppv_static: optically thick mode only");
  if (opts->units == IRT_UNITS_TB)
    return fail(IRT_EUNSUPPORTED, "irt_forward_ppv_static: T_RJ or intensity units only");

  // a grid descriptor on the host stack pointing into the static array
  irt_grid g;
  g.nx = desc->nx; g.ny = desc->ny; g.nz = desc->nz;
  g.dx = desc->cell_cm;
  g.store = store;
  g.bf16_mask = store == ST_H16 ? bf_mask : 0;
  for (int q = 0; q < 5; ++q) g.scale[q] = scale[q];
  g.cell_bytes = (size_t)need;
  g.device = 0;
  irt_job job;
  job.grid = &g;
  job.view = *view;
  job.vaxis = *vaxis;
  job.out = *out;
  st = check_job(job, opts->precision);
  if (st) return st;
  // the record area must hold one block of warps, each with the records of
  // the longest ray (checked here so that no kernel of the call runs)
  const Plan p = plan_job(job, opts->precision, 0);
  {
    const size_t rec = opts->precision == IRT_PREC_F64 ? kRecBytesF64 : kRecBytesF32;
    const size_t stride = ((size_t)p.kmax * rec + 255) & ~(size_t)255;
    const size_t rec_need = stride * kWarpsPerBlock;
    if (rec_need > kStaticRecBytes)
      return fail(IRT_EINVAL,
                  "irt_forward_ppv_static: rays of up to %d samples need %zu bytes of sample "
                  "records (%d warps x %zu B); the static scratch holds %zu bytes (rays of at most "
                  "%zu samples)",
                  p.kmax, rec_need, kWarpsPerBlock, stride, kStaticRecBytes,
                  (kStaticRecBytes / kWarpsPerBlock) / rec);
  }

  void* base = nullptr;
  st = static_scratch_base(&base);
  if (st) return st;
  g.cells = base;
  unsigned char* recs = static_cast<unsigned char*>(base) + kStaticCellBytes;
  g.ctl = reinterpret_cast<unsigned long long*>(recs + kStaticRecBytes);
  cudaStream_t s = (cudaStream_t)cuda_stream;
  // the work-queue counter must start at zero; the array keeps the last call's values
  cudaError_t ce = cudaMemsetAsync(g.ctl, 0, kStaticCtlBytes, s);
  if (ce != cudaSuccess) return cuda_fail(ce, "irt_forward_ppv_static: clear control words");
  int e = launch_pack(store, src, dt, scale, g.cells, ncell, cuda_stream);
  ++g_launches;
  if (e) return cuda_fail(e, "irt_forward_ppv_static: pack kernel");

  const PhysParams P = fold_constants(line, dust, opts);
  JobTable tab;
  std::memset(&tab, 0, sizeof tab);
  tab.j[0] = make_jobdev(job, p);
  tab.j[0].item_begin = 0;
  const long long total = tab.j[0].nitems;
  FwdLaunch L;
  L.total = total;
  L.queue = nullptr;   // one job: round-robin items
  L.grid_blocks = 0;
  L.kmax = p.kmax;
  L.fwmax = 32 * p.ni;
  L.cwmax = p.cw;
  L.flags = opts->flags;
  L.stats = nullptr;
  L.rscr = recs;
  L.rbytes = kStaticRecBytes;
  L.lines = nullptr;
  e = dispatch(opts->precision, opts->integration, store, p.ni, tab, 1, P, to_float(P), L, s);
  ++g_launches;
  if (e) return cuda_fail(e, "irt_forward_ppv_static: forward kernel");
  return IRT_OK;
}

/*
 * irt.h - C ABI of the B300 (sm_103a) IRIS-SO synthetic-observation library.
 *
 * The library turns 3-D gas fields (H2 density, gas and dust temperature,
 * line-of-sight velocity, tracer abundance) into position-position-velocity
 * cubes of a molecular line plus dust continuum, with the five components
 * [T] total, [C] continuum, [D] dust excess, [L] line and [B] background.
 *
 * Method (paper sections):
 *   Sec. 3.1  dI/ds = j - alpha I for the total and the continuum intensity
 *   Sec. 3.2  dust alpha_D = kappa rho_gas with a Planck source B_nu(T_dust)
 *   Sec. 3.3  line j = h nu A n_u phi / 4 pi, alpha = h nu (n_l B_lu - n_u B_ul) phi / 4 pi
 *             with a Gaussian Doppler profile phi
 *   Sec. 3.7  Einstein relations B_ul = c^2 A / (2 h nu^3), B_lu = (g_u/g_l) B_ul
 *   Sec. 5.10 LTE populations n_i = N g_i exp(-E_i / kT) / Z(T)
 *   Sec. 4.3  T_inf cut-off and Doppler-shifted frequencies
 *   Sec. 4.4/4.5 optically thick transfer on a fine velocity grid (step dv/(2f),
 *             Table 4) with a Simpson channel average; continuum and background
 *             at the channel value
 *   Sec. 4.8  formal (exponential) and smooth (trapezoidal first step, BDF2,
 *             ReLU) integration
 *   Sec. 4.9/4.10 Rayleigh-Jeans temperature output; [L] = [T] - [C]
 *
 * Conventions fixed where the paper is silent:
 *   - LTE with E_l = E_u - h nu / k and a rigid-rotor Z(T) with constant B0.
 *   - Frequency of velocity u: nu(u) = nu_ul (1 - u / c), positive = receding.
 *     The Doppler width b^2 = 2 k T / m + 2 sigma_turb^2 (sigma = 1-D rms).
 *   - Channel c spans [v0 + c dv, v0 + (c+1) dv] km/s.  f >= 1: fine points
 *     v0 + g dv/(2f), g = 0 .. 2 f nchan, edges shared by adjacent channels;
 *     f = 0: the channel centre alone.
 *   - Smooth integration puts the background on the first sample node;
 *     formal integration applies K full steps.
 *   - [D] = [C] - [B].  Outputs are Rayleigh-Jeans temperatures at each
 *     channel centre frequency (or cgs intensity with IRT_UNITS_INTENSITY).
 *   - Geometry: view.trilinear = 0 is the z view: pixel (x, y) is the cell
 *     column (x, y), rays travel along +z (background at z = 0, observer
 *     beyond z = nz dx), one sample per cell.  view.trilinear = 1 is an
 *     orthographic view along d = (sin t cos p, sin t sin p, cos t): pixel
 *     (px, py) sits at box_centre + (px - (npx-1)/2) pixel e_t + (py - (npy-1)/2)
 *     pixel e_p with e_t = (cos t cos p, cos t sin p, -sin t), e_p = (-sin p,
 *     cos p, 0); the chord through the box is split into K = ceil(chord/dx)
 *     equal steps sampled at their midpoints with trilinear interpolation of
 *     cell-centred values (indices clamped at the faces).  view.trilinear = 2
 *     is the radial view of an observer-centred spherical tensor (Sec. 2.2)
 *     stored [r][b][l] as [z][y][x]: pixel (x, y) = (l, b), the ray runs
 *     from the far end r = nz - 1 (background) to the observer at r = 0, one
 *     sample per cell with step cell_cm = the radial spacing.
 *
 * All entry points are asynchronous on the given CUDA stream (NULL = legacy
 * default stream) and never throw.  A status other than IRT_OK means that no
 * kernel of the failed call was launched (except IRT_ECUDA after a launch,
 * which reports the CUDA error); irt_last_error() gives a message.
 */
#ifndef IRT_H_
#define IRT_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define IRT_ABI_VERSION 1

typedef enum {
  IRT_OK = 0,
  IRT_EINVAL = 1,          /* invalid argument, detected before any launch */
  IRT_ENOMEM = 2,          /* device allocation failed */
  IRT_ECUDA = 3,           /* CUDA runtime error (message has the CUDA string) */
  IRT_EUNSUPPORTED = 4,    /* valid but not supported combination */
  IRT_ETIMEOUT = 5         /* a bounded device wait gave up */
} irt_status;

typedef enum { IRT_F32 = 0, IRT_F16 = 1, IRT_BF16 = 2, IRT_F64 = 3 } irt_dtype;

typedef enum { IRT_FORMAL = 0, IRT_SMOOTH = 1, IRT_FORMAL_KAHAN = 2 } irt_integration;
/* Output units.  TRJ: Rayleigh-Jeans temperature [K] at each channel's
 * centre frequency; INTENSITY: erg s^-1 cm^-2 Hz^-1 sr^-1; TB: Planck
 * brightness temperature [K] at the channel centre, with the continuum
 * subtracted in that space ([L] = T_B([T]) - T_B([C]), [D] = T_B([C]) -
 * T_B([B]); Sec. 4.9, 4.10).  The adjoint takes TRJ or INTENSITY.  The
 * thick mode with TB renders T_RJ and converts in a second pass, so it needs
 * the T, C and B cubes of every job (IRT_EINVAL otherwise); the graph API and
 * irt_forward_ppv_static take TRJ or INTENSITY. */
typedef enum { IRT_UNITS_TRJ = 0, IRT_UNITS_INTENSITY = 1, IRT_UNITS_TB = 2 } irt_units;
typedef enum { IRT_PREC_F32 = 0, IRT_PREC_F64 = 1 } irt_precision;
/* Transfer modes (Sec. 4.5-4.7).  THICK: line and dust interact at every
 * fine velocity (velocity subsampling f, Simpson channel average).
 * SELECTIVELY_THIN: no subsampling; each channel uses the channel-averaged
 * line profile (Gaussian mass in the channel / channel width); the continuum
 * is solved first and the total sees j_L + j_D - alpha_L I_C with absorption
 * alpha_D (the line does not absorb itself).  THIN: absorption and
 * stimulation ignored, I = I_bg + integral of j (formal: midpoint sum;
 * smooth: Simpson over node pairs, trapezoid on an odd last interval).  The
 * thin modes take IRT_FORMAL or IRT_SMOOTH, ignore subsample_f, and are
 * rendered by irt_forward_ppv only (no graph, static entry or adjoint). */
typedef enum {
  IRT_MODE_THICK = 0,
  IRT_MODE_SELECTIVELY_THIN = 1,
  IRT_MODE_THIN = 2,
  IRT_MODE_DENSITY_TRACING = 3
} irt_transfer_mode;
/* IRT_MODE_DENSITY_TRACING (Sec. 5.10, "simple observation"): the tracer
 * column density per unit velocity [cm^-2 per km/s], each sample spreading
 * x n_H2 h over velocity with the line's Doppler profile (channel-averaged
 * like the thin modes), summed as the optically thin integral (IRT_FORMAL
 * midpoint, IRT_SMOOTH Simpson); no T_inf cut, background or dust; units
 * ignored.  Written to out.T and out.L; out.C, out.D, out.B are zero. */

/* opts.flags */
#define IRT_FLAG_EXPLICIT_CHANNELS 1u  /* evaluate every channel explicitly (no
                                          continuum basis shortcut) */
#define IRT_FLAG_STATS 2u              /* accumulate work counters into the first
                                          job's grid (see irt_grid_stats) */
#define IRT_FLAG_AUTOTUNE 4u           /* time the launch plans for this job mix
                                          (synchronous; not during stream capture)
                                          and cache the fastest */
#define IRT_FLAG_SAVE_CHECKPOINTS 8u   /* one z- or radial-view job, smooth, float: keep
                                          the transfer state every 32 samples in
                                          the grid, for irt_adjoint_ppv of the
                                          same job, which then skips its own
                                          forward sweep */

typedef struct irt_grid irt_grid;   /* opaque */

/* Grid: nx * ny * nz cubic cells of side cell_cm.  dtype[q] is the storage
 * type of field q (order of irt_fields); the physical value of field q is
 * the stored value times scale[q] (0 means 1).  Scales let 16-bit storage
 * hold densities above the fp16 range or abundances below its normal range. */
typedef struct {
  int nx, ny, nz;
  double cell_cm;
  irt_dtype dtype[5];
  double scale[5];
} irt_grid_desc;

/* Field pointers, C order [z][y][x] (x fastest), device memory:
 * n_h2_cm3 [cm^-3], t_gas_k [K], t_dust_k [K], v_los_kms [km/s, + receding],
 * x_tracer (tracer number density / n_H2). */
typedef struct {
  const void *n_h2_cm3, *t_gas_k, *t_dust_k, *v_los_kms, *x_tracer;
} irt_fields;

/* Line constants: frequency [Hz], Einstein A [1/s], upper-level energy [K],
 * rotational constant [Hz], statistical weights, molecular mass [amu],
 * T_inf cut-off [K], 1-D microturbulent dispersion [km/s]. */
typedef struct {
  double nu_ul_hz, a_ul_s, e_u_k, b0_hz, g_u, g_l, mass_amu, t_inf_k, sigma_turb_kms;
} irt_line;

/* Dust: opacity per gram of gas [cm^2/g]; gas mass per H2 molecule [amu]. */
typedef struct {
  double kappa_cm2_per_g_gas, mu_mass_per_h2_amu;
} irt_dust;

typedef struct {
  double theta_rad, phi_rad;
  int npx, npy;        /* image size (z and radial views: must equal nx, ny) */
  double pixel_cm;     /* pixel pitch (oblique views) */
  int trilinear;       /* 0: z view (cell exact), 1: oblique trilinear view,
                          2: radial view of an [r][b][l] tensor (cell exact) */
} irt_view;

typedef struct {
  int nchan;                 /* >= 1 */
  double v_first_edge_kms;   /* lower edge of channel 0 */
  double dv_kms;             /* channel width, > 0 */
  int subsample_f;           /* velocity-subsampling factor f >= 0 */
} irt_vaxis;

typedef struct {
  int mode;            /* irt_transfer_mode */
  int integration;     /* irt_integration */
  int units;           /* irt_units */
  double t_bg_k;       /* background (CMB) temperature [K], >= 0 */
  int precision;       /* irt_precision: arithmetic type of the kernels */
  unsigned flags;      /* IRT_FLAG_* */
} irt_opts;

/* Output cubes, device memory, [nchan][npy][npx].  float for IRT_PREC_F32,
 * double for IRT_PREC_F64.  A NULL entry is not written. */
typedef struct {
  void *T, *C, *D, *L, *B;
} irt_cubes;

typedef struct {
  irt_grid* grid;
  irt_view view;
  irt_vaxis vaxis;
  irt_cubes out;
} irt_job;

/*
 * irt_create_grid - copy the five fields (device pointers, layout above) into
 * a grid owned by the library, in a cell-interleaved layout.  The grid is the
 * library's form of the paper's physical tensor (Sec. 2.2: velocity,
 * density, gas and dust temperature and abundances sampled on a regular
 * lattice; Sec. 2.3 for the gas temperature): here a Cartesian lattice of
 * cubic cells, or the paper's observer-centred [r][b][l] tensor read with
 * its radial axis as z (see irt_view).  Storage: all
 * 16-bit fields stay 16-bit (fp16/bf16 per field); otherwise fields are kept
 * as float, or as double when any field is IRT_F64.  Later edits to the
 * caller's buffers do not affect the grid.  On success *out is a new handle
 * to release with irt_destroy.  IRT_EINVAL for non-positive sizes, a
 * non-positive or non-finite cell size, NULL pointers or an unknown dtype;
 * IRT_ENOMEM if the device allocation fails.
 *
 * Every device allocation of the library (grids, scratch, graphs) fails with
 * IRT_ENOMEM, without calling the CUDA runtime, while the environment
 * variable IRT_FAIL_ALLOC is set to a non-empty value other than "0" (read on
 * every call): host-side fault injection for tests of the IRT_ENOMEM paths.
 */
irt_status irt_create_grid(const irt_grid_desc* desc, const irt_fields* fields,
                           void* cuda_stream, irt_grid** out);

/*
 * irt_update_grid - copy new field values into an existing grid (same size,
 * cell, storage and 16-bit scales as at creation; IRT_EINVAL otherwise),
 * asynchronously on cuda_stream, without any allocation: a caller rendering
 * many snapshots of one shape (a training loop) keeps its grids.  The H2
 * abundance returns to 0.5 and checkpoints kept by earlier renders no longer
 * apply.  Launches using the grid on other streams must have finished.
 */
irt_status irt_update_grid(irt_grid* grid, const irt_grid_desc* desc, const irt_fields* fields,
                           void* cuda_stream);

/*
 * irt_forward_ppv - render njobs >= 1 jobs (Sec. 4.4-4.10).  A work item is
 * one ray with every channel.  njobs == 1 runs one persistent launch whose
 * warps take the rays round-robin; njobs > 1 runs one persistent launch per
 * table of up to 64 jobs, its warps pulling rays from a device work queue
 * (longest rays first).  The output cubes are written completely (every
 * channel of every pixel).  A grid takes part in one launch at a time (its
 * work-queue counter).  IRT_EINVAL before any launch for: njobs < 1, NULL
 * job, grid or constants, nchan < 1, dv <= 0, f < 0, a non-finite or negative
 * constant, a z view whose size differs from the grid or whose angles are
 * non-zero, an oblique view with npx/npy < 1 or pixel <= 0; all output
 * pointers NULL.  IRT_EUNSUPPORTED for IRT_PREC_F64 on a grid that is not
 * stored as double, f > 64, or more than 32000 fine velocities (2 f nchan + 1).
 *
 * IRT_FLAG_SAVE_CHECKPOINTS (njobs == 1, z or radial view, IRT_SMOOTH, float precision,
 * else IRT_EUNSUPPORTED) stores, in a buffer the grid owns (npx x npy x
 * ceil(nz / 32) x 2 x 10 x 32 floats, grown on demand), the transfer state of
 * every ray every 32 samples, with a signature of the job (velocity axis,
 * line, dust, background).  A later irt_adjoint_ppv of the same grid and an
 * identical job on the same stream uses it instead of re-integrating the
 * forward; any other job ignores it.
 *
 * Scratch: the per-warp sample records (and the adjoint's checkpoints) live in
 * device buffers the library keeps per (device, stream) and reuses across
 * grids and calls; they grow on demand (a growth waits for the device) and
 * are held until the process exits.  A call that would grow them during
 * stream capture fails with IRT_EUNSUPPORTED: run it once uncaptured first.
 * Graphs from irt_forward_graph_create own their buffer.
 */
irt_status irt_forward_ppv(const irt_job* jobs, int njobs, const irt_line* line,
                           const irt_dust* dust, const irt_opts* opts, void* cuda_stream);

/*
 * CUDA graph of one irt_forward_ppv call (usually a batch): the queue reset and
 * the persistent kernel with the job table and launch plan baked in.  The
 * grids and output cubes named by the jobs must outlive the graph; launching
 * it re-renders them from the grids' current contents.  With
 * IRT_FLAG_AUTOTUNE the plan is tuned first (synchronously) if the job mix
 * has no cached plan.  Errors as irt_forward_ppv; IRT_ECUDA if capture or
 * instantiation fails.
 */
typedef struct irt_graph irt_graph;
irt_status irt_forward_graph_create(const irt_job* jobs, int njobs, const irt_line* line,
                                    const irt_dust* dust, const irt_opts* opts,
                                    irt_graph** out);
irt_status irt_forward_graph_launch(irt_graph* graph, void* cuda_stream);
irt_status irt_forward_graph_destroy(irt_graph* graph);

/*
 * irt_tuned_plan - the cached plan of a job mix: out = {fine blocks per lane
 * NI (32 NI velocities per channel window), tile width, tile height} in rays,
 * or {0, 0, 0} if the mix was never tuned (the default plan is used).
 */
irt_status irt_tuned_plan(const irt_job* jobs, int njobs, const irt_opts* opts, int out[3]);

/*
 * irt_adjoint_ppv - gradients of a scalar loss with respect to n_H2, T_gas
 * and v_los of every cell for one job (Sec. 4 intro: the observation is
 * differentiable end to end; Sec. 4.8 run in reverse), given the cotangents
 * dLoss/d[T], d[C], d[D], d[L], d[B] (float cubes [nchan][npy][npx], NULL =
 * zero).  grad_* are float [nz][ny][nx], written completely (overwritten, not
 * accumulated; a cell no ray samples gets zero).  Any view, integrator
 * (IRT_FORMAL_KAHAN is differentiated as the formal step it equals), f and
 * channel count.  Two sweeps: smooth jobs of one channel window, on any
 * view, run the fast sweep (line hull in registers, continuum basis; 4
 * register blocks first, then the rays with wider hulls at 9 blocks, then at
 * the job's full width), which hands the rays it cannot take (h alpha_D >
 * 1/2 on some sample, a line window wider than 64 fine velocities) to the
 * general sweep; every other job runs the general sweep alone (every
 * velocity explicit).  Oblique views add each sample's gradients to its
 * eight trilinear cells with atomics, so their sums may differ in the last
 * bits between runs.  The
 * forward state is recomputed from checkpoints every 32 samples held in
 * device scratch kept per (device, stream).  IRT_EINVAL as irt_forward_ppv
 * plus NULL gradients; IRT_EUNSUPPORTED for IRT_PREC_F64, double field
 * storage, the thin modes, T_B units, or rays and channel counts whose
 * per-warp shared memory (52 bytes a sample + 8 bytes a channel) exceeds
 * 110 KiB.
 */
irt_status irt_adjoint_ppv(const irt_job* job, const irt_line* line, const irt_dust* dust,
                           const irt_opts* opts, const irt_cubes* cotangent,
                           float* grad_n_h2, float* grad_t_gas, float* grad_v_los,
                           void* cuda_stream);

/*
 * irt_forward_ppv_static - render one job without allocating device memory.
 * The paper has no counterpart: this entry point exists for callers that may
 * not call cudaMalloc, for example a plugin whose host application owns all
 * device memory and hands it only finished buffers, or a real-time loop that
 * must not block on the allocator or fail with out-of-memory after start-up.
 * The caller passes the fields (device pointers, layout and dtypes as for
 * irt_create_grid) and the output cubes; the packed copy of the fields, the
 * per-warp sample records and the work-queue counter go to one file-scope
 * device array of 32 MiB + 16 MiB + 256 bytes that every device loading the
 * library holds until the process exits (the 16 MiB of records bound the
 * warps the launch keeps resident: each holds the records of its longest
 * ray).  A grid needing more than 32 MiB of packed cells (32, 16 or
 * 64 bytes per cell for float, 16-bit or double storage; e.g. 1,048,576 float
 * cells) is rejected with IRT_EINVAL and a message giving both sizes, and so
 * is a view whose longest ray needs more than the 16 MiB of records for one
 * block of 4 warps (48 bytes a sample in float precision, 64 in double:
 * rays of at most 87,381 or 65,536 samples); both checks come before any
 * CUDA call.  The call issues no cudaMalloc/cudaFree.
 * IRT_FLAG_SAVE_CHECKPOINTS and IRT_FLAG_STATS give IRT_EUNSUPPORTED (no grid
 * keeps checkpoints or work counters).  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress); make that first call before
 * any stream capture.  All calls share the array and it keeps the last call's
 * contents (the counter is cleared by each call): calls whose kernels overlap
 * on the GPU, on different streams or host threads, race and must be
 * serialised by the caller.  Other argument checks and errors as
 * irt_forward_ppv.
 */
irt_status irt_forward_ppv_static(const irt_grid_desc* desc, const irt_fields* fields,
                                  const irt_view* view, const irt_vaxis* vaxis,
                                  const irt_cubes* out, const irt_line* line,
                                  const irt_dust* dust, const irt_opts* opts,
                                  void* cuda_stream);

/*
 * Non-LTE level populations by the optically thin (OT) level balance
 * (Sec. 3.4-3.6) through a precomputed coefficient grid (Sec. 4.2, 4.3).
 *
 * irt_level_model describes the tracer molecule as a molecular data file
 * does (Sec. 4.1): nlev levels (2..64) with energies E_i / k [K] and weights
 * g_i; nrad radiative transitions (rad_up > rad_lo, Einstein A [1/s],
 * frequency [Hz]); npartner collision partners (irt_partner kinds, at most
 * 5), each with ncoll de-excitation transitions (coll_up > coll_lo, indices
 * [partner][c]) and rate coefficients k_ul_cm3_s [partner][c][t] [cm^3/s]
 * tabulated at coll_temp_k [partner][t] (ntemp ascending temperatures; linear
 * interpolation in T, end values held beyond); the excitation rates follow
 * by detailed balance at the gas temperature (Sec. 3.6).  t_rad_k is the
 * blackbody background T-bar of the balance (0 = pure OT), ortho_para the
 * ortho-/para-H2 ratio, x_he the He abundance per H nucleus.  Partner
 * densities at total H density n_H and H2 abundance chi (H2 per H nucleus):
 * H2 chi n_H, para/ortho H2 split by ortho_para, H (1 - 2 chi) n_H, He
 * x_he n_H.  All arrays are host memory, read during the call.
 *
 * irt_ot_axes: the grid nodes, uniform in log10 n_H [cm^-3], in chi and in
 * log10 T [K] (each axis >= 2 nodes; the paper's grid is 128 x 64 x 64).
 */
typedef enum {
  IRT_PARTNER_H2 = 0, IRT_PARTNER_PH2 = 1, IRT_PARTNER_OH2 = 2, IRT_PARTNER_H = 3,
  IRT_PARTNER_HE = 4
} irt_partner;

typedef struct {
  int nlev;
  const double* energy_k;
  const double* g;
  int nrad;
  const int* rad_up;
  const int* rad_lo;
  const double* a_ul_s;
  const double* nu_hz;
  int npartner;
  const int* partner;
  int ntemp;
  const double* coll_temp_k;
  int ncoll;
  const int* coll_up;
  const int* coll_lo;
  const double* k_ul_cm3_s;
  double t_rad_k;
  double ortho_para;
  double x_he;
} irt_level_model;

typedef struct {
  int n_n, n_chi, n_t;
  double log10_nh_min, log10_nh_max;
  double chi_min, chi_max;
  double log10_t_min, log10_t_max;
} irt_ot_axes;

typedef struct irt_ot_table irt_ot_table;   /* opaque */

/*
 * irt_create_ot_table - solve the OT level system at every grid node (one
 * FP64 solve per node on the device, Sec. 4.2) and keep, for each of the
 * nlines (1..8) radiative transitions lines[] of the model, the
 * frequency-integrated line emission and absorption coefficients per tracer
 * molecule, j = (h nu / 4 pi) A f_u and alpha = (h nu / 4 pi)(f_l B_lu -
 * f_u B_ul) (Sec. 3.3, 3.6).  Asynchronous on cuda_stream (the model is
 * copied before the call returns).  IRT_EINVAL for NULL arguments, level or
 * transition indices out of range, non-positive weights, frequencies, A or
 * temperatures, negative rates, unknown partners, axes with fewer than 2
 * nodes or empty ranges, chi outside [0, 0.5]; IRT_EUNSUPPORTED beyond 64
 * levels, 5 partners or 8 lines; IRT_ENOMEM.
 */
irt_status irt_create_ot_table(const irt_level_model* model, const irt_ot_axes* axes,
                               const int* lines, int nlines, void* cuda_stream,
                               irt_ot_table** out);

/* irt_ot_table_values - copy the grid to host memory, synchronously:
 * out[nlines][n_n][n_chi][n_t][2] = (j, alpha) per tracer molecule [cgs]. */
irt_status irt_ot_table_values(const irt_ot_table* table, double* out);

/* irt_destroy_ot_table - free a grid (NULL is a no-op); no launch may still
 * use it. */
irt_status irt_destroy_ot_table(irt_ot_table* table);

/*
 * irt_grid_set_h2_fraction - the H2 abundance chi (H2 molecules per H
 * nucleus, device array [z][y][x] of dtype IRT_F32/F16/BF16/F64) of every
 * cell, kept in the grid beside the five fields (in the grid's storage
 * precision, fp16 for 16-bit grids).  Used only by irt_forward_ppv_ot; a grid
 * whose abundance was never set is fully molecular (chi = 0.5).  Asynchronous
 * on cuda_stream.  IRT_EINVAL for NULL arguments or an unknown dtype.
 */
irt_status irt_grid_set_h2_fraction(irt_grid* grid, const void* chi, int dtype,
                                    void* cuda_stream);

/*
 * irt_forward_ppv_ot - irt_forward_ppv with the line coefficients of the OT
 * level balance: each sample looks up line line_index of the grid at
 * (log10 n_H, chi, log10 T) by trilinear interpolation, the cell index
 * clamped to the grid so that beyond its bounds the edge cell continues
 * linearly (Sec. 4.2), with n_H = n_H2 / chi, and multiplies by the tracer
 * density x n_H2 (Sec. 4.3).  line supplies the profile (mass, sigma_turb),
 * T_inf and the frequency, which must equal the grid line's to 1e-12
 * relative; its a_ul_s, e_u_k, b0_hz, g_u and g_l are not used.  A sample with
 * n_H2, chi or x not positive, or T outside (0, T_inf], has no line.  Modes,
 * precisions, units and errors as irt_forward_ppv; IRT_EINVAL for a NULL
 * table, a line index out of range or a frequency mismatch;
 * IRT_EUNSUPPORTED for IRT_FLAG_SAVE_CHECKPOINTS (the adjoint takes LTE
 * populations only).
 */
irt_status irt_forward_ppv_ot(const irt_job* jobs, int njobs, const irt_ot_table* table,
                              int line_index, const irt_line* line, const irt_dust* dust,
                              const irt_opts* opts, void* cuda_stream);

/*
 * irt_forward_ppv_lines - render nlines (1..4) spectral lines of one job in
 * one persistent launch (Sec. 4.1: one or several lines; Sec. 3.2: each line
 * with its own dust opacity): line q takes its constants lines[q], its dust
 * dusts[q] and writes the cubes outs[q] (job->out is not used).  Each ray's
 * field samples are taken once (cell loads, trilinear blends) and kept for
 * the ray's other lines; the per-sample physics, the transfer and the
 * epilogue run per line.  With table != NULL the lines take their
 * coefficients from the OT grid, line q from grid line table_lines[q] (as
 * irt_forward_ppv_ot).  Each line's cubes equal those of a single-line
 * irt_forward_ppv (or irt_forward_ppv_ot) call with the same arguments.
 * Thick mode, float precision, float or 16-bit storage; units as
 * irt_forward_ppv (T_B by a conversion pass per line).  IRT_EINVAL as
 * irt_forward_ppv per line, and for a NULL table_lines or a frequency
 * mismatch with the table; IRT_EUNSUPPORTED for other modes, precisions or
 * storage, more than 4 lines or IRT_FLAG_SAVE_CHECKPOINTS.
 */
irt_status irt_forward_ppv_lines(const irt_job* job, int nlines, const irt_line* lines,
                                 const irt_dust* dusts, const irt_cubes* outs,
                                 const irt_ot_table* table, const int* table_lines,
                                 const irt_opts* opts, void* cuda_stream);

/* irt_destroy - free the grid and everything it owns (NULL is a no-op).  The
 * caller must make sure no launch using the grid is still running. */
irt_status irt_destroy(irt_grid* grid);

/*
 * irt_grid_stats - copy (synchronously, after the device is idle on all
 * streams) the work counters a forward call with IRT_FLAG_STATS accumulated
 * into this grid, then zero them if reset != 0.  out[6] = work items, ray
 * samples (summed over rays once, whatever the number of channel windows),
 * (sample, 32-velocity block) pairs where the line was evaluated,
 * (sample, block) pairs integrated explicitly, items integrated without the
 * continuum shortcut, and fine-velocity updates of the dense method
 * (samples x fine velocities).  IRT_EINVAL for NULL arguments.
 */
irt_status irt_grid_stats(irt_grid* grid, unsigned long long out[6], int reset);

/* Last error message of the calling thread ("" if none). */
const char* irt_last_error(void);

/* Number of kernel launches the library issued on this thread since the last
 * call (for launch accounting in benchmarks). */
long long irt_launch_count(void);

/*
 * irt_measure_pipe_peaks - microbenchmark of the two pipes that bound the
 * transfer kernels on the current device at its present clock: FP32 fused
 * multiply-adds and special-function (ex2.approx) results, each as lane
 * operations per second (best of three timed launches after a warm-up, about
 * a millisecond of kernels in all, on cuda_stream, synchronised).  The paper
 * has no counterpart: the measurement harness divides by these numbers.
 * Allocates and frees a small device buffer.  IRT_EINVAL for NULL outputs,
 * IRT_ENOMEM, IRT_ECUDA.
 */
irt_status irt_measure_pipe_peaks(double* fp32_ops_per_s, double* mufu_ops_per_s,
                                  void* cuda_stream);

/*
 * Latitude-mean reduction (Sec. 6.1): out[a][c] = mean over b of in[a][b][c]
 * for a C-order [A][B][C] device array (dtype IRT_F32 or IRT_F64, out the
 * same type, [A][C], device memory, not overlapping in).  On a PPV cube
 * [nchan][npy][npx] it is the l-v image u (b = y); on a field [nz][ny][nx]
 * the top-down map t.  Float input is summed in float (8 interleaved partial
 * sums), double in double.  Asynchronous on cuda_stream; the caller owns
 * both arrays.  IRT_EINVAL for NULL arrays or extents < 1, IRT_EUNSUPPORTED
 * for another dtype or A > 65535, IRT_ECUDA for a launch error.
 */
irt_status irt_mean_axis1(const void* in, int dtype, long long A, long long B, long long C,
                          void* out, void* cuda_stream);

/*
 * Gaussian beam convolution (Sec. 4.11) of a [nchan][npy][npx] device cube
 * (dtype IRT_F32 or IRT_F64): each channel image convolved with a separable
 * Gaussian of FWHM fwhm_px pixels (the paper's 30 arcsec divided by the
 * map's angular pixel size); sigma = FWHM / (2 sqrt(2 ln 2)), taps out to
 * ceil(4 sigma) normalised to unit sum, the sky outside the image zero.
 * scratch is a caller-owned cube of the same size (the pass along x lands
 * there); out may equal in.  Asynchronous on cuda_stream.  IRT_EINVAL for
 * NULL arrays, bad extents, FWHM <= 0 or a scratch aliasing in/out;
 * IRT_EUNSUPPORTED for another dtype, more than 64 taps a side or more than
 * 65535 channels.
 */
irt_status irt_beam_convolve(const void* in, int dtype, long long nchan, int npy, int npx,
                             double fwhm_px, void* scratch, void* out, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* IRT_H_ */

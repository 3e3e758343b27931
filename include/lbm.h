/*
 * lbm.h -- C ABI of the GB300 (sm_103a) MRT-Smagorinsky lattice Boltzmann
 * solver for forced homogeneous isotropic turbulence (Khan, Succi &
 * Falcucci, "Validating the Boltzmann approach to the large-eddy simulations
 * of forced homogeneous incompressible turbulence").
 *
 * The library advances the D3Q19 Guo-MRT evolution equation, Eq. (mrt_les_guo)
 * of Sec. 2.3 with the matrices of App. B, on a periodic box: one fused
 * stream + collide kernel per time step, the Smagorinsky relaxation rate
 * 1/s_nu = 1/2 + 3 (nu0 + C |S|) computed per cell from the non-equilibrium
 * moments (Eqs. eddy_visc, les_viscosity, strain_norm, yu_strain), and the
 * forcing of Eq. (forcing_pattern) applied as the Guo source of Eq. (guo_force).
 * Diagnostics (energy, injection, dissipation, the turbulent Knudsen number
 * K_t of Eq. (Kt_definition), the energy spectrum of Eq. (integral_length_scale),
 * structure functions and flatness of Eqs. (structure_function), (flatness))
 * are fused FP64 reductions on the device.
 *
 * Conventions shared by every entry point
 *  - Lattice units: dx = dt = 1, rho0 = 1, cs^2 = 1/3 (App. A).
 *  - Populations are numbered a = 0..18 in the paper's order 1..19 (App. B
 *    table; a = 18 is the rest particle).  They are stored on the device
 *    weight-shifted, f' = f - w_a, in FP32, FP16 or BF16.
 *  - Host arrays are C-contiguous with x fastest:
 *      populations [19][nz][ny][nx], vectors [3][nz][ny][nx], scalars [nz][ny][nx].
 *  - A handle holds one or more independent instances ("ensemble") that
 *    advance together; `inst` selects one (0 for a single-instance handle).
 *  - All pointers to host buffers are owned by the caller; the library never
 *    keeps them after the call returns.  Device memory is owned by the handle.
 *  - Every function returns LBM_OK (0) or a negative LBM_ERR_* code;
 *    lbm_last_error() gives a one-line description.  Errors raised inside a
 *    kernel (non-finite statistics, a device wait that gave up) surface at the
 *    next synchronising call (lbm_sync, lbm_stats, lbm_spectrum, lbm_get_*).
 *  - A handle is bound to one CUDA device and one stream and is not
 *    thread-safe.
 */
#ifndef LBM_GB300_H
#define LBM_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LBM_OK 0
#define LBM_ERR_INVALID_ARG (-1)
#define LBM_ERR_CUDA (-2)
#define LBM_ERR_OOM (-3)
#define LBM_ERR_UNSTABLE (-4)   /* a statistics pass met NaN or Inf */
#define LBM_ERR_TIMEOUT (-5)    /* a bounded device-side wait gave up */
#define LBM_ERR_UNSUPPORTED (-6)

/* Storage precision of the populations (arithmetic is FP32 in every case). */
#define LBM_FP32 0
#define LBM_FP16_SHIFTED 1      /* f - w stored as IEEE binary16 */
#define LBM_BF16_SHIFTED 2      /* f - w stored as bfloat16 */

/* External force F(x). */
#define LBM_FORCE_NONE 0
#define LBM_FORCE_PAPER_SIN 1   /* Eq. (forcing_pattern): Fx = F0 sin(2 pi y/ny),
                                   Fy = F0 sin(2 pi z/nz), Fz = F0 sin(2 pi x/nx);
                                   (i, j, k) read as the 0-based (x, y, z) */
#define LBM_FORCE_CONST 2       /* uniform body_force */
#define LBM_FORCE_KOLMOGOROV 3  /* Fx = F0 sin(2 pi y/ny) only (one mode of the above) */

/* Initial fields for lbm_init_field. Populations become f' = M^-1 m^eq(drho, u)
 * (App. B) with the given u, i.e. the local equilibrium. */
#define LBM_INIT_REST 0         /* u = 0, drho = 0 */
#define LBM_INIT_TGV3D 1        /* u = A sin X cos Y cos Z, v = -A cos X sin Y cos Z,
                                   w = 0, X = 2 pi x / nx (Taylor-Green, Sec. 3.1) */
#define LBM_INIT_TGV2D 2        /* u = A sin X cos Y, v = -A cos X sin Y, w = 0 and
                                   drho = 3 (A^2/4)(cos 2X + cos 2Y) */
#define LBM_INIT_VELOCITY 3     /* u from the caller, drho = 0 */

/* Which quantities lbm_stats computes beyond the fused domain sums. */
#define LBM_STATS_SPECTRUM 1    /* derived scales from E(k) (needs cuFFT) */
#define LBM_STATS_STRUCTURE 2   /* S_p(r), p = 1..6, and F4(r) */

#define LBM_MAX_R 24

typedef struct lbm_params {
  int32_t nx, ny, nz;     /* lattice size, each >= 1 */
  int32_t precision;      /* LBM_FP32 | LBM_FP16_SHIFTED | LBM_BF16_SHIFTED */
  double re;              /* Re = U0 nx / nu0 (Sec. 3.1); used when nu0 <= 0 */
  double u0;              /* characteristic velocity U0 (lu), > 0 when used */
  double nu0;             /* bare viscosity (lu); <= 0: nu0 = u0 nx / re */
  double cs;              /* Smagorinsky constant C of Eq. (eddy_visc), >= 0 */
  double cf;              /* Cf of Eq. (forcing_amplitude) */
  double f0;              /* forcing amplitude; <= 0: F0 = cf u0^2 / nx (rho0 = 1) */
  double body_force[3];   /* LBM_FORCE_CONST */
  int32_t force_mode;     /* LBM_FORCE_* */
  int32_t stats_every;    /* > 0: lbm_step fuses the statistics into every step
                             whose input time t has t % stats_every == 0 and
                             appends a record (lbm_series); 0: never */
  int32_t hist_bins;      /* bins of the theta histogram on [0, hist_max); 0: 4096 */
  int32_t device;         /* CUDA device ordinal */
  double hist_max;        /* <= 0: 0.02 */
  void* stream;           /* cudaStream_t to run on; NULL: the handle creates one */
  int32_t kernel;         /* 0: autotune; 1: direct-load kernel; 2: TMA bulk-copy kernel */
  int32_t tile_rows;      /* rows (of nx cells) per tile; 0: autotune */
  int32_t stages;         /* TMA pipeline stages; 0: autotune */
  int32_t threads;        /* threads per block; 0: autotune.  kernel, tile_rows,
                             stages (TMA) and threads all set: no autotuning */
  int32_t row_align;      /* byte alignment of each x-line (power of two >= 16;
                             0: 16).  Padding costs memory, not bandwidth: only
                             the nx live cells of a line are moved */
  int32_t strain_mode;    /* 0: the strain of Eq. (yu_strain) with the bare shear
                             rate s9 = s_nu0 (explicit); 1: with the local rate
                             s9 = s_nu(|S|) of Eq. (les_viscosity), solved per cell
                             (closed form of the pure-shear quadratic, then two
                             Newton steps: self-consistent) */
  int32_t layout;         /* population array in device memory: 1 population-
                             major [19][nz][ny][nxp], 2 row-interleaved
                             [nz][ny][19][nxp] (the 19 x-lines of a cell row are
                             adjacent, grouped as lbm_device_ptr states: longer
                             contiguous runs for the TMA kernel); 0: the autotuner picks for the TMA kernel,
                             population-major otherwise.  Results do not depend
                             on it. */
  int32_t tma_slots;      /* shared-memory tiles of the TMA kernel: 0 compile-time
                             slots when the tile fits one (the autotuner also
                             tries the runtime stride), 1 always the runtime
                             stride (x-lines of a tile packed; with one-x-line
                             tiles of the row-interleaved array an odd step
                             copies each slot group of a cell row in one piece),
                             2 the compile-time slots sized for two co-resident
                             blocks per SM (two stages of 2880-byte slots) */
} lbm_params;

/* Domain statistics of one instance at one time (all FP64 sums on the device). */
typedef struct lbm_stats_s {
  int64_t step;           /* time t of the state described */
  int64_t cells;
  double mass;            /* sum over cells of drho = rho - 1 */
  double momentum[3];     /* sum of rho u, u = (sum f c + F/2)/rho (Eq. guo_velocity) */
  double E_k;             /* 1/2 <u.u> (Sec. 2.2) */
  double inj;             /* <F.u> (Eq. energy_balance) */
  double eps0;            /* 2 nu0 <S_ij S_ij> = nu0 <|S|^2>, S from Eq. (yu_strain) */
  double eps_sgs;         /* 2 <nu_t S_ij S_ij> */
  double uu[6];           /* <ux ux>, <uy uy>, <uz uz>, <ux uy>, <ux uz>, <uy uz> */
  double theta_mean;      /* theta = tau_e - 1/2 (Sec. 4.1) */
  double theta_var;
  double theta_min, theta_max;
  double theta_p05, theta_p50, theta_p95, theta_p99;  /* from the histogram: bin centres */
  double Kt_mean, Kt_var; /* K_t = sqrt(3) theta / l with l = dx (Eq. Kt_definition) */
  /* LBM_STATS_SPECTRUM, with k_s = 2 pi s / nx (Eqs. integral_length_scale -
   * dissipation_rate, Sec. 3.1); NaN when not requested. */
  double L, eps_spec, eta, lambda, u_rms, Re_lambda;
  /* LBM_STATS_STRUCTURE (Eqs. velocity_increment - flatness); nr = 0 if not requested. */
  int32_t nr;
  int32_t r[LBM_MAX_R];
  double Sp[LBM_MAX_R][6];  /* S_p(r) for p = 1..6, three axes pooled */
  double F4[LBM_MAX_R];
  /* Isotropy (Sec. 3.2, Fig. isotropy_validation) from the fused <u_i u_j>
   * (the mean flow is zero: the forcing sums to zero over the box):
   * E_i / E, b_ij = <u_i u_j>/<u_k u_k> - delta_ij/3 (xx, yy, zz, xy, xz, yz),
   * II_b = -b_ij b_ji / 2, III_b = b_ij b_jk b_ki / 3, and the Lumley
   * coordinates xi = (III_b/2)^(1/3), eta = (-II_b/3)^(1/2). */
  double E_frac[3];
  double b[6];
  double II_b, III_b, lumley_xi, lumley_eta;
} lbm_stats_t;

/* One record of the fused in-step statistics (lbm_params.stats_every). */
typedef struct lbm_record_s {
  int64_t step;
  double mass, momentum[3], E_k, inj, eps0, eps_sgs;
  double theta_mean, theta_var, theta_min, theta_max;
} lbm_record_t;

typedef struct lbm_s* lbm_t;

/* Create a single-instance handle: validates the parameters, derives nu0 from Re
 * (Sec. 3.1), s_nu0 from Eq. (bare_viscosity) and F0 from Eq. (forcing_amplitude),
 * allocates one population array (19 nz ny nxp values, nxp = nx rounded up to 16
 * bytes) and autotunes the step kernel.  The populations start at the rest
 * state.  Errors: INVALID_ARG (sizes < 1, nu0 and re both unusable, C < 0,
 * unknown enum), OOM, CUDA. */
int lbm_create(const lbm_params* params, lbm_t* out);

/* Create a handle with `count` independent instances (params[0..count-1]; sizes,
 * physics and seeds may differ, precision and device must agree).  One launch
 * per time step advances all of them (tiles of every instance in one grid).
 * Errors as lbm_create; UNSUPPORTED if precisions or devices differ. */
int lbm_create_batch(const lbm_params* params, int32_t count, lbm_t* out);

/* The batch entry points under their ensemble names (Sec. 3: statistics of
 * independent forced-HIT runs; no counterpart in the paper's solver, which runs
 * one box): lbm_batch_create is lbm_create_batch; lbm_batch_step(h, n)
 * advances every instance by n steps in the same launches as lbm_step;
 * lbm_batch_stats(h, what, out) fills out[i] (caller-owned, lbm_count(h)
 * entries) with lbm_stats of instance i, stopping at the first error.
 * Errors as the functions they stand for. */
int lbm_batch_create(const lbm_params* params, int32_t count, lbm_t* out);
int lbm_batch_step(lbm_t h, int64_t n);
int lbm_batch_stats(lbm_t h, int32_t what, lbm_stats_t* out);

/* Release every device resource of the handle.  Accepts NULL. */
int lbm_destroy(lbm_t h);

/* Number of instances of the handle. */
int lbm_count(lbm_t h);

/* Set instance `inst` to the local equilibrium f' = M^-1 m^eq(drho, u) (App. B)
 * of an initial field (Sec. 3.1).  mode = LBM_INIT_*; amplitude is A of the
 * Taylor-Green modes; for LBM_INIT_VELOCITY, u points to 3 nz ny nx FP64 values
 * ([3][nz][ny][nx]) in
 *   u_on_device = 0: host memory, copied in bounded chunks through a device
 *                    staging buffer;
 *   u_on_device = 1: device memory of the handle's device;
 *   u_on_device = 2: page-locked host memory (cudaHostAlloc, cudaMallocHost or
 *                    cudaHostRegister) that the initialisation kernel reads in
 *                    place over the host link, no staging copy; both ends of
 *                    the range are checked to be page-locked (INVALID_ARG
 *                    otherwise) and the whole range must be one such block.
 * The caller keeps ownership; the call is asynchronous on the handle's stream,
 * so u must stay valid until the next synchronising call.  Resets the step
 * counter of the handle to 0 when count == 1.  Errors: INVALID_ARG, CUDA. */
int lbm_init_field(lbm_t h, int32_t inst, int32_t mode, double amplitude,
                   const double* u, int32_t u_on_device);

/* LBM_INIT_VELOCITY from an FP32 field u[3][nz][ny][nx] (same layout, same
 * u_on_device values 0 / 1 / 2 and the same checks as lbm_init_field).  The
 * equilibrium is computed from the FP32 rounding of the velocity in either
 * entry point, so an FP32 field gives exactly the populations of the FP64
 * field it was rounded from, with half the bytes to move.  No counterpart in
 * the paper (an input format).  Errors: INVALID_ARG, CUDA. */
int lbm_init_velocity_f32(lbm_t h, int32_t inst, const float* u, int32_t u_on_device);

/* Set instance `inst` to the local equilibrium of a seeded random solenoidal
 * velocity field generated on the device.  The paper's runs start from a
 * Taylor-Green field (Sec. 3.1) and are analysed in a statistically stationary
 * forced state; this field stands in for such states as a synthetic input:
 *   modes 0 < |k| <= kc, kc = max(1, min(n_min/2 - 1, floor(6 k0))), half space
 *   kz > 0 | (kz = 0, ky > 0) | (kz = ky = 0, kx > 0) with conjugate partners;
 *   per mode and component a complex standard normal (Box-Muller of uniforms
 *   from SplitMix64 applied twice to a counter of (seed mod 2^32, k, component,
 *   draw)); projected normal to k (divergence-free); integer shell
 *   s = round(|k|) scaled to the energy s^4 exp(-2 (s/k0)^2); a global factor
 *   so that u_rms = sqrt(<u.u>/3) = urms; u(x) = sum_k u_hat(k) e^{2 pi i k.x/n}
 *   by a cuFFT complex-to-real transform in FP64, rounded to FP32.
 * Deterministic: the same seed gives the same field on every run.  u_out (may
 * be NULL) receives that FP32 velocity [3][nz][ny][nx]: host memory
 * (u_out_on_device = 0) or device memory of the handle's device (1).
 * Allocates its work buffers (about 28 bytes per cell) for the duration of
 * the call and synchronises the handle's stream.  Its cost beyond the
 * transforms grows with kc^3 (under a millisecond for k0 = 4, kc = 24).  Resets the step counter
 * when count == 1.  Errors: INVALID_ARG (urms or k0 not finite and > 0, an
 * extent < 4, u_out_on_device not 0 or 1), OOM, CUDA (cuFFT failures
 * included). */
int lbm_init_random_spectrum(lbm_t h, int32_t inst, uint64_t seed, double urms, double k0,
                             float* u_out, int32_t u_out_on_device);

/* Advance every instance by n >= 0 time steps of Eq. (mrt_les_guo): collide in
 * moment space, stream with periodic wrap (AA pattern: one population array,
 * even steps write in place, odd steps to the neighbours).  Asynchronous on the
 * handle's stream; launches are replayed from captured CUDA graphs.
 * Errors: INVALID_ARG (n < 0), CUDA. */
int lbm_step(lbm_t h, int64_t n);

/* Block until the handle's stream is idle; report device-side errors
 * (UNSTABLE, TIMEOUT) raised since the previous check. */
int lbm_sync(lbm_t h);

/* Time t (number of steps taken since the last init / set). */
int64_t lbm_time(lbm_t h);

/* Statistics of instance `inst` at the current time: one read-only pass of the
 * step kernel computes the same per-cell quantities as a collision (drho, u, |S|,
 * theta) and reduces them in FP64; `what` adds LBM_STATS_SPECTRUM and/or
 * LBM_STATS_STRUCTURE.  Synchronous.  Errors: INVALID_ARG, UNSTABLE, TIMEOUT
 * (a bounded wait of the TMA kernel's pass gave up), CUDA. */
int lbm_stats(lbm_t h, int32_t inst, int32_t what, lbm_stats_t* out);

/* Fused in-step records (params.stats_every > 0) of instance `inst` appended
 * since the previous call, oldest first, at most `max` (the device keeps the
 * last 1024).  *count receives the number written.  Synchronous. */
int lbm_series(lbm_t h, int32_t inst, lbm_record_t* out, int32_t max, int32_t* count);

/* Relative residual of the energy balance of Eq. (energy_balance),
 * eps = -dE_k/dt + <F.u>, along a record series (lbm_series): for the interior
 * records k = 1..n-2, residual[k-1] = (eps_k - (-(E_{k+1} - E_{k-1}) /
 * (t_{k+1} - t_{k-1}) + inj_k)) / eps_k with eps = eps0 + eps_sgs (molecular
 * plus Smagorinsky dissipation).  `at` (may be NULL) receives the record
 * times.  Host arithmetic only (no device call).  Errors: INVALID_ARG
 * (n < 3, null pointers, non-increasing times). */
int lbm_energy_balance(const lbm_record_t* rec, int32_t n, double* residual, int64_t* at);

/* Energy spectrum E(s), s = 0..kmax, of Eq. (integral_length_scale) with
 * |u_hat|^2, u_hat = N^-3 sum_x u exp(-2 pi i k.x/N), integer shells
 * s - 1/2 <= |k| < s + 1/2 (cuFFT R2C in FP32, shell sums in FP64).  E points
 * to kmax + 1 doubles of host memory.  Synchronous.  Errors: INVALID_ARG
 * (kmax < 0), CUDA (cuFFT failures included). */
int lbm_spectrum(lbm_t h, int32_t inst, double* E, int32_t kmax);

/* theta histogram of the last lbm_stats call of `inst`: `bins` counts
 * (bins == params.hist_bins) plus, in counts[bins], the cells at or above hist_max. */
int lbm_histogram(lbm_t h, int32_t inst, uint64_t* counts, int32_t bins);

/* Canonical populations of `inst` at the current time, FP64 host array
 * [19][nz][ny][nx]: weight-shifted f' (shifted = 1) or f = f' + w (shifted = 0).
 * Exact conversion of the stored values.  Synchronous. */
int lbm_get_populations(lbm_t h, int32_t inst, double* host, int32_t shifted);

/* Overwrite the populations of `inst` (same layout as lbm_get_populations,
 * rounded to the storage precision).  Together with lbm_get_populations and
 * lbm_set_time this is checkpoint / resume: a resumed run is bitwise identical
 * to an uninterrupted one. */
int lbm_set_populations(lbm_t h, int32_t inst, const double* host, int32_t shifted);

/* Set the handle's time counter (all instances; only the AA parity and the
 * statistics schedule depend on it).  The stored populations are re-laid out
 * so that the canonical state is unchanged. */
int lbm_set_time(lbm_t h, int64_t t);

/* Per-cell fields of `inst` at the current time (FP64 host arrays, any may be
 * NULL): drho [nz][ny][nx], u [3][nz][ny][nx] (Guo-corrected), |S| and theta =
 * tau_e - 1/2 [nz][ny][nx].  Computed in FP32 by the read-only step pass. */
int lbm_get_fields(lbm_t h, int32_t inst, double* drho, double* u, double* snorm,
                   double* theta);

/* The Guo-corrected velocity u = (sum_a f_a c_a + F/2) / rho (Eq. guo_velocity)
 * of `inst` at the current time into the caller-owned FP64 host array
 * u[3][nz][ny][nx]: lbm_get_fields with only u requested.  Synchronous.
 * Errors: INVALID_ARG (null handle or output, instance out of range), CUDA. */
int lbm_get_velocity(lbm_t h, int32_t inst, double* u);

/* One plane of theta = tau_e - 1/2 (the K_t map of Sec. 4.1): axis 0, 1, 2 =
 * the plane x = index, y = index or z = index; host array of the plane's two
 * other extents (row-major, the faster axis last).  Synchronous.  A z-plane
 * reads that plane's cells only (x- and y-planes cut every tile: the whole
 * lattice); non-finite values appear in the slice as such, the domain-wide
 * check is lbm_stats'.  Errors: INVALID_ARG (null handle or output, instance,
 * axis or index out of range), TIMEOUT, UNSTABLE (x- and y-planes), CUDA. */
int lbm_get_theta_slice(lbm_t h, int32_t inst, int32_t axis, int32_t index, double* host);

/* Device pointer and size in bytes of the population array of `inst`, for
 * zero-copy inspection (read-only by convention), in the AA order of the
 * current parity and in the layout lbm_kernel_config reports:
 * [19][nz][ny][nxp] (population-major, slot a at index a) or
 * [nz][ny][19][nxp] (row-interleaved; the 19 slots of a cell row in the order
 * 0 1 18 11 3 7 8 13 5 15 16 4 14 17 12 2 6 9 10, grouped by the slot's
 * (cy, cz)). */
int lbm_device_ptr(lbm_t h, int32_t inst, void** ptr, size_t* bytes, int32_t* nxp);

/* Effective parameters after derivation: nu0, s_nu0, F0, C of `inst`. */
int lbm_get_params(lbm_t h, int32_t inst, double* nu0, double* s_nu0, double* f0, double* C);

/* Kernel chosen by the autotuner: kind (1 direct, 2 TMA bulk), tile rows,
 * pipeline stages, threads per block, blocks per SM, population layout (1
 * population-major, 2 row-interleaved), shared-memory slot bytes of the TMA
 * tiles (0: runtime stride).  Any pointer may be NULL. */
int lbm_kernel_config(lbm_t h, int32_t* kind, int32_t* tile_rows, int32_t* stages,
                      int32_t* threads, int32_t* blocks_per_sm, int32_t* layout,
                      int32_t* slot_bytes);

/* Test hook for the failure path (no counterpart in the paper): the next
 * TMA-kernel step launch of `h` runs with every device-side wait bounded by
 * wait_seconds, and block 0 never loads its first tile, so that its consumers'
 * wait runs out.  The kernel then records LBM_ERR_TIMEOUT, waits for its copies
 * in flight (at most 4 x wait_seconds; copies still missing then are reported
 * in the error text) and returns; the next synchronising call reports
 * LBM_ERR_TIMEOUT and the handle stays usable (re-initialise the state: the
 * withheld tile was not updated).  Nothing faults or hangs.
 * Errors: INVALID_ARG (wait_seconds outside (0, 10]), UNSUPPORTED (the handle
 * runs the direct kernel). */
int lbm_debug_withhold_load(lbm_t h, double wait_seconds);

/* Structure functions S_p(r), p = 1..6, of a velocity field the caller already
 * holds in device memory, computed without allocating any device memory.  The
 * paper has no counterpart: it is a service for callers that cannot call
 * cudaMalloc, such as code sharing the GPU with a framework whose pool
 * allocator owns the device memory, or pipelines that must not risk the
 * implicit synchronisation of cudaMalloc / cudaFree.
 *   u      device, FP32 [3][nz][ny][nx] (x fastest), on the current device
 *   r      host, nr separations, each >= 1 (periodic wrap)
 *   sp     device, nr x 6 doubles: sp[k][p-1] = <(u_a(x + r_k e_a) - u_a(x))^p>
 *          over cells and the three axes, the same quantity as lbm_stats.Sp
 *   stream cudaStream_t to run on (NULL: the default stream); asynchronous
 * Limit: 1 <= nr <= 24.  The per-block partial sums live in one fixed array of
 * 576 KiB of device memory that each GPU loading the library holds until the
 * process exits; every call shares it, so calls whose work overlaps on the GPU
 * (other streams, other threads) race and must be serialised by the caller.
 * The first call on a device looks up that array's address with the device
 * current; make that first call before any stream capture begins.
 * Before any launch, both ends of u (3 nx ny nz floats) and of sp (nr x 6
 * doubles) are checked to be device or managed memory of the current device
 * (cudaPointerGetAttributes, which allocates nothing).
 * Errors: INVALID_ARG (null pointer, extents < 1, nr outside [1, 24], r < 1,
 * u or sp not device memory of the current device), CUDA; lbm_last_error(NULL)
 * gives the text. */
int lbm_structure_functions_noalloc(const float* u, int32_t nx, int32_t ny, int32_t nz,
                                    const int32_t* r, int32_t nr, double* sp, void* stream);

/* Text of the last error of `h` (or of the last failed create when h is NULL).
 * The pointer stays valid until the next call on the same handle. */
const char* lbm_last_error(lbm_t h);

/* Library version string. */
const char* lbm_version(void);

#ifdef __cplusplus
}
#endif
#endif /* LBM_GB300_H */

/*
 * lym1.h -- C ABI of a GB300 (sm_103a) implementation of one substep of the
 * Lydion M1 method for Lyman-alpha radiative transfer on a 2D grid
 * (arXiv 2606.02711, "Lydion").
 *
 * One substep of length dt (Sec. 2.1, "overall update scheme"), per cell and
 * frequency bin k:
 *   1. explicit finite-volume transport of J and H with the M1 (Levermore)
 *      closure, MinMod-limited reconstruction of J and f = H/J, the
 *      asymptotic-preserving GLF flux for J, the modified GLF flux for K and
 *      upwind advection of uJ/c, uH/c, plus the -grad(u):K/c work term
 *      (Sec. 2.1 step 1);
 *   2. implicit emission / dust absorption / destruction of J and H
 *      (Sec. 2.1 step 2, absorption-step equations);
 *   3. the Lya radiation force f = 4 pi/(c ct) sum_k dnu_k (H' - H'')/dt
 *      (Sec. 2.3, force equation);
 *   4. the implicit (BDF1) frequency diffusion + recoil + Doppler solve per
 *      cell with the exponential scheme, then H <- (J_new/J_old) H
 *      (Sec. 2.1 step 3 and App. A).
 *
 * Geometry: 2D Cartesian, uniform square cells of width dx; the slab has depth
 * dx (cell volume dx^3).  Boundaries: outflow (two ghost layers that copy the
 * edge cell).  State per (bin, cell): J, Hx, Hy in erg cm^-2 s^-1 Hz^-1 sr^-1
 * (frequency-integrated, erg cm^-2 s^-1 sr^-1, for a gray group).
 * Array layout: per-cell fields [ny][nx] (x fastest), state [nb][ny][nx].
 *
 * Memory: the library allocates and owns all device memory of a context.
 * Caller buffers may be host (pageable or pinned) or device pointers: copies
 * use unified addressing.  The library never keeps a caller pointer after a
 * call returns.  A context is bound to one CUDA stream and is not thread-safe.
 *
 * Errors: every function returns LYM1_OK (0) or a negative code below.  On
 * error the context state is unchanged unless stated otherwise.
 */
#ifndef LYM1_H
#define LYM1_H

#ifdef __cplusplus
extern "C" {
#endif

#define LYM1_OK 0
#define LYM1_EINVAL (-1)         /* invalid argument (null pointer, size, option) */
#define LYM1_ENOMEM (-2)         /* device allocation failed */
#define LYM1_ECUDA (-3)          /* a CUDA runtime call or kernel launch failed */
#define LYM1_ENONFINITE (-4)     /* a diagnostic sum is not finite (NaN/Inf in the state) */
#define LYM1_ETIMEOUT (-5)       /* a kernel's bounded wait on its own bulk copies expired (sticky,
                                    reported by lym1_synchronize and lym1_diagnostics) */
#define LYM1_ENOTCONVERGED (-6)  /* substep cap reached before the steady-state test passed */
#define LYM1_ENODEVICE (-7)      /* no CUDA device is usable */
#define LYM1_ERANGE (-8)         /* size beyond the fixed maximum of an allocation-free call */

/* Arithmetic of the substep. */
#define LYM1_FP64_DET 0    /* FP64, fixed operation order, no FMA contraction, own exp/expm1 */
#define LYM1_FP64 1        /* FP64 with FMA and hardware exp/expm1 */
#define LYM1_MIXED 2       /* FP32 state, transport and closure; FP64 implicit steps 2-3 and
                              conservation sums (the force sum: compensated FP32) */
#define LYM1_MIXED_FAST 3  /* FP32 throughout (compensated FP32 sums per cell, FP64 across
                              cells); subtraction-free solve */

typedef struct lym1_ctx lym1_ctx;

typedef struct {
  int nx, ny;      /* cells in x and y, each >= 1 */
  double dx_cm;    /* cell width (cm), > 0 */
  int geometry;    /* 0 = 2D Cartesian slab of depth dx, outflow on all four sides;
                      1 = axisymmetric (R, Z) as in the paper's tests and RHD runs (Sec. 4):
                      x = R from the axis (R = 0 at the left edge), y = Z from the midplane
                      (Z = 0 at the bottom edge); the axis reflects (H_R, u_R mirrored), the
                      midplane is a mirror (H_Z, u_Z mirrored), the outer R and Z edges are
                      outflow; finite volumes per radian with the hoop source of div K; a
                      cell's lum is emitted into its full ring volume 2 pi Vol; energies and
                      force integrals cover the ring volumes of the half-space Z > 0 */
  int bc[4];       /* x-, x+, y-, y+ outflow kind: 0 = zero gradient (two ghost layers copying
                      the edge cell); 1 = outflow into vacuum (the ghosts carry no radiation,
                      opacities and velocities are copied: radiation leaves and never enters,
                      for clouds surrounded by vacuum as in Sec. 4).  The mirrored sides of
                      geometry 1 (x- and y-) ignore their entry. */
} lym1_grid;

typedef struct {
  int n_bins;                  /* bins in edges_dnu_hz (n_bins + 1 edges), ignored if edges is NULL */
  const double *edges_dnu_hz;  /* ascending bin edges in nu - nu_Lya (Hz), host memory, or NULL for
                                  the paper's grid (Sec. 2.1): widths dnu_D(T_min) q^j, |dnu| <=
                                  min(1e5 dnu_D(T_min), 0.99 nu_Lya, nu_LyC - nu_Lya) */
  double q;                    /* growth factor of the paper grid (0 => 1.1) */
  double T_min;                /* resolution temperature of the paper grid, K (0 => 30) */
  int gray;                    /* 1: one gray group with opacity alpha*eta, eta = sum_k w_k <H>_k
                                  over the grid; no frequency step */
} lym1_groups;

typedef struct {
  const double *n_hi;     /* [ny][nx] neutral hydrogen density, cm^-3 (alpha = n_hi sigma0) */
  const double *rho_dust; /* [ny][nx] dust mass density, g cm^-3 */
  const double *p_d;      /* [ny][nx] Lya destruction probability per scattering */
  const double *ux, *uy;  /* [ny][nx] gas velocity, cm/s */
  double temp_K;          /* gas temperature (uniform), K, > 0 */
  double kappa_abs;       /* dust kappa_ext (1 - omega), cm^2/g */
  double kappa_F;         /* dust kappa_ext (1 - omega g), cm^2/g */
  double c_tilde;         /* (reduced) speed of light, cm/s (0 => c) */
  double cfl;             /* CFL_RT (0 => 0.4); dt_RT = cfl/2 * dx / (c_tilde + max|u|) */
  int recoil;             /* 1: atomic recoil term in the frequency step */
  int freq_step;          /* 1: run the frequency step (ignored for a gray group) */
  int precision;          /* LYM1_FP64_DET, LYM1_FP64, LYM1_MIXED or LYM1_MIXED_FAST */
  void *cuda_stream;      /* cudaStream_t the context runs on; NULL = legacy default stream */
  const double *temp_field; /* [ny][nx] gas temperature per cell, K, each > 0 (host or device
                               pointer), or NULL for the uniform temp_K.  With a field the
                               per-bin tables (App. A: <H>_k, Doppler width, a_v, sigma0; Sec. 2.1
                               step 2: emission fractions; the recoil factor h/(k_B T)) are built
                               for every cell's own temperature, once at creation, on the host
                               (the routine of the uniform case, once per distinct value), and
                               held per [bin][cell] on the device.  Contexts with and without a
                               field cannot share a batch. */
} lym1_opacities;

typedef struct {
  int nb;                 /* state bins (1 for a gray group) */
  int precision;
  double dt_cfl;          /* RT time step dt_RT (s) */
  double eta;             /* sum_k w_k <H>_k over the grid */
  double dnu_D, a_v, sigma0;  /* line constants at temp_K */
  double bytes_per_substep;   /* algorithmic HBM bytes of one substep */
  double device_bytes;        /* device memory held by the context */
  long long substeps_done;
} lym1_info;

typedef struct {
  double e_tot;           /* Lya energy in the domain after the last substep, erg */
  double emitted, absorbed, outflow, work;  /* erg, summed over all substeps since the last reset */
  double residual;        /* e_tot - e_start - (emitted - absorbed - outflow - work), erg */
  double e_start;         /* energy when the counters were last reset, erg */
  double max_f;           /* max |H|/J over cells and bins after the last substep (FP32 policies:
                             over (cell, bin) pairs holding >= 1e-8 of the domain energy) */
  double n_unrealisable;  /* (cell, bin) pairs with |H| > J (1 + 1e-6) after the last substep,
                             counted over the same pairs */
  double force_abs;       /* sum |f| dV of the last substep's force, dyn */
  double force_radial;    /* sum f . r_hat dV (r from the box centre), dyn */
  double M_F, M_F_radial; /* force multipliers (Sec. 4 definitions): force / (L_tot / c) */
  double f_esc;           /* outflow / emitted since the last reset */
  double L_tot;           /* total source luminosity, erg/s */
  long long substeps;     /* substeps since the last reset */
} lym1_diag;

/* Human-readable text of a status code (static storage). */
const char *lym1_strerror(int status);

/*
 * Creates a context: copies the per-cell fields (host or device pointers) to
 * the device, builds the per-bin tables on the host (frequency grid, line
 * constants, bin-averaged Voigt profile <H>_k, App. A; emission fractions,
 * Sec. 2.1 step 2) and zeroes the state and the sources.
 * Contexts of different geometries cannot share a batch (lym1_batch_create).
 * Returns LYM1_EINVAL for unsupported geometry/boundaries/precision, fewer than
 * one cell or bin, more than LYM1_MAX_BINS bins, non-positive dx or T;
 * LYM1_ENOMEM if device memory runs out; LYM1_ENODEVICE without a GPU.
 */
int lym1_create(const lym1_grid *grid, const lym1_groups *groups, const lym1_opacities *opac,
                lym1_ctx **out);

#define LYM1_MAX_BINS 1024

/* Frees every device allocation of the context.  Accepts NULL. */
void lym1_destroy(lym1_ctx *ctx);

/*
 * Sets the Lya sources: lum_erg_s[ny][nx] is the luminosity emitted in each
 * cell, spread over the bins with the emission fractions w_k (phi_nu = H/sqrt
 * pi, Sec. 2.1 step 2): j_k = lum w_k / (4 pi dx^3 dnu_k) (axisymmetric grid:
 * the cell's ring volume 2 pi Vol in place of dx^3).  Host or device pointer.
 * The call only enqueues work on the context's stream (the copy, a device sum
 * of the total luminosity that lym1_diagnostics reads back for M_F, and the
 * ring-volume scaling) and returns without waiting: a pinned host buffer must
 * stay unchanged until the stream has passed the copy (pageable memory is
 * staged before the call returns).  The diagnostic counters keep running
 * (emission is booked per substep with the sources in force).  LYM1_EINVAL for
 * a band context (lym1_bands_update sets band emission).
 */
int lym1_set_sources(lym1_ctx *ctx, const double *lum_erg_s);

/* Replaces the state (J, Hx, Hy), each [nb][ny][nx], host or device pointers
 * (FP64; rounded to FP32 in the mixed modes).  Resets the diagnostic counters. */
int lym1_set_state(lym1_ctx *ctx, const double *J, const double *Hx, const double *Hy);

/* Copies the state out as FP64 [nb][ny][nx] into caller buffers (host or device). */
int lym1_get_state(lym1_ctx *ctx, double *J, double *Hx, double *Hy);

/*
 * Halo rows of a y-slab decomposition of one grid over several GPUs (the
 * multi-GPU form of the substep; the paper's own code parallelises with
 * threads on one machine, Sec. 2.2).  The substep's stencil reaches two cells
 * each way (the MinMod face states of Sec. 2.1 step 1) and steps 2 and 3 are
 * cell-local, so a slab rank needs only its neighbours' two edge rows before
 * each substep: these calls move whole rows in the state's own element type,
 * without the FP64 conversion of lym1_get_state / lym1_set_state.
 *
 * lym1_state_elem_size: *bytes = 4 under LYM1_MIXED and LYM1_MIXED_FAST, else 8.
 * lym1_get_rows copies rows [y0, y0 + n_rows) of every bin of J, Hx, Hy into
 * caller buffers laid out [nb][n_rows][nx] of that element type; lym1_set_rows
 * copies such buffers into those rows.  Buffers are host or device memory
 * (unified addressing), owned by the caller.  Both calls only enqueue the
 * copies on the context's stream (one strided copy per array): read a host
 * buffer, or hand a device buffer to another stream, after lym1_synchronize;
 * the buffers of lym1_set_rows must stay unchanged until the stream has
 * passed the copy.  lym1_set_rows leaves the diagnostic counters running.
 * LYM1_EINVAL for a null pointer, n_rows < 0 or rows outside [0, ny);
 * n_rows = 0 copies nothing.
 */
int lym1_state_elem_size(lym1_ctx *ctx, int *bytes);
int lym1_get_rows(lym1_ctx *ctx, int y0, int n_rows, void *J, void *Hx, void *Hy);
int lym1_set_rows(lym1_ctx *ctx, int y0, int n_rows, const void *J, const void *Hx,
                  const void *Hy);

/*
 * Enqueues n substeps of length dt_s on the context's stream (dt_s <= 0 means
 * the CFL step dt_RT).  Asynchronous: returns after the launches; errors of
 * the kernels themselves surface at the next synchronising call.
 */
int lym1_substeps(lym1_ctx *ctx, int n, double dt_s);

/* Advances dt_s in n = ceil(dt_s / dt_RT) equal substeps; *n_substeps_out = n
 * (may be NULL).  Asynchronous like lym1_substeps. */
int lym1_step(lym1_ctx *ctx, double dt_s, int *n_substeps_out);

/* Moments of the current state, [nb][ny][nx], FP64: E = 4 pi J / c
 * (erg cm^-3 Hz^-1), Fx, Fy = 4 pi H (erg cm^-2 s^-1 Hz^-1) (Sec. 2.1).  Any
 * output pointer may be NULL to skip it.  Synchronises the stream. */
int lym1_moments(lym1_ctx *ctx, double *E, double *Fx, double *Fy);

/* Force per unit volume of the last substep, fx, fy [ny][nx], dyn cm^-3
 * (Sec. 2.3).  Synchronises the stream. */
int lym1_force(lym1_ctx *ctx, double *fx, double *fy);

/* Diagnostics (energy bookkeeping with compensated sums, M_F, f_esc).
 * Synchronises the stream; LYM1_ENONFINITE if a sum is NaN or Inf. */
int lym1_diagnostics(lym1_ctx *ctx, lym1_diag *out);

/* Static facts about the context. */
int lym1_get_info(lym1_ctx *ctx, lym1_info *out);

/*
 * Device bytes that lym1_create will allocate for a Lya context on this grid
 * with these groups and precision (temp_field != 0: with a per-cell
 * temperature field), computed on the host from the same allocation list:
 * equal to lym1_info.device_bytes of that context right after creation.  Not
 * included: buffers made on demand later (lym1_spectrum_enable,
 * lym1_set_pruning) and the persistent graph-replayed batch of lym1_substeps
 * (a few kB).  For admission control by a device-memory budget (serving).
 * LYM1_EINVAL for invalid sizes, groups or precision.  No CUDA call.
 */
int lym1_plan_bytes(const lym1_grid *grid, const lym1_groups *groups, int precision, int temp_field,
                    double *bytes);

/* Per-bin tables (host buffers of nb doubles, any may be NULL): bin width
 * dnu_k, absolute centre frequency nubar_k, bin-averaged Voigt <H>_k and the
 * emissivity factor w_k / (4 pi dx^3 dnu_k). */
int lym1_tables(lym1_ctx *ctx, double *dnu, double *nubar, double *Havg, double *gem);

/* Blocks until all work of the context's stream is done; reports kernel errors. */
int lym1_synchronize(lym1_ctx *ctx);

/*
 * Runs substeps until the steady-state test of the serving loop passes or
 * max_substeps is reached: every check_every substeps the domain energy E is
 * compared with the previous check, and the run stops when
 * |E_n - E_{n-m}| / E_n / m < tol (m = check_every).  *n_done receives the
 * substeps run.  Returns LYM1_ENOTCONVERGED (state valid) at the cap.
 */
int lym1_run_to_steady(lym1_ctx *ctx, double tol, int check_every, int max_substeps,
                       int *n_done);

/*
 * Batches: several contexts (clouds of different sizes, luminosities and
 * densities) advanced together.  Each substep of a batch is three launches in
 * total -- one persistent transport kernel over a work list of every
 * context's 16x16 tiles, one persistent frequency-step kernel over every
 * context's cell blocks and one reduction kernel with a block per context --
 * captured once in a CUDA graph and replayed.  The persistent grid size is
 * tuned on the batch's first substeps (each candidate times one substep; the
 * choice does not change any result) and kept in a process-wide cache keyed
 * by device, precision, geometry, table mode, bin count and the power of two
 * of the batch's tile count: a later batch of the same class starts tuned
 * and skips those substeps.  Every context advances with its own
 * dt_RT and its own bookkeeping, exactly as with lym1_substeps.
 * The contexts must share precision, bin count and stream, and not be gray;
 * otherwise LYM1_EINVAL.  A batch holds device pointers of its contexts:
 * destroy the batch before any of them.
 */
typedef struct lym1_batch lym1_batch;
int lym1_batch_create(lym1_ctx *const *ctxs, int n_ctx, lym1_batch **out);
int lym1_batch_substeps(lym1_batch *batch, int n);
/* persistent grid sizes in use (0 until tuned; set at creation when the
 * tuned-grid cache holds the batch's class) */
int lym1_batch_grid(lym1_batch *batch, int *transport_blocks, int *freq_blocks);
/*
 * Tile-shape autotuning of the batched transport.  Besides the persistent grid
 * size, the tuner times the transport's work layouts (no counterpart in the
 * paper, which loops over bins on CPU threads): 16 x 16 tiles (the only one
 * of LYM1_FP64_DET batches, so that they equal solo runs bit for bit), 32 x 8
 * tiles (plain table modes, no pruning or acceptance rule), and the bins of
 * each 16 x 16 tile split over 2, 4 or 8 blocks when the tiles alone do not
 * fill the GPU (small clouds; at least 16 bins a block; the groups' force
 * sums are added in group order by the frequency step).  A layout changes
 * only the summation order of the force and of the transport's bookkeeping,
 * not J or H.  The winner is cached with the grid (see above).
 * lym1_batch_config reports the layout and grids in use (all 0 until tuned):
 * tile width and height, bin groups, transport and frequency-step grids.
 * lym1_batch_configure fixes a layout instead of tuning it: tile_shape 0 =
 * 16 x 16, 1 = 32 x 8 (LYM1_EINVAL with pruning, broad bands or the
 * acceptance rule); bin_groups 1, 2, 4 or 8 (at most the bin count); grid_t
 * persistent transport blocks (0 = all resident).  Call it outside stream
 * capture; it synchronises the batch's stream and drops the captured graph.
 */
int lym1_batch_config(lym1_batch *batch, int *tile_x, int *tile_y, int *bin_groups,
                      int *transport_blocks, int *freq_blocks);
int lym1_batch_configure(lym1_batch *batch, int tile_shape, int bin_groups, int transport_blocks);
void lym1_batch_destroy(lym1_batch *batch);

/* One-shot batch: create, run n substeps, destroy. */
int lym1_substeps_batched(lym1_ctx **ctxs, int n_ctx, int n);

typedef struct {
  double transport_ms;          /* summed device time of the transport + source kernels */
  double freq_ms;               /* summed device time of the frequency-step kernels */
  double finalize_ms;           /* summed device time of the per-substep reduction kernels */
  long long transport_launches, freq_launches, finalize_launches;
} lym1_profile;

/*
 * Kernel timing: while enabled, every kernel launch of a substep is bracketed
 * by CUDA events recorded on the context's stream (no synchronisation is
 * added).  lym1_profile_read synchronises the stream, sums the event-timed
 * durations per kernel since the last reset and optionally resets.
 */
int lym1_profile_enable(lym1_ctx *ctx, int on);

/*
 * Test hook for the failure path of the bounded waits.  The next
 * frequency-step launch arms one bulk-copy stage without issuing its copies,
 * so its wait runs out after ~2 s.  The kernel records the expiry and returns,
 * and the next lym1_synchronize reports LYM1_ETIMEOUT once and clears it.  The
 * state of that substep is not meaningful; the context stays usable.  Only
 * for FP32 contexts whose cell count is a multiple of 4 (LYM1_EINVAL
 * otherwise).
 */
int lym1_debug_expire_wait(lym1_ctx *ctx);

/*
 * Test hook for the FP64 helpers of the LYM1_MIXED kernels (no counterpart in
 * the paper: GB300 runs FP64 arithmetic and FP32 <-> FP64 conversions on a
 * pipe of ~1/70 of the FP32 rate, so those kernels convert on the integer
 * pipe and refine a hardware reciprocal approximation by Newton-Raphson).
 * For i < n (device pointers, caller-owned): wide[i] = xf[i] widened to FP64,
 * narrow[i] = xd[i] narrowed to FP32 (round to nearest even), rcp[i] = 1 /
 * xd[i] (two Newton-Raphson steps), rcp1[i] = 1 / xd[i] from the hardware
 * approximation with one step, and rcpf[i] = 1 / xd[i] as the mixed source
 * step and elimination take it: the FP32 reciprocal of the significand seeds
 * it (exponent in integer bits, any normal xd[i] below 2^1020) and one FP64
 * step refines it; both conversions flush subnormals to zero.  Runs on
 * the legacy default stream and synchronises it.  LYM1_EINVAL for null
 * pointers or n < 0; LYM1_ECUDA if the launch fails.
 */
int lym1_debug_fp64_helpers(const float *xf, const double *xd, long long n, double *wide,
                            float *narrow, double *rcp, double *rcp1, double *rcpf);
int lym1_profile_read(lym1_ctx *ctx, lym1_profile *out, int reset);

/*
 * Allocation-free energy of a caller-owned state.  The paper has no
 * counterpart: this is a service for callers that cannot allocate device
 * memory when they need the number -- for instance a host code whose device
 * memory is owned by another runtime's allocator (a framework that has already
 * reserved most of HBM), or a real-time loop that forbids allocation.
 *
 * Returns in *e_out (host or device pointer) the Lya energy in erg,
 * (4 pi / c) dx^3 sum_cells sum_k dnu_k J_k, of J[nb][nc] (FP64, device
 * memory of the current device) with bin widths dnu[nb] (host pointer, Hz),
 * with the same partition, reduction order and rounding as the energy that
 * lym1_diagnostics reports for a Cartesian FP64 context holding that state.
 * Runs on cuda_stream (NULL = legacy default stream) and synchronises it
 * before returning.
 *
 * Memory: calls no cudaMalloc/cudaFree and no allocating library routine.
 * Its partial sums live in one file-scope device array of
 * (LYM1_NOALLOC_MAX_CELLS / 128 + 1) doubles (1 MiB), which every GPU that
 * loads the library holds until the process exits.  The first call on a
 * device looks up that array's device address (cudaGetSymbolAddress) with
 * the device current; make the first call on each device before any stream
 * capture.  All calls share the array and it keeps the last call's contents:
 * calls that overlap on the GPU (other streams, other host threads) race and
 * must be serialised by the caller.
 * Errors: LYM1_EINVAL for null pointers, nb or nc < 1, dx_cm <= 0, or a J
 * that is not device (or managed) memory of the current device (host arrays
 * included), checked with cudaPointerGetAttributes before any launch;
 * LYM1_ERANGE for nb > LYM1_NOALLOC_MAX_BINS or nc > LYM1_NOALLOC_MAX_CELLS;
 * LYM1_ECUDA if a launch or copy fails.  A CUDA error already pending when
 * the call starts is reported as LYM1_ECUDA and left pending for the caller;
 * an error raised by the call itself is cleared before it returns.
 */
#define LYM1_NOALLOC_MAX_CELLS (1 << 24) /* 16,777,216 cells, e.g. 4096 x 4096 */
#define LYM1_NOALLOC_MAX_BINS 1024
int lym1_energy_noalloc(const double *J, const double *dnu, int nb, long long nc, double dx_cm,
                        double *e_out, void *cuda_stream);

/*
 * Substep acceptance rule of step 2 (Sec. 2.1 step 2 and its footnote), off
 * by default.  With on = 1 every cell subcycles its implicit emission/
 * absorption update: a trial substep is accepted when the cell's Lya energy
 * density changes by |e'' - e'| / (e' + e_floor) < 0.1 (e_floor =
 * 4 pi J_floor / c, J_floor = 1e-15 erg cm^-2 s^-1 sr^-1); otherwise it is
 * halved and redone until the accepted substeps fill dt_RT.  Where the paper
 * gives only the halving: each cell starts with the whole dt_RT, an accepted
 * substep doubles the next trial (capped by what is left), substeps are whole
 * multiples of dt_RT / 2^40 and one of that size is accepted whatever the
 * change, and after 2^16 trials in a substep every further trial is accepted
 * (a bound on the loop).  The force, emission and absorption add up over the
 * accepted substeps; the frequency step follows with dt_RT.  The transport
 * then leaves step 2 to one extra kernel (one thread per cell, a pass over
 * the bins per trial), so a substep costs more where cells subcycle.
 * Lya contexts only (LYM1_EINVAL for broad bands and on other than 0 or 1).
 * A change rebuilds the graph-replayed path; batches made before it refuse to
 * run (LYM1_EINVAL); all contexts of a batch share the setting.
 */
int lym1_set_accept(lym1_ctx *ctx, int on);

/*
 * Emergent spectrum (Sec. 4: the spectra of photons leaving the domain, Test 6
 * at the outer R and Z boundaries; f_esc per bin).  lym1_spectrum_enable(ctx, 1)
 * zeroes and starts the accumulation, over the following substeps, of the
 * energy (erg) leaving through each outer boundary face in each bin: the
 * per-face terms of the outflow bookkeeping of lym1_diagnostics.  Faces are
 * ordered x- (by y), x+ (by y), y- (by x), y+ (by x) for geometry 0, and R outer
 * (by Z), Z outer (by R) for geometry 1 (the axis and midplane are mirrors);
 * the axisymmetric energies are those of the full rings.  (ctx, 0) stops it.
 * Enable before adding the context to a lym1_batch.
 * lym1_spectrum_read copies the [bin][face] array (nb x *n_faces doubles, host
 * or device pointer; out = NULL only reports *n_faces).  LYM1_EINVAL if the
 * spectrum was never enabled.
 */
int lym1_spectrum_enable(lym1_ctx *ctx, int on);
int lym1_spectrum_read(lym1_ctx *ctx, double *out, int *n_faces);

/*
 * Reduced speed of light (Sec. 2.1).  lym1_set_ctilde sets c_tilde (cm/s,
 * 0 < c_tilde <= c) and with it the RT time step dt_RT = cfl/2 dx /
 * (c_tilde + max|u|) reported by lym1_get_info; later substeps use both.
 *
 * lym1_dynamic_ctilde applies the dynamic choice of Sec. 2.1 on the GPU:
 *   c_dyn = eps_rsl max_cells { max[1, (a_v tau_0)^(1/3) f_abs] max[|u|, c_s] },
 *   f_abs = 1 / (1 + (a_v tau_0)^(1/3) tau_c + 0.6 p_d tau_0),
 *   c_tilde = min[max(ct_min, c_dyn), c],
 * then moves c_tilde by at most -25 % (x 0.75) or x 4 from its current value,
 * and sets it as lym1_set_ctilde does.  tau_0 = n_HI sigma0 dx is the cell's
 * line-centre optical depth and tau_c = rho_dust kappa_abs dx its continuum
 * absorption depth, with a_v and sigma0 at the cell's temperature.
 * cs: per-cell sound speed, cm/s, [ny][nx] FP64, host or device pointer, read
 * during the call; NULL takes that of neutral atomic gas at the cell's
 * temperature, sqrt(gamma k_B T / (mu m_H)) with gamma = 5/3, mu = 1.22.
 * The paper's defaults are eps_rsl = 4 and ct_min = 100 km/s = 1e7 cm/s.
 * The new value is written to *c_tilde_out (host pointer, may be NULL).
 * Runs on the context's stream and synchronises it.  A lym1_batch holding
 * the context picks up the new c_tilde before its next substep.
 * Errors: LYM1_EINVAL for a null ctx, eps_rsl <= 0 or not finite, ct_min < 0
 * or > c, c_tilde outside (0, c]; LYM1_ENONFINITE if the reduction met only
 * non-finite terms and left no valid value (c_tilde then stays unchanged);
 * LYM1_ECUDA if a launch or copy fails.
 */
int lym1_set_ctilde(lym1_ctx *ctx, double c_tilde);
int lym1_dynamic_ctilde(lym1_ctx *ctx, const double *cs, double eps_rsl, double ct_min,
                        double *c_tilde_out);

/*
 * Broad bands (Sec. 3: the stellar bands IR, optical, FUV, LW, EUV1-3 are
 * solved, like Lya, with the M1 moment equations of Sec. 2.1 but without the
 * frequency-derivative terms; the IR band's dust emission enters as its
 * emissivity).  A band context advances n_bands frequency-integrated groups
 * with the transport of Sec. 2.1 step 1 (closure, corrected GLF fluxes with
 * each band's own face optical depth, advection and -grad u : K / c) and the
 * implicit absorption/emission of step 2:
 *   (J'' - J') / (c_tilde dt) = j - kappa J'',  (H'' - H') / (c_tilde dt) = -alpha_F H'',
 * and the force of Sec. 2.3 summed over bands.  There is no frequency step.
 * Per-[band][cell] inputs, [n_bands][ny][nx] FP64, host or device pointers,
 * copied during the call, each finite and >= 0:
 *   alpha_F     flux opacity, cm^-1 (absorption plus scattering weighted by 1 - g)
 *   kappa       absorption opacity, cm^-1
 *   emissivity  j, erg s^-1 cm^-3 sr^-1
 * The state J, H of each band is frequency integrated (erg s^-1 cm^-2 sr^-1)
 * and the bin width of every band is 1.  Every other call (substeps, step,
 * state, moments, force, diagnostics with M_F over the total emitted power,
 * spectrum, profiling, set_ctilde) works on a band context as on a Lya one;
 * lym1_set_sources and lym1_dynamic_ctilde return LYM1_EINVAL, and band
 * contexts cannot join a lym1_batch (no frequency step: each substep is one
 * transport launch and one reduction).
 * lym1_bands_update replaces the three inputs (opacities that follow the
 * chemistry and dust between hydro steps); the state is kept.
 * Errors: LYM1_EINVAL for null pointers, n_bands outside 1..LYM1_MAX_BINS, a
 * bad grid or precision, or any input value negative or not finite (an update
 * that fails changes nothing); LYM1_ENOMEM, LYM1_ECUDA, LYM1_ENODEVICE as for
 * lym1_create.
 */
typedef struct {
  int n_bands;
  const double *alpha_F;
  const double *kappa;
  const double *emissivity;
} lym1_bands;
/*
 * New gas temperatures for a context created with a temperature field
 * (lym1_opacities.temp_field), e.g. after each hydro step of a
 * radiation-hydrodynamics run.  Rebuilds on the GPU, one thread per cell, the
 * per-cell tables of App. A and Sec. 2.1 that the field determines: <H>_k over
 * every bin at the cell's Doppler width and a_v, the emission factors
 * w_k / (4 pi V dnu_k) with w_k = <H>_k dx_k normalised to sum 1, sigma0 and
 * alpha = n_HI sigma0, h / (k_B T) and dnu_D^2 / 2.  The steps and their order
 * are those of the tables built at creation on the host; the device's exp,
 * erf and erfc make the two agree to about 1e-15 relative, not bit for bit.
 * temp_field: [ny][nx] K, host or device pointer, each value finite and > 0.
 * The state J, H and the diagnostic counters are kept.  Synchronises the
 * context's stream; takes a temporary device buffer of one cell plane.
 * Errors: LYM1_EINVAL for a null pointer, a context made without a temperature
 * field, or any temperature <= 0 or not finite (nothing is changed);
 * LYM1_ENOMEM, LYM1_ECUDA.
 */
int lym1_set_temperature(lym1_ctx *ctx, const double *temp_field);

/*
 * Active-bin pruning (Sec. 2.2): with cut > 0 (the paper uses 1e-10) each
 * substep first takes, on the GPU, the energy of every bin, dnu_k sum_cells
 * V_cell J_k, and advects only the bins holding more than cut of the total;
 * the others skip step 1 (no fluxes, advection, work or hoop terms: J' = J,
 * H' = H) and still take steps 2 and 3.  cut = 0 (the default) advects every
 * bin.  Pruning changes results where it skips a bin.  On GB300 it does not
 * make substeps faster: the transport variant that can skip bins runs slower
 * per advected bin than the default one, and the per-bin energies take a pass
 * over the state (with half the bins of a 512^2 x 194 state pruned, 1.93 ms a
 * substep against 1.74 ms without).  A lym1_batch captures the
 * setting of its contexts at creation: after a change of the cut, create the
 * batch anew (lym1_batch_substeps returns LYM1_EINVAL until then).
 * Errors: LYM1_EINVAL for a null ctx or cut outside [0, 1); LYM1_ENOMEM.
 */
int lym1_set_pruning(lym1_ctx *ctx, double cut);

int lym1_create_bands(const lym1_grid *grid, const lym1_bands *bands, const double *ux,
                      const double *uy, double c_tilde, double cfl, int precision,
                      void *cuda_stream, lym1_ctx **out);
int lym1_bands_update(lym1_ctx *ctx, const double *alpha_F, const double *kappa,
                      const double *emissivity);

#ifdef __cplusplus
}
#endif

#endif /* LYM1_H */

/*
 * ehd.h -- C ABI of the GB300 library for the coupled time step of the
 * segregated electroconvection solver of Guan & Novosselov (arXiv:1812.05711):
 * a two-relaxation-time (TRT) D2Q9 lattice Boltzmann scheme for the fluid (f)
 * and the space charge (g), coupled every step to a fast Poisson solver for
 * the electric potential (FFT along the periodic x, tridiagonal in y).
 *
 * Conventions for every entry point:
 *   - Plain C types only.  Host pointers are marked "host"; the library owns
 *     all device memory of a run.  No entry point takes ownership of a
 *     caller's buffer.
 *   - Every call returns an ehd_status; on failure ehd_last_error() gives a
 *     thread-local message.  No C++ exception crosses this boundary.
 *   - Work is enqueued on the run's CUDA stream and is asynchronous unless the
 *     comment says the call synchronises.  A run is not thread-safe; distinct
 *     runs may be driven from distinct host threads.
 *   - Grids: Nx columns (periodic in x, a power of two, 16..2048), Ny node rows
 *     (2..8192).  Node row j sits at y = j + 1/2; the injector electrode
 *     (phi = 1, rho_c = rho0) is the wall y = 0 and the collector (phi = 0) the
 *     wall y = H = Ny.  Host field arrays are FP64, row-major, x fastest:
 *     [Ny][Nx] per field, [9][Ny][Nx] per population set.
 *   - D2Q9 numbering: c0=(0,0) c1=(1,0) c2=(0,1) c3=(-1,0) c4=(0,-1)
 *     c5=(1,1) c6=(-1,1) c7=(-1,-1) c8=(1,-1).
 */
#ifndef EHD_H
#define EHD_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ehd_run ehd_run;     /* opaque, owned by the library */
typedef struct ehd_batch ehd_batch; /* opaque, owned by the library */

typedef enum {
  EHD_OK = 0,
  EHD_EINVAL = -1,     /* invalid argument (size, parameter, mask, pointer) */
  EHD_ENOMEM = -2,     /* device or host allocation failed */
  EHD_ECUDA = -3,      /* a CUDA runtime call failed */
  EHD_EDIVERGED = -4,  /* a non-finite density or charge was produced */
  EHD_ETIMEOUT = -5,   /* a bounded device wait gave up (reported by the next
                          synchronising call, like EHD_EDIVERGED) */
  EHD_EBUSY = -6       /* reserved: capacity exhausted */
} ehd_status;

/* Storage type of the populations.  F64 storage with F64 compute is the plain
 * double-precision path of the paper (Sec. IV.4); every other combination
 * computes in FP32 on populations stored shifted by their rest equilibrium
 * (f_i - w_i rho_hydrostatic(y) and g_i - w_i rho_c,hydrostatic(y)). */
typedef enum {
  EHD_STORE_F64 = 0,
  EHD_STORE_F32 = 1,
  EHD_STORE_BF16 = 2,
  EHD_STORE_F16 = 3
} ehd_storage;

typedef enum { EHD_COMPUTE_F64 = 0, EHD_COMPUTE_F32 = 1 } ehd_compute;

#define EHD_MAX_PERT_MODES 16
#define EHD_NDIAG 8

/* Field mask bits for ehd_fields (output order follows the bit order). */
#define EHD_FIELD_RHO (1u << 0)   /* fluid density, Eq. 5 */
#define EHD_FIELD_UX (1u << 1)    /* velocity with half force, Eq. 7 */
#define EHD_FIELD_UY (1u << 2)
#define EHD_FIELD_RHOC (1u << 3)  /* charge density, Eq. 6 */
#define EHD_FIELD_PHI (1u << 4)   /* electric potential, Eq. 4 */
#define EHD_FIELD_EX (1u << 5)    /* E = -grad phi (central differences; E_x spectral with ex_spectral) */
#define EHD_FIELD_EY (1u << 6)
#define EHD_FIELD_ALL 0x7Fu

typedef struct {
  int storage;      /* ehd_storage; default EHD_STORE_F32 */
  int compute;      /* ehd_compute; default EHD_COMPUTE_F32.  F64 compute needs
                       F64 storage. */
  double lambda_g;  /* charge magic parameter Lambda_g of Eq. 17; default 1e-6
                       (Sec. IV.2) */
  double u_ion;     /* lattice ion drift speed mu_b dphi0 / H; sets the lattice
                       scale of the Eq. 26 groups.  Default 2e-3. */
  int wall_mode;    /* 0: halfway walls, Poisson mirror ghost
                       phi_{-1} = 2 phi_w - phi_0 (default).
                       1: Dirichlet on the extra nodes j = -1, Ny (the odd
                       extension of Eq. 21 as printed). */
  int n_modes;      /* initial perturbation: number of x-modes of Eq. 29
                       (mode k has k+1 periods across the channel); 0 = none */
  double pert_amp[EHD_MAX_PERT_MODES];   /* amplitude in units of u_ion */
  double pert_phase[EHD_MAX_PERT_MODES]; /* x-phase, radians */
  void* stream;     /* cudaStream_t to run on; NULL = a stream the library
                       creates and owns */
  int step_kernel;  /* 0: march form -- a warp walks a slab of rows, pulls the
                       populations through registers and writes the new
                       charge density itself; 1: one thread per node, push
                       form, charge density summed by a separate kernel.
                       Same results up to rounding order.  -1 (default):
                       the march form, except plain FP64 runs (FP64 compute)
                       without spectral E_x, which take the push form: there
                       the FP64 arithmetic of a warp's row walk is latency
                       bound and one thread per node is faster at every size
                       (128x104: 52 vs 112 us per step). */
  int x_symbol;     /* x second derivative of the Poisson solve: 0 spectral,
                       -(2 pi m / Nx)^2 (Eq. 20, default); 1 the 3-point
                       difference -4 sin^2(pi m / Nx), so that the solve
                       inverts the 5-point Laplacian. */
  int ex_spectral;  /* E_x = -d phi / dx: 0 central difference (default);
                       1 spectral, the inverse x-transform of -i k_m phi_m
                       (k_m = 2 pi m / Nx, Nyquist mode dropped), formed by the
                       Poisson solve into a plane that the march form reads.
                       Needs the march form with 2 columns per lane and ring
                       depth 2; refused in batches.  The run then holds one
                       more [Ny][P] array beyond ehd_footprint. */
  int perturbation; /* FP32 compute only: 0 (default) stores the charge
                       populations shifted by w_i rho_c,hydrostatic(y); 1
                       advances an x-uniform base state of both population
                       sets exactly, in FP64 (its collision, streaming in y,
                       wall rules and mean-mode potential, on a second
                       stream), and stores and collides only the charge
                       populations' departure from it in FP32, with the
                       departure of the equilibrium written out term by term.
                       FP32 then resolves the charge populations' odd
                       non-equilibrium part, which it otherwise does not at
                       Fe of order 10^3 (omega_g- close to 2), so that growth
                       rates of small rolls match the FP64 oracle.  Needs the
                       march form (two columns per lane, cp.async staging) and
                       central-difference E_x.  Batches take such runs
                       beside plain ones (their base states advance on the
                       batch's second stream). */
  int dc_printed;   /* charge relaxation rates: 0 (default) D_c = cs2
                       (tau_g- - 1/2), the antisymmetric rate carrying the
                       charge flux; 1 Eq. 16 as printed, D_c = cs2 (tau_g+ -
                       1/2), tau_g- then from lambda_g (Eq. 17), so the
                       scheme's own diffusivity is cs2 lambda_g / (tau_g+ -
                       1/2) rather than D_c.  For measuring what the printed
                       assignment does to the results. */
} ehd_options;

/* Fill *opt with the defaults above. */
void ehd_default_options(ehd_options* opt);

/* Create a run: map the non-dimensional groups of Eq. 26 (T, C, M, Fe) to
 * lattice units (rho = 1, dphi0 = 1, H = Ny, mu_b = u_ion H), set the TRT rates
 * of Eqs. 16-17 (nu from tau+, D_c from tau_g-, Lambda for the fluid as given,
 * Lambda_g from opt), allocate the device state and initialise it to the
 * hydrostatic profile of Eqs. 27-28 plus the Eq. 29 perturbation, then solve
 * phi (ehd_poisson).  Synchronises the stream.
 * Errors: EHD_EINVAL for a bad size or non-positive T, C, M, Fe, Lambda,
 * lambda_g, u_ion, tau+ > 50 or an unsupported storage/compute pair;
 * EHD_ENOMEM, EHD_ECUDA.  *out is NULL on failure. */
ehd_status ehd_create(int Nx, int Ny, double T, double C, double M, double Fe,
                      double Lambda, const ehd_options* opt, ehd_run** out);

/* Solve the Poisson equation (Eq. 4; discretised as Eqs. 18-20 with the
 * Dirichlet walls of Table I) for phi from the current charge density
 * rho_c = sum_i g_i (Eq. 6): real FFT of every row, one tridiagonal solve per
 * wavenumber (the mean mode in FP64), inverse FFT.  Asynchronous. */
ehd_status ehd_poisson(ehd_run* run);

/* Advance n >= 0 coupled steps (Eqs. 5-17, Table I).  Per step: E = -grad phi;
 * fused fluid TRT collision with the electric force -rho_c grad phi (Eq. 7
 * half-force velocity, Eqs. 8, 10, 12, 13, 15); charge TRT collision with the
 * drift u + mu_b E (Eqs. 9, 11, 14); streaming with halfway bounce-back of f
 * on both walls, anti-bounce-back injection of rho0 and zero-gradient outflow
 * of g; then the Poisson solve for the new charge.  Asynchronous; a
 * non-finite density or charge is reported by the next synchronising call. */
ehd_status ehd_step(ehd_run* run, long n);

/* Instrumented stepping: advance n steps with one launch per kernel (no
 * graph) and CUDA events on the run's stream around each phase; the paper has
 * no counterpart (measurement only).  host ms_out[EHD_NPROFILE]: summed
 * milliseconds of [0] the fused collide-stream kernel, [1] the charge-moment
 * kernel (0 when the step kernel writes the charge itself), [2] the Poisson
 * solve (forward FFT, tridiagonal modes, inverse FFT; the mean mode runs
 * beside them on a second stream and is joined before the event), [3] whole
 * steps, [4] = n, and inside [2]: [5] the forward row FFT, [6] the solves of
 * the wavenumbers m >= 1, [7] the inverse row FFT, [8] the mean mode m = 0
 * (on its own stream, concurrent with [6]).  Synchronises. */
#define EHD_NPROFILE 9
ehd_status ehd_step_profile(ehd_run* run, long n, double* ms_out);

/* Launch-shape tuning of a run (the paper has no counterpart; results do
 * not change beyond rounding order).  param: EHD_TUNE_SLAB_ROWS (rows each
 * warp of the march form walks, 1..Ny), EHD_TUNE_RING_DEPTH (rows staged
 * ahead by cp.async: 2, 3, 4 or 6; with 2 columns per lane only 2, 3, 4),
 * EHD_TUNE_STEP_KERNEL (0 march form, 1 node-parallel form),
 * EHD_TUNE_COLS_PER_LANE (march form: 1 or 2 adjacent nodes per lane),
 * EHD_TUNE_TILE_MODES (wavenumbers per CTA of the mode solve: 1, 2, 4, 8;
 * 0 = the largest whose tile fits in shared memory; other widths change the
 * scans' chunking, so results then differ from batch members' in rounding), EHD_TUNE_PDL (a mask
 * of the Poisson kernels launched with programmatic dependent launch, so that
 * each is resident and waiting when its predecessor ends: 1 the forward row
 * transform, 2 the wavenumber solve, 4 the inverse transform, 8 the step
 * kernel (march form: it stages its first rows' populations before waiting
 * for phi); the default is 7 up to 2^18 nodes and from 2^21 (2048 x 1680:
 * 114.1 us per step against 114.3 with 11, 114.7 with 3, 116.9 with none),
 * 11 between them (1024 x 840: 41.2 against 41.7 with 7) and 11 for
 * perturbation-form runs at every size (2048 x 1680: 120.2 against 121.1
 * with 3 and 135.4 with 7, whose early-resident inverse-transform CTAs
 * starve the base chain on the third stream); results are the same for
 * every mask),
 * EHD_TUNE_FFT_CTA (FP32 rows
 * of 2048: 1, the default, one CTA of 64 threads per row; 0, one warp per
 * row), EHD_TUNE_Y_SOLVER (the y solve of the wavenumbers m >= 1: 0, the
 * default, one tridiagonal per wavenumber (Eq. 18); 1, the literal form of
 * Sec. IV.3: odd extension of each spectrum column in y to NE = 2 Ny points
 * (walls halfway, the default) or 2 Ny + 2 (walls on nodes) (Eqs. 21-22), a
 * complex FFT of length NE, division by -(kappa_m + 4 sin^2(pi k / NE))
 * (Eqs. 20, 24), inverse FFT, first Ny points (Eq. 25); NE must have no
 * prime factor above 13 and one column must fit in shared memory, and
 * runs in a batch keep 0; the mean mode m = 0 is solved as before),
 * EHD_TUNE_MARCH_TMA (march form, FP32 storage and compute, 128 <= Nx <=
 * 2048: 0, the default, per-lane 8-byte cp.async staging and 8-byte
 * stores; 1, each row of a strip staged by tensor copies
 * (cp.async.bulk.tensor, 9 planes per copy) with mbarrier completion;
 * 2, the same and completed rows written by tensor stores from a
 * shared-memory tile; 3, tensor copies two rows ahead (three stages); the
 * same results bit for bit), EHD_TUNE_TILE_THREADS (threads per CTA of the
 * mode solve, FP32 compute: 256, 512 or 1024; 0 = the default; more threads
 * cut each wavenumber's rows into shorter chunks, so results differ in
 * rounding order), EHD_TUNE_TILE_CLUSTER (FP32 compute with 8 wavenumbers
 * per tile: 1, each tile solved by a cluster of two CTAs that stage half the
 * rows each and exchange their chunk maps through distributed shared memory;
 * 0, the default, one CTA per tile, which is faster (2048 x 1680: 118.9-120.2
 * against 121.5 us per step); the same results bit for bit), EHD_TUNE_TILE_TMA
 * (FP32 compute with 8 wavenumbers per tile: 1, each tile's spectrum and
 * pivots staged by tensor copies of 256-row boxes with mbarrier completion;
 * 0, the default, by 16-byte cp.async chunks from all threads, which is
 * faster for these 64- and 32-byte rows (2048 x 1680: 117.2-117.9 against
 * 118.4 us per step); the same results bit for bit), EHD_TUNE_SLAB_SHIFT
 * (march form with two columns per lane and cp.async staging: rows d by
 * which the slab partition advances each step, 0..Ny; step k of the
 * sequence (k = step number mod 16, the graph length) uses slabs that start
 * at rows b S - (k d mod S), so each slab begins on the rows that the slab
 * below it wrote last in the step before, which are then still in L2; 0
 * keeps one partition; the default is 4 for runs whose populations exceed
 * the L2 size and 0 otherwise; results differ in rounding order only, where
 * a row's charge is summed from slab-boundary partials).
 * Drops the run's captured graphs.  EHD_EINVAL for an unknown parameter or
 * value. */
#define EHD_TUNE_SLAB_ROWS 1
#define EHD_TUNE_RING_DEPTH 2
#define EHD_TUNE_STEP_KERNEL 3
#define EHD_TUNE_COLS_PER_LANE 4
#define EHD_TUNE_TILE_MODES 5
#define EHD_TUNE_PDL 6
#define EHD_TUNE_FFT_CTA 7
#define EHD_TUNE_Y_SOLVER 8
#define EHD_TUNE_MARCH_TMA 9
#define EHD_TUNE_TILE_THREADS 10
#define EHD_TUNE_TILE_CLUSTER 11
#define EHD_TUNE_TILE_TMA 12
#define EHD_TUNE_SLAB_SHIFT 13
ehd_status ehd_tune(ehd_run* run, int param, int value);

/* Current value of a tuning parameter (-1 for an unknown one or NULL run). */
int ehd_tune_get(ehd_run* run, int param);

/* Copy fields of the current state to host_out (host, FP64, caller-owned,
 * popcount(mask) * Ny * Nx doubles, one [Ny][Nx] plane per set bit in bit
 * order).  Synchronises the stream.  EHD_EINVAL for mask == 0, a mask bit
 * above EHD_FIELD_ALL or host_out == NULL. */
ehd_status ehd_fields(ehd_run* run, unsigned mask, double* host_out);

/* Diagnostics of the current state, FP64 reductions on the device
 * (host out[EHD_NDIAG]): total mass sum rho, total charge sum rho_c, charge
 * injected and collected since creation (sums of the wall fluxes of every
 * step), kinetic energy sum rho |u|^2 / 2, max |u_y|, max |u|, step count.
 * Synchronises; EHD_EDIVERGED if the state holds a non-finite value. */
ehd_status ehd_diagnostics(ehd_run* run, double* out);

/* Replace the populations (host, FP64 [9][Ny][Nx] each) and re-solve phi.
 * For shifted storages the values are shifted and rounded on the device.
 * Synchronises.  The step counter and flux sums are kept. */
ehd_status ehd_load(ehd_run* run, const double* f_host, const double* g_host);

/* Copy the populations out (host, FP64 [9][Ny][Nx] each, unshifted).
 * Either pointer may be NULL.  Synchronises. */
ehd_status ehd_save(ehd_run* run, double* f_host, double* g_host);

/* Lattice parameters of a run (host out[16]): Nx, Ny, H, mu_b, eps, nu, rho0,
 * D_c, tau+, tau-, tau_g+, tau_g-, rho_a, y_a, storage, compute. */
ehd_status ehd_params(ehd_run* run, double* out);

/* Device bytes a run of this size and storage holds (for admission). */
ehd_status ehd_footprint(int Nx, int Ny, int storage, size_t* bytes);

/* Block the host until the run's stream is idle; EHD_EDIVERGED if a step has
 * produced a non-finite density or charge. */
ehd_status ehd_sync(ehd_run* run);

/* The cudaStream_t the run enqueues on. */
void* ehd_stream(ehd_run* run);

/* Poisson solve on caller-owned device buffers that allocates no device
 * memory.  The paper has no counterpart; this exists for callers that cannot
 * call cudaMalloc while they run -- a process whose device memory is all
 * reserved up front by a framework's own pool, or a latency-critical loop
 * that cannot accept the implicit device synchronisation of cudaMalloc and
 * cudaFree.  It solves the same discrete problem as ehd_poisson
 * (d2/dx2 spectral, second differences in y, phi = phi0 at the injector
 * wall and 0 at the collector, wall placement per wall_mode as in
 * ehd_options) for the charge density the caller passes:
 *   rhoc  device, FP32, [Ny][Nx] row-major, read only
 *   phi   device, FP32, [Ny][Nx] row-major, written (the full potential)
 *   eps   lattice permittivity (the equation is lap phi = -rho_c / eps)
 *   stream  cudaStream_t to enqueue on (NULL = the legacy default stream).
 * Every intermediate (half spectrum, Thomas pivots, twiddles, FP64 mean
 * profile) lives in one fixed 8 MiB __device__ array inside the library;
 * every GPU that loads the library holds it until the process exits.  With
 * CUDA's default lazy module loading the array is placed on a device when
 * the library's code is first used there, at the latest by the first call of
 * this function: make that first call on each device before a pool reserves
 * the rest of that device's memory.  Sizes whose intermediates do not fit
 * (beyond about 1024 x 840 nodes; Nx a power of two up to 2048, Ny up to
 * 4096) return EHD_EINVAL with a message, as do NULL pointers and eps <= 0.
 * Every call looks up the array's device address with the calling device
 * current.  The first call on a device builds the twiddle and pivot tables
 * for the sizes given; make that first call before any stream capture.
 * Later calls rebuild the tables only when Nx, Ny or wall_mode change,
 * except that a call made while its stream is being captured always
 * enqueues the rebuild, and after one such call every later call on that
 * device rebuilds them too.  All calls share the one array and it keeps the
 * last call's contents (each call writes everything it reads, so nothing
 * needs clearing): calls that overlap on the GPU, e.g. on two streams, race.
 * Asynchronous. */
ehd_status ehd_poisson_noalloc(int Nx, int Ny, double eps, double phi0,
                               int wall_mode, const float* rhoc, float* phi,
                               void* stream);

/* Free the run and its device memory (synchronises first).  NULL is a no-op. */
void ehd_destroy(ehd_run* run);

/* ------------------------------------------------------------------ batches
 * A batch advances many runs of uneven sizes together (the paper runs one
 * channel at a time; batching is this library's addition for parameter
 * sweeps).  Every phase of the coupled step -- collide-and-stream, forward row
 * FFT, FP32 wavenumber systems, float-float mean mode, inverse row FFT -- is
 * one persistent kernel over work lists that cover all member runs; a tick of
 * k steps is captured once per k as a CUDA graph.  Members must be
 * FP32-storage, FP32-compute runs in the march form with 64 <= Nx <= max_nx,
 * Ny <= max_ny.  Each member's result is the one it gets alone (the kernels
 * are the single-run ones, applied per run). */

/* Create a batch for up to max_runs runs whose device state together holds
 * at most hbm_budget bytes (the sum of the members' ehd_footprint; 0 = no
 * limit), with max_nx a power of two in [64, 2048] and max_ny in [2, 4096]
 * small enough that max_ny rows of 8 wavenumbers fit one CTA's shared memory
 * beside 16 KB (2250 rows on a GPU with 227 KB); stream = cudaStream_t or
 * NULL for an own stream.  The batch's own work lists (a few MB for
 * thousands of runs) are not counted in hbm_budget.
 * EHD_EINVAL / EHD_ENOMEM / EHD_ECUDA. */
ehd_status ehd_batch_create(int max_runs, size_t hbm_budget, int max_nx,
                            int max_ny, void* stream, ehd_batch** out);

/* Add a run with a budget of `steps` further steps.  Synchronises the run's
 * own stream.  EHD_EBUSY if the batch is full or the run's footprint does not
 * fit what is left of the HBM budget; EHD_EINVAL for a run of the wrong kind
 * or size, or one that is already in a batch.  While a member, the run is
 * advanced only by ehd_batch_tick (ehd_step returns EHD_EBUSY); its fields,
 * diagnostics and checkpoints stay readable. */
ehd_status ehd_batch_add(ehd_batch* batch, ehd_run* run, long steps);

/* Admission query for a run not yet created (a server's check before it
 * allocates one): EHD_OK if a run of Nx x Ny nodes and this storage would be
 * admitted now, EHD_EBUSY if it would have to wait for a slot or for memory
 * held by members, EHD_EINVAL if it can never be admitted (outside the
 * batch's size limits or the storage it takes, or a footprint above the
 * whole HBM budget).  Changes nothing. */
ehd_status ehd_batch_admits(ehd_batch* batch, int Nx, int Ny, int storage);

/* Bytes the members' device state holds (sum of their ehd_footprint) and the
 * batch's HBM budget (0 = no limit); either pointer (host) may be NULL. */
ehd_status ehd_batch_memory(ehd_batch* batch, size_t* used, size_t* budget);

/* Remove a run (synchronises the batch stream).  EHD_EINVAL if not a member. */
ehd_status ehd_batch_remove(ehd_batch* batch, ehd_run* run);

/* Advance every member by min(steps, its remaining budget); steps is even
 * and >= 2.  Asynchronous on the batch stream. */
ehd_status ehd_batch_tick(ehd_batch* batch, int steps);

/* Steps a member still has in its budget (-1 if not a member). */
long ehd_batch_remaining(ehd_batch* batch, ehd_run* run);

/* Number of member runs (-1 for NULL). */
int ehd_batch_size(ehd_batch* batch);

/* Wait for the batch stream; EHD_EDIVERGED if a member holds a non-finite
 * density or charge. */
ehd_status ehd_batch_sync(ehd_batch* batch);

/* The cudaStream_t the batch enqueues on. */
void* ehd_batch_stream(ehd_batch* batch);

/* Launch-shape tuning of a batch (results unchanged): EHD_BATCH_SLAB_ROWS
 * (rows per march warp item; 0 = chosen from the membership so the march
 * items fill about one wave), EHD_BATCH_MARCH_CTAS / EHD_BATCH_ROW_CTAS /
 * EHD_BATCH_TILE_CTAS (fixed grid of the persistent march, row-FFT and
 * wavenumber kernels), EHD_BATCH_PDL (a mask of the phase kernels launched
 * with programmatic dependent launch: 1 the forward transforms, the default,
 * 2 the wavenumber tiles, 4 the inverse transforms).  Drops the captured
 * graphs.  EHD_EINVAL otherwise. */
#define EHD_BATCH_SLAB_ROWS 1
#define EHD_BATCH_MARCH_CTAS 2
#define EHD_BATCH_ROW_CTAS 3
#define EHD_BATCH_TILE_CTAS 4
#define EHD_BATCH_PDL 5
ehd_status ehd_batch_tune(ehd_batch* batch, int param, int value);

/* Current value of a batch tuning parameter (-1 if unknown). */
int ehd_batch_tune_get(ehd_batch* batch, int param);

/* Free the batch (synchronises); its members become ordinary runs. */
void ehd_batch_destroy(ehd_batch* batch);

/* Message of the last failure on this host thread ("" if none). */
const char* ehd_last_error(void);

/* Route the library's device allocations through caller functions (e.g. a
 * framework's caching allocator).  alloc returns a device pointer aligned to
 * 256 bytes or NULL; free releases it.  Pass NULLs to return to cudaMalloc.
 * Affects runs created afterwards. */
ehd_status ehd_set_allocator(void* (*alloc)(size_t bytes, void* ctx),
                             void (*free_fn)(void* ptr, void* ctx), void* ctx);

#ifdef __cplusplus
}
#endif

#endif /* EHD_H */

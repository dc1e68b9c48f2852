// ehd_dev.cuh -- device-side types shared by the kernels and the host code of
// the GB300 electroconvection library (D2Q9 TRT lattice Boltzmann for fluid f
// and charge g, FFT/tridiagonal Poisson solve; arXiv:1812.05711).
//
// Memory layout of one run in HBM (all planes row-major, x fastest, rows
// padded to a pitch P that is a multiple of 32 elements = 128 B for FP32):
//   f[2], g[2]   population ping-pong buffers, [9][Ny][P] of the storage type
//   dphi         potential minus its row mean, [Ny][P] of the compute type R
//   phibar       row mean of the potential (the m = 0 mode), [Ny] FP64
//   Ebar         mean-mode field E_y per row, [Ny] of R
//   spec         half spectrum of every row, [Ny][Mh] complex R, Mh = Nx/2+1
//   spec0        mean-mode right-hand side / solution, [Ny] FP64
//   rfac         reciprocal Thomas pivots, mode-major [Mh][Ny] of R
//   rfac0        the same for m = 0, [Ny] FP64
//   tw           twiddles exp(-2 pi i k / Nx), k < Nx/2, complex R
//   rch          per-row charge shift (hydrostatic rho_c rounded to FP32), [Ny]
#pragma once

#include <cuda.h>  // CUtensorMap (types only; the encoder is reached through the runtime)
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace ehd {

// D2Q9 numbering: c0=(0,0) c1=(1,0) c2=(0,1) c3=(-1,0) c4=(0,-1)
// c5=(1,1) c6=(-1,1) c7=(-1,-1) c8=(1,-1); weights 4/9, 1/9, 1/36.
constexpr double kW0 = 4.0 / 9.0;
constexpr double kW1 = 1.0 / 9.0;
constexpr double kW2 = 1.0 / 36.0;

// ------------------------------------------------------------ storage ---
template <class S> struct Store;
template <> struct Store<double> {
  template <class R> __device__ __forceinline__ static R ld(const double* p) { return (R)__ldg(p); }
  template <class R> __device__ __forceinline__ static void st(double* p, R v) { *p = (double)v; }
  template <class R> __device__ __forceinline__ static R rt(R v) { return v; }
};
template <> struct Store<float> {
  template <class R> __device__ __forceinline__ static R ld(const float* p) { return (R)__ldg(p); }
  template <class R> __device__ __forceinline__ static void st(float* p, R v) { *p = (float)v; }
  template <class R> __device__ __forceinline__ static R rt(R v) { return (R)(float)v; }
};
template <> struct Store<__nv_bfloat16> {
  template <class R> __device__ __forceinline__ static R ld(const __nv_bfloat16* p) {
    return (R)__bfloat162float(__ldg(p));
  }
  template <class R> __device__ __forceinline__ static void st(__nv_bfloat16* p, R v) {
    *p = __float2bfloat16_rn((float)v);
  }
  template <class R> __device__ __forceinline__ static R rt(R v) {
    return (R)__bfloat162float(__float2bfloat16_rn((float)v));
  }
};
// FP16 keeps the shifted populations scaled by 2^12: they are small (of the
// order of the flow's departure from the hydrostatic state, 1e-7 .. 1e-2)
// and would otherwise fall below FP16's normal range (6.1e-5); the scaled
// values stay far below its largest finite value.  Powers of two scale exactly.
constexpr float kHalfScale = 4096.0f, kHalfUnscale = 1.0f / 4096.0f;
template <> struct Store<__half> {
  template <class R> __device__ __forceinline__ static R ld(const __half* p) {
    return (R)(__half2float(__ldg(p)) * kHalfUnscale);
  }
  template <class R> __device__ __forceinline__ static void st(__half* p, R v) {
    *p = __float2half_rn((float)v * kHalfScale);
  }
  template <class R> __device__ __forceinline__ static R rt(R v) {
    return (R)(__half2float(__float2half_rn((float)v * kHalfScale)) * kHalfUnscale);
  }
};

template <class R> struct Cplx { R re, im; };

// ----------------------------------------------------------- kernel args ---
// Programmatic dependent launch.  A kernel launched with pdl = true may
// start while the previous kernel of its stream is still running; it must
// call grid_dep_wait() before touching anything that kernel writes or reads
// (only tables that no kernel of the step writes may be read before it), and
// calls grid_dep_launch() after that wait, so that when a kernel starts,
// every kernel two or more launches back has completed.  Both instructions
// are no-ops in a kernel launched without the attribute.
__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }
__device__ __forceinline__ void grid_dep_launch() { asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory"); }

template <class... P, class... A>
cudaError_t launch_ex(bool pdl, void (*kernel)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                      A&&... args) {
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t c = {};
  c.gridDim = grid;
  c.blockDim = block;
  c.dynamicSmemBytes = smem;
  c.stream = s;
  c.attrs = at;
  c.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&c, kernel, static_cast<A&&>(args)...);
}

// Tensor maps of a run's spectrum [Ny][Mp] complex and pivots [Ny][Mp] (FP32)
// for staging a tile of 8 wavenumbers: boxes of 256 rows and one box of the
// last Ny % 256 rows.
struct ModesTma {
  CUtensorMap spec_full, spec_tail, rf_full, rf_tail;
  int nfull, tail;
};
// a 2-D FP32 tensor map: inner x outer elements, rows row_bytes apart
cudaError_t tma_encode_2d(CUtensorMap* m, const void* base, unsigned long long inner, unsigned long long outer,
                          unsigned long long row_bytes, unsigned box_inner, unsigned box_outer);
cudaError_t modes_tma_encode(ModesTma* t, const void* spec, const void* rfac, int Ny, int Mp);

struct StepArgs {
  int Nx, Ny, P;
  long long plane;           // elements per population plane (Ny * P)
  const void* fin;
  const void* gin;
  void* fout;
  void* gout;
  const void* dphi;          // R [Ny][P]
  const void* Ebar;          // R [Ny]
  const float* rch;          // [Ny] charge shift, nullptr for unshifted storage
  double* flux_part;         // [2][nxb] per-CTA injected / collected charge
  int* err;                  // bit 0: non-finite density or charge
  double wp, wm, gwp, gwm;   // omega+, omega-, omega_g+, omega_g-
  double mub, rho0;          // ion mobility, injected density
  double fb, fd, fdq;        // f shift r(y) = fb + fd y (fd an FP32 value), and -fd / omega- (0 when unshifted)
  const void* ex;            // R [Ny][P]: spectral E_x, or nullptr for central differences of dphi
  int wall_mode;
  // march form only
  void* rhoc_out;            // R [Ny][P]: rho_c of the new state (slab-boundary rows: partial, see rhoc_dn)
  void* rhoc_dn;             // R [nslab][P]: row y0(b) - 1, charge of the populations pushed down by slab b
  void* rhoc_up;             // R [nslab][P]: row y0(b), charge of the populations pushed up by slab b - 1
  int slab_rows;             // rows per warp slab
  int slab_off;              // slab b covers rows [b*slab_rows - slab_off, (b+1)*slab_rows - slab_off) within
                             // [0, Ny), 0 <= slab_off < slab_rows (cp.async march, two columns per lane only)
  int nstrips;               // 32-column strips (30 owned columns each)
  int ring_depth;            // rows staged ahead by cp.async (2, 3, 4 or 6)
  int cols_per_lane;         // 1: 32-column strips (30 owned); 2: 64-column strips (60 owned)
  int pdl;                   // launch with programmatic dependent launch (see launch_ex)
  const float* base_tab;     // perturbation form: the march table of time t ([Ny][4]); nullptr otherwise
};

struct PoissonArgs {
  int Nx, Ny, P, Mh, log2Nx;
  int Mp;                    // row pitch of the spectrum and pivot tables (Mh rounded up to 4)
  const void* rhoc;          // charge density, R [Ny][P]
  const void* rhoc_dn;       // slab-boundary partials of the march form (see StepArgs), added to rhoc
  const void* rhoc_up;
  int xslab;                 // slab height of those partials; 0: rhoc is complete
  int xoff;                  // slab_off of the step kernel that wrote them
  double inv_eps;            // 1 / eps
  void* spec;                // half spectrum, complex R [Ny][Mp]
  void* spec0;               // row sums (m = 0), [Ny]: double, or float (hi, lo) pairs when R = float
  const void* rfac;          // reciprocal pivots, R [Ny][Mp] (m >= 1 used)
  const void* rfac0;         // reciprocal pivots of m = 0, [Ny]: double, or float (hi, lo) pairs
  const void* tw;            // complex R [Nx]: exp(-2 pi i q / Nx)
  void* dphi;                // R [Ny][P]
  void* phibar;              // row-mean potential [Ny]: double, or float (hi, lo) pairs when R = float
  void* Ebar;                // R [Ny]
  double phi0;               // injector potential (collector is 0)
  // mean-mode (m = 0) constants, formed on the host: the injector wall value
  // W = Nx phi0 in spectral units and the closure factor 1 / (2 Ny) (walls
  // halfway) or 1 / (Ny + 1) (walls on nodes); in FP64 and split into
  // float-float (hi, lo) pairs, hi = fl32(v), lo = fl32(v - hi)
  double mW, mC;
  float mWf[2], mCf[2];
  int wall_mode;
  const double* flux_part;   // [2][nflux] wall-flux partials of the last step, or nullptr
  int nflux;
  double* flux_acc;          // [2] FP64 totals of injected / collected charge
  int tile_modes;            // wavenumbers per CTA of the mode solve (8, 4, 2, 1; 0 = largest that fits)
  int tile_threads;          // threads per CTA of the mode solve (FP32: 256, 512, 1024; 0 = 256)
  int tile_cluster;          // FP32, 8 wavenumbers per tile: two-CTA clusters per tile (same bits)
  int tile_tma;              // FP32, 8 wavenumbers per tile: tiles staged by tensor copies (same bits)
  const struct ModesTma* mtma;  // host pointer to the run's tensor maps of spec and rfac (or nullptr)
  int* err;                  // device error word (bit 2: a bounded wait gave up)
  int pdl;                   // programmatic dependent launch, a mask: 1 forward transform, 2 wavenumber
                             // solve, 4 inverse transform
  int fft_cta;               // rows of 2048: one CTA of 64 threads per row (else one warp per row)
  // y solve of the wavenumbers m >= 1: 0 per-wavenumber tridiagonal (k_modes_tile),
  // 1 odd-extension transform of length NE (k_modes_oddext, Eqs. 21-25)
  int y_solver;
  int NE, nfac;              // odd-extension length, number of its radices
  int fac[16];               // radices of NE in stage order
  const void* twy;           // complex R [NE]: exp(-2 pi i t / NE)
  const void* symy;          // R [NE]: 4 sin^2(pi k / NE)
  const void* kap;           // R [Mh]: kappa_m, the x symbol of wavenumber m
  void* ex;                  // R [Ny][P]: spectral E_x written after phi, or nullptr
};

// Charge density of row y as the Poisson solve sees it: the step kernel's
// march form leaves, at each slab boundary, the populations that cross it to
// the slab that computed them, together with their share of the new charge
// density (rhoc_dn for the row below the boundary, rhoc_up for the row
// above).  The readers add main + dn + up, in this order.
template <class R>
__device__ __forceinline__ void rhoc_partials(const PoissonArgs& a, int y, const R*& dn, const R*& up) {
  dn = nullptr;
  up = nullptr;
  if (a.xslab > 0) {
    // slab b starts at row b S - off (b >= 1): row y closes a slab when
    // y + 1 + off is a multiple of S and opens one when y + off is
    const int S = a.xslab, yd = y + 1 + a.xoff, yu = y + a.xoff;
    if (yd % S == 0 && y + 1 < a.Ny) dn = static_cast<const R*>(a.rhoc_dn) + (long long)(yd / S) * a.P;
    if (yu % S == 0 && y > 0) up = static_cast<const R*>(a.rhoc_up) + (long long)(yu / S) * a.P;
  }
}

struct FieldArgs {
  int Nx, Ny, P;
  long long plane;
  const void* f;
  const void* g;
  const void* dphi;
  const void* phibar;        // double, or float (hi, lo) pairs when R = float
  const void* Ebar;
  const float* rch;
  const void* ex;            // R [Ny][P]: spectral E_x, or nullptr
  double fb, fd;             // f shift r(y) = fb + fd y
  double mub;
  int wall_mode;
  const double* base_g;      // perturbation form: [9][Ny] base g added to the stored departures (else nullptr)
  const double* phiB;        // [Ny] base potential and field added to the departure's
  const double* EB;
};

// Row-mean potential as stored: a double, or a float-float (hi, lo) pair on
// the FP32 path (kept off the slow scalar FP64 units during the step).
template <class R>
__device__ __forceinline__ double load_phibar(const void* p, int j) {
  if constexpr (sizeof(R) == 8) {
    return static_cast<const double*>(p)[j];
  } else {
    const float2 v = static_cast<const float2*>(p)[j];
    return (double)v.x + (double)v.y;
  }
}

// ------------------------------------------------ perturbation form ---
// FP32-compute runs may advance the charge populations as departures from an
// x-uniform base state that is advanced exactly, in FP64: g = B_g(y, t) + d.
// The base (both population sets, [9][Ny] FP64 each) follows the method's
// own dynamics restricted to x-uniform fields -- collision, streaming in y,
// the wall rules and the mean mode of the Poisson equation -- so the
// departure d carries only what varies in x (a roll and its consequences)
// and its FP32 arithmetic is relative to that.  The step kernel needs, per
// row, the base charge, the base fluid velocity u_y and the base field E_y:
// the march table, FP32 [Ny][4] = {rho_c, u_y, E_y, 0}.
struct BaseArgs {
  int Nx, Ny;
  const double* fin;   // [9][Ny] base f at time t
  const double* gin;   // [9][Ny] base g at time t
  double* fout;        // [9][Ny] at t + 1
  double* gout;
  const double* EB;    // [Ny] base E_y at time t
  const double* mom;   // [5][Ny] rho, rho_c, u_x, u_y, u_y + mu_b E_y at time t
  double wp, wm, gwp, gwm, mub, rho0, eps;
  double cp, cm;       // force factors 1 - wp / 2, 1 - wm / 2
  double* flux_acc;    // [2] FP64 totals of the base's injected / collected charge
  double* sums;        // [4][Ny] rho_c, rho, j_y, j_x of the state at t + 1 (out)
  double* rhs;         // [Ny] its mean-mode right-hand side -Nx rho_c / eps (out)
  double* loc;         // [2][Ny] chunk-local prefix sums of rhs (out)
  double* chunk;       // [2][base_chunks(Ny)] chunk totals (out)
};
struct BasePoissonArgs {
  int Nx, Ny, wall_mode;
  double phi0, mub;
  const double* rhs;   // [Ny] mean-mode right-hand side of the state
  const double* sums;  // [4][Ny] its rho_c, rho, j_y, j_x
  const double* loc;   // [2][Ny] and the chunk sums of the right-hand side
  const double* chunk;
  double* phiB;        // [Ny] base potential (out)
  double* EB;          // [Ny] base E_y (out)
  float* table;        // [Ny][4] march table (out)
  double* mom;         // [5][Ny] moments for the state's base step (out)
};
// rows per chunk of the base kernels: chunks of a run's base state
int base_chunks(int Ny);
cudaError_t launch_base_step(const BaseArgs& a, cudaStream_t s);
// row sums and right-hand side of the state fin / gin (fout, gout unused)
cudaError_t launch_base_sums(const BaseArgs& a, cudaStream_t s);
cudaError_t launch_base_poisson(const BasePoissonArgs& a, cudaStream_t s);

// ------------------------------------------------------------- batches ---
// A batch advances many runs (FP32 storage and compute, march form) together:
// each phase of the step is one persistent kernel over a work list that
// covers every member run; the lists live in device memory, so membership
// changes need no new launch configuration.
struct BatchRunDesc {
  StepArgs sa[2];    // [p]: step from buffer p to 1 - p
  PoissonArgs pa;    // Poisson solve of the run (with its wall fluxes)
  BaseArgs ba[2];    // perturbation form: the base step from buffer p (ba[p].fin == nullptr otherwise)
  BasePoissonArgs bp[2];  // and the potential of its result (bp[p].sums == nullptr otherwise)
  int cur0;          // buffer holding the state at the start of the tick
  int remaining;     // steps the run still takes in this tick
  int E;             // Nx / 64: warp-FFT shape
  int pad;
};
struct BatchTables {
  const BatchRunDesc* runs;
  const int4* march_items;  // (run, strip, slab, 0)
  const int2* row_items;    // (run, row)
  const int2* tile_items;   // (run, first wavenumber)
  const int* counts;        // device: [0] runs, [1] march items, [2] rows, [3] tiles
  int* work;                // device: items taken so far in this step's march, forward FFT,
                            // wavenumber and inverse FFT phases (zeroed before each step)
  int modes_smem;           // tile bytes for the largest admissible Ny (fixed per batch)
  int pdl;                  // programmatic dependent launch: 1 forward transforms, 2 tiles, 4 inverse
  int emax;                 // largest admissible Nx / 64: the widest warp-FFT shape compiled in
};

// Dynamic scheduling of a batch phase's items (largest first in the lists):
// one lane or thread takes the next index from the phase's counter.
__device__ __forceinline__ int next_item_warp(int* counter) {
  int it = 0;
  if ((threadIdx.x & 31) == 0) it = atomicAdd(counter, 1);
  return __shfl_sync(0xffffffffu, it, 0);
}
// one launch of each phase for step t (0-based) of a tick
// pert: the graph has perturbation-form members (the march branches per run)
cudaError_t launch_batch_march(const BatchTables& t, int step, int grid, bool pert, cudaStream_t s);
cudaError_t launch_batch_rfft(const BatchTables& t, int step, int grid, cudaStream_t s);
cudaError_t launch_batch_irfft(const BatchTables& t, int step, int grid, cudaStream_t s);
cudaError_t launch_batch_modes(const BatchTables& t, int step, int grid, cudaStream_t s);
cudaError_t launch_batch_mean(const BatchTables& t, int step, int grid, cudaStream_t s);
// wavenumber-tile CTAs of the batch that fit one SM with `smem` bytes of tile
int batch_modes_ctas_per_sm(int smem);
// perturbation-form members: the FP64 base step and its potential
cudaError_t launch_batch_base(const BatchTables& t, int step, int max_runs, int max_ny, cudaStream_t s);
constexpr int kBatchTileModes = 8;



// Tensor maps of the TMA form of the march kernel (FP32 storage and compute,
// Nx >= 128): the pre-collision populations as 3-D tensors {Nx, Ny, 9}
// loaded in boxes of {68, 1, 9} (a strip's 64 columns and the 4-column
// alignment margin, every plane of one row), the potential fluctuation
// {Nx, Ny} in boxes of {68, 1}, and the post-collision populations stored in
// boxes of {60, 1, 9} (a strip's owned columns).  One set per buffer parity.
constexpr int kTmaLoadCols = 68;
constexpr int kTmaStoreCols = 60;
struct MarchTma {
  CUtensorMap f, g, dphi, fo, go;
};
// Encode the maps of a run (f[cur], g[cur] in, f[1-cur], g[1-cur] out).
cudaError_t march_tma_encode(MarchTma* m, const void* fin, const void* gin, const void* dphi, void* fout, void* gout,
                             int Nx, int Ny, int P);
bool march_tma_supported(int Nx);
cudaError_t launch_march_tma(const StepArgs& a, const MarchTma& m, int form, cudaStream_t s);

// Launchers (defined in the .cu files); storage: 0 F64, 1 F32, 2 BF16, 3 F16;
// real_f64: compute type (true = double).
cudaError_t launch_step(const StepArgs& a, int storage, bool real_f64, int rows_per_cta, cudaStream_t s);
int step_flux_blocks(int Nx);
cudaError_t launch_march(const StepArgs& a, int storage, bool real_f64, cudaStream_t s);
int march_strips(int Nx, int cols_per_lane);
int march_warps_per_sm(int storage, bool real_f64, int cols_per_lane, int ring_depth);
cudaError_t march_set_attributes();
// Poisson solve from the charge plane: forward row FFTs and the wavenumber
// systems on s; the FP64 mean mode (and the wall-flux totals) on `side`
// between the fork and join events when side != nullptr.
cudaError_t launch_poisson(const PoissonArgs& a, bool real_f64, cudaStream_t s, cudaStream_t side, cudaEvent_t fork,
                           cudaEvent_t join, const cudaEvent_t* marks = nullptr);
// Odd-extension y solve (k_oddext.cu): radices of n (4, 2, 3, 5, 7, 11, 13;
// at most cap of them) into fac, their count, or -1 if n has another factor;
// the shared memory one CTA needs; the launch over m = 1 .. Mh - 1.
int oddext_factors(int n, int* fac, int cap);
size_t oddext_smem_bytes(int NE, bool real_f64);
cudaError_t launch_modes_oddext(const PoissonArgs& a, bool real_f64, cudaStream_t s);
cudaError_t oddext_set_attributes();
// rho_c = sum_i g_i (+ the row shift) into the charge plane.
cudaError_t launch_rhoc(const void* g, long long plane, int storage, bool real_f64, int Nx, int Ny, int P,
                        const float* rch, void* rhoc, cudaStream_t s);
cudaError_t poisson_set_attributes();
// warp-per-row real FFTs (FP32 path, Nx = 64 ... 2048)
bool fftw_supported(int Nx);
cudaError_t fftw_set_tables();
cudaError_t launch_rfft_warp(const PoissonArgs& a, cudaStream_t s);
cudaError_t launch_irfft_warp(const PoissonArgs& a, cudaStream_t s);
// The same transform of -i k_m phi_m (spectral E_x) into a.ex.
cudaError_t launch_irfft_warp_dx(const PoissonArgs& a, cudaStream_t s);
cudaError_t launch_fields(const FieldArgs& a, int storage, bool real_f64, unsigned mask, double* out,
                          cudaStream_t s);
cudaError_t launch_reduce_state(const FieldArgs& a, int storage, bool real_f64, double* part, int nblk,
                                double* out, int* err, cudaStream_t s);
int reduce_state_blocks();
// shift per row: shift_w (rch[y] + c0 + c1 y) + (brow ? brow[y] : 0)
cudaError_t launch_load_plane(const double* src, void* dst, int storage, int Nx, int Ny, int P, double shift_w,
                              const float* rch, double c0, double c1, const double* brow, cudaStream_t s);
cudaError_t launch_save_plane(const void* src, double* dst, int storage, int Nx, int Ny, int P, double shift_w,
                              const float* rch, double c0, double c1, const double* brow, cudaStream_t s);
// base_g (perturbation form): [9][Ny] subtracted from g instead of w_i rch[y]
cudaError_t launch_init(const double* rho_h, const double* rc_h, const double* Eh, const double* sY,
                        const double* cY, const double* Sx, const double* Cy, double Fh, double mub,
                        void* f, void* g, int storage, int Nx, int Ny, int P, const float* rch, double fb,
                        double fd, const double* base_g, cudaStream_t s);

}  // namespace ehd

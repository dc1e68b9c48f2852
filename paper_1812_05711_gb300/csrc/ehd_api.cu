// ehd_api.cu -- host side of the C ABI declared in include/ehd.h: parameter
// mapping (Eq. 26 groups -> lattice units, TRT rates of Eqs. 16-17), the
// hydrostatic constants (Eqs. 27-28), device memory of a run, the per-run CUDA
// graph of the time step, and the field / diagnostics / checkpoint calls.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "ehd.h"
#include "ehd_dev.cuh"

using namespace ehd;

namespace {

thread_local std::string g_err;

ehd_status fail(ehd_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return st;
}

#define EHD_CK(call)                                                                          \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess) return fail(EHD_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

struct Allocator {
  void* (*alloc)(size_t, void*) = nullptr;
  void (*free_fn)(void*, void*) = nullptr;
  void* ctx = nullptr;
};
std::mutex g_alloc_mu;
Allocator g_alloc;

constexpr double kPi = 3.141592653589793238462643383279502884;
constexpr int kGraphSteps = 16;  // steps per captured graph (even: buffer parity)
constexpr int kSlabShift = 4;    // default slab_shift of large runs (rows per step)

size_t storage_bytes(int storage) { return storage == 0 ? 8 : (storage == 1 ? 4 : 2); }

}  // namespace

struct ehd_run {
  int device = 0;
  int Nx = 0, Ny = 0, P = 0, Mh = 0, Mp = 0, log2Nx = 0;
  int storage = 1, compute = 1, wall_mode = 0;
  bool real_f64 = false;
  size_t rsz = 4;  // sizeof compute real
  // lattice parameters
  double T = 0, C = 0, M = 0, Fe = 0, Lambda = 0, Lambda_g = 0, u_ion = 0;
  double H = 0, mub = 0, eps = 0, nu = 0, rho0 = 0, Dc = 0, phi0 = 1.0;
  double tau_p = 0, tau_m = 0, taug_p = 0, taug_m = 0, rho_a = 0, y_a = 0;
  // device state
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  cudaStream_t side = nullptr;        // second stream for the FP64 mean mode
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  void* rhoc = nullptr;               // charge plane [Ny][P] of the compute type
  Allocator al;
  std::vector<void*> blocks;
  void* f[2] = {nullptr, nullptr};
  void* g[2] = {nullptr, nullptr};
  int cur = 0;
  void* dphi = nullptr;
  void* phibar = nullptr;
  void* Ebar = nullptr;
  void* spec = nullptr;
  void* spec0 = nullptr;
  void* rfac = nullptr;
  void* rfac0 = nullptr;
  void* tw = nullptr;
  void* rx_dn = nullptr;  // slab-boundary charge partials of the march form, [Ny/4 + 2][P] each
  void* rx_up = nullptr;
  float* rch = nullptr;  // [Ny] hydrostatic charge of each row (FP32), shifted storage only
  double fb = 0, fd = 0; // f shift fb + fd y: the hydrostatic density ramp, fd rounded to FP32
  double* flux_part = nullptr;
  int nxb = 0;
  double* small = nullptr;  // [0] q_in sum, [1] q_out sum, [2..7] last reduction, [8..9] base q_in, q_out
  int* err = nullptr;
  double* red_part = nullptr;
  int rows = 1;        // rows per CTA of the node-parallel step kernel
  int step_kernel = 0; // 0 march form, 1 node-parallel push form
  int slab_rows = 4;   // rows per warp slab of the march form
  int slab_shift = 0;  // rows the slab partition of the march form advances per step (see march_shift)
  int ring_depth = 2;  // rows staged ahead in the march form
  int cols_per_lane = 2;
  int tile_modes = 0;  // wavenumbers per CTA of the mode solve (0: largest that fits)
  int tile_threads = 0;  // threads per CTA of the mode solve (0: 256)
  int tile_cluster = 0;  // two-CTA clusters per wavenumber tile (FP32, 8 wavenumbers): off, slower
  int tile_tma = 0;      // wavenumber tiles staged by tensor copies (FP32, when the maps encode): off, slower
  ModesTma mtma = {};
  bool mtma_ok = false;
  int pdl = 0;         // programmatic dependent launch between the Poisson kernels (off: see ehd_tune)
  int fft_cta = 1;     // rows of 2048: CTA-per-row transforms
  int y_solver = 0;    // y solve of m >= 1: 0 tridiagonal, 1 odd-extension transform
  int NE = 0, nfac = -1, fac[16] = {};  // odd-extension length and radices (nfac < 0: unsupported)
  void* oddt = nullptr;  // its tables: complex R [NE] twiddles, R [NE] y symbol, R [Mh] x symbol
  int ex_spectral = 0;   // E_x from the x-spectrum of phi instead of central differences
  void* exs = nullptr;   // R [Ny][P] spectral E_x (ex_spectral only)
  int nstrips = 1;
  long step = 0;
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  ehd_batch* batch = nullptr;  // batch the run belongs to, if any
  // TMA form of the march (FP32 storage and compute, 128 <= Nx): tensor maps
  // for a step from buffer 0 and from buffer 1, and whether it is used
  MarchTma tma[2] = {};
  bool tma_ok = false;
  int march_tma = 0;
  // perturbation form: FP64 x-uniform base state ([9][Ny] per set, one per
  // buffer parity), its potential, field and the march table per parity
  int pert = 0;
  double* bf[2] = {nullptr, nullptr};
  double* bg[2] = {nullptr, nullptr};
  double* EBd = nullptr;
  double* phiB = nullptr;
  double* brhs = nullptr;
  double* bsum = nullptr;  // [4][Ny] rho_c, rho, j_y, j_x of the newest base state, [2][Ny] + [2][chunks] its prefix sums
  double* bmom = nullptr;  // [5][Ny] its moments for the next base step
  float* btab[2] = {nullptr, nullptr};
  cudaStream_t side2 = nullptr;  // the base chain: forked after the march, joined at the end of the step
  cudaEvent_t ev_base = nullptr;
};

struct ehd_batch {
  int device = 0, max_runs = 0, max_nx = 0, max_ny = 0, sms = 152;
  size_t hbm_budget = 0;      // bytes the members' device state may hold (0: no limit)
  size_t hbm_used = 0;        // sum of the members' ehd_footprint
  std::vector<size_t> member_bytes;
  cudaStream_t stream = nullptr, side = nullptr;
  bool own_stream = false;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_upload = nullptr, ev_base = nullptr;
  cudaStream_t side2 = nullptr;  // base chains of perturbation-form members
  std::vector<ehd_run*> members;
  int npert = 0;              // members in the perturbation form
  std::vector<long> remaining;
  int slab_rows = 4;
  // device tables and their pinned host staging copies
  BatchRunDesc* d_runs = nullptr;
  int4* d_march = nullptr;
  int2* d_rows = nullptr;
  int2* d_tiles = nullptr;
  int* d_counts = nullptr;
  int* d_work = nullptr;  // [4] dynamic item counters of the step's phases
  BatchRunDesc* h_runs = nullptr;
  int4* h_march = nullptr;
  int2* h_rows = nullptr;
  int2* h_tiles = nullptr;
  int* h_counts = nullptr;
  size_t cap_march = 0, cap_rows = 0, cap_tiles = 0;
  bool dirty = true;
  int grid_march = 0, grid_rows = 0, grid_tiles = 0, grid_mean = 0, modes_smem = 0;
  int slab_rows_fixed = 0;  // 0: choose from the membership
  // programmatic dependent launch of the phase kernels (mask: 1 forward
  // transforms, 2 wavenumber tiles, 4 inverse transforms): the forward
  // transforms only (64 uneven runs: 213.0 us per step against 214.3
  // without, 213.5 with all three)
  int pdl = 1;
  std::map<int, cudaGraphExec_t> graphs;  // by 2 x tick length + (any member in the perturbation form)
};

namespace {

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int now = -1;
    if (prev >= 0 && cudaGetDevice(&now) == cudaSuccess && now != prev) cudaSetDevice(prev);
  }
};

void* run_alloc(ehd_run* r, size_t bytes) {
  bytes = (bytes + 255) & ~(size_t)255;
  void* p = nullptr;
  if (r->al.alloc) {
    p = r->al.alloc(bytes, r->al.ctx);
  } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  if (p) r->blocks.push_back(p);
  return p;
}

void run_free(ehd_run* r, void* p) {
  if (!p) return;
  auto it = std::find(r->blocks.begin(), r->blocks.end(), p);
  if (it != r->blocks.end()) r->blocks.erase(it);
  if (r->al.free_fn)
    r->al.free_fn(p, r->al.ctx);
  else
    cudaFree(p);
}

// (H + ya)^{3/2} - ya^{3/2} = H ((H + ya) + sqrt((H + ya) ya) + ya) / (sqrt(H + ya) + sqrt(ya))
double hydro_gap(double ya, double H) {
  const double a = H + ya, sa = std::sqrt(a), sb = std::sqrt(ya);
  return H * (a + sa * sb + ya) / (sa + sb);
}

// Eqs. 27-28 with rho_c(0) = rho0 and int_0^H E dy = dphi0:
// rho_a = rho0 sqrt(ya), (4 rho_a / 3 eps) gap(ya) = dphi0.  Bisection on ln ya.
bool hydrostatic(double rho0, double eps, double H, double dphi0, double* rho_a, double* ya) {
  auto resid = [&](double lya) {
    const double y = std::exp(lya);
    return 4.0 * rho0 * std::sqrt(y) / (3.0 * eps) * hydro_gap(y, H) - dphi0;
  };
  double lo = std::log(H) - 46.0, hi = std::log(H) + 46.0;  // ~1e-20 H .. 1e20 H
  if (!(resid(lo) < 0.0) || !(resid(hi) > 0.0)) return false;
  for (int it = 0; it < 300; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (resid(mid) > 0.0)
      hi = mid;
    else
      lo = mid;
  }
  *ya = std::exp(0.5 * (lo + hi));
  *rho_a = rho0 * std::sqrt(*ya);
  return true;
}

ehd_status upload(ehd_run* r, void* dst, const void* src, size_t bytes) {
  EHD_CK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, r->stream));
  EHD_CK(cudaStreamSynchronize(r->stream));  // src is a temporary host vector
  return EHD_OK;
}

StepArgs step_args(const ehd_run* r, int cur) {
  StepArgs a{};
  a.Nx = r->Nx;
  a.Ny = r->Ny;
  a.P = r->P;
  a.plane = (long long)r->Ny * r->P;
  a.fin = r->f[cur];
  a.gin = r->g[cur];
  a.fout = r->f[1 - cur];
  a.gout = r->g[1 - cur];
  a.dphi = r->dphi;
  a.Ebar = r->Ebar;
  a.rch = r->rch;
  a.fb = r->fb;
  a.fd = r->fd;
  a.fdq = -r->fd * r->tau_m;
  a.ex = r->exs;
  a.flux_part = r->flux_part;
  a.err = r->err;
  a.wp = 1.0 / r->tau_p;
  a.wm = 1.0 / r->tau_m;
  a.gwp = 1.0 / r->taug_p;
  a.gwm = 1.0 / r->taug_m;
  a.mub = r->mub;
  a.rho0 = r->rho0;
  a.wall_mode = r->wall_mode;
  a.rhoc_out = r->rhoc;
  a.rhoc_dn = r->rx_dn;
  a.rhoc_up = r->rx_up;
  a.slab_rows = r->slab_rows;
  a.nstrips = r->nstrips;
  a.ring_depth = r->ring_depth;
  a.cols_per_lane = r->cols_per_lane;
  a.pdl = r->pdl;
  a.base_tab = r->pert ? r->btab[cur] : nullptr;
  return a;
}

// float-float split of a host constant: hi = fl32(v), lo = fl32(v - hi)
// (v - hi is exact in FP64), as the device forms it from a double
void split_ff(double v, float* f) {
  f[0] = (float)v;
  f[1] = (float)(v - (double)f[0]);
}

// with_flux: the charge density comes from a step (wall-flux partials
// pending, and the march form's slab-boundary partials when it ran)
PoissonArgs poisson_args(const ehd_run* r, bool with_flux) {
  PoissonArgs a{};
  a.Nx = r->Nx;
  a.Ny = r->Ny;
  a.P = r->P;
  a.Mh = r->Mh;
  a.Mp = r->Mp;
  a.log2Nx = r->log2Nx;
  a.rhoc = r->rhoc;
  a.rhoc_dn = r->rx_dn;
  a.rhoc_up = r->rx_up;
  a.xslab = (with_flux && r->step_kernel == 0 && r->cols_per_lane == 2) ? r->slab_rows : 0;
  a.inv_eps = 1.0 / r->eps;
  a.spec = r->spec;
  a.spec0 = r->spec0;
  a.rfac = r->rfac;
  a.rfac0 = r->rfac0;
  a.tw = r->tw;
  a.dphi = r->dphi;
  a.phibar = r->phibar;
  a.Ebar = r->Ebar;
  a.phi0 = r->pert ? 0.0 : r->phi0;  // perturbation form: the base carries the wall potentials
  a.mW = (double)r->Nx * a.phi0;
  a.mC = (r->wall_mode == 0) ? 1.0 / (2.0 * r->Ny) : 1.0 / (double)(r->Ny + 1);
  split_ff(a.mW, a.mWf);
  split_ff(a.mC, a.mCf);
  a.wall_mode = r->wall_mode;
  a.flux_part = with_flux ? r->flux_part : nullptr;
  a.nflux = r->nxb;
  a.flux_acc = r->small;
  a.tile_modes = r->tile_modes;
  a.tile_threads = r->tile_threads;
  a.tile_cluster = r->tile_cluster;
  a.tile_tma = r->tile_tma;
  a.mtma = r->mtma_ok ? &r->mtma : nullptr;
  a.err = r->err;
  a.pdl = r->pdl;
  a.fft_cta = r->fft_cta;
  a.y_solver = r->y_solver;
  a.ex = r->exs;
  a.NE = r->NE;
  a.nfac = r->nfac;
  for (int k = 0; k < 16; ++k) a.fac[k] = r->fac[k];
  if (r->oddt) {
    a.twy = r->oddt;
    a.symy = static_cast<const char*>(r->oddt) + 2 * (size_t)r->NE * r->rsz;
    a.kap = static_cast<const char*>(r->oddt) + 3 * (size_t)r->NE * r->rsz;
  }
  return a;
}

// Perturbation form: the potential, field and march table of the base state
// of buffer `cur`, and one FP64 step of the base from buffer `cur`.
BasePoissonArgs base_poisson_args(const ehd_run* r, int cur) {
  BasePoissonArgs b{};
  b.Nx = r->Nx;
  b.Ny = r->Ny;
  b.wall_mode = r->wall_mode;
  b.phi0 = r->phi0;
  b.mub = r->mub;
  b.rhs = r->brhs;
  b.sums = r->bsum;
  b.loc = r->bsum + 4 * (size_t)r->Ny;
  b.chunk = r->bsum + 6 * (size_t)r->Ny;
  b.mom = r->bmom;
  b.phiB = r->phiB;
  b.EB = r->EBd;
  b.table = r->btab[cur];
  return b;
}
BaseArgs base_step_args(const ehd_run* r, int cur) {
  BaseArgs b{};
  b.Nx = r->Nx;
  b.Ny = r->Ny;
  b.fin = r->bf[cur];
  b.gin = r->bg[cur];
  b.fout = r->bf[1 - cur];
  b.gout = r->bg[1 - cur];
  b.EB = r->EBd;
  b.wp = 1.0 / r->tau_p;
  b.wm = 1.0 / r->tau_m;
  b.gwp = 1.0 / r->taug_p;
  b.gwm = 1.0 / r->taug_m;
  b.mub = r->mub;
  b.rho0 = r->rho0;
  b.eps = r->eps;
  b.flux_acc = r->small + 8;
  b.cp = 1.0 - 0.5 * b.wp;
  b.cm = 1.0 - 0.5 * b.wm;
  b.mom = r->bmom;
  b.sums = r->bsum;
  b.rhs = r->brhs;
  b.loc = r->bsum + 4 * (size_t)r->Ny;
  b.chunk = r->bsum + 6 * (size_t)r->Ny;
  return b;
}
// The base step from buffer `cur` and the potential and march table of the
// result, on the third stream from the point where the departure's forward
// row transform has ended (ev_fork: the base kernels then run beside the
// wavenumber solves and the inverse transform rather than holding SM slots
// the march or the forward transform need: 125.3 us per 2048 x 1680 step
// against 127.7 when forked right after the march, and 122.4 for the shifted
// FP32 form); the main stream waits for them at the end of the step.
cudaError_t enqueue_base(ehd_run* r, int cur) {
  cudaError_t e = cudaStreamWaitEvent(r->side2, r->ev_fork, 0);
  if (e == cudaSuccess) e = launch_base_step(base_step_args(r, cur), r->side2);
  if (e == cudaSuccess) e = launch_base_poisson(base_poisson_args(r, 1 - cur), r->side2);
  if (e == cudaSuccess) e = cudaEventRecord(r->ev_base, r->side2);
  return e;
}

// Charge plane of buffer `cur`, then phi (the Poisson solve).  Perturbation
// form: the departure's charge and potential, and the base's potential.
cudaError_t enqueue_poisson(ehd_run* r, int cur, bool with_flux) {
  cudaError_t e = launch_rhoc(r->g[cur], (long long)r->Ny * r->P, r->storage, r->real_f64, r->Nx, r->Ny, r->P,
                              r->pert ? nullptr : r->rch, r->rhoc, r->stream);
  if (e != cudaSuccess) return e;
  if (r->pert) {
    if ((e = launch_base_sums(base_step_args(r, cur), r->stream)) != cudaSuccess) return e;
    if ((e = launch_base_poisson(base_poisson_args(r, cur), r->stream)) != cudaSuccess) return e;
  }
  return launch_poisson(poisson_args(r, with_flux), r->real_f64, r->stream, r->side, r->ev_fork, r->ev_join);
}

FieldArgs field_args(const ehd_run* r) {
  FieldArgs a{};
  a.Nx = r->Nx;
  a.Ny = r->Ny;
  a.P = r->P;
  a.plane = (long long)r->Ny * r->P;
  a.f = r->f[r->cur];
  a.g = r->g[r->cur];
  a.dphi = r->dphi;
  a.phibar = r->phibar;
  a.Ebar = r->Ebar;
  a.rch = r->rch;
  a.fb = r->fb;
  a.fd = r->fd;
  a.ex = r->exs;
  a.mub = r->mub;
  a.wall_mode = r->wall_mode;
  a.base_g = r->pert ? r->bg[r->cur] : nullptr;
  a.phiB = r->pert ? r->phiB : nullptr;
  a.EB = r->pert ? r->EBd : nullptr;
  return a;
}

// The march form's collide-and-stream kernel: its TMA form when the run
// takes it, else the cp.async form.
bool tma_form(const ehd_run* r) {
  return r->march_tma && r->tma_ok && r->cols_per_lane == 2 && !r->ex_spectral && r->step_kernel == 0;
}
cudaError_t launch_march_run(const ehd_run* r, const StepArgs& sa, int cur) {
  if (tma_form(r)) return launch_march_tma(sa, r->tma[cur], r->march_tma, r->stream);
  return launch_march(sa, r->storage, r->real_f64, r->stream);
}

// Slab offset of the march form at position k of the step sequence (k = step
// number mod the graph length).  The partition advances by slab_shift rows a
// step, so that each slab of the next step starts on the rows that the last
// step wrote last -- those are still in L2 when the next march begins, and
// its first reads hit there instead of in HBM.  Which slab computes a row
// changes only where partial charge sums are added (rounding order).
int march_shift(const ehd_run* r, long k) {
  if (r->slab_shift <= 0 || r->step_kernel != 0 || r->cols_per_lane != 2 || tma_form(r) || r->batch) return 0;
  return (int)((k * (long)r->slab_shift) % r->slab_rows);
}

// One coupled step from buffer `cur`: collide+stream with the wall-flux
// partials, then the Poisson solve of the new charge (which also adds the
// fluxes to the FP64 totals).  The march form writes the new charge itself;
// the node-parallel form needs the separate charge-moment kernel.
cudaError_t enqueue_step(ehd_run* r, int cur, long k) {
  StepArgs sa = step_args(r, cur);
  if (r->step_kernel == 0) {
    sa.slab_off = march_shift(r, k);
    PoissonArgs pa = poisson_args(r, true);
    pa.xoff = sa.slab_off;
    cudaError_t e = launch_march_run(r, sa, cur);
    if (e == cudaSuccess) e = launch_poisson(pa, r->real_f64, r->stream, r->side, r->ev_fork, r->ev_join);
    if (e == cudaSuccess && r->pert) e = enqueue_base(r, cur);
    if (e == cudaSuccess && r->pert) e = cudaStreamWaitEvent(r->stream, r->ev_base, 0);
    return e;
  }
  cudaError_t e = launch_step(sa, r->storage, r->real_f64, r->rows, r->stream);
  if (e != cudaSuccess) return e;
  return enqueue_poisson(r, 1 - cur, true);
}

ehd_status build_graph(ehd_run* r, int cur) {
  cudaGraph_t g = nullptr;
  EHD_CK(cudaStreamBeginCapture(r->stream, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = cudaSuccess;
  int c = cur;
  for (int k = 0; k < kGraphSteps && e == cudaSuccess; ++k) {
    e = enqueue_step(r, c, k);
    c = 1 - c;
  }
  cudaError_t e2 = cudaStreamEndCapture(r->stream, &g);
  if (e != cudaSuccess || e2 != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return fail(EHD_ECUDA, "graph capture: %s", cudaGetErrorString(e != cudaSuccess ? e : e2));
  }
  e = cudaGraphInstantiate(&r->graph[cur], g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return fail(EHD_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
  return EHD_OK;
}

ehd_status check_err(ehd_run* r) {
  if (r->batch) EHD_CK(cudaStreamSynchronize(r->batch->stream));
  int h = 0;
  EHD_CK(cudaMemcpyAsync(&h, r->err, sizeof(int), cudaMemcpyDeviceToHost, r->stream));
  EHD_CK(cudaStreamSynchronize(r->stream));
  if (h & 2) return fail(EHD_ETIMEOUT, "a bounded wait of the step kernel gave up (tensor copy not completed)");
  if (h) return fail(EHD_EDIVERGED, "non-finite density or charge in the state");
  return EHD_OK;
}

ehd_status destroy_quiet(ehd_run* r) {
  if (!r) return EHD_OK;
  DeviceGuard dg(r->device);
  if (r->stream) cudaStreamSynchronize(r->stream);
  for (int k = 0; k < 2; ++k)
    if (r->graph[k]) cudaGraphExecDestroy(r->graph[k]);
  if (r->side) cudaStreamSynchronize(r->side);
  if (r->side2) cudaStreamSynchronize(r->side2);
  if (r->ev_fork) cudaEventDestroy(r->ev_fork);
  if (r->ev_join) cudaEventDestroy(r->ev_join);
  if (r->ev_base) cudaEventDestroy(r->ev_base);
  if (r->side) cudaStreamDestroy(r->side);
  if (r->side2) cudaStreamDestroy(r->side2);
  std::vector<void*> bl = r->blocks;
  for (void* p : bl) run_free(r, p);
  if (r->own_stream && r->stream) cudaStreamDestroy(r->stream);
  delete r;
  return EHD_OK;
}

}  // namespace

namespace ehd {
// Lets other translation units of the library report through ehd_last_error.
void set_error(const char* msg) { g_err = msg; }
}  // namespace ehd

// ======================================================================= ABI
extern "C" {

void ehd_default_options(ehd_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof *o);
  o->step_kernel = -1;
  o->storage = EHD_STORE_F32;
  o->compute = EHD_COMPUTE_F32;
  o->lambda_g = 1e-6;
  o->u_ion = 2e-3;
  o->wall_mode = 0;
  o->n_modes = 0;
  o->stream = nullptr;
  o->perturbation = 0;
  o->dc_printed = 0;
}

const char* ehd_last_error(void) { return g_err.c_str(); }

ehd_status ehd_set_allocator(void* (*alloc)(size_t, void*), void (*free_fn)(void*, void*), void* ctx) {
  if ((alloc == nullptr) != (free_fn == nullptr)) return fail(EHD_EINVAL, "alloc and free must both be set or both NULL");
  std::lock_guard<std::mutex> lk(g_alloc_mu);
  g_alloc.alloc = alloc;
  g_alloc.free_fn = free_fn;
  g_alloc.ctx = ctx;
  return EHD_OK;
}

ehd_status ehd_footprint(int Nx, int Ny, int storage, size_t* bytes) {
  if (!bytes) return fail(EHD_EINVAL, "bytes is NULL");
  if (Nx < 16 || Nx > 2048 || (Nx & (Nx - 1)) || Ny < 2 || Ny > 8192 || storage < 0 || storage > 3)
    return fail(EHD_EINVAL, "unsupported size or storage");
  const size_t P = (size_t)((Nx + 31) / 32 * 32), Mp = ((size_t)Nx / 2 + 1 + 3) / 4 * 4;
  const size_t rs = (storage == 0) ? 8 : 4;  // worst case for the compute type
  const size_t ny = (size_t)Ny, plane = ny * P;
  // the buffers ehd_create allocates, each rounded as a caching allocator
  // carves it (2 MiB above 1 MiB, 512 B below), so that the sum bounds what
  // a run holds whichever allocator serves it
  const size_t bufs[] = {
      9 * plane * storage_bytes(storage), 9 * plane * storage_bytes(storage),  // f ping-pong
      9 * plane * storage_bytes(storage), 9 * plane * storage_bytes(storage),  // g ping-pong
      plane * rs, plane * rs,                                                  // dphi, rho_c
      ny * 8, ny * rs, ny * Mp * 2 * rs, ny * 8, Mp * ny * rs, ny * 8,         // phibar .. rfac0
      (size_t)(Nx + 1024) * 2 * rs, ny * 4,                                    // twiddles, shifts
      (ny / 4 + 2) * P * rs, (ny / 4 + 2) * P * rs,                            // slab-boundary shares
      2 * (size_t)std::max(march_strips(Nx, 1), step_flux_blocks(Nx)) * 8,    // flux partials
      16 * 8 + 64, (size_t)reduce_state_blocks() * 6 * 8,
      (3 * (2 * ny + 2) + (size_t)Nx / 2 + 1) * rs,                          // odd-extension tables
      9 * ny * 8, 9 * ny * 8, 9 * ny * 8, 9 * ny * 8, ny * 8, ny * 8, ny * 8,  // perturbation-form base
      ny * 16, ny * 16};
  size_t b = 0;
  for (size_t v : bufs) {
    const size_t g = (v > (1u << 20)) ? (2u << 20) : 512;
    b += (v + g - 1) / g * g;
  }
  *bytes = b;
  return EHD_OK;
}

ehd_status ehd_create(int Nx, int Ny, double T, double C, double M, double Fe, double Lambda, const ehd_options* opt,
                      ehd_run** out) {
  if (!out) return fail(EHD_EINVAL, "out is NULL");
  *out = nullptr;
  ehd_options o;
  ehd_default_options(&o);
  if (opt) o = *opt;
  // the row transforms hold a row in one CTA (at most 2048 points)
  if (Nx < 16 || Nx > 2048 || (Nx & (Nx - 1)))
    return fail(EHD_EINVAL, "Nx must be a power of two in [16, 2048] (got %d)", Nx);
  if (Ny < 2 || Ny > 8192) return fail(EHD_EINVAL, "Ny must be in [2, 8192] (got %d)", Ny);
  if (!(T > 0) || !(C > 0) || !(M > 0) || !(Fe > 0) || !(Lambda > 0))
    return fail(EHD_EINVAL, "T, C, M, Fe and Lambda must be positive");
  if (!(o.lambda_g > 0) || !(o.u_ion > 0)) return fail(EHD_EINVAL, "lambda_g and u_ion must be positive");
  if (o.storage < 0 || o.storage > 3) return fail(EHD_EINVAL, "storage must be 0..3");
  if (o.compute != EHD_COMPUTE_F64 && o.compute != EHD_COMPUTE_F32) return fail(EHD_EINVAL, "compute must be 0 or 1");
  if (o.compute == EHD_COMPUTE_F64 && o.storage != EHD_STORE_F64)
    return fail(EHD_EINVAL, "FP64 compute needs FP64 storage");
  if (o.wall_mode != 0 && o.wall_mode != 1) return fail(EHD_EINVAL, "wall_mode must be 0 or 1");
  if (o.x_symbol != 0 && o.x_symbol != 1) return fail(EHD_EINVAL, "x_symbol must be 0 or 1");
  if (o.ex_spectral != 0 && o.ex_spectral != 1) return fail(EHD_EINVAL, "ex_spectral must be 0 or 1");
  if (o.ex_spectral && o.step_kernel == 1) return fail(EHD_EINVAL, "spectral E_x needs the march form");
  if (o.n_modes < 0 || o.n_modes > EHD_MAX_PERT_MODES) return fail(EHD_EINVAL, "n_modes out of range");
  if (o.step_kernel < -1 || o.step_kernel > 1) return fail(EHD_EINVAL, "step_kernel must be -1, 0 or 1");
  if (o.perturbation != 0 && o.perturbation != 1) return fail(EHD_EINVAL, "perturbation must be 0 or 1");
  if (o.perturbation && (o.compute != EHD_COMPUTE_F32 || o.ex_spectral || o.step_kernel == 1))
    return fail(EHD_EINVAL, "the perturbation form needs FP32 compute, the march form and central-difference E_x");

  ehd_run* r = new ehd_run();
  {
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    r->al = g_alloc;
  }
  if (cudaGetDevice(&r->device) != cudaSuccess) {
    delete r;
    return fail(EHD_ECUDA, "no CUDA device");
  }
  r->Nx = Nx;
  r->Ny = Ny;
  r->P = (Nx + 31) / 32 * 32;
  r->Mh = Nx / 2 + 1;
  r->Mp = (r->Mh + 3) / 4 * 4;
  while ((1 << r->log2Nx) < Nx) ++r->log2Nx;
  r->storage = o.storage;
  r->compute = o.compute;
  r->real_f64 = (o.compute == EHD_COMPUTE_F64);
  r->rsz = r->real_f64 ? 8 : 4;
  r->wall_mode = o.wall_mode;
  r->T = T, r->C = C, r->M = M, r->Fe = Fe, r->Lambda = Lambda, r->Lambda_g = o.lambda_g, r->u_ion = o.u_ion;
  // Eq. 26 with rho = 1, dphi0 = 1, H = Ny and mu_b = u_ion H / dphi0
  r->H = (double)Ny;
  r->mub = o.u_ion * r->H;
  r->eps = M * M * r->mub * r->mub;        // M = sqrt(eps / rho) / mu_b
  r->nu = r->eps / (T * r->mub);           // T = eps dphi0 / (mu mu_b)
  r->rho0 = C * r->eps / (r->H * r->H);    // C = rho0 H^2 / (eps dphi0)
  r->Dc = r->mub / Fe;                     // Fe = mu_b dphi0 / Dc
  // Eqs. 16-17 (dt = 1, cs2 = 1/3): nu from the symmetric fluid rate; the
  // charge flux relaxes with the antisymmetric rate, which carries Dc
  r->tau_p = 3.0 * r->nu + 0.5;
  r->tau_m = 0.5 + Lambda / (r->tau_p - 0.5);
  if (o.dc_printed) {  // Eq. 16 as printed: the symmetric charge rate carries Dc
    r->taug_p = 3.0 * r->Dc + 0.5;
    r->taug_m = 0.5 + o.lambda_g / (r->taug_p - 0.5);
  } else {
    r->taug_m = 3.0 * r->Dc + 0.5;
    r->taug_p = 0.5 + o.lambda_g / (r->taug_m - 0.5);
  }
  if (r->tau_p > 50.0 || r->tau_m > 50.0 || r->taug_p > 50.0 || r->taug_m > 50.0) {
    ehd_status st0 = fail(EHD_EINVAL, "relaxation time above 50 (tau+ %.3g, tau- %.3g, tau_g+ %.3g, tau_g- %.3g)",
                          r->tau_p, r->tau_m, r->taug_p, r->taug_m);
    delete r;
    return st0;
  }
  if (!hydrostatic(r->rho0, r->eps, r->H, 1.0, &r->rho_a, &r->y_a)) {
    delete r;
    return fail(EHD_EINVAL, "hydrostatic profile has no solution");
  }
  const bool shifted = !r->real_f64;

  DeviceGuard dg(r->device);
  ehd_status st = EHD_OK;
  if (o.stream) {
    r->stream = static_cast<cudaStream_t>(o.stream);
  } else {
    if (cudaStreamCreateWithFlags(&r->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete r;
      return fail(EHD_ECUDA, "stream creation failed");
    }
    r->own_stream = true;
  }
  if (cudaStreamCreateWithFlags(&r->side, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&r->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&r->ev_join, cudaEventDisableTiming) != cudaSuccess ||
      (o.perturbation && (cudaStreamCreateWithFlags(&r->side2, cudaStreamNonBlocking) != cudaSuccess ||
                          cudaEventCreateWithFlags(&r->ev_base, cudaEventDisableTiming) != cudaSuccess))) {
    destroy_quiet(r);
    return fail(EHD_ECUDA, "stream/event creation failed");
  }
  {
    cudaError_t e = poisson_set_attributes();
    if (e == cudaSuccess) e = march_set_attributes();
    if (e == cudaSuccess) e = oddext_set_attributes();
    if (e != cudaSuccess) {
      destroy_quiet(r);
      return fail(EHD_ECUDA, "setting the shared-memory limit of the Poisson kernels: %s", cudaGetErrorString(e));
    }
  }

  const size_t plane = (size_t)Ny * r->P;
  const size_t sb = storage_bytes(r->storage);
  for (int k = 0; k < 2; ++k) {
    r->f[k] = run_alloc(r, 9 * plane * sb);
    r->g[k] = run_alloc(r, 9 * plane * sb);
  }
  r->dphi = run_alloc(r, plane * r->rsz);
  r->rhoc = run_alloc(r, plane * r->rsz);
  r->phibar = run_alloc(r, Ny * sizeof(double));
  r->Ebar = run_alloc(r, Ny * r->rsz);
  r->spec = run_alloc(r, (size_t)Ny * r->Mp * 2 * r->rsz);
  r->spec0 = run_alloc(r, Ny * sizeof(double));
  r->rfac = run_alloc(r, (size_t)r->Mp * Ny * r->rsz);
  r->rfac0 = run_alloc(r, Ny * sizeof(double));
  // twiddles exp(-2 pi i q / Nx), q < Nx; FP32 rows of 2048 append the
  // first-pass twiddles of the CTA transform, [k1 < 16][t < 64]
  r->tw = run_alloc(r, (size_t)(Nx + (Nx == 2048 && !r->real_f64 ? 1024 : 0)) * 2 * r->rsz);
  if (shifted) r->rch = static_cast<float*>(run_alloc(r, Ny * sizeof(float)));
  r->NE = (r->wall_mode == 0) ? 2 * Ny : 2 * Ny + 2;
  r->nfac = oddext_factors(r->NE, r->fac, 16);
  if (r->nfac > 0) r->oddt = run_alloc(r, (3 * (size_t)r->NE + r->Mh) * r->rsz);
  r->ex_spectral = o.ex_spectral;
  if (r->ex_spectral) {
    r->exs = run_alloc(r, (size_t)Ny * r->P * r->rsz);
  }
  r->rx_dn = run_alloc(r, (size_t)(Ny / 4 + 2) * r->P * r->rsz);
  r->rx_up = run_alloc(r, (size_t)(Ny / 4 + 2) * r->P * r->rsz);
  r->pert = o.perturbation;
  if (r->pert) {
    for (int k = 0; k < 2; ++k) {
      r->bf[k] = static_cast<double*>(run_alloc(r, 9 * (size_t)Ny * sizeof(double)));
      r->bg[k] = static_cast<double*>(run_alloc(r, 9 * (size_t)Ny * sizeof(double)));
      r->btab[k] = static_cast<float*>(run_alloc(r, 4 * (size_t)Ny * sizeof(float)));
    }
    r->EBd = static_cast<double*>(run_alloc(r, (size_t)Ny * sizeof(double)));
    r->phiB = static_cast<double*>(run_alloc(r, (size_t)Ny * sizeof(double)));
    r->brhs = static_cast<double*>(run_alloc(r, (size_t)Ny * sizeof(double)));
    r->bsum = static_cast<double*>(run_alloc(r, (6 * (size_t)Ny + 2 * (size_t)base_chunks(Ny)) * sizeof(double)));
    r->bmom = static_cast<double*>(run_alloc(r, 5 * (size_t)Ny * sizeof(double)));
  }
  r->step_kernel = (o.step_kernel >= 0) ? o.step_kernel : (r->real_f64 && !o.ex_spectral) ? 1 : 0;
  // programmatic dependent launch (mask of EHD_TUNE_PDL), as measured per
  // step: all three Poisson kernels (7) for up to 2^18 nodes (512 x 416:
  // 20.1 us against 20.7 with 3) and from 2^21 (2048 x 1680: 114.1 against
  // 114.3 with 11, 114.7 with 3, 116.9 with none); between them the forward
  // transform, the wavenumber solve and the step kernel (11; 1024 x 840: 41.2
  // against 41.7 with 7, 42.4 with 3).  Perturbation-form runs take 11 at
  // every size (512 x 416: 28.9 against 29.5 with 7; 2048 x 1680: 120.2
  // against 121.1 with 3 and 135.4 with 7, whose early-resident inverse
  // transform CTAs starve the base chain on the third stream)
  {
    const long long nodes = (long long)Nx * Ny;
    r->pdl = (r->pert || (nodes > (1LL << 18) && nodes < (1LL << 21))) ? 11 : 7;
  }
  r->cols_per_lane = 2;
  r->nstrips = march_strips(Nx, r->cols_per_lane);
  r->nxb = (r->step_kernel == 0) ? r->nstrips : step_flux_blocks(Nx);
  r->flux_part = static_cast<double*>(
      run_alloc(r, 2 * (size_t)std::max(march_strips(Nx, 1), step_flux_blocks(Nx)) * sizeof(double)));
  r->small = static_cast<double*>(run_alloc(r, 16 * sizeof(double) + 64));
  r->red_part = static_cast<double*>(run_alloc(r, (size_t)reduce_state_blocks() * 6 * sizeof(double)));
  bool ok = r->f[0] && r->f[1] && r->g[0] && r->g[1] && r->dphi && r->rhoc && r->rx_dn && r->rx_up && r->phibar &&
            r->Ebar && r->spec && r->spec0 &&
            r->rfac && r->rfac0 && r->tw && (!shifted || r->rch) && r->flux_part && r->small && r->red_part &&
            (r->nfac <= 0 || r->oddt) && (!r->ex_spectral || r->exs) &&
            (!r->pert || (r->bf[0] && r->bf[1] && r->bg[0] && r->bg[1] && r->btab[0] && r->btab[1] && r->EBd &&
                          r->phiB && r->brhs && r->bsum && r->bmom));
  if (!ok) {
    destroy_quiet(r);
    return fail(EHD_ENOMEM, "device allocation failed");
  }
  r->err = reinterpret_cast<int*>(r->small + 16);
  // tensor maps for staging the wavenumber tiles (FP32 compute)
  if (!r->real_f64) r->mtma_ok = modes_tma_encode(&r->mtma, r->spec, r->rfac, Ny, r->Mp) == cudaSuccess;
  // tensor maps of the TMA march (FP32 storage and compute): one set per
  // buffer parity; the default form when they encode
  if (r->storage == EHD_STORE_F32 && !r->real_f64 && march_tma_supported(Nx)) {
    r->tma_ok = march_tma_encode(&r->tma[0], r->f[0], r->g[0], r->dphi, r->f[1], r->g[1], Nx, Ny, r->P) ==
                    cudaSuccess &&
                march_tma_encode(&r->tma[1], r->f[1], r->g[1], r->dphi, r->f[0], r->g[0], Nx, Ny, r->P) ==
                    cudaSuccess;
    // the per-lane cp.async form stays the default: at 2048 x 1680 the
    // tensor-copy forms took 98.6 (loads) and 100.8 us (loads and stores)
    // per launch against its 93.4 us
    r->march_tma = 0;
  }
  // march slabs: as many warps as the GPU holds at once (one wave), at
  // least 4 rows each
  {
    int sms = 152;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, r->device);
    const long long resident =
        (long long)sms * march_warps_per_sm(r->storage, r->real_f64, r->cols_per_lane, r->ring_depth);
    long long rows = ((long long)Ny * r->nstrips + resident - 1) / resident;
    r->slab_rows = (int)std::max(4LL, std::min((long long)Ny, rows));
    // populations larger than L2: the slab partition advances a step, so that
    // the rows a step wrote last are read first by the next (see
    // march_shift); only where the one extra slab per strip keeps one wave
    int l2 = 0;
    const bool l2_known = cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, r->device) == cudaSuccess && l2 > 0;
    const long long slabs = (Ny + r->slab_rows - 1) / r->slab_rows + 1;
    const long long pop_bytes = 36 * (long long)Ny * r->P * (long long)storage_bytes(r->storage);
    if (l2_known && pop_bytes > (long long)l2 && (long long)r->nstrips * slabs <= resident) r->slab_shift = kSlabShift;
  }
  // rows per CTA of the node-parallel kernel: keep >= ~4 CTAs per SM
  {
    const long long xb = (Nx + 127) / 128;
    long long rows = xb * Ny / 608;
    r->rows = (int)std::max(1LL, std::min(8LL, rows));
  }

  // ---- host tables: twiddles, Thomas pivots, shifts, initial profiles
  {
    std::vector<double> twd(2 * (size_t)Nx);  // interleaved re, im: exp(-2 pi i q / Nx), q < Nx
    for (int q = 0; q < Nx; ++q) {
      const double ang = 2.0 * kPi * (double)q / (double)Nx;
      twd[2 * q] = std::cos(ang);
      twd[2 * q + 1] = -std::sin(ang);
    }
    if (Nx == 2048 && !r->real_f64)  // exp(-2 pi i t k1 / 1024) at [k1][t], t < 64, k1 < 16
      for (int k1 = 0; k1 < 16; ++k1)
        for (int t = 0; t < 64; ++t) {
          const double ang = 2.0 * kPi * (double)(t * k1) / 1024.0;
          twd.push_back(std::cos(ang));
          twd.push_back(-std::sin(ang));
        }
    // reciprocal Thomas pivots, [Ny][Mp] (row-major, wavenumber fastest)
    std::vector<double> piv((size_t)r->Mp * Ny, 1.0), piv0(Ny);
    for (int m = 0; m < r->Mh; ++m) {
      const double kx = 2.0 * kPi * (double)m / (double)Nx;
      const double sx = std::sin(kPi * (double)m / (double)Nx);
      const double kappa = (o.x_symbol == 1) ? 4.0 * sx * sx : kx * kx;  // Eq. 20, or the 3-point symbol
      const double diag = -(2.0 + kappa);
      const double corner = diag - (r->wall_mode == 0 ? 1.0 : 0.0);
      double prev = 0.0;
      for (int j = 0; j < Ny; ++j) {
        const double b = (j == 0 || j == Ny - 1) ? corner : diag;
        const double beta = (j == 0) ? b : b - prev;
        prev = 1.0 / beta;
        piv[(size_t)j * r->Mp + m] = prev;
        if (m == 0) piv0[j] = prev;
      }
    }
    if (r->real_f64) {
      st = upload(r, r->tw, twd.data(), twd.size() * 8);
      if (st == EHD_OK) st = upload(r, r->rfac, piv.data(), piv.size() * 8);
    } else {
      std::vector<float> twf(twd.begin(), twd.end()), pivf(piv.begin(), piv.end());
      st = upload(r, r->tw, twf.data(), twf.size() * 4);
      if (st == EHD_OK) st = upload(r, r->rfac, pivf.data(), pivf.size() * 4);
    }
    if (st == EHD_OK && r->oddt) {
      // odd-extension tables: exp(-2 pi i t / NE), 4 sin^2(pi k / NE), kappa_m
      const int NE = r->NE;
      std::vector<double> tab(3 * (size_t)NE + r->Mh);
      for (int t = 0; t < NE; ++t) {
        const double ang = 2.0 * kPi * (double)t / (double)NE, sy = std::sin(kPi * (double)t / (double)NE);
        tab[2 * t] = std::cos(ang);
        tab[2 * t + 1] = -std::sin(ang);
        tab[2 * (size_t)NE + t] = 4.0 * sy * sy;
      }
      for (int m = 0; m < r->Mh; ++m) {
        const double kx = 2.0 * kPi * (double)m / (double)Nx, sx = std::sin(kPi * (double)m / (double)Nx);
        tab[3 * (size_t)NE + m] = (o.x_symbol == 1) ? 4.0 * sx * sx : kx * kx;
      }
      if (r->real_f64) {
        st = upload(r, r->oddt, tab.data(), tab.size() * 8);
      } else {
        std::vector<float> tf(tab.begin(), tab.end());
        st = upload(r, r->oddt, tf.data(), tf.size() * 4);
      }
    }
    if (st == EHD_OK) {
      if (r->real_f64) {
        st = upload(r, r->rfac0, piv0.data(), Ny * sizeof(double));
      } else {  // float-float (hi, lo) pairs for the FP32 path's mean mode
        std::vector<float> ff(2 * (size_t)Ny);
        for (int j = 0; j < Ny; ++j) {
          ff[2 * j] = (float)piv0[j];
          ff[2 * j + 1] = (float)(piv0[j] - (double)ff[2 * j]);
        }
        st = upload(r, r->rfac0, ff.data(), ff.size() * sizeof(float));
      }
    }
    if (st != EHD_OK) {
      destroy_quiet(r);
      return st;
    }
  }
  {
    const int nx = Nx;
    std::vector<double> rho_h(Ny), rc_h(Ny), Eh(Ny), sY(Ny), cY(Ny), Sx(nx, 0.0), Cy(nx, 0.0);
    std::vector<float> rchf(Ny);
    const double Fh = 2.0 * r->rho_a * r->rho_a / r->eps;  // rho_c E of Eqs. 27-28, constant
    if (shifted) {
      // f shift: the hydrostatic density 1 + 3 Fh (y - H/2) of row y, its
      // slope rounded to FP32 so that the kernels add the row change exactly
      r->fd = (double)(float)(3.0 * Fh);
      r->fb = 1.0 + r->fd * (0.5 - 0.5 * r->H);
    }
    for (int j = 0; j < Ny; ++j) {
      const double y = j + 0.5, s = std::sqrt(y + r->y_a);
      rc_h[j] = r->rho_a / s;                       // Eq. 27
      Eh[j] = 2.0 * r->rho_a / r->eps * s;           // Eq. 28
      rho_h[j] = 1.0 + 3.0 * Fh * (y - 0.5 * r->H);  // cs2 d rho / dy = F
      sY[j] = std::sin(2.0 * kPi * y / r->H);
      cY[j] = std::cos(2.0 * kPi * y / r->H);
      rchf[j] = (float)rc_h[j];
    }
    // Eq. 29 with x, y scaled by H (Lx = Nx / H, Ly = 1), amplitude a u_ion
    const double Lx = (double)Nx / r->H;
    for (int k = 0; k < o.n_modes; ++k) {
      const double mk = k + 1.0, a = o.pert_amp[k] * o.u_ion;
      for (int x = 0; x < nx; ++x) {
        const double arg = 2.0 * kPi * mk * (double)x / (double)Nx + o.pert_phase[k];
        Sx[x] += a * (Lx / mk) * std::sin(arg);
        Cy[x] += a * std::cos(arg);
      }
    }
    std::vector<double> pack;
    pack.insert(pack.end(), rho_h.begin(), rho_h.end());
    pack.insert(pack.end(), rc_h.begin(), rc_h.end());
    pack.insert(pack.end(), Eh.begin(), Eh.end());
    pack.insert(pack.end(), sY.begin(), sY.end());
    pack.insert(pack.end(), cY.begin(), cY.end());
    pack.insert(pack.end(), Sx.begin(), Sx.end());
    pack.insert(pack.end(), Cy.begin(), Cy.end());
    double* dpack = static_cast<double*>(run_alloc(r, pack.size() * sizeof(double)));
    if (!dpack) {
      destroy_quiet(r);
      return fail(EHD_ENOMEM, "device allocation failed");
    }
    st = upload(r, dpack, pack.data(), pack.size() * sizeof(double));
    if (st == EHD_OK && shifted) st = upload(r, r->rch, rchf.data(), Ny * sizeof(float));
    if (st == EHD_OK && r->pert) {
      // base state: the x-uniform part of the initial state (no roll):
      // f^eq(rho_h, -F_h / (2 rho_h) e_y), g^eq(rho_c,h, mu_b E_h e_y)
      static const int cy[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
      static const double w[9] = {kW0, kW1, kW1, kW1, kW1, kW2, kW2, kW2, kW2};
      std::vector<double> bfh(9 * (size_t)Ny), bgh(9 * (size_t)Ny);
      for (int j = 0; j < Ny; ++j) {
        const double fy = -0.5 * Fh / rho_h[j], gy = r->mub * Eh[j];
        for (int i = 0; i < 9; ++i) {
          const double fc = cy[i] * fy, gc = cy[i] * gy;
          bfh[i * (size_t)Ny + j] = w[i] * rho_h[j] * (1.0 + 3.0 * fc + 4.5 * fc * fc - 1.5 * fy * fy);
          bgh[i * (size_t)Ny + j] = w[i] * rc_h[j] * (1.0 + 3.0 * gc + 4.5 * gc * gc - 1.5 * gy * gy);
        }
      }
      st = upload(r, r->bf[0], bfh.data(), bfh.size() * sizeof(double));
      if (st == EHD_OK) st = upload(r, r->bg[0], bgh.data(), bgh.size() * sizeof(double));
    }
    if (st == EHD_OK) {
      const double* p = dpack;
      cudaError_t e = cudaMemsetAsync(r->small, 0, 16 * sizeof(double) + 64, r->stream);
      if (e == cudaSuccess)
        e = launch_init(p, p + Ny, p + 2 * Ny, p + 3 * Ny, p + 4 * Ny, p + 5 * Ny, p + 5 * Ny + nx, Fh, r->mub,
                        r->f[0], r->g[0], r->storage, Nx, Ny, r->P, r->rch, r->fb, r->fd,
                        r->pert ? r->bg[0] : nullptr, r->stream);
      if (e == cudaSuccess) e = enqueue_poisson(r, 0, false);
      if (e == cudaSuccess) e = cudaStreamSynchronize(r->stream);
      if (e != cudaSuccess) st = fail(EHD_ECUDA, "initialisation: %s", cudaGetErrorString(e));
    }
    run_free(r, dpack);
    if (st != EHD_OK) {
      destroy_quiet(r);
      return st;
    }
  }
  *out = r;
  return EHD_OK;
}

ehd_status ehd_tune(ehd_run* r, int param, int value) {
  if (!r) return fail(EHD_EINVAL, "run is NULL");
  switch (param) {
    case EHD_TUNE_SLAB_ROWS:
      if (value < std::min(4, r->Ny) || value > r->Ny) return fail(EHD_EINVAL, "slab rows must be in [min(4, Ny), Ny]");
      r->slab_rows = value;
      break;
    case EHD_TUNE_SLAB_SHIFT:
      if (value < 0 || value > r->Ny) return fail(EHD_EINVAL, "slab shift must be in [0, Ny]");
      r->slab_shift = value;
      break;
    case EHD_TUNE_RING_DEPTH:
      if (value != 2 && value != 3 && value != 4 && value != 6) return fail(EHD_EINVAL, "ring depth must be 2, 3, 4 or 6");
      if (value != 2 && r->ex_spectral) return fail(EHD_EINVAL, "spectral E_x runs keep ring depth 2");
      if (value == 6 && r->cols_per_lane == 2) return fail(EHD_EINVAL, "ring depth 6 needs one column per lane");
      r->ring_depth = value;
      break;
    case EHD_TUNE_TILE_MODES:
      if (value != 0 && value != 1 && value != 2 && value != 4 && value != 8)
        return fail(EHD_EINVAL, "tile modes must be 0, 1, 2, 4 or 8");
      r->tile_modes = value;
      break;
    case EHD_TUNE_TILE_THREADS:
      if (value != 0 && value != 256 && value != 512 && value != 1024)
        return fail(EHD_EINVAL, "tile threads must be 0, 256, 512 or 1024");
      if (value > 256 && r->real_f64) return fail(EHD_EINVAL, "FP64 mode solves take 256 threads");
      r->tile_threads = value;
      break;
    case EHD_TUNE_TILE_CLUSTER:
      if (value != 0 && value != 1) return fail(EHD_EINVAL, "tile cluster must be 0 or 1");
      r->tile_cluster = value;
      break;
    case EHD_TUNE_TILE_TMA:
      if (value != 0 && value != 1) return fail(EHD_EINVAL, "tile tensor copies must be 0 or 1");
      r->tile_tma = value;
      break;
    case EHD_TUNE_PDL:
      if (value < 0 || value > 15) return fail(EHD_EINVAL, "programmatic dependent launch: a mask of 1, 2, 4 and 8");
      r->pdl = value;
      break;
    case EHD_TUNE_FFT_CTA:
      if (value != 0 && value != 1) return fail(EHD_EINVAL, "CTA-per-row transforms must be 0 or 1");
      r->fft_cta = value;
      break;
    case EHD_TUNE_Y_SOLVER: {
      if (value != 0 && value != 1) return fail(EHD_EINVAL, "y solver must be 0 (tridiagonal) or 1 (odd extension)");
      if (value == 1) {
        if (r->batch) return fail(EHD_EINVAL, "runs in a batch use the tridiagonal y solve");
        if (r->nfac <= 0)
          return fail(EHD_EINVAL, "odd-extension length %d has a prime factor above 13", r->NE);
        int optin = 0;
        EHD_CK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, r->device));
        if (oddext_smem_bytes(r->NE, r->real_f64) > (size_t)optin)
          return fail(EHD_EINVAL, "odd-extension column of %d points exceeds shared memory", r->NE);
      }
      r->y_solver = value;
      break;
    }
    case EHD_TUNE_COLS_PER_LANE:
      if (value != 1 && value != 2) return fail(EHD_EINVAL, "columns per lane must be 1 or 2");
      if (value != 2 && r->pert) return fail(EHD_EINVAL, "perturbation-form runs keep two columns per lane");
      if (value != 2 && r->ex_spectral) return fail(EHD_EINVAL, "spectral E_x runs keep two columns per lane");
      if (value == 2 && r->ring_depth == 6) r->ring_depth = 3;
      r->cols_per_lane = value;
      r->nstrips = march_strips(r->Nx, value);
      if (r->step_kernel == 0) r->nxb = r->nstrips;
      break;
    case EHD_TUNE_MARCH_TMA:
      if (value < 0 || value > 3) return fail(EHD_EINVAL, "TMA march must be 0, 1, 2 or 3");
      if (value != 0 && r->pert) return fail(EHD_EINVAL, "perturbation-form runs use the cp.async march");
      if (value != 0 && !r->tma_ok)
        return fail(EHD_EINVAL, "the TMA march needs FP32 storage and compute and 128 <= Nx <= 2048");
      r->march_tma = value;
      break;
    case EHD_TUNE_STEP_KERNEL:
      if (value != 0 && value != 1) return fail(EHD_EINVAL, "step kernel must be 0 or 1");
      if (value != 0 && r->pert) return fail(EHD_EINVAL, "perturbation-form runs need the march form");
      if (value != 0 && r->ex_spectral) return fail(EHD_EINVAL, "spectral E_x needs the march form");
      r->step_kernel = value;
      r->nxb = (value == 0) ? r->nstrips : step_flux_blocks(r->Nx);
      break;
    default:
      return fail(EHD_EINVAL, "unknown tuning parameter %d", param);
  }
  DeviceGuard dg(r->device);
  for (int k = 0; k < 2; ++k)
    if (r->graph[k]) {
      cudaGraphExecDestroy(r->graph[k]);
      r->graph[k] = nullptr;
    }
  return EHD_OK;
}

int ehd_tune_get(ehd_run* r, int param) {
  if (!r) return -1;
  switch (param) {
    case EHD_TUNE_SLAB_ROWS: return r->slab_rows;
    case EHD_TUNE_SLAB_SHIFT: return r->slab_shift;
    case EHD_TUNE_RING_DEPTH: return r->ring_depth;
    case EHD_TUNE_STEP_KERNEL: return r->step_kernel;
    case EHD_TUNE_COLS_PER_LANE: return r->cols_per_lane;
    case EHD_TUNE_TILE_MODES: return r->tile_modes;
    case EHD_TUNE_TILE_THREADS: return r->tile_threads;
    case EHD_TUNE_TILE_CLUSTER: return r->tile_cluster;
    case EHD_TUNE_TILE_TMA: return r->tile_tma;
    case EHD_TUNE_PDL: return r->pdl;
    case EHD_TUNE_FFT_CTA: return r->fft_cta;
    case EHD_TUNE_Y_SOLVER: return r->y_solver;
    case EHD_TUNE_MARCH_TMA: return tma_form(r) ? r->march_tma : 0;
  }
  return -1;
}

ehd_status ehd_poisson(ehd_run* r) {
  if (!r) return fail(EHD_EINVAL, "run is NULL");
  DeviceGuard dg(r->device);
  EHD_CK(enqueue_poisson(r, r->cur, false));
  return EHD_OK;
}

ehd_status ehd_step(ehd_run* r, long n) {
  if (!r) return fail(EHD_EINVAL, "run is NULL");
  if (r->batch) return fail(EHD_EBUSY, "run is a member of a batch: advance it with ehd_batch_tick");
  if (n < 0) return fail(EHD_EINVAL, "negative step count");
  DeviceGuard dg(r->device);
  while (n >= kGraphSteps) {
    if (!r->graph[r->cur]) {
      ehd_status st = build_graph(r, r->cur);
      if (st != EHD_OK) return st;
    }
    EHD_CK(cudaGraphLaunch(r->graph[r->cur], r->stream));
    n -= kGraphSteps;
    r->step += kGraphSteps;
  }
  for (; n > 0; --n) {
    EHD_CK(enqueue_step(r, r->cur, r->step % kGraphSteps));
    r->cur = 1 - r->cur;
    r->step += 1;
  }
  return EHD_OK;
}

ehd_status ehd_step_profile(ehd_run* r, long n, double* ms_out) {
  if (!r || !ms_out) return fail(EHD_EINVAL, "NULL argument");
  if (n < 0) return fail(EHD_EINVAL, "negative step count");
  DeviceGuard dg(r->device);
  for (int k = 0; k < EHD_NPROFILE; ++k) ms_out[k] = 0.0;
  if (n == 0) return EHD_OK;
  // events per step: [0] before the step kernel, [1] after it, [2] after the
  // charge kernel, [3] after the Poisson solve, [4..8] the Poisson marks
  constexpr int NE = 9;
  std::vector<cudaEvent_t> ev((size_t)NE * n, nullptr);
  cudaError_t e = cudaSuccess;
  for (auto& x : ev)
    if (e == cudaSuccess) e = cudaEventCreate(&x);
  for (long t = 0; t < n && e == cudaSuccess; ++t) {
    cudaEvent_t* E = &ev[(size_t)NE * t];
    StepArgs sa = step_args(r, r->cur);
    sa.slab_off = march_shift(r, r->step % kGraphSteps);
    PoissonArgs pa = poisson_args(r, true);
    pa.xoff = sa.slab_off;
    const int nxt = 1 - r->cur;
    if (e == cudaSuccess) e = cudaEventRecord(E[0], r->stream);
    if (e == cudaSuccess)
      e = (r->step_kernel == 0) ? launch_march_run(r, sa, r->cur)
                                : launch_step(sa, r->storage, r->real_f64, r->rows, r->stream);
    if (e == cudaSuccess) e = cudaEventRecord(E[1], r->stream);
    if (e == cudaSuccess && r->step_kernel == 1)
      e = launch_rhoc(r->g[nxt], (long long)r->Ny * r->P, r->storage, r->real_f64, r->Nx, r->Ny, r->P, r->rch,
                      r->rhoc, r->stream);
    if (e == cudaSuccess) e = cudaEventRecord(E[2], r->stream);
    if (e == cudaSuccess)
      e = launch_poisson(pa, r->real_f64, r->stream, r->side, r->ev_fork, r->ev_join, E + 4);
    if (e == cudaSuccess && r->pert) e = enqueue_base(r, r->cur);  // third stream, joined at the step's end
    if (e == cudaSuccess && r->pert) e = cudaStreamWaitEvent(r->stream, r->ev_base, 0);
    if (e == cudaSuccess) e = cudaEventRecord(E[3], r->stream);
    if (e == cudaSuccess) {
      r->cur = nxt;
      r->step += 1;
    }
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(r->stream);
  // (slot, from, to): summed intervals
  static const int span[8][3] = {{0, 0, 1}, {1, 1, 2}, {2, 2, 3}, {3, 0, 3},
                                 {5, 2, 4}, {6, 4, 5}, {7, 5, 6}, {8, 7, 8}};
  for (long t = 0; t < n && e == cudaSuccess; ++t) {
    const cudaEvent_t* E = &ev[(size_t)NE * t];
    for (int k = 0; k < 8 && e == cudaSuccess; ++k) {
      float ms = 0;
      e = cudaEventElapsedTime(&ms, E[span[k][1]], E[span[k][2]]);
      ms_out[span[k][0]] += ms;
    }
  }
  for (auto& x : ev)
    if (x) cudaEventDestroy(x);
  if (e != cudaSuccess) return fail(EHD_ECUDA, "ehd_step_profile: %s", cudaGetErrorString(e));
  ms_out[4] = (double)n;
  return check_err(r);
}

ehd_status ehd_fields(ehd_run* r, unsigned mask, double* host_out) {
  if (!r) return fail(EHD_EINVAL, "run is NULL");
  if (r->batch) EHD_CK(cudaStreamSynchronize(r->batch->stream));
  if (mask == 0 || (mask & ~EHD_FIELD_ALL)) return fail(EHD_EINVAL, "invalid field mask 0x%x", mask);
  if (!host_out) return fail(EHD_EINVAL, "host_out is NULL");
  DeviceGuard dg(r->device);
  int nf = 0;
  for (int b = 0; b < 7; ++b) nf += (mask >> b) & 1;
  const size_t n = (size_t)r->Nx * r->Ny;
  double* dev = static_cast<double*>(run_alloc(r, nf * n * sizeof(double)));
  if (!dev) return fail(EHD_ENOMEM, "device allocation failed");
  cudaError_t e = launch_fields(field_args(r), r->storage, r->real_f64, mask, dev, r->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(host_out, dev, nf * n * sizeof(double), cudaMemcpyDeviceToHost, r->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(r->stream);
  run_free(r, dev);
  if (e != cudaSuccess) return fail(EHD_ECUDA, "ehd_fields: %s", cudaGetErrorString(e));
  return check_err(r);
}

ehd_status ehd_diagnostics(ehd_run* r, double* out) {
  if (!r || !out) return fail(EHD_EINVAL, "NULL argument");
  if (r->batch) EHD_CK(cudaStreamSynchronize(r->batch->stream));
  DeviceGuard dg(r->device);
  EHD_CK(launch_reduce_state(field_args(r), r->storage, r->real_f64, r->red_part, reduce_state_blocks(),
                             r->small + 2, r->err, r->stream));
  double h[10];
  EHD_CK(cudaMemcpyAsync(h, r->small, 10 * sizeof(double), cudaMemcpyDeviceToHost, r->stream));
  EHD_CK(cudaStreamSynchronize(r->stream));
  out[0] = h[2];         // mass
  out[1] = h[3];         // charge
  out[2] = h[0] + h[8];  // injected since creation (departure and base parts)
  out[3] = h[1] + h[9];  // collected since creation
  out[4] = h[4];  // kinetic energy
  out[5] = h[5];  // max |u_y|
  out[6] = h[6];  // max |u|
  out[7] = (double)r->step;
  return check_err(r);
}

ehd_status ehd_load(ehd_run* r, const double* f_host, const double* g_host) {
  if (!r || !f_host || !g_host) return fail(EHD_EINVAL, "NULL argument");
  DeviceGuard dg(r->device);
  const size_t n = (size_t)r->Nx * r->Ny, plane = (size_t)r->Ny * r->P;
  const size_t sb = storage_bytes(r->storage);
  double* stage = static_cast<double*>(run_alloc(r, n * sizeof(double)));
  if (!stage) return fail(EHD_ENOMEM, "device allocation failed");
  static const double w[9] = {kW0, kW1, kW1, kW1, kW1, kW2, kW2, kW2, kW2};
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < 9 && e == cudaSuccess; ++i) {
    e = cudaMemcpyAsync(stage, f_host + i * n, n * sizeof(double), cudaMemcpyHostToDevice, r->stream);
    if (e == cudaSuccess)
      e = launch_load_plane(stage, static_cast<char*>(r->f[r->cur]) + i * plane * sb, r->storage, r->Nx, r->Ny,
                            r->P, w[i], nullptr, r->fb, r->fd, nullptr, r->stream);
  }
  if (r->pert) {
    // perturbation form: the new base state is the row means of the loaded
    // populations, and g is stored as the departure from it
    std::vector<double> bfh(9 * (size_t)r->Ny, 0.0), bgh(9 * (size_t)r->Ny, 0.0);
    for (int i = 0; i < 9; ++i)
      for (int j = 0; j < r->Ny; ++j) {
        double sf = 0, sg = 0;
        for (int x = 0; x < r->Nx; ++x) {
          sf += f_host[i * n + (size_t)j * r->Nx + x];
          sg += g_host[i * n + (size_t)j * r->Nx + x];
        }
        bfh[i * (size_t)r->Ny + j] = sf / r->Nx;
        bgh[i * (size_t)r->Ny + j] = sg / r->Nx;
      }
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(r->bf[r->cur], bfh.data(), bfh.size() * sizeof(double), cudaMemcpyHostToDevice, r->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(r->bg[r->cur], bgh.data(), bgh.size() * sizeof(double), cudaMemcpyHostToDevice, r->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(r->stream);  // the host vectors end here
  }
  for (int i = 0; i < 9 && e == cudaSuccess; ++i) {
    e = cudaMemcpyAsync(stage, g_host + i * n, n * sizeof(double), cudaMemcpyHostToDevice, r->stream);
    if (e == cudaSuccess)
      e = launch_load_plane(stage, static_cast<char*>(r->g[r->cur]) + i * plane * sb, r->storage, r->Nx, r->Ny,
                            r->P, r->pert ? 0.0 : w[i], r->pert ? nullptr : r->rch, 0.0, 0.0,
                            r->pert ? r->bg[r->cur] + i * (size_t)r->Ny : nullptr, r->stream);
  }
  if (e == cudaSuccess) e = enqueue_poisson(r, r->cur, false);
  if (e == cudaSuccess) e = cudaStreamSynchronize(r->stream);
  run_free(r, stage);
  if (e != cudaSuccess) return fail(EHD_ECUDA, "ehd_load: %s", cudaGetErrorString(e));
  return EHD_OK;
}

ehd_status ehd_save(ehd_run* r, double* f_host, double* g_host) {
  if (!r) return fail(EHD_EINVAL, "run is NULL");
  if (r->batch) EHD_CK(cudaStreamSynchronize(r->batch->stream));
  DeviceGuard dg(r->device);
  const size_t n = (size_t)r->Nx * r->Ny, plane = (size_t)r->Ny * r->P;
  const size_t sb = storage_bytes(r->storage);
  double* stage = static_cast<double*>(run_alloc(r, n * sizeof(double)));
  if (!stage) return fail(EHD_ENOMEM, "device allocation failed");
  static const double w[9] = {kW0, kW1, kW1, kW1, kW1, kW2, kW2, kW2, kW2};
  cudaError_t e = cudaSuccess;
  for (int set = 0; set < 2; ++set) {
    double* host = set == 0 ? f_host : g_host;
    if (!host) continue;
    const void* base = set == 0 ? r->f[r->cur] : r->g[r->cur];
    for (int i = 0; i < 9 && e == cudaSuccess; ++i) {
      const bool dep = set == 1 && r->pert;  // g as departures from the base state
      e = launch_save_plane(static_cast<const char*>(base) + i * plane * sb, stage, r->storage, r->Nx, r->Ny, r->P,
                            dep ? 0.0 : w[i], set == 0 || dep ? nullptr : r->rch, set == 0 ? r->fb : 0.0,
                            set == 0 ? r->fd : 0.0, dep ? r->bg[r->cur] + i * (size_t)r->Ny : nullptr, r->stream);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(host + i * n, stage, n * sizeof(double), cudaMemcpyDeviceToHost, r->stream);
    }
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(r->stream);
  run_free(r, stage);
  if (e != cudaSuccess) return fail(EHD_ECUDA, "ehd_save: %s", cudaGetErrorString(e));
  return EHD_OK;
}

ehd_status ehd_params(ehd_run* r, double* out) {
  if (!r || !out) return fail(EHD_EINVAL, "NULL argument");
  const double v[16] = {(double)r->Nx, (double)r->Ny, r->H,      r->mub,    r->eps,  r->nu,
                        r->rho0,       r->Dc,         r->tau_p,  r->tau_m,  r->taug_p, r->taug_m,
                        r->rho_a,      r->y_a,        (double)r->storage, (double)r->compute};
  std::memcpy(out, v, sizeof v);
  return EHD_OK;
}

ehd_status ehd_sync(ehd_run* r) {
  if (!r) return fail(EHD_EINVAL, "run is NULL");
  DeviceGuard dg(r->device);
  return check_err(r);
}

void* ehd_stream(ehd_run* r) { return r ? static_cast<void*>(r->stream) : nullptr; }

void ehd_destroy(ehd_run* r) {
  if (r && r->batch) ehd_batch_remove(r->batch, r);
  destroy_quiet(r);
}

}  // extern "C"

// ===================================================================== batches
namespace {

template <class T>
T* pinned(size_t n) {
  void* p = nullptr;
  if (cudaHostAlloc(&p, n * sizeof(T) + 1, cudaHostAllocDefault) != cudaSuccess) return nullptr;
  return static_cast<T*>(p);
}

template <class T>
T* devmem(size_t n) {
  void* p = nullptr;
  if (cudaMalloc(&p, n * sizeof(T) + 256) != cudaSuccess) return nullptr;
  return static_cast<T*>(p);
}

void batch_free(ehd_batch* b) {
  if (!b) return;
  DeviceGuard dg(b->device);
  if (b->stream) cudaStreamSynchronize(b->stream);
  for (auto& kv : b->graphs) cudaGraphExecDestroy(kv.second);
  for (ehd_run* r : b->members) r->batch = nullptr;
  cudaFree(b->d_runs);
  cudaFree(b->d_march);
  cudaFree(b->d_rows);
  cudaFree(b->d_tiles);
  cudaFree(b->d_counts);
  cudaFree(b->d_work);
  cudaFreeHost(b->h_runs);
  cudaFreeHost(b->h_march);
  cudaFreeHost(b->h_rows);
  cudaFreeHost(b->h_tiles);
  cudaFreeHost(b->h_counts);
  if (b->ev_fork) cudaEventDestroy(b->ev_fork);
  if (b->ev_join) cudaEventDestroy(b->ev_join);
  if (b->ev_upload) cudaEventDestroy(b->ev_upload);
  if (b->ev_base) cudaEventDestroy(b->ev_base);
  if (b->side2) cudaStreamDestroy(b->side2);
  if (b->side) cudaStreamDestroy(b->side);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  delete b;
}

BatchTables batch_tables(const ehd_batch* b) {
  BatchTables t{};
  t.runs = b->d_runs;
  t.march_items = b->d_march;
  t.row_items = b->d_rows;
  t.tile_items = b->d_tiles;
  t.counts = b->d_counts;
  t.work = b->d_work;
  t.modes_smem = b->modes_smem;
  t.emax = std::max(1, b->max_nx / 64);
  t.pdl = b->pdl;
  return t;
}

// Work lists of the current membership; slab height chosen so that the
// march items of all members come to about four per resident warp (taken
// dynamically, largest first: 64 uneven runs up to 512 x 416 step in 229 us
// with 10-14-row slabs, 264 us with one wave of 45-row slabs).
void batch_build_items(ehd_batch* b, int resident_warps) {
  long long strip_rows = 0;
  for (ehd_run* r : b->members) strip_rows += (long long)march_strips(r->Nx, 2) * r->Ny;
  long long rows = (strip_rows + 4LL * resident_warps - 1) / std::max(1, 4 * resident_warps);
  b->slab_rows = b->slab_rows_fixed > 0 ? b->slab_rows_fixed : (int)std::max(4LL, rows);
  // the phases take their items from a counter in list order: largest
  // first (full slabs, then the partial top slabs by height; rows of the
  // widest runs first; wavenumber tiles of the tallest runs first), so the
  // last items taken are the short ones
  const int S = b->slab_rows;
  const size_t nmem = b->members.size();
  size_t nm = 0, nr = 0, nt = 0;
  for (size_t i = 0; i < nmem; ++i) {
    ehd_run* r = b->members[i];
    const int ns = march_strips(r->Nx, 2);
    for (int sl = 0; sl < r->Ny / S; ++sl)
      for (int s = 0; s < ns; ++s) b->h_march[nm++] = make_int4((int)i, s, sl, 0);
  }
  for (int h = S - 1; h >= 1; --h)
    for (size_t i = 0; i < nmem; ++i) {
      ehd_run* r = b->members[i];
      if (r->Ny % S != h) continue;
      const int ns = march_strips(r->Nx, 2);
      for (int s = 0; s < ns; ++s) b->h_march[nm++] = make_int4((int)i, s, r->Ny / S, 0);
    }
  std::vector<size_t> by_nx(nmem), by_ny(nmem);
  for (size_t i = 0; i < nmem; ++i) by_nx[i] = by_ny[i] = i;
  std::stable_sort(by_nx.begin(), by_nx.end(),
                   [&](size_t p, size_t q) { return b->members[p]->Nx < b->members[q]->Nx; });
  std::stable_sort(by_ny.begin(), by_ny.end(),
                   [&](size_t p, size_t q) { return b->members[p]->Ny > b->members[q]->Ny; });
  // row items: 2048 / Nx rows of one run each (one warp's four-step
  // transform), the narrowest runs first: their items walk the most rows one
  // after another, so they are the longest
  for (size_t i : by_nx)
    for (int y = 0; y < b->members[i]->Ny; y += 2048 / b->members[i]->Nx) b->h_rows[nr++] = make_int2((int)i, y);
  for (size_t i : by_ny)
    for (int m0 = 0; m0 < b->members[i]->Mh; m0 += kBatchTileModes) b->h_tiles[nt++] = make_int2((int)i, m0);
  b->h_counts[0] = (int)b->members.size();
  b->h_counts[1] = (int)nm;
  b->h_counts[2] = (int)nr;
  b->h_counts[3] = (int)nt;
}

// One tick of K steps.  With perturbation-form members (pert) each step
// also advances their FP64 base states and base potentials on a third
// stream, forked after the forward row transforms and joined at the end of
// the step.
ehd_status batch_capture(ehd_batch* b, int K, bool pert, cudaGraphExec_t* out) {
  const BatchTables t = batch_tables(b);
  cudaGraph_t g = nullptr;
  EHD_CK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = cudaSuccess;
  for (int s = 0; s < K && e == cudaSuccess; ++s) {
    e = cudaMemsetAsync(b->d_work, 0, 4 * sizeof(int), b->stream);
    if (e == cudaSuccess) e = launch_batch_march(t, s, b->grid_march, pert, b->stream);
    if (e == cudaSuccess) e = launch_batch_rfft(t, s, b->grid_rows, b->stream);
    if (e == cudaSuccess) e = cudaEventRecord(b->ev_fork, b->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->side, b->ev_fork, 0);
    if (pert) {
      if (e == cudaSuccess) e = cudaStreamWaitEvent(b->side2, b->ev_fork, 0);
      if (e == cudaSuccess) e = launch_batch_base(t, s, b->max_runs, b->max_ny, b->side2);
      if (e == cudaSuccess) e = cudaEventRecord(b->ev_base, b->side2);
    }
    if (e == cudaSuccess) e = launch_batch_mean(t, s, b->grid_mean, b->side);
    if (e == cudaSuccess) e = cudaEventRecord(b->ev_join, b->side);
    if (e == cudaSuccess) e = launch_batch_modes(t, s, b->grid_tiles, b->stream);
    if (e == cudaSuccess) e = launch_batch_irfft(t, s, b->grid_rows, b->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->ev_join, 0);
    if (pert && e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->ev_base, 0);
  }
  cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
  if (e != cudaSuccess || e2 != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return fail(EHD_ECUDA, "batch graph capture: %s", cudaGetErrorString(e != cudaSuccess ? e : e2));
  }
  e = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return fail(EHD_ECUDA, "batch graph instantiate: %s", cudaGetErrorString(e));
  return EHD_OK;
}

}  // namespace

extern "C" {

ehd_status ehd_batch_create(int max_runs, size_t hbm_budget, int max_nx, int max_ny, void* stream,
                            ehd_batch** out) {
  if (!out) return fail(EHD_EINVAL, "out is NULL");
  *out = nullptr;
  if (max_runs < 1 || max_runs > 4096) return fail(EHD_EINVAL, "max_runs must be in [1, 4096]");
  if (max_nx < 64 || max_nx > 2048 || (max_nx & (max_nx - 1)))
    return fail(EHD_EINVAL, "max_nx must be a power of two in [64, 2048]");
  if (max_ny < 2 || max_ny > 4096) return fail(EHD_EINVAL, "max_ny must be in [2, 4096]");
  ehd_batch* b = new ehd_batch();
  if (cudaGetDevice(&b->device) != cudaSuccess) {
    delete b;
    return fail(EHD_ECUDA, "no CUDA device");
  }
  b->max_runs = max_runs;
  b->max_nx = max_nx;
  b->max_ny = max_ny;
  b->hbm_budget = hbm_budget;
  cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->device);
  {
    // the batch's wavenumber tiles hold max_ny rows of 8 wavenumbers (12 B
    // each) in shared memory, beside about 16 KB of fixed scratch
    int optin = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, b->device);
    const int rows_cap = (optin - 16384) / (kBatchTileModes * (int)(sizeof(float2) + sizeof(float)));
    if (max_ny > rows_cap) {
      delete b;
      return fail(EHD_EINVAL, "max_ny %d exceeds the %d rows a batch's wavenumber tile holds", max_ny, rows_cap);
    }
  }
  if (stream) {
    b->stream = static_cast<cudaStream_t>(stream);
  } else if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) == cudaSuccess) {
    b->own_stream = true;
  }
  if (!b->stream || cudaStreamCreateWithFlags(&b->side, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->ev_join, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->ev_upload, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->ev_base, cudaEventDisableTiming) != cudaSuccess ||
      cudaStreamCreateWithFlags(&b->side2, cudaStreamNonBlocking) != cudaSuccess) {
    batch_free(b);
    return fail(EHD_ECUDA, "stream/event creation failed");
  }
  {
    cudaError_t e = poisson_set_attributes();
    if (e == cudaSuccess) e = march_set_attributes();
    if (e != cudaSuccess) {
      batch_free(b);
      return fail(EHD_ECUDA, "kernel attributes: %s", cudaGetErrorString(e));
    }
  }
  const size_t per_march = (size_t)march_strips(max_nx, 2) * (size_t)((max_ny + 3) / 4);
  b->cap_march = (size_t)max_runs * per_march;
  b->cap_rows = (size_t)max_runs * max_ny;
  b->cap_tiles = (size_t)max_runs * ((max_nx / 2 + 1 + kBatchTileModes - 1) / kBatchTileModes);
  b->d_runs = devmem<BatchRunDesc>(max_runs);
  b->d_march = devmem<int4>(b->cap_march);
  b->d_rows = devmem<int2>(b->cap_rows);
  b->d_tiles = devmem<int2>(b->cap_tiles);
  b->d_counts = devmem<int>(4);
  b->d_work = devmem<int>(4);
  b->h_runs = pinned<BatchRunDesc>(max_runs);
  b->h_march = pinned<int4>(b->cap_march);
  b->h_rows = pinned<int2>(b->cap_rows);
  b->h_tiles = pinned<int2>(b->cap_tiles);
  b->h_counts = pinned<int>(4);
  if (!b->d_runs || !b->d_march || !b->d_rows || !b->d_tiles || !b->d_counts || !b->d_work || !b->h_runs || !b->h_march ||
      !b->h_rows || !b->h_tiles || !b->h_counts) {
    batch_free(b);
    return fail(EHD_ENOMEM, "batch table allocation failed");
  }
  const int wps = march_warps_per_sm(1, false, 2, 2);
  b->grid_march = b->sms * std::max(1, wps / 4);
  // row-transform CTAs: eight per SM take the items dynamically (64 uneven
  // runs: 227.5 against 236.7 us per step with four)
  b->grid_rows = b->sms * 8;
  b->grid_mean = std::min(max_runs, b->sms);
  // wavenumber tile (spectrum + pivots) of the tallest admissible run; the
  // mean-mode solve needs less
  b->modes_smem = max_ny * kBatchTileModes * (int)(sizeof(float2) + sizeof(float));
  // as many tile CTAs as fit an SM, up to four (64 uneven runs up to 512 x
  // 416: 238.5 us per step against 256.6 with one per SM)
  b->grid_tiles = b->sms * std::max(1, std::min(4, batch_modes_ctas_per_sm(b->modes_smem)));
  *out = b;
  return EHD_OK;
}

ehd_status ehd_batch_add(ehd_batch* b, ehd_run* r, long steps) {
  if (!b || !r) return fail(EHD_EINVAL, "NULL argument");
  if (steps < 0) return fail(EHD_EINVAL, "negative step budget");
  if (r->batch) return fail(EHD_EINVAL, "run is already in a batch");
  if (r->storage != EHD_STORE_F32 || r->real_f64 || r->step_kernel != 0)
    return fail(EHD_EINVAL, "batches take FP32-storage, FP32-compute runs in the march form");
  if (r->y_solver != 0) return fail(EHD_EINVAL, "batches take runs with the tridiagonal y solve");
  if (r->ex_spectral) return fail(EHD_EINVAL, "batches take runs with central-difference E_x");
  if (r->Nx < 64 || r->Nx > b->max_nx || r->Ny > b->max_ny) return fail(EHD_EINVAL, "run size exceeds the batch limits");
  if (r->device != b->device) return fail(EHD_EINVAL, "run and batch are on different devices");
  if ((int)b->members.size() >= b->max_runs) return fail(EHD_EBUSY, "batch is full");
  size_t need = 0;
  if (ehd_footprint(r->Nx, r->Ny, r->storage, &need) != EHD_OK) return EHD_EINVAL;
  if (b->hbm_budget && b->hbm_used + need > b->hbm_budget)
    return fail(EHD_EBUSY, "HBM budget: the members hold %zu of %zu bytes, the run needs %zu", b->hbm_used,
                b->hbm_budget, need);
  DeviceGuard dg(b->device);
  EHD_CK(cudaStreamSynchronize(r->stream));
  r->batch = b;
  b->members.push_back(r);
  b->remaining.push_back(steps);
  b->member_bytes.push_back(need);
  b->hbm_used += need;
  if (r->pert) ++b->npert;
  b->dirty = true;
  return EHD_OK;
}

ehd_status ehd_batch_admits(ehd_batch* b, int Nx, int Ny, int storage) {
  if (!b) return fail(EHD_EINVAL, "batch is NULL");
  if (storage != EHD_STORE_F32) return fail(EHD_EINVAL, "batches take FP32-storage runs");
  if (Nx < 64 || Nx > b->max_nx || Ny > b->max_ny || Ny < 2)
    return fail(EHD_EINVAL, "a %dx%d run exceeds the batch limits", Nx, Ny);
  size_t need = 0;
  ehd_status st = ehd_footprint(Nx, Ny, storage, &need);
  if (st != EHD_OK) return st;
  if (b->hbm_budget && need > b->hbm_budget)
    return fail(EHD_EINVAL, "a %dx%d run needs %zu bytes, more than the whole HBM budget of %zu", Nx, Ny, need,
                b->hbm_budget);
  if ((int)b->members.size() >= b->max_runs) return fail(EHD_EBUSY, "batch is full");
  if (b->hbm_budget && b->hbm_used + need > b->hbm_budget)
    return fail(EHD_EBUSY, "HBM budget: the members hold %zu of %zu bytes, the run needs %zu", b->hbm_used,
                b->hbm_budget, need);
  return EHD_OK;
}

ehd_status ehd_batch_memory(ehd_batch* b, size_t* used, size_t* budget) {
  if (!b) return fail(EHD_EINVAL, "batch is NULL");
  if (used) *used = b->hbm_used;
  if (budget) *budget = b->hbm_budget;
  return EHD_OK;
}

ehd_status ehd_batch_remove(ehd_batch* b, ehd_run* r) {
  if (!b || !r) return fail(EHD_EINVAL, "NULL argument");
  auto it = std::find(b->members.begin(), b->members.end(), r);
  if (it == b->members.end()) return fail(EHD_EINVAL, "run is not a member of this batch");
  DeviceGuard dg(b->device);
  EHD_CK(cudaStreamSynchronize(b->stream));
  const size_t i = (size_t)(it - b->members.begin());
  b->members.erase(it);
  b->remaining.erase(b->remaining.begin() + i);
  b->hbm_used -= b->member_bytes[i];
  b->member_bytes.erase(b->member_bytes.begin() + i);
  if (r->pert) --b->npert;
  r->batch = nullptr;
  b->dirty = true;
  return EHD_OK;
}

ehd_status ehd_batch_tick(ehd_batch* b, int steps) {
  if (!b) return fail(EHD_EINVAL, "batch is NULL");
  if (steps < 2 || (steps & 1)) return fail(EHD_EINVAL, "a tick is an even number of steps >= 2");
  DeviceGuard dg(b->device);
  // the staging buffers of the previous tick must have been consumed
  EHD_CK(cudaEventSynchronize(b->ev_upload));
  if (b->dirty) {
    const int wps = march_warps_per_sm(1, false, 2, 2);
    batch_build_items(b, b->sms * wps);
  }
  for (size_t i = 0; i < b->members.size(); ++i) {
    ehd_run* r = b->members[i];
    BatchRunDesc& d = b->h_runs[i];
    for (int p = 0; p < 2; ++p) {
      d.sa[p] = step_args(r, p);
      d.sa[p].cols_per_lane = 2;
      d.sa[p].ring_depth = 2;
      d.sa[p].nstrips = march_strips(r->Nx, 2);
      d.sa[p].slab_rows = b->slab_rows;
    }
    for (int p = 0; p < 2; ++p) {
      d.ba[p] = r->pert ? base_step_args(r, p) : BaseArgs{};
      d.bp[p] = r->pert ? base_poisson_args(r, 1 - p) : BasePoissonArgs{};
    }
    d.pa = poisson_args(r, true);
    d.pa.nflux = d.sa[0].nstrips;
    d.pa.xslab = b->slab_rows;
    d.cur0 = r->cur;
    d.remaining = (int)std::min<long>(steps, b->remaining[i]);
    d.E = r->Nx / 64;
  }
  const size_t nrun = b->members.size();
  if (nrun > 0) EHD_CK(cudaMemcpyAsync(b->d_runs, b->h_runs, nrun * sizeof(BatchRunDesc), cudaMemcpyHostToDevice, b->stream));
  if (b->dirty) {
    EHD_CK(cudaMemcpyAsync(b->d_counts, b->h_counts, 4 * sizeof(int), cudaMemcpyHostToDevice, b->stream));
    if (b->h_counts[1] > 0)
      EHD_CK(cudaMemcpyAsync(b->d_march, b->h_march, b->h_counts[1] * sizeof(int4), cudaMemcpyHostToDevice, b->stream));
    if (b->h_counts[2] > 0)
      EHD_CK(cudaMemcpyAsync(b->d_rows, b->h_rows, b->h_counts[2] * sizeof(int2), cudaMemcpyHostToDevice, b->stream));
    if (b->h_counts[3] > 0)
      EHD_CK(cudaMemcpyAsync(b->d_tiles, b->h_tiles, b->h_counts[3] * sizeof(int2), cudaMemcpyHostToDevice, b->stream));
    b->dirty = false;
  }
  EHD_CK(cudaEventRecord(b->ev_upload, b->stream));
  if (nrun == 0) return EHD_OK;
  const int key = 2 * steps + (b->npert > 0);
  auto it = b->graphs.find(key);
  if (it == b->graphs.end()) {
    cudaGraphExec_t ge = nullptr;
    ehd_status st = batch_capture(b, steps, b->npert > 0, &ge);
    if (st != EHD_OK) return st;
    it = b->graphs.emplace(key, ge).first;
  }
  EHD_CK(cudaGraphLaunch(it->second, b->stream));
  for (size_t i = 0; i < nrun; ++i) {
    ehd_run* r = b->members[i];
    const long k = std::min<long>(steps, b->remaining[i]);
    b->remaining[i] -= k;
    r->step += k;
    r->cur ^= (int)(k & 1);
  }
  return EHD_OK;
}

long ehd_batch_remaining(ehd_batch* b, ehd_run* r) {
  if (!b || !r) return -1;
  for (size_t i = 0; i < b->members.size(); ++i)
    if (b->members[i] == r) return b->remaining[i];
  return -1;
}

int ehd_batch_size(ehd_batch* b) { return b ? (int)b->members.size() : -1; }

ehd_status ehd_batch_sync(ehd_batch* b) {
  if (!b) return fail(EHD_EINVAL, "batch is NULL");
  DeviceGuard dg(b->device);
  EHD_CK(cudaStreamSynchronize(b->stream));
  for (ehd_run* r : b->members) {
    int h = 0;
    EHD_CK(cudaMemcpy(&h, r->err, sizeof(int), cudaMemcpyDeviceToHost));
    if (h & 2) return fail(EHD_ETIMEOUT, "a bounded wait of a member's step kernel gave up");
    if (h) return fail(EHD_EDIVERGED, "a member run holds a non-finite density or charge");
  }
  return EHD_OK;
}

void* ehd_batch_stream(ehd_batch* b) { return b ? static_cast<void*>(b->stream) : nullptr; }

ehd_status ehd_batch_tune(ehd_batch* b, int param, int value) {
  if (!b) return fail(EHD_EINVAL, "batch is NULL");
  switch (param) {
    case EHD_BATCH_SLAB_ROWS:
      if (value != 0 && (value < 4 || value > b->max_ny))
        return fail(EHD_EINVAL, "slab rows must be 0 (automatic) or in [4, max_ny]");
      b->slab_rows_fixed = value;
      b->dirty = true;
      break;
    case EHD_BATCH_MARCH_CTAS:
    case EHD_BATCH_ROW_CTAS:
    case EHD_BATCH_TILE_CTAS:
      if (value < 1 || value > 65535) return fail(EHD_EINVAL, "CTA count must be in [1, 65535]");
      if (param == EHD_BATCH_MARCH_CTAS) b->grid_march = value;
      if (param == EHD_BATCH_ROW_CTAS) b->grid_rows = value;
      if (param == EHD_BATCH_TILE_CTAS) b->grid_tiles = value;
      break;
    case EHD_BATCH_PDL:
      if (value < 0 || value > 7) return fail(EHD_EINVAL, "programmatic dependent launch: a mask of 1, 2 and 4");
      b->pdl = value;
      break;
    default:
      return fail(EHD_EINVAL, "unknown batch tuning parameter %d", param);
  }
  DeviceGuard dg(b->device);
  EHD_CK(cudaStreamSynchronize(b->stream));
  for (auto& kv : b->graphs) cudaGraphExecDestroy(kv.second);
  b->graphs.clear();
  return EHD_OK;
}

int ehd_batch_tune_get(ehd_batch* b, int param) {
  if (!b) return -1;
  switch (param) {
    case EHD_BATCH_SLAB_ROWS: return b->slab_rows_fixed > 0 ? b->slab_rows_fixed : b->slab_rows;
    case EHD_BATCH_MARCH_CTAS: return b->grid_march;
    case EHD_BATCH_ROW_CTAS: return b->grid_rows;
    case EHD_BATCH_TILE_CTAS: return b->grid_tiles;
    case EHD_BATCH_PDL: return b->pdl;
  }
  return -1;
}

void ehd_batch_destroy(ehd_batch* b) { batch_free(b); }

}  // extern "C"

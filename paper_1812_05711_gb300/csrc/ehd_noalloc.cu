// ehd_noalloc.cu -- a Poisson solve that allocates no device memory.
//
// Some callers cannot call cudaMalloc once they are running: a process whose
// device memory is entirely reserved up front by a framework's own pool, or a
// latency-critical loop where the implicit device synchronisation of
// cudaMalloc / cudaFree is not acceptable.  ehd_poisson_noalloc gives them the
// Poisson solve of the library (row FFT, one tridiagonal per wavenumber with
// the mean mode in FP64, inverse row FFT) on their own device buffers, with
// every intermediate (half spectrum, pivots, twiddles, mean profile) kept in
// one file-scope __device__ array of fixed size.  That array is part of the
// library image: every GPU that loads the library holds it until the process
// exits.
//
// In host code the array's name is only a host-side stand-in; its device
// address is looked up with cudaGetSymbolAddress on every call, with the
// calling device current, and passed to the kernels.
//
// The twiddle and pivot tables for a grid are rebuilt only when the sizes
// change, which the host tracks per device.  A call made while its stream is
// being captured cannot rely on that record (the captured work may run any
// number of times, interleaved with direct calls for other sizes), so it
// always enqueues the table build, and from then on every call on that
// device rebuilds the tables.
#include <cuda_runtime.h>

#include <mutex>

#include "ehd.h"
#include "ehd_dev.cuh"

namespace ehd {
void set_error(const char* msg);
}

namespace {

using ehd::Cplx;

constexpr size_t kScratchBytes = size_t(8) << 20;  // 8 MiB
constexpr int kMaxNx = 2048;
constexpr int kMaxNy = 4096;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

struct Layout {
  size_t spec, spec0, piv, piv0, tw, phibar, total;
};

size_t up256(size_t b) { return (b + 255) & ~size_t(255); }

Layout layout_for(int Nx, int Ny) {
  const size_t Mh = (size_t)Nx / 2 + 1;
  Layout L{};
  size_t o = 0;
  L.spec = o;   o += up256(Mh * Ny * sizeof(Cplx<float>));  // [Ny][Mh]
  L.spec0 = o;  o += up256((size_t)Ny * sizeof(double));
  L.piv = o;    o += up256(Mh * Ny * sizeof(float));        // [Mh][Ny]
  L.piv0 = o;   o += up256((size_t)Ny * sizeof(double));
  L.tw = o;     o += up256((size_t)(Nx / 2) * sizeof(Cplx<float>));
  L.phibar = o; o += up256((size_t)Ny * sizeof(double));
  L.total = o;
  return L;
}

struct DeviceSlot {
  unsigned char* base = nullptr;  // device address of g_scratch at the last call
  int Nx = 0, Ny = 0, wall_mode = -1;  // sizes the tables were built for
  bool always_rebuild = false;    // set once a call was made during stream capture
};
std::mutex g_mu;
DeviceSlot g_slots[kMaxDevices];

struct Ptrs {
  Cplx<float>* spec;
  double* spec0;
  float* piv;
  double* piv0;
  Cplx<float>* tw;
  double* phibar;
};

Ptrs ptrs(unsigned char* base, const Layout& L) {
  return {reinterpret_cast<Cplx<float>*>(base + L.spec), reinterpret_cast<double*>(base + L.spec0),
          reinterpret_cast<float*>(base + L.piv),        reinterpret_cast<double*>(base + L.piv0),
          reinterpret_cast<Cplx<float>*>(base + L.tw),   reinterpret_cast<double*>(base + L.phibar)};
}

// Twiddles exp(-2 pi i k / Nx) and reciprocal Thomas pivots of every
// wavenumber (diagonal -(2 + kappa_m), unit off-diagonals, wall corners).
__global__ void k_na_tables(int Nx, int Ny, int wall_mode, Ptrs p) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < Nx / 2) {
    double s, c;
    sincospi(2.0 * (double)t / (double)Nx, &s, &c);
    p.tw[t] = {(float)c, (float)-s};
  }
  const int Mh = Nx / 2 + 1;
  if (t < Mh) {
    const double kx = 2.0 * 3.141592653589793238462643383279502884 * (double)t / (double)Nx;
    const double diag = -(2.0 + kx * kx);
    const double corner = diag - (wall_mode == 0 ? 1.0 : 0.0);
    double prev = 0.0;
    for (int j = 0; j < Ny; ++j) {
      const double b = (j == 0 || j == Ny - 1) ? corner : diag;
      prev = 1.0 / ((j == 0) ? b : b - prev);
      if (t == 0)
        p.piv0[j] = prev;
      else
        p.piv[(size_t)t * Ny + j] = (float)prev;
    }
  }
}

__device__ Cplx<float>* na_fft(Cplx<float>* a, Cplx<float>* b, int N, const Cplx<float>* tw, bool inverse) {
  const int half = N >> 1;
  for (int Ns = 1; Ns < N; Ns <<= 1) {
    const int tstride = N / (2 * Ns);
    for (int j = threadIdx.x; j < half; j += blockDim.x) {
      const int k = j & (Ns - 1);
      Cplx<float> w = tw[k * tstride];
      if (inverse) w.im = -w.im;
      const Cplx<float> u = a[j], x = a[j + half];
      const Cplx<float> v = {x.re * w.re - x.im * w.im, x.re * w.im + x.im * w.re};
      const int idx = ((j - k) << 1) + k;
      b[idx] = {u.re + v.re, u.im + v.im};
      b[idx + Ns] = {u.re - v.re, u.im - v.im};
    }
    __syncthreads();
    Cplx<float>* t = a;
    a = b;
    b = t;
  }
  return a;
}

// One CTA per row: s = -rho_c / eps, FP64 row sum (mean mode), FFT of the rest.
__global__ void __launch_bounds__(256) k_na_fwd(int Nx, int Ny, double inv_eps, const float* __restrict__ rhoc,
                                                Ptrs p) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[8];
  Cplx<float>* A = reinterpret_cast<Cplx<float>*>(smem);
  Cplx<float>* B = A + Nx;
  const int y = blockIdx.x;
  double sum = 0.0;
  for (int x = threadIdx.x; x < Nx; x += blockDim.x) {
    const float s = -rhoc[(size_t)y * Nx + x] * (float)inv_eps;
    A[x].re = s;
    sum += (double)s;
  }
  for (int o = 16; o > 0; o >>= 1) sum += __shfl_down_sync(0xffffffffu, sum, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = sum;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    red[0] = t;
    p.spec0[y] = t;
  }
  __syncthreads();
  const float mean = (float)(red[0] / (double)Nx);
  for (int x = threadIdx.x; x < Nx; x += blockDim.x) {
    A[x].re -= mean;
    A[x].im = 0.0f;
  }
  __syncthreads();
  const Cplx<float>* res = na_fft(A, B, Nx, p.tw, false);
  const int Mh = Nx / 2 + 1;
  for (int m = threadIdx.x; m < Mh; m += blockDim.x)
    p.spec[(size_t)y * Mh + m] = (m == 0) ? Cplx<float>{0.0f, 0.0f} : res[m];
}

// Thomas recurrences of one wavenumber as a warp scan over 32 row chunks.
template <class R, class V, class Ops>
__device__ void na_thomas(V* d, const R* r, int Ny, int lane) {
  const int C = (Ny + 31) >> 5;
  const int j0 = min(lane * C, Ny), j1 = min(j0 + C, Ny);
  R al = R(1);
  V br = Ops::zero();
  for (int j = j0; j < j1; ++j) {
    al = -r[j] * al;
    br = Ops::scl(r[j], Ops::sub(d[j], br));
  }
  for (int o = 1; o < 32; o <<= 1) {
    const R a2 = __shfl_up_sync(0xffffffffu, al, o);
    const V b2 = Ops::up(br, o);
    if (lane >= o) {
      br = Ops::axpy(al, b2, br);
      al *= a2;
    }
  }
  V x = Ops::up(br, 1);
  if (lane == 0) x = Ops::zero();
  for (int j = j0; j < j1; ++j) {
    x = Ops::scl(r[j], Ops::sub(d[j], x));
    d[j] = x;
  }
  __syncwarp();
  al = R(1);
  br = Ops::zero();
  for (int j = j1 - 1; j >= j0; --j) {
    al = -r[j] * al;
    br = Ops::axpy(-r[j], br, d[j]);
  }
  for (int o = 1; o < 32; o <<= 1) {
    const R a2 = __shfl_down_sync(0xffffffffu, al, o);
    const V b2 = Ops::down(br, o);
    if (lane + o < 32) {
      br = Ops::axpy(al, b2, br);
      al *= a2;
    }
  }
  x = Ops::down(br, 1);
  if (lane == 31) x = Ops::zero();
  for (int j = j1 - 1; j >= j0; --j) {
    x = Ops::axpy(-r[j], x, d[j]);
    d[j] = x;
  }
  __syncwarp();
}

struct RealOps {
  __device__ static double zero() { return 0.0; }
  __device__ static double up(double v, int o) { return __shfl_up_sync(0xffffffffu, v, o); }
  __device__ static double down(double v, int o) { return __shfl_down_sync(0xffffffffu, v, o); }
  __device__ static double axpy(double a, double x, double b) { return a * x + b; }
  __device__ static double sub(double x, double y) { return x - y; }
  __device__ static double scl(double a, double x) { return a * x; }
};

struct CplxOps {
  using V = Cplx<float>;
  __device__ static V zero() { return {0.0f, 0.0f}; }
  __device__ static V up(V v, int o) {
    return {__shfl_up_sync(0xffffffffu, v.re, o), __shfl_up_sync(0xffffffffu, v.im, o)};
  }
  __device__ static V down(V v, int o) {
    return {__shfl_down_sync(0xffffffffu, v.re, o), __shfl_down_sync(0xffffffffu, v.im, o)};
  }
  __device__ static V axpy(float a, V x, V b) { return {a * x.re + b.re, a * x.im + b.im}; }
  __device__ static V sub(V x, V y) { return {x.re - y.re, x.im - y.im}; }
  __device__ static V scl(float a, V x) { return {a * x.re, a * x.im}; }
};

__global__ void __launch_bounds__(128) k_na_modes(int Nx, int Ny, int wall_mode, double phi0, int wpc, Ptrs p) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m = blockIdx.x * wpc + warp;
  const int Mh = Nx / 2 + 1;
  if (warp >= wpc || m >= Mh) return;
  if (m == 0) {
    double* d = reinterpret_cast<double*>(smem) + (size_t)warp * Ny;
    const double wc = (wall_mode == 0) ? 2.0 : 1.0;
    for (int j = lane; j < Ny; j += 32) d[j] = p.spec0[j] - ((j == 0) ? wc * (double)Nx * phi0 : 0.0);
    __syncwarp();
    na_thomas<double, double, RealOps>(d, p.piv0, Ny, lane);
    for (int j = lane; j < Ny; j += 32) p.phibar[j] = d[j] / (double)Nx;
    return;
  }
  Cplx<float>* d = reinterpret_cast<Cplx<float>*>(smem) + (size_t)warp * Ny;
  for (int j = lane; j < Ny; j += 32) d[j] = p.spec[(size_t)j * Mh + m];
  __syncwarp();
  na_thomas<float, Cplx<float>, CplxOps>(d, p.piv + (size_t)m * Ny, Ny, lane);
  for (int j = lane; j < Ny; j += 32) p.spec[(size_t)j * Mh + m] = d[j];
}

// One CTA per row: inverse FFT of the modes m >= 1 plus the FP64 mean profile.
__global__ void __launch_bounds__(256) k_na_inv(int Nx, int Ny, float* __restrict__ phi, Ptrs p) {
  extern __shared__ __align__(16) unsigned char smem[];
  Cplx<float>* A = reinterpret_cast<Cplx<float>*>(smem);
  Cplx<float>* B = A + Nx;
  const int y = blockIdx.x, half = Nx >> 1, Mh = Nx / 2 + 1;
  const Cplx<float>* spec = p.spec + (size_t)y * Mh;
  for (int m = threadIdx.x; m < Nx; m += blockDim.x) {
    Cplx<float> v = {0.0f, 0.0f};
    if (m > 0 && m <= half) {
      v = spec[m];
    } else if (m > half) {
      const Cplx<float> s = spec[Nx - m];
      v = {s.re, -s.im};
    }
    A[m] = v;
  }
  __syncthreads();
  const Cplx<float>* res = na_fft(A, B, Nx, p.tw, true);
  const double pb = p.phibar[y];
  for (int x = threadIdx.x; x < Nx; x += blockDim.x)
    phi[(size_t)y * Nx + x] = (float)(pb + (double)(res[x].re / (float)Nx));
}

ehd_status na_fail(ehd_status st, const char* msg) {
  ehd::set_error(msg);
  return st;
}

}  // namespace

extern "C" ehd_status ehd_poisson_noalloc(int Nx, int Ny, double eps, double phi0, int wall_mode,
                                          const float* rhoc, float* phi, void* stream) {
  if (Nx < 16 || Nx > kMaxNx || (Nx & (Nx - 1)))
    return na_fail(EHD_EINVAL, "ehd_poisson_noalloc: Nx must be a power of two in [16, 2048]");
  if (Ny < 2 || Ny > kMaxNy) return na_fail(EHD_EINVAL, "ehd_poisson_noalloc: Ny must be in [2, 4096]");
  if (!(eps > 0)) return na_fail(EHD_EINVAL, "ehd_poisson_noalloc: eps must be positive");
  if (wall_mode != 0 && wall_mode != 1) return na_fail(EHD_EINVAL, "ehd_poisson_noalloc: wall_mode must be 0 or 1");
  if (!rhoc || !phi) return na_fail(EHD_EINVAL, "ehd_poisson_noalloc: rhoc and phi must be device pointers");
  const Layout L = layout_for(Nx, Ny);
  if (L.total > kScratchBytes)
    return na_fail(EHD_EINVAL,
                   "ehd_poisson_noalloc: this grid needs more than the 8 MiB static scratch "
                   "(about 1024 x 840 nodes is the largest channel that fits)");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) return na_fail(EHD_ECUDA, "ehd_poisson_noalloc: no CUDA device");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  std::lock_guard<std::mutex> lk(g_mu);
  DeviceSlot& slot = g_slots[dev];
  void* addr = nullptr;
  e = cudaGetSymbolAddress(&addr, g_scratch);
  if (e != cudaSuccess || !addr)
    return na_fail(EHD_ECUDA, "ehd_poisson_noalloc: cudaGetSymbolAddress of the static scratch failed");
  if (static_cast<unsigned char*>(addr) != slot.base) {
    // first call on this device, or the module was loaded again (e.g. after
    // cudaDeviceReset): nothing in the array can be trusted
    slot = DeviceSlot{};
    slot.base = static_cast<unsigned char*>(addr);
  }
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) {
    (void)cudaGetLastError();
    cap = cudaStreamCaptureStatusActive;  // unknown: take the safe path
  }
  if (cap != cudaStreamCaptureStatusNone) slot.always_rebuild = true;
  const Ptrs p = ptrs(slot.base, L);
  if (slot.always_rebuild || slot.Nx != Nx || slot.Ny != Ny || slot.wall_mode != wall_mode) {
    const int n = Nx / 2 + 1;
    k_na_tables<<<(n + 127) / 128, 128, 0, s>>>(Nx, Ny, wall_mode, p);
    if ((e = cudaGetLastError()) != cudaSuccess) return na_fail(EHD_ECUDA, "ehd_poisson_noalloc: table kernel launch failed");
    slot.Nx = Nx;
    slot.Ny = Ny;
    slot.wall_mode = wall_mode;
  }
  const size_t row_smem = 2 * (size_t)Nx * sizeof(Cplx<float>);
  k_na_fwd<<<Ny, 256, row_smem, s>>>(Nx, Ny, 1.0 / eps, rhoc, p);
  int wpc = (int)((48u * 1024u) / ((size_t)Ny * sizeof(Cplx<float>)));
  wpc = wpc < 1 ? 1 : (wpc > 4 ? 4 : wpc);
  k_na_modes<<<(Nx / 2 + 1 + wpc - 1) / wpc, 32 * wpc, (size_t)wpc * Ny * sizeof(Cplx<float>), s>>>(
      Nx, Ny, wall_mode, phi0, wpc, p);
  k_na_inv<<<Ny, 256, row_smem, s>>>(Nx, Ny, phi, p);
  if ((e = cudaGetLastError()) != cudaSuccess) return na_fail(EHD_ECUDA, "ehd_poisson_noalloc: kernel launch failed");
  return EHD_OK;
}

// k_poisson.cu -- fast Poisson solver of Sec. IV.3 (arXiv:1812.05711) on the
// GB300: [Dx^2 + Dy^2] phi = s, s = -rho_c / eps (Eqs. 4, 18).  Spectral in x
// (Eqs. 19-20), second-order finite differences in y with Dirichlet walls,
// i.e. one constant-coefficient tridiagonal system per wavenumber (its
// eigenvalues are the -4 sin^2 symbols of Eq. 24, so this equals the
// odd-extension transform of Eqs. 21-25).
//
//   K1 k_rows_fwd  one CTA per row: rho_c = sum_i g_i (Eq. 6), the row mean in
//                  FP64 (the m = 0 mode), Stockham radix-2 FFT of the
//                  fluctuation in shared memory, half spectrum out.
//   K2 k_modes     one warp per wavenumber: Thomas recurrences with the
//                  precomputed reciprocal pivots, written as a warp-parallel
//                  scan of affine maps (32 lanes x Ny/32 rows each); the
//                  m = 0 mode carries the wall potential and runs in FP64.
//   K3 k_rows_inv  one CTA per row: inverse FFT -> phi minus its row mean.
#include "ehd_dev.cuh"

namespace ehd {

namespace {

template <class R>
__device__ __forceinline__ Cplx<R> cmul(Cplx<R> a, Cplx<R> b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}

// Stockham autosort radix-2 FFT of length N (power of two) in shared memory,
// ping-ponging between a and b.  tw[k] = exp(-2 pi i k / N), k < N/2.
// Returns the buffer holding the result.  All threads of the block call it.
template <class R>
__device__ Cplx<R>* fft_shared(Cplx<R>* a, Cplx<R>* b, int N, const Cplx<R>* __restrict__ tw, bool inverse) {
  const int half = N >> 1;
  for (int Ns = 1; Ns < N; Ns <<= 1) {
    const int tstride = N / (2 * Ns);
    for (int j = threadIdx.x; j < half; j += blockDim.x) {
      const int k = j & (Ns - 1);
      Cplx<R> w = tw[k * tstride];
      if (inverse) w.im = -w.im;
      const Cplx<R> u = a[j];
      const Cplx<R> v = cmul(a[j + half], w);
      const int idx = ((j - k) << 1) + k;
      b[idx] = {u.re + v.re, u.im + v.im};
      b[idx + Ns] = {u.re - v.re, u.im - v.im};
    }
    __syncthreads();
    Cplx<R>* t = a;
    a = b;
    b = t;
  }
  return a;
}

__device__ __forceinline__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0) {
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];  // fixed order
    red[0] = t;
  }
  __syncthreads();
  t = red[0];
  __syncthreads();
  return t;
}

}  // namespace

// --------------------------------------------------------------------- K1 ---
template <class S, class R>
__global__ void __launch_bounds__(256) k_rows_fwd(PoissonArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[8];
  Cplx<R>* A = reinterpret_cast<Cplx<R>*>(smem_raw);
  Cplx<R>* B = A + a.Nx;
  const int y = blockIdx.x;
  const int N = a.Nx;
  const S* __restrict__ g = static_cast<const S*>(a.gin);
  const R sg = a.rch ? (R)a.rch[y] : R(0);
  const R ieps = (R)a.inv_eps;
  double sum = 0.0;
  for (int x = threadIdx.x; x < N; x += blockDim.x) {
    const long long c = (long long)y * a.P + x;
    R rc = R(0);
#pragma unroll
    for (int i = 0; i < 9; ++i) rc += Store<S>::template ld<R>(g + i * a.plane + c);
    const R s = -(rc + sg) * ieps;  // Eq. 4 source
    A[x].re = s;
    sum += (double)s;
  }
  const double total = block_sum(sum, red);  // DFT coefficient m = 0 (Eq. 19)
  if (threadIdx.x == 0) a.spec0[y] = total;
  const R mean = (R)(total / (double)N);
  for (int x = threadIdx.x; x < N; x += blockDim.x) {
    A[x].re -= mean;
    A[x].im = R(0);
  }
  __syncthreads();
  const Cplx<R>* res = fft_shared<R>(A, B, N, static_cast<const Cplx<R>*>(a.tw), false);
  Cplx<R>* spec = static_cast<Cplx<R>*>(a.spec) + (long long)y * a.Mh;
  for (int m = threadIdx.x; m < a.Mh; m += blockDim.x) spec[m] = (m == 0) ? Cplx<R>{R(0), R(0)} : res[m];
}

// --------------------------------------------------------------------- K2 ---
namespace {

// Thomas for one system with unit off-diagonals, d'_j = r_j (d_j - d'_{j-1}),
// x_j = d'_j - r_j x_{j+1}, each recurrence evaluated as a warp scan of the
// affine maps of the lanes' contiguous chunks [j0, j1).
template <class R, class V>
struct Scan;

template <class R>
struct Scan<R, R> {
  __device__ static R shup(R v, int o) { return __shfl_up_sync(0xffffffffu, v, o); }
  __device__ static R shdn(R v, int o) { return __shfl_down_sync(0xffffffffu, v, o); }
  __device__ static R zero() { return R(0); }
  __device__ static R axpy(R a, R x, R b) { return a * x + b; }   // a x + b
  __device__ static R sub(R x, R y) { return x - y; }
  __device__ static R scl(R a, R x) { return a * x; }
};

template <class R>
struct Scan<R, Cplx<R>> {
  using V = Cplx<R>;
  __device__ static V shup(V v, int o) {
    return {__shfl_up_sync(0xffffffffu, v.re, o), __shfl_up_sync(0xffffffffu, v.im, o)};
  }
  __device__ static V shdn(V v, int o) {
    return {__shfl_down_sync(0xffffffffu, v.re, o), __shfl_down_sync(0xffffffffu, v.im, o)};
  }
  __device__ static V zero() { return {R(0), R(0)}; }
  __device__ static V axpy(R a, V x, V b) { return {a * x.re + b.re, a * x.im + b.im}; }
  __device__ static V sub(V x, V y) { return {x.re - y.re, x.im - y.im}; }
  __device__ static V scl(R a, V x) { return {a * x.re, a * x.im}; }
};

template <class R, class V>
__device__ void warp_thomas(V* d, const R* __restrict__ r, int Ny, int lane) {
  using Op = Scan<R, V>;
  const int C = (Ny + 31) >> 5;
  const int j0 = min(lane * C, Ny), j1 = min(j0 + C, Ny);
  // forward elimination: chunk map x -> al x + br
  R al = R(1);
  V br = Op::zero();
  for (int j = j0; j < j1; ++j) {
    const R rj = r[j];
    al = -rj * al;
    br = Op::scl(rj, Op::sub(d[j], br));
  }
  for (int o = 1; o < 32; o <<= 1) {
    const R a2 = __shfl_up_sync(0xffffffffu, al, o);
    const V b2 = Op::shup(br, o);
    if (lane >= o) {
      br = Op::axpy(al, b2, br);
      al = al * a2;
    }
  }
  V x = Op::shup(br, 1);
  if (lane == 0) x = Op::zero();
  for (int j = j0; j < j1; ++j) {
    x = Op::scl(r[j], Op::sub(d[j], x));
    d[j] = x;
  }
  __syncwarp();
  // back substitution, chunks composed from the top lane down
  al = R(1);
  br = Op::zero();
  for (int j = j1 - 1; j >= j0; --j) {
    const R rj = r[j];
    al = -rj * al;
    br = Op::axpy(-rj, br, d[j]);
  }
  for (int o = 1; o < 32; o <<= 1) {
    const R a2 = __shfl_down_sync(0xffffffffu, al, o);
    const V b2 = Op::shdn(br, o);
    if (lane + o < 32) {
      br = Op::axpy(al, b2, br);
      al = al * a2;
    }
  }
  x = Op::shdn(br, 1);
  if (lane == 31) x = Op::zero();
  for (int j = j1 - 1; j >= j0; --j) {
    x = Op::axpy(-r[j], x, d[j]);
    d[j] = x;
  }
  __syncwarp();
}

}  // namespace

template <class R>
__global__ void __launch_bounds__(128) k_modes(PoissonArgs a, int warps_per_cta) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m = blockIdx.x * warps_per_cta + warp;
  if (warp >= warps_per_cta || m >= a.Mh) return;  // warp-uniform exit
  const int Ny = a.Ny;
  if (m == 0) {
    // mean mode in FP64 with the wall potentials lifted into the right-hand
    // side: mirror ghost phi_{-1} = 2 phi_w - phi_0 (or phi_w on node walls)
    double* d = reinterpret_cast<double*>(smem_raw) + (size_t)warp * Ny * (sizeof(Cplx<R>) / sizeof(double));
    const double wc = (a.wall_mode == 0) ? 2.0 : 1.0;
    for (int j = lane; j < Ny; j += 32) {
      double v = a.spec0[j];
      if (j == 0) v -= wc * (double)a.Nx * a.phi0;
      d[j] = v;
    }
    __syncwarp();
    warp_thomas<double, double>(d, a.rfac0, Ny, lane);
    const double inN = 1.0 / (double)a.Nx;
    R* Ebar = static_cast<R*>(a.Ebar);
    for (int j = lane; j < Ny; j += 32) {
      const double pc = d[j] * inN;
      const double pd = (j > 0) ? d[j - 1] * inN : ((a.wall_mode == 0) ? 2.0 * a.phi0 - pc : a.phi0);
      const double pu = (j < Ny - 1) ? d[j + 1] * inN : ((a.wall_mode == 0) ? -pc : 0.0);
      a.phibar[j] = pc;
      Ebar[j] = (R)(-0.5 * (pu - pd));
    }
    return;
  }
  Cplx<R>* d = reinterpret_cast<Cplx<R>*>(smem_raw) + (size_t)warp * Ny;
  Cplx<R>* spec = static_cast<Cplx<R>*>(a.spec);
  const R* r = static_cast<const R*>(a.rfac) + (long long)m * Ny;
  for (int j = lane; j < Ny; j += 32) d[j] = spec[(long long)j * a.Mh + m];
  __syncwarp();
  warp_thomas<R, Cplx<R>>(d, r, Ny, lane);
  for (int j = lane; j < Ny; j += 32) spec[(long long)j * a.Mh + m] = d[j];
}

// --------------------------------------------------------------------- K3 ---
template <class R>
__global__ void __launch_bounds__(256) k_rows_inv(PoissonArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Cplx<R>* A = reinterpret_cast<Cplx<R>*>(smem_raw);
  Cplx<R>* B = A + a.Nx;
  const int y = blockIdx.x;
  const int N = a.Nx, half = N >> 1;
  const Cplx<R>* spec = static_cast<const Cplx<R>*>(a.spec) + (long long)y * a.Mh;
  for (int m = threadIdx.x; m < N; m += blockDim.x) {
    Cplx<R> v;
    if (m == 0) {
      v = {R(0), R(0)};  // the mean is carried by phibar
    } else if (m <= half) {
      v = spec[m];
    } else {
      const Cplx<R> s = spec[N - m];  // Hermitian symmetry of a real row
      v = {s.re, -s.im};
    }
    A[m] = v;
  }
  __syncthreads();
  const Cplx<R>* res = fft_shared<R>(A, B, N, static_cast<const Cplx<R>*>(a.tw), true);
  R* dphi = static_cast<R*>(a.dphi) + (long long)y * a.P;
  const R inN = R(1) / (R)N;
  for (int x = threadIdx.x; x < N; x += blockDim.x) dphi[x] = res[x].re * inN;
}

// ---------------------------------------------------------------- launch ---
namespace {

int modes_warps_per_cta(int Ny, size_t cplx_bytes) {
  const size_t per_warp = (size_t)Ny * cplx_bytes;
  int w = (int)((200u * 1024u) / per_warp);
  return w < 1 ? 1 : (w > 4 ? 4 : w);
}

template <class S, class R>
cudaError_t poisson_t(const PoissonArgs& a, cudaStream_t s) {
  const size_t row_smem = 2 * (size_t)a.Nx * sizeof(Cplx<R>);
  k_rows_fwd<S, R><<<a.Ny, 256, row_smem, s>>>(a);
  const int wpc = modes_warps_per_cta(a.Ny, sizeof(Cplx<R>));
  const size_t mode_smem = (size_t)wpc * a.Ny * sizeof(Cplx<R>);
  k_modes<R><<<(a.Mh + wpc - 1) / wpc, 32 * wpc, mode_smem, s>>>(a, wpc);
  k_rows_inv<R><<<a.Ny, 256, row_smem, s>>>(a);
  return cudaGetLastError();
}

template <class K>
cudaError_t allow_max_dynamic_smem(K kernel) {
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  cudaFuncAttributes fa;
  e = cudaFuncGetAttributes(&fa, kernel);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
}

template <class S, class R>
cudaError_t set_attrs_t() {
  cudaError_t e = allow_max_dynamic_smem(k_rows_fwd<S, R>);
  if (e != cudaSuccess) return e;
  e = allow_max_dynamic_smem(k_modes<R>);
  if (e != cudaSuccess) return e;
  return allow_max_dynamic_smem(k_rows_inv<R>);
}

}  // namespace

cudaError_t poisson_set_attributes() {
  cudaError_t e;
  if ((e = set_attrs_t<double, double>()) != cudaSuccess) return e;
  if ((e = set_attrs_t<double, float>()) != cudaSuccess) return e;
  if ((e = set_attrs_t<float, float>()) != cudaSuccess) return e;
  if ((e = set_attrs_t<__nv_bfloat16, float>()) != cudaSuccess) return e;
  return set_attrs_t<__half, float>();
}

cudaError_t launch_poisson(const PoissonArgs& a, int storage, bool real_f64, cudaStream_t s) {
  if (real_f64) {
    if (storage != 0) return cudaErrorInvalidValue;
    return poisson_t<double, double>(a, s);
  }
  switch (storage) {
    case 0: return poisson_t<double, float>(a, s);
    case 1: return poisson_t<float, float>(a, s);
    case 2: return poisson_t<__nv_bfloat16, float>(a, s);
    case 3: return poisson_t<__half, float>(a, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace ehd

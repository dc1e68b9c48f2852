// k_oddext.cu -- the y-direction solve of the Poisson equation in the literal
// form of Sec. IV.3 (Eqs. 21-25), as an alternative to the per-wavenumber
// tridiagonal of k_modes_tile: for each x-wavenumber m >= 1 the column
// s_m(y) of the half spectrum is extended oddly in y to NE points (Eqs. 21-22:
// NE = 2 Ny antisymmetric about the half node when the walls sit halfway
// between nodes, NE = 2 Ny + 2 with zeros on the wall nodes otherwise),
// transformed by a complex FFT of length NE, divided by the symbol of the
// discrete Laplacian -(kappa_m + 4 sin^2(pi k / NE)) (Eqs. 20, 24), transformed
// back, and its first Ny points kept (Eq. 25).  The mean mode m = 0, which
// also carries the wall potential and the flux totals, stays on k_mean_mode.
//
// One CTA per wavenumber.  The column lives in shared memory (two buffers of
// NE complex values) and is transformed by a Stockham autosort FFT: stage s of
// radix P reads x[j + r N/P], twiddles by exp(-2 pi i r (j mod Ns) / (Ns P)),
// applies a P-point DFT in registers and writes y[(j / Ns) Ns P + (j mod Ns)
// + r Ns], Ns being the product of the earlier radices.  Radices 4, 2, 3, 5,
// 7, 11, 13 cover every NE the run accepts; the twiddles come from a table of
// exp(-2 pi i t / NE) built on the host in double precision.
#include "ehd_dev.cuh"

namespace ehd {

namespace {

constexpr int kOddThreads = 256;

template <class R>
__device__ __forceinline__ Cplx<R> cmul(Cplx<R> a, Cplx<R> b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}

// table entry t of exp(-2 pi i t / N), conjugated for the inverse transform
template <class R, bool INV>
__device__ __forceinline__ Cplx<R> root(const Cplx<R>* __restrict__ tw, int t) {
  Cplx<R> w = tw[t];
  if (INV) w.im = -w.im;
  return w;
}

// P-point DFT of v in registers: o_q = sum_r v_r w^(r q), w = exp(-+2 pi i / P);
// wp[t] = w^t (loaded once per stage)
template <class R, int P, bool INV>
__device__ __forceinline__ void dft_p(const Cplx<R> (&v)[P], Cplx<R> (&o)[P], const Cplx<R> (&wp)[P]) {
  if constexpr (P == 2) {
    o[0] = {v[0].re + v[1].re, v[0].im + v[1].im};
    o[1] = {v[0].re - v[1].re, v[0].im - v[1].im};
  } else if constexpr (P == 4) {
    // w = -i forward, +i inverse
    const Cplx<R> a0 = {v[0].re + v[2].re, v[0].im + v[2].im}, a1 = {v[0].re - v[2].re, v[0].im - v[2].im};
    const Cplx<R> b0 = {v[1].re + v[3].re, v[1].im + v[3].im}, d = {v[1].re - v[3].re, v[1].im - v[3].im};
    const Cplx<R> b1 = INV ? Cplx<R>{-d.im, d.re} : Cplx<R>{d.im, -d.re};
    o[0] = {a0.re + b0.re, a0.im + b0.im};
    o[2] = {a0.re - b0.re, a0.im - b0.im};
    o[1] = {a1.re + b1.re, a1.im + b1.im};
    o[3] = {a1.re - b1.re, a1.im - b1.im};
  } else {
#pragma unroll
    for (int k = 0; k < P; ++k) {
      Cplx<R> s = v[0];
#pragma unroll
      for (int r = 1; r < P; ++r) {
        const Cplx<R> t = cmul(v[r], wp[(r * k) % P]);
        s.re += t.re;
        s.im += t.im;
      }
      o[k] = s;
    }
  }
}

// Twiddles of butterfly kk: w1 = exp(-+2 pi i kk / (Ns P)) from the table;
// in FP32 its powers w1^r by repeated products (one table load per butterfly
// instead of P - 1; the powers lose at most P - 2 roundings), in FP64 from
// the table (FP64 products cost more than the loads on this GPU).
template <class R, int P, bool INV>
__device__ void stage(const Cplx<R>* __restrict__ x, Cplx<R>* __restrict__ y, int N, int Ns,
                      const Cplx<R>* __restrict__ tw) {
  const int nb = N / P, tstep = N / (Ns * P);
  Cplx<R> wp[P];
#pragma unroll
  for (int t = 0; t < P; ++t) wp[t] = root<R, INV>(tw, t * (N / P));
  for (int j = threadIdx.x; j < nb; j += blockDim.x) {
    const int kk = j % Ns;
    Cplx<R> v[P], o[P];
    v[0] = x[j];
    if constexpr (sizeof(R) == 4) {
      const Cplx<R> w1 = root<R, INV>(tw, kk * tstep);
      Cplx<R> w = w1;
#pragma unroll
      for (int r = 1; r < P; ++r) {
        v[r] = cmul(x[j + r * nb], w);
        if (r + 1 < P) w = cmul(w, w1);
      }
    } else {
#pragma unroll
      for (int r = 1; r < P; ++r) v[r] = cmul(x[j + r * nb], root<R, INV>(tw, r * kk * tstep));
    }
    dft_p<R, P, INV>(v, o, wp);
    const int base = (j / Ns) * Ns * P + kk;
#pragma unroll
    for (int r = 0; r < P; ++r) y[base + r * Ns] = o[r];
  }
}

// MAXP: the largest radix compiled in (7 or 13); the 11- and 13-point
// DFTs double the kernel's registers, so lengths without those factors use
// the MAXP = 7 instance (64 registers: four CTAs per SM instead of two)
template <class R, bool INV, int MAXP>
__device__ void run_stage(int P, const Cplx<R>* x, Cplx<R>* y, int N, int Ns, const Cplx<R>* tw) {
  switch (P) {
    case 2: stage<R, 2, INV>(x, y, N, Ns, tw); break;
    case 3: stage<R, 3, INV>(x, y, N, Ns, tw); break;
    case 4: stage<R, 4, INV>(x, y, N, Ns, tw); break;
    case 5: stage<R, 5, INV>(x, y, N, Ns, tw); break;
    default:
      if constexpr (MAXP > 7) {
        if (P == 11) {
          stage<R, 11, INV>(x, y, N, Ns, tw);
          break;
        }
        if (P == 13) {
          stage<R, 13, INV>(x, y, N, Ns, tw);
          break;
        }
      }
      stage<R, 7, INV>(x, y, N, Ns, tw);
      break;
  }
}

// FFT of the NE points in buf[0] (buf[1] scratch); returns the buffer that
// holds the result
template <class R, bool INV, int MAXP>
__device__ Cplx<R>* fft_column(const PoissonArgs& a, Cplx<R>* b0, Cplx<R>* b1, const Cplx<R>* tw) {
  Cplx<R>* x = b0;
  Cplx<R>* y = b1;
  int Ns = 1;
  for (int s = 0; s < a.nfac; ++s) {
    run_stage<R, INV, MAXP>(a.fac[s], x, y, a.NE, Ns, tw);
    Ns *= a.fac[s];
    Cplx<R>* t = x;
    x = y;
    y = t;
    __syncthreads();
  }
  return x;
}

template <class R, int MAXP>
__global__ void __launch_bounds__(kOddThreads) k_modes_oddext(PoissonArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  grid_dep_wait();
  grid_dep_launch();
  const int m = 1 + blockIdx.x;  // uniform over the CTA
  if (m >= a.Mh) return;
  const int Ny = a.Ny, NE = a.NE, Mp = a.Mp;
  Cplx<R>* b0 = reinterpret_cast<Cplx<R>*>(smem_raw);
  Cplx<R>* b1 = b0 + NE;
  Cplx<R>* spec = static_cast<Cplx<R>*>(a.spec);
  const Cplx<R>* tw = static_cast<const Cplx<R>*>(a.twy);
  const int off = (a.wall_mode == 0) ? 0 : 1;  // extended index of row 0
  // odd extension (Eqs. 21-22): point off + j holds s_j, point NE - 1 - j
  // holds -s_j; with walls on nodes, points 0 and Ny + 1 are the zero walls
  if (off && threadIdx.x == 0) {
    b0[0] = {R(0), R(0)};
    b0[Ny + 1] = {R(0), R(0)};
  }
  for (int j = threadIdx.x; j < Ny; j += blockDim.x) {
    const Cplx<R> s = spec[(long long)j * Mp + m];
    b0[off + j] = s;
    b0[NE - 1 - j] = {-s.re, -s.im};
  }
  __syncthreads();
  Cplx<R>* X = fft_column<R, false, MAXP>(a, b0, b1, tw);
  // divide by the symbol (Eqs. 20, 24) and by NE for the inverse
  {
    const R kap = static_cast<const R*>(a.kap)[m];
    const R* __restrict__ sym = static_cast<const R*>(a.symy);
    for (int k = threadIdx.x; k < NE; k += blockDim.x) {
      const R q = R(-1) / ((R)NE * (kap + sym[k]));
      X[k] = {X[k].re * q, X[k].im * q};
    }
  }
  __syncthreads();
  Cplx<R>* Y = fft_column<R, true, MAXP>(a, X, X == b0 ? b1 : b0, tw);
  for (int j = threadIdx.x; j < Ny; j += blockDim.x) spec[(long long)j * Mp + m] = Y[off + j];
}

template <class R>
size_t oddext_smem(int NE) {
  return 2 * (size_t)NE * sizeof(Cplx<R>);
}

}  // namespace

int oddext_factors(int n, int* fac, int cap) {
  int nf = 0;
  static const int radix[] = {4, 2, 3, 5, 7, 11, 13};
  for (int p : radix)
    while (n > 1 && n % p == 0) {
      if (nf == cap) return -1;
      fac[nf++] = p;
      n /= p;
    }
  return n == 1 ? nf : -1;
}

size_t oddext_smem_bytes(int NE, bool real_f64) {
  return real_f64 ? oddext_smem<double>(NE) : oddext_smem<float>(NE);
}

cudaError_t launch_modes_oddext(const PoissonArgs& a, bool real_f64, cudaStream_t s) {
  if (a.Mh <= 1) return cudaSuccess;
  const dim3 grid(a.Mh - 1), block(kOddThreads);
  const bool pdl = (a.pdl & 2) != 0;
  bool small = true;  // every radix <= 7
  for (int k = 0; k < a.nfac; ++k) small = small && a.fac[k] <= 7;
  if (real_f64)
    return small ? launch_ex(pdl, k_modes_oddext<double, 7>, grid, block, oddext_smem<double>(a.NE), s, a)
                 : launch_ex(pdl, k_modes_oddext<double, 13>, grid, block, oddext_smem<double>(a.NE), s, a);
  return small ? launch_ex(pdl, k_modes_oddext<float, 7>, grid, block, oddext_smem<float>(a.NE), s, a)
               : launch_ex(pdl, k_modes_oddext<float, 13>, grid, block, oddext_smem<float>(a.NE), s, a);
}

cudaError_t oddext_set_attributes() {
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_modes_oddext<double, 7>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_modes_oddext<double, 13>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_modes_oddext<float, 7>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_modes_oddext<float, 13>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
}

}  // namespace ehd

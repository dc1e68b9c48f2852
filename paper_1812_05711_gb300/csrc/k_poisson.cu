// k_poisson.cu -- fast Poisson solver of Sec. IV.3 (arXiv:1812.05711) on the
// GB300: [Dx^2 + Dy^2] phi = s, s = -rho_c / eps (Eqs. 4, 18).  Spectral in x
// (Eqs. 19-20), second-order finite differences in y with Dirichlet walls:
// one constant-coefficient tridiagonal system per wavenumber (its eigenvalues
// are the -4 sin^2 symbols of Eq. 24, so this equals the odd-extension
// transform of Eqs. 21-25).
//
//   k_rhoc        rho_c = sum_i g_i (Eq. 6) from the populations, when the
//                 step kernel did not already write it.
//   k_rfft_rows   1024/L rows per CTA (L = Nx/2): the row's N real samples are
//                 packed as L complex values, transformed by a radix-4
//                 Stockham FFT in shared memory and untangled into the half
//                 spectrum (Eq. 19).  The row mean (the m = 0 mode) is summed
//                 in FP32 pairs with a compensated tree and removed first.
//   k_modes_tile  8 wavenumbers x Ny rows per CTA held in shared memory; the
//                 Thomas recurrences of each wavenumber (reciprocal pivots
//                 precomputed) run as 32 chunk-parallel affine scans.
//   k_mean_mode   128 threads: the m = 0 system in FP64 with the wall
//                 potentials lifted into the right-hand side; also adds the
//                 step's wall-flux partials to the run's FP64 totals.  It
//                 runs on a second stream, beside k_modes_tile/k_rfft_inv.
//   k_irfft_rows  inverse of k_rfft_rows -> phi minus its row mean.
#include <algorithm>

#include <cooperative_groups.h>

#include "ehd_dev.cuh"

namespace cg = cooperative_groups;

namespace ehd {

namespace {

template <class R>
__device__ __forceinline__ Cplx<R> cmul(Cplx<R> a, Cplx<R> b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <class R>
__device__ __forceinline__ Cplx<R> cadd(Cplx<R> a, Cplx<R> b) { return {a.re + b.re, a.im + b.im}; }
template <class R>
__device__ __forceinline__ Cplx<R> csub(Cplx<R> a, Cplx<R> b) { return {a.re - b.re, a.im - b.im}; }
template <class R>
__device__ __forceinline__ Cplx<R> cconj(Cplx<R> a) { return {a.re, -a.im}; }

// Radix-4 Stockham FFT of length L (power of two, L >= 2) for the rows of a
// CTA, T = max(L/4, 1) threads per row; a/b point at this row's two buffers
// (padded indexing).  tw[q] = exp(-2 pi i q / N) with N = 2L, in shared
// memory; W_L^q = tw[2q].  Every thread of the CTA must call it (it
// synchronises).  Returns the buffer with the result.
template <class R>
__device__ Cplx<R>* fft_rows(Cplx<R>* a, Cplx<R>* b, int L, int T, int tr, const Cplx<R>* tw, bool inverse);

// shared-memory index with one complex of padding every 16 (bank spread)
__device__ __forceinline__ int pidx(int c) { return c + (c >> 4); }

template <int BYTES>
__device__ __forceinline__ void cp_async_chunk(void* smem_dst, const void* gsrc) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  if constexpr (BYTES == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gsrc));
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(d), "l"(gsrc), "n"(BYTES));
}
__device__ __forceinline__ void cp_async_all() {
  asm volatile("cp.async.commit_group;\n" ::);
  asm volatile("cp.async.wait_group 0;\n" ::);
}

// error-free sum of two floats (Knuth): s + e == a + b exactly
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

template <class R>
__device__ Cplx<R>* fft_rows(Cplx<R>* a, Cplx<R>* b, int L, int T, int tr, const Cplx<R>* tw, bool inverse) {
  int Ns = 1;
  int log2L = 0;
  while ((1 << log2L) < L) ++log2L;
  if (log2L & 1) {  // one radix-2 stage
    const int half = L >> 1;
    for (int j = tr; j < half; j += T) {
      const int k = j & (Ns - 1);
      Cplx<R> w = tw[2 * k * (L / (2 * Ns))];
      if (inverse) w.im = -w.im;
      const Cplx<R> u = a[pidx(j)], v = cmul(a[pidx(j + half)], w);
      const int idx = ((j - k) << 1) + k;
      b[pidx(idx)] = cadd(u, v);
      b[pidx(idx + Ns)] = csub(u, v);
    }
    __syncthreads();
    Cplx<R>* t = a;
    a = b;
    b = t;
    Ns = 2;
  }
  const int q = L >> 2;
  while (Ns < L) {
    for (int j = tr; j < q; j += T) {
      const int k = j & (Ns - 1);
      const int st = 2 * (L / (4 * Ns)) * k;
      Cplx<R> w1 = tw[st], w2 = tw[2 * st], w3 = tw[3 * st];
      if (inverse) {
        w1.im = -w1.im;
        w2.im = -w2.im;
        w3.im = -w3.im;
      }
      const Cplx<R> v0 = a[pidx(j)], v1 = cmul(a[pidx(j + q)], w1), v2 = cmul(a[pidx(j + 2 * q)], w2),
                    v3 = cmul(a[pidx(j + 3 * q)], w3);
      const Cplx<R> t0 = cadd(v0, v2), t1 = csub(v0, v2), t2 = cadd(v1, v3);
      const Cplx<R> d = csub(v1, v3);
      const Cplx<R> t3 = inverse ? Cplx<R>{-d.im, d.re} : Cplx<R>{d.im, -d.re};  // (+-i)(v1 - v3)
      const int idx = (j - k) * 4 + k;
      b[pidx(idx)] = cadd(t0, t2);
      b[pidx(idx + Ns)] = cadd(t1, t3);
      b[pidx(idx + 2 * Ns)] = csub(t0, t2);
      b[pidx(idx + 3 * Ns)] = csub(t1, t3);
    }
    __syncthreads();
    Cplx<R>* t = a;
    a = b;
    b = t;
    Ns <<= 2;
  }
  return a;
}

// padded complex elements per row buffer
__host__ __device__ __forceinline__ int row_len_padded(int L) { return L + (L >> 4) + 1; }

}  // namespace

// ----------------------------------------------------------------- rho_c ---
template <class S, class R>
__global__ void k_rhoc(const S* __restrict__ g, long long plane, int Nx, int Ny, int P, const float* __restrict__ rch,
                       R* __restrict__ rhoc) {
  const long long n = (long long)Nx * Ny;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(k % Nx), y = (int)(k / Nx);
    const long long c = (long long)y * P + x;
    R v = rch ? (R)rch[y] : R(0);
    R s = R(0);
#pragma unroll
    for (int i = 0; i < 9; ++i) s += Store<S>::template ld<R>(g + i * plane + c);
    rhoc[c] = v + s;
  }
}

// ------------------------------------------------------------ forward FFT ---
// Shared memory: twiddle table (N complex), then per row two padded buffers.
template <class R>
__global__ void __launch_bounds__(256) k_rfft_rows(PoissonArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ float wred_hi[8], wred_lo[8];
  __shared__ double wred_d[8];
  const int N = a.Nx, L = N >> 1;
  const int T = (L >= 4) ? (L >> 2) : 1;  // threads per row
  const int rows = 256 / T;
  const int lr = threadIdx.x / T, tr = threadIdx.x % T;
  const int y = blockIdx.x * rows + lr;
  const bool live = (y < a.Ny);
  const int LP = row_len_padded(L);
  Cplx<R>* stw = reinterpret_cast<Cplx<R>*>(smem_raw);
  Cplx<R>* A = stw + N + (size_t)lr * LP;
  Cplx<R>* B = stw + N + (size_t)rows * LP + (size_t)lr * LP;
  const Cplx<R>* gtw = static_cast<const Cplx<R>*>(a.tw);
  for (int q = threadIdx.x; q < N; q += 256) stw[q] = gtw[q];
  const R* __restrict__ rc = static_cast<const R*>(a.rhoc) + (long long)(live ? y : 0) * a.P;
  const R *rdn, *rup;
  rhoc_partials<R>(a, live ? y : 0, rdn, rup);
  const R ieps = (R)a.inv_eps;
  // s = -rho_c / eps packed as complex pairs; per-thread partial sum
  R part = R(0);
  for (int n = tr; n < L; n += T) {
    R s0 = R(0), s1 = R(0);
    if (live) {
      R v0 = rc[2 * n], v1 = rc[2 * n + 1];
      if (rdn) {
        v0 += rdn[2 * n];
        v1 += rdn[2 * n + 1];
      }
      if (rup) {
        v0 += rup[2 * n];
        v1 += rup[2 * n + 1];
      }
      s0 = -v0 * ieps;
      s1 = -v1 * ieps;
    }
    A[pidx(n)] = {s0, s1};
    part += s0 + s1;
  }
  // row sum (the m = 0 DFT coefficient) over the row's T threads: shuffles
  // within segments of min(T, 32) lanes, then the row's warps
  const int W = T < 32 ? T : 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float shi = 0.0f, slo = 0.0f;  // FP32 path: float-float
  double sd = 0.0;               // FP64 path
  if constexpr (sizeof(R) == 8) {
    sd = (double)part;
    for (int o = W >> 1; o > 0; o >>= 1) sd += __shfl_down_sync(0xffffffffu, sd, o, W);
    if (T > 32) {
      if (lane == 0) wred_d[warp] = sd;
      __syncthreads();
      if (tr == 0)
        for (int w = 1; w < T / 32; ++w) sd += wred_d[warp + w];
    }
  } else {
    shi = (float)part;
    for (int o = W >> 1; o > 0; o >>= 1) {
      const float h2 = __shfl_down_sync(0xffffffffu, shi, o, W), l2 = __shfl_down_sync(0xffffffffu, slo, o, W);
      float s_, e_;
      two_sum(shi, h2, s_, e_);
      shi = s_;
      slo = slo + l2 + e_;
    }
    if (T > 32) {
      if (lane == 0) {
        wred_hi[warp] = shi;
        wred_lo[warp] = slo;
      }
      __syncthreads();
      if (tr == 0)
        for (int w = 1; w < T / 32; ++w) {
          float s_, e_;
          two_sum(shi, wred_hi[warp + w], s_, e_);
          shi = s_;
          slo = slo + wred_lo[warp + w] + e_;
        }
    }
  }
  __shared__ R rmean[256 / 2];  // rows per CTA <= 128
  if (tr == 0) {
    if constexpr (sizeof(R) == 8) {
      if (live) static_cast<double*>(a.spec0)[y] = sd;
      rmean[lr] = (R)(sd / (double)N);
    } else {
      float h, l;  // renormalise
      two_sum(shi, slo, h, l);
      if (live) static_cast<float2*>(a.spec0)[y] = make_float2(h, l);
      rmean[lr] = h / (float)N;
    }
  }
  __syncthreads();
  const R mean = rmean[lr];
  for (int n = tr; n < L; n += T) {
    A[pidx(n)].re -= mean;
    A[pidx(n)].im -= mean;
  }
  __syncthreads();
  const Cplx<R>* Z = fft_rows<R>(A, B, L, T, tr, stw, false);
  // untangle: S[k] = (Z[k] + Z*[L-k]) / 2 - i W^k (Z[k] - Z*[L-k]) / 2
  if (live) {
    Cplx<R>* spec = static_cast<Cplx<R>*>(a.spec) + (long long)y * a.Mp;
    for (int k = tr; k <= L; k += T) {
      if (k == 0) {
        spec[0] = {R(0), R(0)};
        continue;
      }
      const Cplx<R> zk = Z[pidx(k == L ? 0 : k)], zc = cconj(Z[pidx(L - k)]);
      const Cplx<R> E = {R(0.5) * (zk.re + zc.re), R(0.5) * (zk.im + zc.im)};
      const Cplx<R> Dm = {R(0.5) * (zk.re - zc.re), R(0.5) * (zk.im - zc.im)};
      const Cplx<R> O = {Dm.im, -Dm.re};  // D / i
      spec[k] = cadd(E, cmul(stw[k], O));
    }
  }
}

// ------------------------------------------------------------ inverse FFT ---
// DX: the transform of E_x = -d phi / dx instead, coefficient k read as
// -i k_k phi_k (k_k = 2 pi k / N, the Nyquist coefficient dropped), into a.ex
template <class R, bool DX>
__device__ __forceinline__ Cplx<R> spec_coef(const Cplx<R>* spec, int k, int L) {
  const Cplx<R> v = spec[k];
  if constexpr (!DX) {
    return v;
  } else {
    if (k == L) return {R(0), R(0)};
    const R kk = (R(3.141592653589793238462643383279502884) / (R)L) * (R)k;
    return {kk * v.im, -kk * v.re};
  }
}

template <class R, bool DX = false>
__global__ void __launch_bounds__(256) k_irfft_rows(PoissonArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int N = a.Nx, L = N >> 1;
  const int T = (L >= 4) ? (L >> 2) : 1;
  const int rows = 256 / T;
  const int lr = threadIdx.x / T, tr = threadIdx.x % T;
  const int y = blockIdx.x * rows + lr;
  const bool live = (y < a.Ny);
  const int LP = row_len_padded(L);
  Cplx<R>* stw = reinterpret_cast<Cplx<R>*>(smem_raw);
  Cplx<R>* A = stw + N + (size_t)lr * LP;
  Cplx<R>* B = stw + N + (size_t)rows * LP + (size_t)lr * LP;
  const Cplx<R>* gtw = static_cast<const Cplx<R>*>(a.tw);
  for (int q = threadIdx.x; q < N; q += 256) stw[q] = gtw[q];
  __syncthreads();
  const Cplx<R>* spec = static_cast<const Cplx<R>*>(a.spec) + (long long)(live ? y : 0) * a.Mp;
  // Z[k] = E[k] + i O[k], E = (S[k] + S*[L-k]) / 2, O = (S[k] - S*[L-k]) / (2 W^k);
  // the mean S[0] is excluded (it lives in phibar)
  for (int k = tr; k < L; k += T) {
    Cplx<R> z = {R(0), R(0)};
    if (live) {
      const Cplx<R> sk = (k == 0) ? Cplx<R>{R(0), R(0)} : spec_coef<R, DX>(spec, k, L);
      const Cplx<R> sc = cconj(spec_coef<R, DX>(spec, L - k, L));
      const Cplx<R> E = {R(0.5) * (sk.re + sc.re), R(0.5) * (sk.im + sc.im)};
      const Cplx<R> D = {R(0.5) * (sk.re - sc.re), R(0.5) * (sk.im - sc.im)};
      const Cplx<R> O = cmul(D, cconj(stw[k]));  // D / W^k
      z = {E.re - O.im, E.im + O.re};            // E + i O
    }
    A[pidx(k)] = z;
  }
  __syncthreads();
  const Cplx<R>* zr = fft_rows<R>(A, B, L, T, tr, stw, true);
  if (live) {
    R* dphi = static_cast<R*>(DX ? a.ex : a.dphi) + (long long)y * a.P;
    const R inL = R(1) / (R)L;
    for (int n = tr; n < L; n += T) {
      const Cplx<R> v = zr[pidx(n)];
      if constexpr (sizeof(R) == 4)
        reinterpret_cast<float2*>(dphi)[n] = make_float2(v.re * inL, v.im * inL);
      else
        reinterpret_cast<double2*>(dphi)[n] = make_double2(v.re * inL, v.im * inL);
    }
  }
}

// ---------------------------------------------------------- mode systems ---
// Thomas with unit off-diagonals and reciprocal pivots r_j:
//   forward  d'_j = r_j (d_j - d'_{j-1})      (affine in d'_{j-1})
//   backward x_j  = d'_j - r_j x_{j+1}         (affine in x_{j+1})
// A CTA holds MB wavenumbers x Ny rows in shared memory; thread (chunk, mode)
// composes the affine maps of its chunk of rows, the chunk maps are combined
// in order, then each chunk is evaluated from its carried-in value.
template <class R, int MB, int NT>
struct TileScratch {
  R al[NT / MB][MB];
  Cplx<R> br[NT / MB][MB];
  Cplx<R> carry[NT / MB][MB];
  R wa[MB][NT / 32 / MB];  // per-warp composed maps, chained across the warps of one mode
  Cplx<R> wb[MB][NT / 32 / MB];
};

// Exclusive scan of the chunk maps x -> al x + br over the NT / MB chunks of
// each of the MB wavenumbers: carry[c][m] = the value entering chunk c, in
// chunk order 0, 1, ... (forward sweep) or from the last chunk down
// (backward sweep).  One warp composes 32 consecutive maps of one wavenumber
// with a shuffle scan; the NT / 32 / MB warps of a wavenumber are chained
// through shared memory.  Called by all NT threads.
template <class R, int MB, int NT, bool BACK>
__device__ __forceinline__ void chunk_carries(TileScratch<R, MB, NT>& ts) {
  constexpr int CH = NT / MB, WPM = CH / 32;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int mo = w / WPM, seg = w % WPM;
  const int q = seg * 32 + lane;
  const int c = BACK ? CH - 1 - q : q;
  R al = ts.al[c][mo];
  Cplx<R> br = ts.br[c][mo];
  for (int o = 1; o < 32; o <<= 1) {
    const R a2 = __shfl_up_sync(0xffffffffu, al, o);
    const R b2r = __shfl_up_sync(0xffffffffu, br.re, o), b2i = __shfl_up_sync(0xffffffffu, br.im, o);
    if (lane >= o) {  // the earlier maps first: x -> al (a2 x + b2) + br
      br = {al * b2r + br.re, al * b2i + br.im};
      al = al * a2;
    }
  }
  R ea = __shfl_up_sync(0xffffffffu, al, 1);
  Cplx<R> eb = {__shfl_up_sync(0xffffffffu, br.re, 1), __shfl_up_sync(0xffffffffu, br.im, 1)};
  if (lane == 0) {
    ea = R(1);
    eb = {R(0), R(0)};
  }
  Cplx<R> vin = {R(0), R(0)};
  if constexpr (WPM > 1) {
    if (lane == 31) {
      ts.wa[mo][seg] = al;
      ts.wb[mo][seg] = br;
    }
    __syncthreads();
    for (int k = 0; k < seg; ++k) {
      const R ak = ts.wa[mo][k];
      const Cplx<R> bk = ts.wb[mo][k];
      vin = {ak * vin.re + bk.re, ak * vin.im + bk.im};
    }
  }
  ts.carry[c][mo] = {ea * vin.re + eb.re, ea * vin.im + eb.im};
}

// One CTA solves wavenumbers m0 .. m0 + MB - 1 of run a (smem_raw: tile
// storage, ts: chunk-map scratch).  The m = 0 column of tile 0 holds zeros
// and is never stored.
template <class R, int MB, int NT>
__device__ __forceinline__ void modes_tile_sweeps(const PoissonArgs& a, int m0, Cplx<R>* d, const R* rt,
                                                  TileScratch<R, MB, NT>& ts);

// PDL: the kernel was launched with programmatic dependent launch; the
// constant pivots are staged before the wait for the forward transform, the
// spectrum after it.
template <class R, int MB, int NT, bool PDL = false>
__device__ __forceinline__ void modes_tile_body(const PoissonArgs& a, int m0, unsigned char* smem_raw,
                                                TileScratch<R, MB, NT>& ts) {
  const int Ny = a.Ny, Mp = a.Mp;
  Cplx<R>* d = reinterpret_cast<Cplx<R>*>(smem_raw);                          // [Ny][MB]
  R* rt = reinterpret_cast<R*>(smem_raw + (size_t)Ny * MB * sizeof(Cplx<R>));  // [Ny][MB]
  Cplx<R>* spec = static_cast<Cplx<R>*>(a.spec);
  const R* __restrict__ rf = static_cast<const R*>(a.rfac);  // [Ny][Mp]
  {
    // stage both tiles with cp.async chunks (rows are Mp-pitched, 16-B aligned)
    constexpr int CB = (MB * (int)sizeof(Cplx<R>) < 16) ? MB * (int)sizeof(Cplx<R>) : 16;
    constexpr int RB = (MB * (int)sizeof(R) < 16) ? MB * (int)sizeof(R) : 16;
    constexpr int CPR = MB * (int)sizeof(Cplx<R>) / CB;  // chunks per row, spectrum
    constexpr int RPR = MB * (int)sizeof(R) / RB;        // chunks per row, pivots
    constexpr int CE = CB / (int)sizeof(Cplx<R>) > 0 ? CB / (int)sizeof(Cplx<R>) : 1;
    constexpr int RE = RB / (int)sizeof(R);
    for (int idx = threadIdx.x; idx < Ny * RPR; idx += NT) {
      const int j = idx / RPR, c = idx % RPR;
      const int m = m0 + c * RE;
      if (m < Mp) cp_async_chunk<RB>(rt + j * MB + c * RE, rf + (long long)j * Mp + m);
    }
    if constexpr (PDL) {
      grid_dep_wait();
      grid_dep_launch();
    }
    for (int idx = threadIdx.x; idx < Ny * CPR; idx += NT) {
      const int j = idx / CPR, c = idx % CPR;
      const int m = m0 + c * CE;
      if (m < Mp) cp_async_chunk<CB>(d + j * MB + c * CE, spec + (long long)j * Mp + m);
    }
    cp_async_all();
  }
  __syncthreads();
  modes_tile_sweeps<R, MB, NT>(a, m0, d, rt, ts);
}

// The three sweeps of a staged tile (d: spectrum [Ny][MB], rt: reciprocal
// pivots [Ny][MB]) and the store of its wavenumbers 1 <= m < Mh.
template <class R, int MB, int NT>
__device__ __forceinline__ void modes_tile_sweeps(const PoissonArgs& a, int m0, Cplx<R>* d, const R* rt,
                                                  TileScratch<R, MB, NT>& ts) {
  constexpr int CH = NT / MB;
  auto& s_al = ts.al;
  auto& s_br = ts.br;
  auto& s_carry = ts.carry;
  const int Ny = a.Ny, Mh = a.Mh, Mp = a.Mp;
  Cplx<R>* spec = static_cast<Cplx<R>*>(a.spec);
  const int mo = threadIdx.x % MB, ch = threadIdx.x / MB;
  const int C = (Ny + CH - 1) / CH;
  const int j0 = min(ch * C, Ny), j1 = min(j0 + C, Ny);
  // forward: compose chunk map
  R al = R(1);
  Cplx<R> br = {R(0), R(0)};
  for (int j = j0; j < j1; ++j) {
    const R r = rt[j * MB + mo];
    const Cplx<R> dj = d[j * MB + mo];
    al = -r * al;
    br = {r * (dj.re - br.re), r * (dj.im - br.im)};
  }
  s_al[ch][mo] = al;
  s_br[ch][mo] = br;
  __syncthreads();
  chunk_carries<R, MB, NT, false>(ts);  // value entering each chunk
  __syncthreads();
  // forward evaluation; compose the backward chunk map on the way
  Cplx<R> x = s_carry[ch][mo];
  R ab = R(1);
  Cplx<R> bb = {R(0), R(0)};
  for (int j = j0; j < j1; ++j) {
    const R r = rt[j * MB + mo];
    const Cplx<R> dj = d[j * MB + mo];
    x = {r * (dj.re - x.re), r * (dj.im - x.im)};
    d[j * MB + mo] = x;
    bb = {bb.re + ab * x.re, bb.im + ab * x.im};
    ab = -ab * r;
  }
  __syncthreads();
  s_al[ch][mo] = ab;
  s_br[ch][mo] = bb;
  __syncthreads();
  chunk_carries<R, MB, NT, true>(ts);  // value just above each chunk, from the top down
  __syncthreads();
  // backward evaluation, each solved value stored as it is formed (a warp's
  // store covers 8 wavenumbers of 4 rows, 64 contiguous bytes each); the
  // stores issue while the sweep's dependent chain waits
  x = s_carry[ch][mo];
  const int m = m0 + mo;
  const bool put = m >= 1 && m < Mh;
  Cplx<R>* col = spec + m;
  for (int j = j1 - 1; j >= j0; --j) {
    const R r = rt[j * MB + mo];
    const Cplx<R> dj = d[j * MB + mo];
    x = {dj.re - r * x.re, dj.im - r * x.im};
    if (put) col[(long long)j * Mp] = x;
  }
}

// threads per CTA of the wavenumber solves: NT / MB chunks per wavenumber
constexpr int kTileThreads = 256;

// The same solve with the tile staged by tensor copies (FP32, 8 wavenumbers):
// one thread issues a box of 256 rows x 8 pivots and of 256 rows x 8
// complex values per copy (the last box holds the remaining rows) into the
// layout the sweeps read, completing on two mbarriers, instead of the CTA
// issuing 16-byte chunks with their address arithmetic.  The pivots (constant
// per run) are requested before the wait for the forward transform.  Waits
// are bounded: one that gives up sets bit 2 of the run's error word, waits
// (bounded again) for the copies in flight and leaves the tile unsolved.
// Measured slower than the CTA's own 16-byte chunks (2048 x 1680: 118.4
// against 117.2-117.9 us per step: a box of 256 rows of 64 or 32 bytes is
// fetched row by row by the SM's one copy engine), so it is an option
// (EHD_TUNE_TILE_TMA).
namespace mt {
constexpr unsigned kWaitLimit = 1u << 22;
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned mbar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(mbar) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned mbar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(mbar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_wait(unsigned mbar, unsigned parity) {
  for (unsigned it = 0; it < kWaitLimit; ++it) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}
__device__ __forceinline__ void load2d(unsigned dst, const CUtensorMap* map, int x, int y, unsigned mbar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n" ::"r"(dst),
      "l"(map), "r"(x), "r"(y), "r"(mbar)
      : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory"); }
}  // namespace mt

// shared memory of the tensor-copy tile: spectrum [Ny][8] complex, pivots [Ny][8]
__host__ __device__ constexpr size_t modes_tma_pivot_offset(int Ny) { return ((size_t)Ny * 64 + 127) / 128 * 128; }

__global__ void __launch_bounds__(kTileThreads) k_modes_tile_tma(PoissonArgs a, const __grid_constant__ ModesTma tm) {
  constexpr int MB = 8, NT = kTileThreads;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ TileScratch<float, MB, NT> ts;
  __shared__ __align__(8) unsigned long long mbar[2];
  const int Ny = a.Ny, m0 = blockIdx.x * MB;
  // tensor-copy destinations 128-byte aligned (the launch adds 128 bytes)
  unsigned char* base = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 127) & ~(uintptr_t)127);
  Cplx<float>* d = reinterpret_cast<Cplx<float>*>(base);
  float* rt = reinterpret_cast<float*>(base + modes_tma_pivot_offset(Ny));
  const unsigned mb_rf = mt::smem_u32(&mbar[0]), mb_sp = mt::smem_u32(&mbar[1]);
  if (threadIdx.x == 0) {
    mt::mbar_init(mb_rf);
    mt::mbar_init(mb_sp);
    mt::fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    mt::mbar_expect_tx(mb_rf, (unsigned)Ny * 32u);
    for (int k = 0; k < tm.nfull; ++k)
      mt::load2d(mt::smem_u32(rt + (size_t)k * 256 * MB), &tm.rf_full, m0, 256 * k, mb_rf);
    if (tm.tail) mt::load2d(mt::smem_u32(rt + (size_t)tm.nfull * 256 * MB), &tm.rf_tail, m0, 256 * tm.nfull, mb_rf);
  }
  grid_dep_wait();  // the forward transform has written the spectrum
  grid_dep_launch();
  if (threadIdx.x == 0) {
    mt::mbar_expect_tx(mb_sp, (unsigned)Ny * 64u);
    for (int k = 0; k < tm.nfull; ++k)
      mt::load2d(mt::smem_u32(d + (size_t)k * 256 * MB), &tm.spec_full, 2 * m0, 256 * k, mb_sp);
    if (tm.tail) mt::load2d(mt::smem_u32(d + (size_t)tm.nfull * 256 * MB), &tm.spec_tail, 2 * m0, 256 * tm.nfull, mb_sp);
  }
  bool ok = mt::mbar_wait(mb_rf, 0u);
  ok = mt::mbar_wait(mb_sp, 0u) && ok;
  if (__syncthreads_or(!ok)) {
    if (threadIdx.x == 0) {
      atomicOr(a.err, 2);
      mt::mbar_wait(mb_rf, 0u);  // the copies in flight land before the CTA leaves
      mt::mbar_wait(mb_sp, 0u);
    }
    __syncthreads();
    return;
  }
  modes_tile_sweeps<float, MB, NT>(a, m0, d, rt, ts);
}

cudaError_t modes_tma_encode(ModesTma* t, const void* spec, const void* rfac, int Ny, int Mp) {
  *t = ModesTma{};
  t->nfull = Ny / 256;
  t->tail = Ny % 256;
  cudaError_t e = cudaSuccess;
  if (t->nfull > 0) {
    if ((e = tma_encode_2d(&t->spec_full, spec, 2ull * Mp, Ny, 8ull * Mp, 16, 256)) != cudaSuccess) return e;
    if ((e = tma_encode_2d(&t->rf_full, rfac, (unsigned long long)Mp, Ny, 4ull * Mp, 8, 256)) != cudaSuccess) return e;
  }
  if (t->tail > 0) {
    if ((e = tma_encode_2d(&t->spec_tail, spec, 2ull * Mp, Ny, 8ull * Mp, 16, (unsigned)t->tail)) != cudaSuccess)
      return e;
    if ((e = tma_encode_2d(&t->rf_tail, rfac, (unsigned long long)Mp, Ny, 4ull * Mp, 8, (unsigned)t->tail)) !=
        cudaSuccess)
      return e;
  }
  return cudaSuccess;
}

// The same solve by a cluster of two CTAs (on two SMs, or two slots of one):
// CTA rank c stages and sweeps only the rows of chunks [16 c, 16 c + 16) --
// half of the tile's shared memory and staging traffic per CTA, and twice
// as many CTAs in flight.  The chunk maps of both halves are written into
// both CTAs' scratch through distributed shared memory, so that each CTA
// runs the single-CTA scan over all 32 chunk maps: chunk boundaries, the
// per-chunk arithmetic and the scan order are those of modes_tile_body, and
// the results are bit for bit the same (a batch, whose CTAs solve whole
// tiles, gives a run the bits it gets alone).  Cluster barriers: after each
// exchange of maps, and before the backward maps overwrite the peer's
// forward ones.  Measured slower than one CTA per tile (2048 x 1680: 121.5
// against 118.9-120.2 us per step; the three cluster barriers cost more than
// the halved staging saves), so it is an option (EHD_TUNE_TILE_CLUSTER).
template <int MB>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kTileThreads) k_modes_tile2(PoissonArgs a) {
  constexpr int NT = kTileThreads, CH = NT / MB, HALF = CH / 2;
  static_assert(CH == 32, "one warp of chunk maps per wavenumber");
  using R = float;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ TileScratch<R, MB, NT> ts;
  grid_dep_wait();
  grid_dep_launch();
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  TileScratch<R, MB, NT>* peer = cl.map_shared_rank(&ts, rank ^ 1);
  const int m0 = (blockIdx.x >> 1) * MB;
  const int Ny = a.Ny, Mh = a.Mh, Mp = a.Mp;
  const int C = (Ny + CH - 1) / CH;
  const int R0 = min(HALF * rank * C, Ny), R1 = min(HALF * (rank + 1) * C, Ny);
  const int rows = R1 - R0;
  Cplx<R>* d = reinterpret_cast<Cplx<R>*>(smem_raw);                              // [rows][MB]
  R* rt = reinterpret_cast<R*>(smem_raw + (size_t)HALF * C * MB * sizeof(Cplx<R>));  // [rows][MB]
  Cplx<R>* spec = static_cast<Cplx<R>*>(a.spec);
  const R* __restrict__ rf = static_cast<const R*>(a.rfac);
  {
    constexpr int CB = 16, RB = 16;
    constexpr int CPR = MB * (int)sizeof(Cplx<R>) / CB, RPR = MB * (int)sizeof(R) / RB;
    constexpr int CE = CB / (int)sizeof(Cplx<R>), RE = RB / (int)sizeof(R);
    for (int idx = threadIdx.x; idx < rows * CPR; idx += NT) {
      const int j = idx / CPR, c = idx % CPR;
      const int m = m0 + c * CE;
      if (m < Mp) cp_async_chunk<CB>(d + j * MB + c * CE, spec + (long long)(R0 + j) * Mp + m);
    }
    for (int idx = threadIdx.x; idx < rows * RPR; idx += NT) {
      const int j = idx / RPR, c = idx % RPR;
      const int m = m0 + c * RE;
      if (m < Mp) cp_async_chunk<RB>(rt + j * MB + c * RE, rf + (long long)(R0 + j) * Mp + m);
    }
    cp_async_all();
  }
  __syncthreads();
  const int mo = threadIdx.x % MB, ch = threadIdx.x / MB;
  const bool own = (ch / HALF) == rank;
  const int j0 = min(ch * C, Ny), j1 = min(j0 + C, Ny);
  if (own) {
    R al = R(1);
    Cplx<R> br = {R(0), R(0)};
    for (int j = j0; j < j1; ++j) {
      const R r = rt[(j - R0) * MB + mo];
      const Cplx<R> dj = d[(j - R0) * MB + mo];
      al = -r * al;
      br = {r * (dj.re - br.re), r * (dj.im - br.im)};
    }
    ts.al[ch][mo] = al;
    ts.br[ch][mo] = br;
    peer->al[ch][mo] = al;
    peer->br[ch][mo] = br;
  }
  cl.sync();
  chunk_carries<R, MB, NT, false>(ts);
  __syncthreads();
  R ab = R(1);
  Cplx<R> bb = {R(0), R(0)};
  if (own) {
    Cplx<R> x = ts.carry[ch][mo];
    for (int j = j0; j < j1; ++j) {
      const R r = rt[(j - R0) * MB + mo];
      const Cplx<R> dj = d[(j - R0) * MB + mo];
      x = {r * (dj.re - x.re), r * (dj.im - x.im)};
      d[(j - R0) * MB + mo] = x;
      bb = {bb.re + ab * x.re, bb.im + ab * x.im};
      ab = -ab * r;
    }
  }
  cl.sync();  // both CTAs have scanned the forward maps
  if (own) {
    ts.al[ch][mo] = ab;
    ts.br[ch][mo] = bb;
    peer->al[ch][mo] = ab;
    peer->br[ch][mo] = bb;
  }
  cl.sync();
  chunk_carries<R, MB, NT, true>(ts);
  __syncthreads();
  if (own) {
    Cplx<R> x = ts.carry[ch][mo];
    for (int j = j1 - 1; j >= j0; --j) {
      const R r = rt[(j - R0) * MB + mo];
      const Cplx<R> dj = d[(j - R0) * MB + mo];
      x = {dj.re - r * x.re, dj.im - r * x.im};
      d[(j - R0) * MB + mo] = x;
    }
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < rows * MB; idx += NT) {
    const int j = idx / MB, mo2 = idx % MB;
    const int m = m0 + mo2;
    if (m >= 1 && m < Mh) spec[(long long)(R0 + j) * Mp + m] = d[idx];
  }
}

template <class R, int MB, int NT = kTileThreads>
__global__ void __launch_bounds__(NT) k_modes_tile(PoissonArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ TileScratch<R, MB, NT> ts;
  modes_tile_body<R, MB, NT, true>(a, blockIdx.x * MB, smem_raw, ts);
}

// Float-float ("double-single") numbers for the FP32 path: value = hi + lo
// with |lo| <= ulp(hi)/2, about 48 significant bits, on the FP32 pipes (scalar
// FP64 is slow on this part).  Error-free transformations: Knuth's two-sum
// and the FMA two-product.
struct ff {
  float hi, lo;
};
__device__ __forceinline__ ff ff_from(double v) {
  const float h = (float)v;
  return {h, (float)(v - (double)h)};
}
__device__ __forceinline__ double ff_to(ff a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ ff ff_add(ff a, ff b) {
  const float s = a.hi + b.hi;
  const float bb = s - a.hi;
  const float e = (a.hi - (s - bb)) + (b.hi - bb) + a.lo + b.lo;
  const float h = s + e;
  return {h, e - (h - s)};
}
__device__ __forceinline__ ff ff_neg(ff a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ ff ff_mul(ff a, ff b) {
  const float p = a.hi * b.hi;
  const float e = fmaf(a.hi, b.hi, -p) + (a.hi * b.lo + a.lo * b.hi);
  const float h = p + e;
  return {h, e - (h - p)};
}
__device__ __forceinline__ ff ff_shfl_up(ff a, int o) {
  return {__shfl_up_sync(0xffffffffu, a.hi, o), __shfl_up_sync(0xffffffffu, a.lo, o)};
}
__device__ __forceinline__ ff ff_shfl_down(ff a, int o) {
  return {__shfl_down_sync(0xffffffffu, a.hi, o), __shfl_down_sync(0xffffffffu, a.lo, o)};
}

// Mean-mode arithmetic: native double, or float-float.
template <class R>
struct MeanNum;
template <>
struct MeanNum<double> {
  using T = double;
  __device__ static T from(double v) { return v; }
  __device__ static T from_f(float v) { return (double)v; }
  __device__ static T from_i(int v) { return (double)v; }
  __device__ static T pair(double d, float, float) { return d; }
  __device__ static double to(T v) { return v; }
  __device__ static T add(T a, T b) { return a + b; }
  __device__ static T mul(T a, T b) { return a * b; }
  __device__ static T neg(T a) { return -a; }
  __device__ static T up(T a, int o) { return __shfl_up_sync(0xffffffffu, a, o); }
  __device__ static T down(T a, int o) { return __shfl_down_sync(0xffffffffu, a, o); }
};
template <>
struct MeanNum<float> {
  using T = ff;
  __device__ static T from(double v) { return ff_from(v); }
  __device__ static T from_f(float v) { return {v, 0.0f}; }
  // exact for |v| <= 2^24, and then equal to ff_from((double)v)
  __device__ static T from_i(int v) { return {(float)v, 0.0f}; }
  // a constant the host split into (hi, lo): equal to ff_from(d)
  __device__ static T pair(double, float hi, float lo) { return {hi, lo}; }
  __device__ static double to(T v) { return ff_to(v); }
  __device__ static T add(T a, T b) { return ff_add(a, b); }
  __device__ static T mul(T a, T b) { return ff_mul(a, b); }
  __device__ static T neg(T a) { return ff_neg(a); }
  __device__ static T up(T a, int o) { return ff_shfl_up(a, o); }
  __device__ static T down(T a, int o) { return ff_shfl_down(a, o); }
};

// m = 0 (the row means) + the step's wall fluxes.  For m = 0 the system of
// Eq. 25 is the 1-D discrete Poisson equation phi_{j-1} - 2 phi_j + phi_{j+1}
// = s_j with the wall ghosts of the closure, whose solution is a double
// prefix sum: with D_j = phi_{j+1} - phi_j (j = -1 .. Ny-1),
//   D_j = D_{-1} + S_j,  S_j = sum_{k<=j} s_k,
//   phi_j = phi_{-1} + (j+1) D_{-1} + T_j,  T_j = sum_{k<j} S_k,
// and the two wall conditions fix phi_{-1} and D_{-1}.  Both sums are block
// scans (per-thread chunks, warp shuffles, one warp over the warp totals).
// Arithmetic: FP64 on the plain FP64 path, float-float on the FP32 path.
// Barrier among the first NT threads of the CTA (all of it when the CTA has
// NT threads): the mean mode may run on a sub-block of a larger CTA.
template <int NT>
__device__ __forceinline__ void sub_sync() {
  asm volatile("bar.sync 1, %0;\n" ::"n"(NT) : "memory");
}

template <class R, int NT>
struct MeanScratch {
  static constexpr int NW = NT / 32;
  typename MeanNum<R>::T wsum[NW], woff[NW], tot[2];
  double fq[2][NW];
};

// Inclusive prefix sum of v[0..Ny) in place (all NT threads; chunk [j0, j1)
// per thread); returns the total.
template <class R, int NT>
__device__ __forceinline__ typename MeanNum<R>::T block_prefix_sum(typename MeanNum<R>::T* v, int j0, int j1,
                                                                   MeanScratch<R, NT>& ms) {
  using N = MeanNum<R>;
  using T = typename N::T;
  constexpr int NW = NT / 32;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  T acc = N::from_f(0.0f);
  for (int j = j0; j < j1; ++j) {
    acc = N::add(acc, v[j]);
    v[j] = acc;
  }
  T incl = acc;  // inclusive scan of the chunk totals over the warp
  for (int o = 1; o < 32; o <<= 1) {
    const T u = N::up(incl, o);
    if (lane >= o) incl = N::add(incl, u);
  }
  if (lane == 31) ms.wsum[warp] = incl;
  sub_sync<NT>();
  if (warp == 0) {
    T w = lane < NW ? ms.wsum[lane] : N::from_f(0.0f);
    for (int o = 1; o < NW; o <<= 1) {
      const T u = N::up(w, o);
      if (lane >= o) w = N::add(w, u);
    }
    T ex = N::up(w, 1);
    if (lane == 0) ex = N::from_f(0.0f);
    if (lane < NW) ms.woff[lane] = ex;
    if (lane == NW - 1) ms.tot[0] = w;
  }
  sub_sync<NT>();
  T ex = N::up(incl, 1);  // chunks of the earlier lanes of this warp
  if (lane == 0) ex = N::from_f(0.0f);
  const T off = N::add(ms.woff[warp], ex);
  for (int j = j0; j < j1; ++j) v[j] = N::add(v[j], off);
  const T total = ms.tot[0];
  sub_sync<NT>();
  return total;
}

template <class R, int NT>
__device__ __forceinline__ void mean_mode_body(const PoissonArgs& a, unsigned char* smem_raw,
                                               MeanScratch<R, NT>& ms) {
  using N = MeanNum<R>;
  using T = typename N::T;
  constexpr int NW = NT / 32;
  T* v = reinterpret_cast<T*>(smem_raw);  // [Ny]: s, then S, then T
  const int Ny = a.Ny, t = threadIdx.x, lane = t & 31, warp = t >> 5;
  if (a.flux_part) {
    // FP64 totals of the wall fluxes: a shuffle tree over the strips, in the
    // warps that hold partials (the others' totals would be +0, whose
    // addition changes nothing; FP64 issue is slow on this part)
    const int nfw = min(NW, (a.nflux + 31) / 32);
    double qi = 0.0, qo = 0.0;
    if (warp < nfw) {
      for (int b = t; b < a.nflux; b += NT) {
        qi += a.flux_part[b];
        qo += a.flux_part[a.nflux + b];
      }
      for (int o = 16; o > 0; o >>= 1) {
        qi += __shfl_down_sync(0xffffffffu, qi, o);
        qo += __shfl_down_sync(0xffffffffu, qo, o);
      }
    }
    auto& fq = ms.fq;
    if (lane == 0 && warp < nfw) {
      fq[0][warp] = qi;
      fq[1][warp] = qo;
    }
    sub_sync<NT>();
    if (t == 0) {
      double si = 0.0, so = 0.0;
      for (int w = 0; w < nfw; ++w) {
        si += fq[0][w];
        so += fq[1][w];
      }
      a.flux_acc[0] += si;
      a.flux_acc[1] += so;
    }
  }
  for (int j = t; j < Ny; j += NT) {
    if constexpr (sizeof(R) == 8) {
      v[j] = static_cast<const double*>(a.spec0)[j];
    } else {
      v[j] = {static_cast<const float2*>(a.spec0)[j].x, static_cast<const float2*>(a.spec0)[j].y};
    }
  }
  sub_sync<NT>();
  const int C = (Ny + NT - 1) / NT;
  const int j0 = min(t * C, Ny), j1 = min(j0 + C, Ny);
  T* Sv = v + Ny;  // [Ny]: copy of S
  // S_j (inclusive), kept in Sv; then v[j] = sum_{k<=j} S_k = T_{j+1}
  block_prefix_sum<R, NT>(v, j0, j1, ms);
  for (int j = j0; j < j1; ++j) Sv[j] = v[j];
  const T T_all = block_prefix_sum<R, NT>(v, j0, j1, ms);   // T_Ny
  const T T_last = (Ny >= 2) ? v[Ny - 2] : N::from_f(0.0f);  // T_{Ny-1}
  // wall values in spectral units: W = Nx phi0 at the injector, 0 at the
  // collector; W and the closure factor come from the host
  const T W = N::pair(a.mW, a.mWf[0], a.mWf[1]);
  T Dm, Pm;  // D_{-1}, phi_{-1}
  if (a.wall_mode == 0) {
    // phi_{-1} + phi_0 = 2W, phi_Ny + phi_{Ny-1} = 0: D_{-1} = -(2W + T_Ny + T_{Ny-1}) / (2 Ny)
    const T num = N::add(N::add(W, W), N::add(T_all, T_last));
    Dm = N::mul(N::neg(num), N::pair(a.mC, a.mCf[0], a.mCf[1]));
    Pm = N::add(W, N::neg(N::mul(Dm, N::from_f(0.5f))));
  } else {
    // phi_{-1} = W, phi_Ny = 0: D_{-1} = -(W + T_Ny) / (Ny + 1)
    Dm = N::mul(N::neg(N::add(W, T_all)), N::pair(a.mC, a.mCf[0], a.mCf[1]));
    Pm = W;
  }
  // phi_j = phi_{-1} + (j+1) D_{-1} + T_j,  E_j = -(2 D_{-1} + S_j + S_{j-1}) / 2
  const T inN = N::from_f(1.0f / (float)a.Nx);
  R* Ebar = static_cast<R*>(a.Ebar);
  const T mhalf = N::from_f(-0.5f);
  for (int j = j0; j < j1; ++j) {
    const T Tj = (j > 0) ? v[j - 1] : N::from_f(0.0f);
    const T Sj = Sv[j], Sjm1 = (j > 0) ? Sv[j - 1] : N::from_f(0.0f);
    const T phi = N::add(N::add(Pm, N::mul(N::from_i(j + 1), Dm)), Tj);
    const T ey = N::mul(mhalf, N::add(N::add(Dm, Dm), N::add(Sj, Sjm1)));
    const T pc = N::mul(phi, inN), ec = N::mul(ey, inN);
    if constexpr (sizeof(R) == 8) {
      static_cast<double*>(a.phibar)[j] = pc;
      Ebar[j] = ec;
    } else {
      static_cast<float2*>(a.phibar)[j] = make_float2(pc.hi, pc.lo);
      Ebar[j] = ec.hi + ec.lo;
    }
  }
}

// threads of the mean mode: 128 up to 1024 rows (shorter scans over the
// warps), 512 above (shorter per-thread chunks)
constexpr int kMeanThreads = 512;
constexpr int kMeanThreadsSmall = 128;
constexpr int kMeanSmallRows = 1024;

template <class R, int NT>
__global__ void __launch_bounds__(NT) k_mean_mode(PoissonArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ MeanScratch<R, NT> ms;
  mean_mode_body<R, NT>(a, smem_raw, ms);
}

// Batch kernels: CTAs take (run, tile) items / one CTA per run.
__global__ void __launch_bounds__(kTileThreads) k_batch_modes(BatchTables t, int step) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  grid_dep_wait();  // programmatic dependent launch (t.pdl): the forward transforms have ended
  grid_dep_launch();
  __shared__ TileScratch<float, kBatchTileModes, kTileThreads> ts;
  __shared__ int s_it;
  const int n = t.counts[3];
  for (;;) {
    // the CTA takes the next tile (tallest runs first) from the step's counter
    if (threadIdx.x == 0) s_it = atomicAdd(t.work + 2, 1);
    __syncthreads();
    const int it = s_it;
    __syncthreads();
    if (it >= n) break;
    const int2 w = t.tile_items[it];
    const BatchRunDesc& rd = t.runs[w.x];
    if (step >= rd.remaining) continue;  // whole CTA
    const PoissonArgs a = rd.pa;
    modes_tile_body<float, kBatchTileModes, kTileThreads>(a, w.y, smem_raw, ts);
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kMeanThreads) k_batch_mean(BatchTables t, int step) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ MeanScratch<float, kMeanThreads> ms;
  __shared__ MeanScratch<float, kMeanThreadsSmall> ms_small;
  const int n = t.counts[0];
  for (int r = blockIdx.x; r < n; r += gridDim.x) {
    const BatchRunDesc& rd = t.runs[r];
    if (step >= rd.remaining) continue;
    const PoissonArgs& a = rd.pa;
    if (a.Ny <= kMeanSmallRows) {  // the same thread count as the run alone
      if (threadIdx.x < kMeanThreadsSmall) mean_mode_body<float, kMeanThreadsSmall>(a, smem_raw, ms_small);
    } else {
      mean_mode_body<float, kMeanThreads>(a, smem_raw, ms);
    }
    __syncthreads();
  }
}


// --------------------------------------------------- perturbation form ---
// One step of the x-uniform base state in FP64: the moments (Eqs. 5-7,
// E_x = 0), the fluid TRT collision with the force rho_c E_y (Eqs. 8, 10,
// 12, 13, 15) and the charge TRT collision with the drift u + mu_b E
// (Eqs. 9, 11, 14), then streaming in y (an x-uniform state does not change
// under the x shifts) with the wall rules: halfway bounce-back of f,
// anti-bounce-back injection of rho0 with the wall-node drift, zero-gradient
// outflow of g (Table I).  The two wall rows add their charge fluxes, times
// Nx, to the base's own FP64 totals.
//
// A CTA of four warps takes kBaseRows rows; lane l holds row y0 - 1 + l, so
// lanes 0 and 31 are the halo rows whose post-collision populations stream
// into the CTA.  Warp w collides one population group -- {0, 1, 3}, {2, 4},
// {5, 7}, {6, 8}: each with its opposite, as the TRT split needs -- so the
// FP64 work of a row is spread over four warps, and the new populations are
// pulled from shared memory.  The row moments (rho, rho_c, u, the drift
// velocity) come from the potential kernel of the previous step, which has
// E_y; the CTA sums the new rows' rho_c, rho, j_x, j_y in population order.
// (FP64 runs at a small fraction of the FP32 rate on this GPU: the split and
// the precomputed moments keep each warp's FP64 instruction count low.)
namespace {
__device__ __forceinline__ double bw(int i) { return i == 0 ? kW0 : (i < 5 ? kW1 : kW2); }
__device__ __forceinline__ int bcx(int i) { return (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0); }
__device__ __forceinline__ int bcy(int i) { return (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0); }
__device__ __forceinline__ int bopp(int i) { return i == 0 ? 0 : (i < 5 ? ((i + 1) & 3) + 1 : ((i - 3) & 3) + 5); }
// c_q . v with the lattice direction known at compile time
template <int Q>
__device__ __forceinline__ double bcdot(double vx, double vy) {
  constexpr int cx = (Q == 1 || Q == 5 || Q == 8) ? 1 : ((Q == 3 || Q == 6 || Q == 7) ? -1 : 0);
  constexpr int cy = (Q == 2 || Q == 5 || Q == 6) ? 1 : ((Q == 4 || Q == 7 || Q == 8) ? -1 : 0);
  if constexpr (cx == 0 && cy == 0) return 0.0;
  else if constexpr (cx == 0) return cy > 0 ? vy : -vy;
  else if constexpr (cy == 0) return cx > 0 ? vx : -vx;
  else return (cx > 0 ? vx : -vx) + (cy > 0 ? vy : -vy);
}
// equilibrium (Eq. 12 / 14) with |v|^2 passed in
template <int Q>
__device__ __forceinline__ double beq(double dens, double vx, double vy, double v2) {
  const double cu = bcdot<Q>(vx, vy);
  return bw(Q) * dens * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * v2);
}
constexpr int kBaseRows = 30;
// the groups' populations: {0, 1, 3}, {2, 4}, {5, 7}, {6, 8}
__device__ __forceinline__ int bgroup_pop(int grp, int k) {
  constexpr int pops[4][3] = {{0, 1, 3}, {2, 4, -1}, {5, 7, -1}, {6, 8, -1}};
  return pops[grp][k];
}
}  // namespace

struct BaseSmem {
  double fp[9][32], gp[9][32];  // post-collision populations of the CTA's rows
  double nf[9][32], ng[9][32];  // populations of t + 1 of its output rows
  double qin[3];                // injected-charge terms of the populations 2, 5, 6
};

// The TRT collision of the population pair (I, O = opposite of I; I == O
// for the rest population).  The odd parts of the pair are equal and
// opposite, so one set of half sums serves both.  The force has no x part
// (E_x = 0 in an x-uniform state): F_i = w_i (3 (c_iy - u_y) + 9 (c_i.u) c_iy) F_y.
struct BaseRow {
  double rho, rc, ux, uy, vy, Fy, u2, v2;
};
template <int I, int O>
__device__ __forceinline__ void base_collide_pair(const BaseArgs& a, const BaseRow& b, int y, BaseSmem& sm,
                                                  int lane) {
  const int Ny = a.Ny;
  const double fI = a.fin[I * Ny + y], fO = a.fin[O * Ny + y];
  const double gI = a.gin[I * Ny + y], gO = a.gin[O * Ny + y];
  const double feqI = beq<I>(b.rho, b.ux, b.uy, b.u2), feqO = beq<O>(b.rho, b.ux, b.uy, b.u2);
  const double geqI = beq<I>(b.rc, b.ux, b.vy, b.v2), geqO = beq<O>(b.rc, b.ux, b.vy, b.v2);
  constexpr int cyI = (I == 2 || I == 5 || I == 6) ? 1 : ((I == 4 || I == 7 || I == 8) ? -1 : 0);
  const double cuI = bcdot<I>(b.ux, b.uy);
  // F_O = w (3 (-c_y - u_y) + 9 (-c.u)(-c_y)) F_y
  double FiI, FiO;
  if constexpr (cyI == 0) {
    FiI = bw(I) * ((0.0 - b.uy) * 3.0 * b.Fy);
    FiO = bw(O) * ((0.0 - b.uy) * 3.0 * b.Fy);
  } else {
    const double c = (double)cyI;
    FiI = bw(I) * (((c - b.uy) * 3.0 + cuI * c * 9.0) * b.Fy);
    FiO = bw(O) * (((-c - b.uy) * 3.0 + cuI * c * 9.0) * b.Fy);
  }
  const double fpl = 0.5 * (fI + fO), fmi = 0.5 * (fI - fO);
  const double epl = 0.5 * (feqI + feqO), emi = 0.5 * (feqI - feqO);
  const double Fpl = 0.5 * (FiI + FiO), Fmi = 0.5 * (FiI - FiO);
  const double ev = a.wp * (fpl - epl), od = a.wm * (fmi - emi);
  const double Fe = a.cp * Fpl, Fo = a.cm * Fmi;
  sm.fp[I][lane] = fI - ev - od + Fe + Fo;
  const double gpl = 0.5 * (gI + gO), gmi = 0.5 * (gI - gO);
  const double hpl = 0.5 * (geqI + geqO), hmi = 0.5 * (geqI - geqO);
  const double gev = a.gwp * (gpl - hpl), god = a.gwm * (gmi - hmi);
  sm.gp[I][lane] = gI - gev - god;
  if constexpr (I != O) {
    sm.fp[O][lane] = fO - ev + od + Fe - Fo;
    sm.gp[O][lane] = gO - gev + god;
  }
}

// The mean mode of the base's Poisson equation is a double prefix sum of the
// right-hand side s over the rows (S_j = sum_{k<=j} s_k, T_j = sum_{k<j} S_k;
// see mean_mode_body).  It is split over chunks of kBaseRows rows: the warp
// that holds a chunk (lanes 1 .. kBaseRows, s = 0 on the other lanes) keeps
// per row the chunk-local sums Sl_j, Tl_j, and per chunk its totals sigma =
// sum of s and tau = sum of Sl; the potential kernel adds the sums of the
// chunks before.
__device__ __forceinline__ void base_chunk_scan(double s, bool valid, int lane, int c, int y, double* loc,
                                                double* chunk, int Ny) {
  double S = s;
  for (int o = 1; o < 32; o <<= 1) {
    const double u = __shfl_up_sync(0xffffffffu, S, o);
    if (lane >= o) S += u;
  }
  const double Sm = valid ? S : 0.0;
  double Ti = Sm;
  for (int o = 1; o < 32; o <<= 1) {
    const double u = __shfl_up_sync(0xffffffffu, Ti, o);
    if (lane >= o) Ti += u;
  }
  double Tl = __shfl_up_sync(0xffffffffu, Ti, 1);
  if (lane == 0) Tl = 0.0;
  if (valid) {
    loc[y] = S;
    loc[Ny + y] = Tl;
  }
  if (lane == 31) {
    chunk[2 * c] = S;
    chunk[2 * c + 1] = Ti;
  }
}

__device__ __noinline__ void base_step_cta(const BaseArgs& a, int y0, BaseSmem& sm) {
  const int lane = threadIdx.x & 31, grp = threadIdx.x >> 5, Ny = a.Ny;
  const int y = y0 - 1 + lane;
  const int npop = grp == 0 ? 3 : 2;
  if (y >= 0 && y < Ny) {
    BaseRow b;
    b.rho = a.mom[y];
    b.rc = a.mom[Ny + y];
    b.ux = a.mom[2 * Ny + y];
    b.uy = a.mom[3 * Ny + y];
    b.vy = a.mom[4 * Ny + y];
    b.Fy = b.rc * a.EB[y];
    b.u2 = b.ux * b.ux + b.uy * b.uy;
    b.v2 = b.ux * b.ux + b.vy * b.vy;
    switch (grp) {
      case 0:
        base_collide_pair<0, 0>(a, b, y, sm, lane);
        base_collide_pair<1, 3>(a, b, y, sm, lane);
        break;
      case 1: base_collide_pair<2, 4>(a, b, y, sm, lane); break;
      case 2: base_collide_pair<5, 7>(a, b, y, sm, lane); break;
      default: base_collide_pair<6, 8>(a, b, y, sm, lane); break;
    }
  }
  __syncthreads();
  const bool out = lane >= 1 && lane <= kBaseRows && y < Ny;
  if (out) {
    for (int k = 0; k < npop; ++k) {
      const int i = bgroup_pop(grp, k), cy = bcy(i);
      double nf, ng;
      if (cy == 0) {
        nf = sm.fp[i][lane];
        ng = sm.gp[i][lane];
      } else if (cy > 0) {
        if (y >= 1) {
          nf = sm.fp[i][lane - 1];
          ng = sm.gp[i][lane - 1];
        } else {
          // injector: bounce-back of f; anti-bounce-back of g with the wall drift (0, mu_b E_y)
          const int d = bopp(i);
          nf = sm.fp[d][lane];
          const double wvy = a.mub * a.EB[0];
          const double cv = bcy(i) * wvy;
          const double even = bw(i) * a.rho0 * (1.0 + 4.5 * cv * cv - 1.5 * (wvy * wvy));
          ng = -sm.gp[d][lane] + 2.0 * even;
          sm.qin[i == 2 ? 0 : (i == 5 ? 1 : 2)] = ng - sm.gp[d][lane];
        }
      } else {
        if (y <= Ny - 2) {
          nf = sm.fp[i][lane + 1];
          ng = sm.gp[i][lane + 1];
        } else {
          // collector: bounce-back of f; the up-movers leave, the down-movers
          // entering the top row are its own (zero-gradient outflow)
          nf = sm.fp[bopp(i)][lane];
          ng = sm.gp[i][lane];
        }
      }
      a.fout[i * Ny + y] = nf;
      a.gout[i * Ny + y] = ng;
      sm.nf[i][lane] = nf;
      sm.ng[i][lane] = ng;
    }
  }
  __syncthreads();
  if (grp == 2) {
    double s = 0.0;
    if (out) {
      double rc = 0;
      for (int i = 0; i < 9; ++i) rc += sm.ng[i][lane];
      a.sums[y] = rc;
      s = -(double)a.Nx * rc / a.eps;
      a.rhs[y] = s;
    }
    base_chunk_scan(s, out, lane, y0 / kBaseRows, y, a.loc, a.chunk, Ny);
  }
  if (out) {
    if (grp == 0) {
      double rho = 0;
      for (int i = 0; i < 9; ++i) rho += sm.nf[i][lane];
      a.sums[Ny + y] = rho;
    } else if (grp == 1) {
      double jy = 0;
      for (int i = 0; i < 9; ++i) jy += bcy(i) * sm.nf[i][lane];
      a.sums[2 * Ny + y] = jy;
    } else if (grp == 3) {
      double jx = 0;
      for (int i = 0; i < 9; ++i) jx += bcx(i) * sm.nf[i][lane];
      a.sums[3 * Ny + y] = jx;
    }
    if (grp == 3 && y == 0) {
      // injected charge: the down-movers 4, 7, 8 reflected into 2, 5, 6
      double qin = 0.0;
      for (int k = 0; k < 3; ++k) qin += sm.qin[k];
      a.flux_acc[0] += (double)a.Nx * qin;
    }
    if (grp == 3 && y == Ny - 1) {
      // collected charge: up-movers out, minus the outflow's down-movers, in population order
      const double qout = ((((sm.gp[2][lane] - sm.gp[4][lane]) + sm.gp[5][lane]) + sm.gp[6][lane]) - sm.gp[7][lane]) -
                          sm.gp[8][lane];
      a.flux_acc[1] += (double)a.Nx * qout;
    }
  }
}

__global__ void __launch_bounds__(128) k_base_step(BaseArgs a) {
  __shared__ BaseSmem sm;
  base_step_cta(a, blockIdx.x * kBaseRows, sm);
}

// Row sums of a base state (at creation and after a load): rho_c, rho, j_y,
// the mean-mode right-hand side and its chunk sums, as the step leaves them
// (one warp per chunk of kBaseRows rows).
__global__ void __launch_bounds__(32) k_base_sums(BaseArgs a) {
  const int lane = threadIdx.x, Ny = a.Ny, c = blockIdx.x;
  const int y = c * kBaseRows - 1 + lane;
  const bool valid = lane >= 1 && lane <= kBaseRows && y < Ny;
  double s = 0.0;
  if (valid) {
    double rho = 0, jy = 0, jx = 0, rc = 0;
    for (int i = 0; i < 9; ++i) rho += a.fin[i * Ny + y];
    for (int i = 0; i < 9; ++i) jy += bcy(i) * a.fin[i * Ny + y];
    for (int i = 0; i < 9; ++i) jx += bcx(i) * a.fin[i * Ny + y];
    for (int i = 0; i < 9; ++i) rc += a.gin[i * Ny + y];
    a.sums[y] = rc;
    a.sums[Ny + y] = rho;
    a.sums[2 * Ny + y] = jy;
    a.sums[3 * Ny + y] = jx;
    s = -(double)a.Nx * rc / a.eps;
    a.rhs[y] = s;
  }
  base_chunk_scan(s, valid, lane, c, y, a.loc, a.chunk, Ny);
}

// Potential of the base state (the mean mode of Eqs. 18-20 with the wall
// potentials, from the chunk sums: each warp scans the chunk totals, takes
// the wall conditions as mean_mode_body does and writes phi, E_y for its
// chunk's rows), and the march table of the state: per row the base
// charge, the base fluid velocity u_y (Eq. 7; its numerator in FP64, the
// quotient in FP32) and the base field E_y.
__device__ __noinline__ void base_potential_warp(const BasePoissonArgs& b, int c) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31, Ny = b.Ny;
  const int nch = (Ny + kBaseRows - 1) / kBaseRows;
  const int K = (nch + 31) / 32;
  const int c0 = min(lane * K, nch), c1 = min(c0 + K, nch);
  // S0_c = sum of sigma over the chunks before c
  double acc = 0.0;
  for (int cc = c0; cc < c1; ++cc) acc += b.chunk[2 * cc];
  double incl = acc;
  for (int o = 1; o < 32; o <<= 1) {
    const double u = __shfl_up_sync(FULL, incl, o);
    if (lane >= o) incl += u;
  }
  double s0 = __shfl_up_sync(FULL, incl, 1);
  if (lane == 0) s0 = 0.0;
  // T0_c = sum over the chunks before c of (rows x S0 + tau)
  double uacc = 0.0;
  {
    double sc = s0;
    for (int cc = c0; cc < c1; ++cc) {
      const int n = min(kBaseRows, Ny - cc * kBaseRows);
      uacc += (double)n * sc + b.chunk[2 * cc + 1];
      sc += b.chunk[2 * cc];
    }
  }
  double uincl = uacc;
  for (int o = 1; o < 32; o <<= 1) {
    const double u = __shfl_up_sync(FULL, uincl, o);
    if (lane >= o) uincl += u;
  }
  double t0 = __shfl_up_sync(FULL, uincl, 1);
  if (lane == 0) t0 = 0.0;
  // S0, T0 of chunk c and of the last chunk, from the lanes that hold them
  double S0c = 0, T0c = 0, S0L = 0, T0L = 0;
  {
    double sc = s0, tc = t0;
    for (int cc = c0; cc < c1; ++cc) {
      if (cc == c) {
        S0c = sc;
        T0c = tc;
      }
      if (cc == nch - 1) {
        S0L = sc;
        T0L = tc;
      }
      const int n = min(kBaseRows, Ny - cc * kBaseRows);
      tc += (double)n * sc + b.chunk[2 * cc + 1];
      sc += b.chunk[2 * cc];
    }
  }
  S0c = __shfl_sync(FULL, S0c, c / K);
  T0c = __shfl_sync(FULL, T0c, c / K);
  S0L = __shfl_sync(FULL, S0L, (nch - 1) / K);
  T0L = __shfl_sync(FULL, T0L, (nch - 1) / K);
  // wall conditions (as mean_mode_body): T_{Ny-1}, S_{Ny-1}, T_Ny
  const int jL = (nch - 1) * kBaseRows;
  const double S_last = S0L + b.loc[Ny - 1];
  const double T_last = (T0L + (double)(Ny - 1 - jL) * S0L) + b.loc[Ny + Ny - 1];
  const double T_all = T_last + S_last;
  const double W = (double)b.Nx * b.phi0;
  double Dm, Pm;
  if (b.wall_mode == 0) {
    const double num = (W + W) + (T_all + T_last);
    Dm = -num * (1.0 / (2.0 * Ny));
    Pm = W + -(Dm * 0.5);
  } else {
    Dm = -(W + T_all) * (1.0 / (double)(Ny + 1));
    Pm = W;
  }
  const int j0 = c * kBaseRows, j = j0 + lane;
  const bool valid = lane < kBaseRows && j < Ny;
  const double Sj = valid ? S0c + b.loc[j] : 0.0;
  double Sjm1 = __shfl_up_sync(FULL, Sj, 1);
  if (lane == 0) Sjm1 = (j > 0) ? S0c : 0.0;
  if (valid) {
    const double Tj = (T0c + (double)(j - j0) * S0c) + b.loc[Ny + j];
    const double phi = (Pm + (double)(j + 1) * Dm) + Tj;
    const double ey = -0.5 * ((Dm + Dm) + (Sj + Sjm1));
    const double inN = 1.0 / (double)b.Nx;
    b.phiB[j] = phi * inN;
    const double Ey = ey * inN;
    b.EB[j] = Ey;
    // moments of the state for its next base step (Eq. 7 with F = rho_c E_y e_y)
    const double rc = b.sums[j], rho = b.sums[Ny + j], jy = b.sums[2 * Ny + j], jx = b.sums[3 * Ny + j];
    const double ux = jx / rho, uy = (jy + 0.5 * (rc * Ey)) / rho;
    b.mom[j] = rho;
    b.mom[Ny + j] = rc;
    b.mom[2 * Ny + j] = ux;
    b.mom[3 * Ny + j] = uy;
    b.mom[4 * Ny + j] = uy + b.mub * Ey;
    b.table[4 * j + 0] = (float)rc;
    b.table[4 * j + 1] = (float)uy;
    b.table[4 * j + 2] = (float)Ey;
    b.table[4 * j + 3] = 0.0f;
  }
}

__global__ void __launch_bounds__(32) k_base_poisson(BasePoissonArgs b) { base_potential_warp(b, blockIdx.x); }

// Batch: the base step of every perturbation-form member (CTA (x, r): rows
// kBaseRows x .. of member r), then one CTA per member for its potential.
__global__ void __launch_bounds__(128) k_batch_base_step(BatchTables t, int step) {
  __shared__ BaseSmem sm;
  const int r = blockIdx.y;
  if (r >= t.counts[0]) return;
  const BatchRunDesc& rd = t.runs[r];
  if (step >= rd.remaining) return;
  const BaseArgs& a = rd.ba[rd.cur0 ^ (step & 1)];
  if (!a.fin || (int)blockIdx.x * kBaseRows >= a.Ny) return;
  base_step_cta(a, blockIdx.x * kBaseRows, sm);
}

__global__ void __launch_bounds__(32) k_batch_base_poisson(BatchTables t, int step) {
  const int r = blockIdx.y;
  if (r >= t.counts[0]) return;
  const BatchRunDesc& rd = t.runs[r];
  if (step >= rd.remaining) return;
  const BasePoissonArgs& b = rd.bp[rd.cur0 ^ (step & 1)];
  if (!b.sums || (int)blockIdx.x * kBaseRows >= b.Ny) return;
  base_potential_warp(b, blockIdx.x);
}

cudaError_t launch_batch_base(const BatchTables& t, int step, int maxr, int max_ny, cudaStream_t s) {
  const int nch = (max_ny + kBaseRows - 1) / kBaseRows;
  k_batch_base_step<<<dim3(nch, maxr), 128, 0, s>>>(t, step);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_batch_base_poisson<<<dim3(nch, maxr), 32, 0, s>>>(t, step);
  return cudaGetLastError();
}

int base_chunks(int Ny) { return (Ny + kBaseRows - 1) / kBaseRows; }

cudaError_t launch_base_step(const BaseArgs& a, cudaStream_t s) {
  k_base_step<<<base_chunks(a.Ny), 128, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_base_sums(const BaseArgs& a, cudaStream_t s) {
  k_base_sums<<<base_chunks(a.Ny), 32, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_base_poisson(const BasePoissonArgs& a, cudaStream_t s) {
  k_base_poisson<<<base_chunks(a.Ny), 32, 0, s>>>(a);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- launch ---
namespace {

constexpr size_t kSmemCap = 200 * 1024;

// wavenumbers per CTA: the spectrum and pivot tiles of all rows must fit
// (8, as the batch's wavenumber tiles, so that a run gives the same bits
// alone and in a batch: the tile width sets the scans' chunking)
int tile_modes(int Ny, size_t cbytes, size_t rbytes) {
  int mb = 8;
  while (mb > 1 && (size_t)Ny * mb * (cbytes + rbytes) > kSmemCap) mb >>= 1;
  return mb;
}

template <class R>
cudaError_t launch_modes(const PoissonArgs& a, cudaStream_t s) {
  int mb = tile_modes(a.Ny, sizeof(Cplx<R>), sizeof(R));
  if (a.tile_modes > 0 && a.tile_modes < mb) mb = a.tile_modes;
  const size_t sm = (size_t)a.Ny * mb * (sizeof(Cplx<R>) + sizeof(R));
  const int nm = a.Mh;  // tiles start at m = 0
  const bool pdl = (a.pdl & 2) != 0;
  if constexpr (sizeof(R) == 4) {
    if (a.tile_tma && a.mtma && mb == 8 && a.tile_threads <= 256 && !a.tile_cluster) {
      const size_t sm3 = modes_tma_pivot_offset(a.Ny) + (size_t)a.Ny * 32 + 128;
      return launch_ex(pdl, k_modes_tile_tma, dim3((nm + 7) / 8), dim3(kTileThreads), sm3, s, a, *a.mtma);
    }
    if (a.tile_cluster && mb == 8 && a.tile_threads <= 256 && a.Ny >= 64) {
      const int C = (a.Ny + 31) / 32;
      const size_t sm2 = (size_t)16 * C * 8 * (sizeof(Cplx<R>) + sizeof(R));
      return launch_ex(pdl, k_modes_tile2<8>, dim3(2 * ((nm + 7) / 8)), dim3(kTileThreads), sm2, s, a);
    }
    if (a.tile_threads == 512 || a.tile_threads == 1024) {
      const bool big = a.tile_threads == 1024;
      switch (mb) {
        case 8:
          return big ? launch_ex(pdl, k_modes_tile<R, 8, 1024>, dim3((nm + 7) / 8), dim3(1024), sm, s, a)
                     : launch_ex(pdl, k_modes_tile<R, 8, 512>, dim3((nm + 7) / 8), dim3(512), sm, s, a);
        case 4:
          return big ? launch_ex(pdl, k_modes_tile<R, 4, 1024>, dim3((nm + 3) / 4), dim3(1024), sm, s, a)
                     : launch_ex(pdl, k_modes_tile<R, 4, 512>, dim3((nm + 3) / 4), dim3(512), sm, s, a);
        case 2:
          return big ? launch_ex(pdl, k_modes_tile<R, 2, 1024>, dim3((nm + 1) / 2), dim3(1024), sm, s, a)
                     : launch_ex(pdl, k_modes_tile<R, 2, 512>, dim3((nm + 1) / 2), dim3(512), sm, s, a);
        default: break;
      }
    }
  }
  switch (mb) {
    case 8: return launch_ex(pdl, k_modes_tile<R, 8>, dim3((nm + 7) / 8), dim3(kTileThreads), sm, s, a);
    case 4: return launch_ex(pdl, k_modes_tile<R, 4>, dim3((nm + 3) / 4), dim3(kTileThreads), sm, s, a);
    case 2: return launch_ex(pdl, k_modes_tile<R, 2>, dim3((nm + 1) / 2), dim3(kTileThreads), sm, s, a);
    default: return launch_ex(pdl, k_modes_tile<R, 1>, dim3(nm), dim3(kTileThreads), sm, s, a);
  }
}

template <class R>
size_t row_smem(int Nx) {
  const int L = Nx / 2, T = (L >= 4) ? L / 4 : 1, rows = 256 / T;
  return ((size_t)Nx + 2 * (size_t)rows * row_len_padded(L)) * sizeof(Cplx<R>);
}

template <class R>
int row_blocks(int Nx, int Ny) {
  const int L = Nx / 2, T = (L >= 4) ? L / 4 : 1, rows = 256 / T;
  return (Ny + rows - 1) / rows;
}

template <class R>
cudaError_t poisson_t(const PoissonArgs& a, cudaStream_t s, cudaStream_t side, cudaEvent_t fork, cudaEvent_t join,
                      const cudaEvent_t* marks) {
  const bool warp_fft = (sizeof(R) == 4) && fftw_supported(a.Nx);
  cudaError_t e;
  if (warp_fft) {
    e = launch_rfft_warp(a, s);
  } else {
    k_rfft_rows<R><<<row_blocks<R>(a.Nx, a.Ny), 256, row_smem<R>(a.Nx), s>>>(a);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return e;
  // optional timing marks: [0] after the forward FFT, [1] after the m >= 1
  // solve, [2] after the inverse FFT (all on s); [3], [4] around the mean mode
  auto mark = [&](int k, cudaStream_t st) { return marks ? cudaEventRecord(marks[k], st) : cudaSuccess; };
  if ((e = mark(0, s)) != cudaSuccess) return e;
  if (side) {
    if ((e = cudaEventRecord(fork, s)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(side, fork, 0)) != cudaSuccess) return e;
  }
  const cudaStream_t ms = side ? side : s;
  if ((e = mark(3, ms)) != cudaSuccess) return e;
  const size_t msm = 2 * (size_t)a.Ny * sizeof(typename MeanNum<R>::T);
  if (a.Ny <= kMeanSmallRows)
    k_mean_mode<R, kMeanThreadsSmall><<<1, kMeanThreadsSmall, msm, ms>>>(a);
  else
    k_mean_mode<R, kMeanThreads><<<1, kMeanThreads, msm, ms>>>(a);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = mark(4, ms)) != cudaSuccess) return e;
  if (side && (e = cudaEventRecord(join, side)) != cudaSuccess) return e;
  e = (a.y_solver == 1) ? launch_modes_oddext(a, sizeof(R) == 8, s) : launch_modes<R>(a, s);
  if (e != cudaSuccess) return e;
  if ((e = mark(1, s)) != cudaSuccess) return e;
  if (warp_fft) {
    e = launch_irfft_warp(a, s);
  } else {
    k_irfft_rows<R><<<row_blocks<R>(a.Nx, a.Ny), 256, row_smem<R>(a.Nx), s>>>(a);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return e;
  if (a.ex) {
    // spectral E_x: the inverse row transform of -i k_m phi_m, formed as it
    // reads the solved spectrum
    if (warp_fft) {
      e = launch_irfft_warp_dx(a, s);
    } else {
      k_irfft_rows<R, true><<<row_blocks<R>(a.Nx, a.Ny), 256, row_smem<R>(a.Nx), s>>>(a);
      e = cudaGetLastError();
    }
    if (e != cudaSuccess) return e;
  }
  if ((e = mark(2, s)) != cudaSuccess) return e;
  if (side && (e = cudaStreamWaitEvent(s, join, 0)) != cudaSuccess) return e;
  return cudaSuccess;
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

template <class R>
cudaError_t set_attrs_t() {
  cudaError_t e;

  if ((e = allow_max_dynamic_smem(k_rfft_rows<R>)) != cudaSuccess) return e;
  if ((e = allow_max_dynamic_smem(k_irfft_rows<R>)) != cudaSuccess) return e;
  if ((e = allow_max_dynamic_smem(k_irfft_rows<R, true>)) != cudaSuccess) return e;
  if ((e = allow_max_dynamic_smem(k_mean_mode<R, kMeanThreads>)) != cudaSuccess) return e;
  if ((e = allow_max_dynamic_smem(k_mean_mode<R, kMeanThreadsSmall>)) != cudaSuccess) return e;
  if constexpr (sizeof(R) == 4) {
    if ((e = allow_max_dynamic_smem(k_modes_tile2<8>)) != cudaSuccess) return e;
    if ((e = allow_max_dynamic_smem(k_modes_tile_tma)) != cudaSuccess) return e;
    if ((e = allow_max_dynamic_smem(k_modes_tile<R, 8, 512>)) != cudaSuccess) return e;
    if ((e = allow_max_dynamic_smem(k_modes_tile<R, 4, 512>)) != cudaSuccess) return e;
    if ((e = allow_max_dynamic_smem(k_modes_tile<R, 2, 512>)) != cudaSuccess) return e;
    if ((e = allow_max_dynamic_smem(k_modes_tile<R, 8, 1024>)) != cudaSuccess) return e;
    if ((e = allow_max_dynamic_smem(k_modes_tile<R, 4, 1024>)) != cudaSuccess) return e;
    if ((e = allow_max_dynamic_smem(k_modes_tile<R, 2, 1024>)) != cudaSuccess) return e;
  }
  if ((e = allow_max_dynamic_smem(k_modes_tile<R, 8>)) != cudaSuccess) return e;
  if ((e = allow_max_dynamic_smem(k_modes_tile<R, 4>)) != cudaSuccess) return e;
  if ((e = allow_max_dynamic_smem(k_modes_tile<R, 2>)) != cudaSuccess) return e;
  return allow_max_dynamic_smem(k_modes_tile<R, 1>);
}

template <class S, class R>
cudaError_t rhoc_t(const void* g, long long plane, int Nx, int Ny, int P, const float* rch, void* rhoc,
                   cudaStream_t s) {
  k_rhoc<S, R><<<1216, 256, 0, s>>>(static_cast<const S*>(g), plane, Nx, Ny, P, rch, static_cast<R*>(rhoc));
  return cudaGetLastError();
}

}  // namespace

int batch_modes_ctas_per_sm(int smem) {
  int blocks = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_batch_modes, kTileThreads, (size_t)smem) !=
      cudaSuccess)
    return 1;
  return blocks;
}

cudaError_t launch_batch_modes(const BatchTables& t, int step, int grid, cudaStream_t s) {
  return launch_ex((t.pdl & 2) != 0, k_batch_modes, dim3(grid), dim3(kTileThreads), (size_t)t.modes_smem, s, t, step);
}

cudaError_t launch_batch_mean(const BatchTables& t, int step, int grid, cudaStream_t s) {
  k_batch_mean<<<grid, kMeanThreads, t.modes_smem, s>>>(t, step);
  return cudaGetLastError();
}

cudaError_t poisson_set_attributes() {
  cudaError_t e = fftw_set_tables();
  if (e != cudaSuccess) return e;
  if ((e = allow_max_dynamic_smem(k_batch_modes)) != cudaSuccess) return e;
  if ((e = allow_max_dynamic_smem(k_batch_mean)) != cudaSuccess) return e;
  e = set_attrs_t<double>();
  if (e != cudaSuccess) return e;
  return set_attrs_t<float>();
}

cudaError_t launch_rhoc(const void* g, long long plane, int storage, bool real_f64, int Nx, int Ny, int P,
                        const float* rch, void* rhoc, cudaStream_t s) {
  if (real_f64) return storage == 0 ? rhoc_t<double, double>(g, plane, Nx, Ny, P, rch, rhoc, s) : cudaErrorInvalidValue;
  switch (storage) {
    case 0: return rhoc_t<double, float>(g, plane, Nx, Ny, P, rch, rhoc, s);
    case 1: return rhoc_t<float, float>(g, plane, Nx, Ny, P, rch, rhoc, s);
    case 2: return rhoc_t<__nv_bfloat16, float>(g, plane, Nx, Ny, P, rch, rhoc, s);
    case 3: return rhoc_t<__half, float>(g, plane, Nx, Ny, P, rch, rhoc, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_poisson(const PoissonArgs& a, bool real_f64, cudaStream_t s, cudaStream_t side, cudaEvent_t fork,
                           cudaEvent_t join, const cudaEvent_t* marks) {
  return real_f64 ? poisson_t<double>(a, s, side, fork, join, marks) : poisson_t<float>(a, s, side, fork, join, marks);
}

}  // namespace ehd

// k_fftw.cu -- warp-per-row real FFTs of the Poisson solve (FP32 path) for
// rows of N = 64 E real samples, E in {1, 2, 4, 8, 16, 32} (Nx = 64 ... 2048).
//
// A row of N reals is packed as L = N/2 = 32 E complex values z[n]
// (Eq. 19 via the half-length transform) and transformed by the four-step
// factorisation L = 32 x E with n = n1 + 32 n2 and k = k2 + E k1:
//   X[k] = sum_n1 W_32^(n1 k1) W_L^(n1 k2) sum_n2 z[n1 + 32 n2] W_E^(n2 k2)
// Lane n1 holds its E values in registers (E-point FFT), multiplies by
// W_L^(n1 k2), the warp transposes through shared memory (padded rows), and
// lane k2 finishes with a 32-point FFT in registers.  No CTA-wide barrier.
// The inverse uses IFFT(Z) = conj(FFT(conj(Z))) / L.
#include <cmath>

#include "ehd_dev.cuh"

namespace ehd {

namespace {

__constant__ float2 c_w32[32];  // exp(-2 pi i k / 32)
__constant__ float2 c_w64[64];  // exp(-2 pi i k / 64)

__host__ __device__ constexpr int bitrev(int i, int n) {
  int r = 0;
  for (int b = 1; b < n; b <<= 1) {
    r = (r << 1) | (i & 1);
    i >>= 1;
  }
  return r;
}

// in-register radix-2 FFT of length M <= 32 (forward, natural order in/out);
// every index is a compile-time constant so the arrays stay in registers
template <int M, int LEN>
struct FftStage {
  __device__ __forceinline__ static void run(float (&re)[M], float (&im)[M]) {
#pragma unroll
    for (int b = 0; b < M / LEN; ++b) {
#pragma unroll
      for (int k = 0; k < LEN / 2; ++k) {
        const float2 w = c_w32[k * (32 / LEN)];
        const int u = b * LEN + k, v = u + LEN / 2;
        const float tr = re[v] * w.x - im[v] * w.y;
        const float ti = re[v] * w.y + im[v] * w.x;
        re[v] = re[u] - tr;
        im[v] = im[u] - ti;
        re[u] += tr;
        im[u] += ti;
      }
    }
    FftStage<M, LEN * 2>::run(re, im);
  }
};
template <int M>
struct FftStage<M, M * 2> {
  __device__ __forceinline__ static void run(float (&)[M], float (&)[M]) {}
};

template <int M>
__device__ __forceinline__ void fft_reg(float (&re)[M], float (&im)[M]) {
#pragma unroll
  for (int i = 0; i < M; ++i) {
    const int j = bitrev(i, M);
    if (j > i) {
      const float tr = re[i], ti = im[i];
      re[i] = re[j];
      im[i] = im[j];
      re[j] = tr;
      im[j] = ti;
    }
  }
  FftStage<M, 2>::run(re, im);
}

__device__ __forceinline__ float2 cm(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

__device__ __forceinline__ void two_sum_f(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// Four-step forward FFT of the warp's row held as (re[n2], im[n2]) in lane
// n1; on return lane k2 < E holds X[k2 + E k1] in (ore[k1], oim[k1]).
// tw: exp(-2 pi i q / N) for q < N (global); sm: this warp's E x 33 buffer.
template <int E>
__device__ __forceinline__ void four_step(float (&re)[E], float (&im)[E], float (&ore)[32], float (&oim)[32],
                                          const float2* __restrict__ tw, float2* sm, int lane) {
  fft_reg<E>(re, im);
  // twiddle W_L^(n1 k2) = W_N^(2 n1 k2): powers of W_N^(2 n1), resynchronised
  // from the table every 4 steps
  constexpr int N = 64 * E;
  const float2 base = tw[(2 * lane) & (N - 1)];
  float2 w = make_float2(1.0f, 0.0f);
#pragma unroll
  for (int k2 = 0; k2 < E; ++k2) {
    if (k2 > 0) w = ((k2 & 3) == 0) ? tw[(2 * lane * k2) & (N - 1)] : cm(w, base);
    const float2 v = cm(make_float2(re[k2], im[k2]), w);
    sm[k2 * 33 + lane] = v;
  }
  __syncwarp();
  const int src = (E == 32) ? lane : (lane & (E - 1));
#pragma unroll
  for (int n1 = 0; n1 < 32; ++n1) {
    const float2 v = sm[src * 33 + n1];
    ore[n1] = v.x;
    oim[n1] = v.y;
  }
  __syncwarp();
  fft_reg<32>(ore, oim);
}

}  // namespace

// Forward transform of row y by one warp; sm: the warp's E x 33 buffer.
template <int E>
__device__ __forceinline__ void rfft_warp_body(const PoissonArgs& a, int y, float2* sm) {
  const int lane = threadIdx.x & 31;
  constexpr int L = 32 * E, N = 2 * L;
  const float2* __restrict__ tw = static_cast<const float2*>(a.tw);
  const float2* rc2 = reinterpret_cast<const float2*>(static_cast<const float*>(a.rhoc) + (long long)y * a.P);
  const float ieps = (float)a.inv_eps;
  float re[E], im[E];
  float shi = 0.0f, slo = 0.0f;
#pragma unroll
  for (int n2 = 0; n2 < E; ++n2) {
    const float2 v = rc2[lane + 32 * n2];
    re[n2] = -v.x * ieps;
    im[n2] = -v.y * ieps;
    float s, e;
    two_sum_f(shi, re[n2], s, e);
    slo += e;
    two_sum_f(s, im[n2], shi, e);
    slo += e;
  }
  // row sum over the warp (float-float): the m = 0 DFT coefficient
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float h2 = __shfl_xor_sync(0xffffffffu, shi, o), l2 = __shfl_xor_sync(0xffffffffu, slo, o);
    float s, e;
    two_sum_f(shi, h2, s, e);
    shi = s;
    slo = slo + l2 + e;
  }
  {
    float h, l;
    two_sum_f(shi, slo, h, l);
    if (lane == 0) static_cast<float2*>(a.spec0)[y] = make_float2(h, l);
    const float mean = h / (float)N;
#pragma unroll
    for (int n2 = 0; n2 < E; ++n2) {
      re[n2] -= mean;
      im[n2] -= mean;
    }
  }
  float xr[32], xi[32];
  four_step<E>(re, im, xr, xi, tw, sm, lane);
  // untangle into the half spectrum: S[k] = E_k + W_N^k O_k,
  // E_k = (Z[k] + Z*[L-k]) / 2, O_k = (Z[k] - Z*[L-k]) / (2i); lane k2 holds
  // k = k2 + E k1, whose partner L - k sits in lane (E - k2) mod E at 31 - k1
  // (lane 0: its own register (32 - k1) mod 32)
  float2* spec = static_cast<float2*>(a.spec) + (long long)y * a.Mp;
  const int partner = (E - lane) & (E - 1);
  const float2 wk2 = tw[lane & (E - 1)];
#pragma unroll
  for (int k1 = 0; k1 < 32; ++k1) {
    float pr = __shfl_sync(0xffffffffu, xr[31 - k1], partner);
    float pi = __shfl_sync(0xffffffffu, xi[31 - k1], partner);
    if (lane == 0) {
      pr = xr[(32 - k1) & 31];
      pi = xi[(32 - k1) & 31];
    }
    const float2 zk = make_float2(xr[k1], xi[k1]);
    const float2 zc = make_float2(pr, -pi);
    const float2 Ev = make_float2(0.5f * (zk.x + zc.x), 0.5f * (zk.y + zc.y));
    const float2 Dv = make_float2(0.5f * (zk.x - zc.x), 0.5f * (zk.y - zc.y));
    const float2 O = make_float2(Dv.y, -Dv.x);
    const float2 wk = cm(wk2, c_w64[k1]);  // W_N^(k2 + E k1) = W_N^k2 W_64^k1
    const float2 Sk = make_float2(Ev.x + (wk.x * O.x - wk.y * O.y), Ev.y + (wk.x * O.y + wk.y * O.x));
    const int k = lane + E * k1;
    if (lane < E) spec[k] = (k == 0) ? make_float2(0.0f, 0.0f) : Sk;
  }
  if (lane == 0) spec[L] = make_float2(xr[0] - xi[0], 0.0f);  // Nyquist: Re Z0 - Im Z0
}

// Inverse transform of row y by one warp -> phi minus its row mean.
template <int E>
__device__ __forceinline__ void irfft_warp_body(const PoissonArgs& a, int y, float2* sm) {
  const int lane = threadIdx.x & 31;
  constexpr int L = 32 * E;
  const float2* __restrict__ tw = static_cast<const float2*>(a.tw);
  const float2* spec = static_cast<const float2*>(a.spec) + (long long)y * a.Mp;
  // conj(Z[n]) for n = lane + 32 n2, Z[k] = E_k + i O_k,
  // E_k = (S[k] + S*[L-k]) / 2, O_k = (S[k] - S*[L-k]) / (2 W_N^k), S[0] := 0
  const float2 wl = tw[lane];
  float re[E], im[E];
#pragma unroll
  for (int n2 = 0; n2 < E; ++n2) {
    const int k = lane + 32 * n2;
    const float2 sk = (k == 0) ? make_float2(0.0f, 0.0f) : spec[k];
    const float2 sp = spec[L - k];
    const float2 sc = make_float2(sp.x, -sp.y);
    const float2 Ev = make_float2(0.5f * (sk.x + sc.x), 0.5f * (sk.y + sc.y));
    const float2 Dv = make_float2(0.5f * (sk.x - sc.x), 0.5f * (sk.y - sc.y));
    const float2 wk = cm(wl, tw[32 * n2]);                         // W_N^k
    const float2 O = cm(Dv, make_float2(wk.x, -wk.y));             // D / W^k
    re[n2] = Ev.x - O.y;                                           // Re(E + i O)
    im[n2] = -(Ev.y + O.x);                                        // -Im: conjugate
  }
  float xr[32], xi[32];
  four_step<E>(re, im, xr, xi, tw, sm, lane);
  if (lane < E) {
    float2* dphi2 = reinterpret_cast<float2*>(static_cast<float*>(a.dphi) + (long long)y * a.P);
    const float inL = 1.0f / (float)L;
#pragma unroll
    for (int k1 = 0; k1 < 32; ++k1) dphi2[lane + E * k1] = make_float2(xr[k1] * inL, -xi[k1] * inL);
  }
}

template <int E>
__global__ void __launch_bounds__(128) k_rfft_warp(PoissonArgs a) {
  __shared__ float2 smem[4][E * 33];
  const int warp = threadIdx.x >> 5;
  const int y = blockIdx.x * 4 + warp;
  if (y < a.Ny) rfft_warp_body<E>(a, y, smem[warp]);
}

template <int E>
__global__ void __launch_bounds__(128) k_irfft_warp(PoissonArgs a) {
  __shared__ float2 smem[4][E * 33];
  const int warp = threadIdx.x >> 5;
  const int y = blockIdx.x * 4 + warp;
  if (y < a.Ny) irfft_warp_body<E>(a, y, smem[warp]);
}

// Batch: warps of a fixed grid take row items (run, y); the row length picks
// the transform shape.
template <bool INV>
__global__ void __launch_bounds__(128) k_batch_fft(BatchTables t, int step) {
  __shared__ float2 smem[4][32 * 33];
  const int warp = threadIdx.x >> 5;
  const int nw = gridDim.x * 4;
  const int n = t.counts[2];
  for (int it = blockIdx.x * 4 + warp; it < n; it += nw) {
    const int2 w = t.row_items[it];
    const BatchRunDesc& rd = t.runs[w.x];
    if (step >= rd.remaining) continue;
    const PoissonArgs a = rd.pa;
    float2* sm = smem[warp];
    switch (rd.E) {
      case 1: INV ? irfft_warp_body<1>(a, w.y, sm) : rfft_warp_body<1>(a, w.y, sm); break;
      case 2: INV ? irfft_warp_body<2>(a, w.y, sm) : rfft_warp_body<2>(a, w.y, sm); break;
      case 4: INV ? irfft_warp_body<4>(a, w.y, sm) : rfft_warp_body<4>(a, w.y, sm); break;
      case 8: INV ? irfft_warp_body<8>(a, w.y, sm) : rfft_warp_body<8>(a, w.y, sm); break;
      case 16: INV ? irfft_warp_body<16>(a, w.y, sm) : rfft_warp_body<16>(a, w.y, sm); break;
      default: INV ? irfft_warp_body<32>(a, w.y, sm) : rfft_warp_body<32>(a, w.y, sm); break;
    }
  }
}

cudaError_t launch_batch_rfft(const BatchTables& t, int step, int grid, cudaStream_t s) {
  k_batch_fft<false><<<grid, 128, 0, s>>>(t, step);
  return cudaGetLastError();
}

cudaError_t launch_batch_irfft(const BatchTables& t, int step, int grid, cudaStream_t s) {
  k_batch_fft<true><<<grid, 128, 0, s>>>(t, step);
  return cudaGetLastError();
}

cudaError_t fftw_set_tables() {
  float2 w32[32], w64[64];
  const double pi = 3.141592653589793238462643383279502884;
  for (int k = 0; k < 32; ++k) w32[k] = make_float2((float)std::cos(2 * pi * k / 32), (float)-std::sin(2 * pi * k / 32));
  for (int k = 0; k < 64; ++k) w64[k] = make_float2((float)std::cos(2 * pi * k / 64), (float)-std::sin(2 * pi * k / 64));
  cudaError_t e = cudaMemcpyToSymbol(c_w32, w32, sizeof w32);
  if (e != cudaSuccess) return e;
  return cudaMemcpyToSymbol(c_w64, w64, sizeof w64);
}

bool fftw_supported(int Nx) { return Nx >= 64 && Nx <= 2048; }

cudaError_t launch_rfft_warp(const PoissonArgs& a, cudaStream_t s) {
  const unsigned g = (unsigned)((a.Ny + 3) / 4);
  switch (a.Nx) {
    case 64: k_rfft_warp<1><<<g, 128, 0, s>>>(a); break;
    case 128: k_rfft_warp<2><<<g, 128, 0, s>>>(a); break;
    case 256: k_rfft_warp<4><<<g, 128, 0, s>>>(a); break;
    case 512: k_rfft_warp<8><<<g, 128, 0, s>>>(a); break;
    case 1024: k_rfft_warp<16><<<g, 128, 0, s>>>(a); break;
    case 2048: k_rfft_warp<32><<<g, 128, 0, s>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_irfft_warp(const PoissonArgs& a, cudaStream_t s) {
  const unsigned g = (unsigned)((a.Ny + 3) / 4);
  switch (a.Nx) {
    case 64: k_irfft_warp<1><<<g, 128, 0, s>>>(a); break;
    case 128: k_irfft_warp<2><<<g, 128, 0, s>>>(a); break;
    case 256: k_irfft_warp<4><<<g, 128, 0, s>>>(a); break;
    case 512: k_irfft_warp<8><<<g, 128, 0, s>>>(a); break;
    case 1024: k_irfft_warp<16><<<g, 128, 0, s>>>(a); break;
    case 2048: k_irfft_warp<32><<<g, 128, 0, s>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace ehd

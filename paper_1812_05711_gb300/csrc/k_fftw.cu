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
        // the pair's sum and difference as packed two-float adds
        const float2 a = make_float2(re[u], im[u]);
        const float2 lo = __fadd2_rn(a, make_float2(-tr, -ti)), hi = __fadd2_rn(a, make_float2(tr, ti));
        re[v] = lo.x;
        im[v] = lo.y;
        re[u] = hi.x;
        im[u] = hi.y;
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

// Four-step forward FFT of rows of L = 32 E complex values, R <= 32 / E rows
// per warp (R = 32 / E: every lane works in both stages).  First stage, per row r:
// lane n1 holds z[n1 + 32 n2] (n2 < E) in (re, im), transforms over n2,
// multiplies by W_L^(n1 k2) = W_N^(2 n1 k2) and writes row r E + k2 of the
// warp's [32][33] buffer.  Second stage: lane r E + k2 reads its buffer row
// and finishes with a 32-point FFT, holding X_r[k2 + E k1] in (ore[k1],
// oim[k1]).  Per row the arithmetic is that of the one-row-per-warp form.
// tw: exp(-2 pi i q / N) for q < N (global).

// the first stage's twiddles of lane n1: powers of W_N^(2 n1), resynchronised
// from the table every 4 steps
template <int E>
__device__ __forceinline__ void four_step_twiddles(const float2* __restrict__ tw, int lane, float2 (&w)[E]) {
  constexpr int N = 64 * E;
  const float2 base = tw[(2 * lane) & (N - 1)];
  float2 c = make_float2(1.0f, 0.0f);
#pragma unroll
  for (int k2 = 0; k2 < E; ++k2) {
    if (k2 > 0) c = ((k2 & 3) == 0) ? tw[(2 * lane * k2) & (N - 1)] : cm(c, base);
    w[k2] = c;
  }
}

template <int E>
__device__ __forceinline__ void four_step_first(float (&re)[E], float (&im)[E], const float2 (&w)[E], float2* sm,
                                                int r, int lane) {
  fft_reg<E>(re, im);
#pragma unroll
  for (int k2 = 0; k2 < E; ++k2) sm[(r * E + k2) * 33 + lane] = cm(make_float2(re[k2], im[k2]), w[k2]);
}

// RE = R E rows of the buffer are written; lanes above them repeat a row (and
// their results are not used), so the buffer needs only RE rows
template <int RE>
__device__ __forceinline__ void four_step_second(float (&ore)[32], float (&oim)[32], const float2* sm, int lane) {
  __syncwarp();
  const int src = lane & (RE - 1);
#pragma unroll
  for (int n1 = 0; n1 < 32; ++n1) {
    const float2 v = sm[src * 33 + n1];
    ore[n1] = v.x;
    oim[n1] = v.y;
  }
  __syncwarp();  // the buffer is free for the warp's next rows
  fft_reg<32>(ore, oim);
}

}  // namespace

// Forward transform of rows y0 .. y0 + R - 1 (those below Ny; R <= 32 / E)
// by one warp; sm: the warp's buffer of R E rows of 33.
template <int E, int R>
__device__ __forceinline__ void rfft_warp_rows(const PoissonArgs& a, int y0, float2* sm) {
  static_assert(R >= 1 && R * E <= 32, "rows per warp");
  const int lane = threadIdx.x & 31;
  constexpr int L = 32 * E, N = 2 * L;
  const float2* __restrict__ tw = static_cast<const float2*>(a.tw);
  const float nieps = -(float)a.inv_eps;
  float2 w[E];
  four_step_twiddles<E>(tw, lane, w);
  float myc0 = 0.0f;  // lane r keeps row r's constant
  for (int r = 0; r < R; ++r) {
    const int y = y0 + r;
    if (y >= a.Ny) break;
    const float2* rc2 = reinterpret_cast<const float2*>(static_cast<const float*>(a.rhoc) + (long long)y * a.P);
    const float *rdn, *rup;
    rhoc_partials<float>(a, y, rdn, rup);
    // A row constant c0 is taken out before the transform (the differences
    // are exact and small, so the rounding scales with the row's variation);
    // only the m = 0 bin depends on it, and it is restored there in
    // float-float.
    const float* row = reinterpret_cast<const float*>(rc2);
    float c0 = row[0];
    if (rdn) c0 += rdn[0];
    if (rup) c0 += rup[0];
    float re[E], im[E];
#pragma unroll
    for (int n2 = 0; n2 < E; ++n2) {
      float2 v = rc2[lane + 32 * n2];
      if (rdn) {
        const float2 d = reinterpret_cast<const float2*>(rdn)[lane + 32 * n2];
        v.x += d.x;
        v.y += d.y;
      }
      if (rup) {
        const float2 u = reinterpret_cast<const float2*>(rup)[lane + 32 * n2];
        v.x += u.x;
        v.y += u.y;
      }
      re[n2] = (v.x - c0) * nieps;
      im[n2] = (v.y - c0) * nieps;
    }
    four_step_first<E>(re, im, w, sm, r, lane);
    if (lane == r) myc0 = c0;
  }
  float xr[32], xi[32];
  four_step_second<R * E>(xr, xi, sm, lane);
  const int r = lane / E, k2 = lane & (E - 1), y = y0 + r;
  const bool live = r < R && y < a.Ny;
  const float c0 = __shfl_sync(0xffffffffu, myc0, r < R ? r : 0);
  if (k2 == 0 && live) {
    // m = 0 coefficient (Z0 sits in lane k2 = 0 of the row's group, k1 = 0),
    // float-float: (Re Z0 + Im Z0) + N c0 (-1/eps), the product exact by the
    // FMA two-product, N a power of two
    float s, e;
    two_sum_f(xr[0], xi[0], s, e);
    const float p = c0 * nieps, pe = fmaf(c0, nieps, -p);
    const float P = p * (float)N, PE = pe * (float)N;
    float h, l;
    two_sum_f(s, P, h, l);
    l += e + PE;
    two_sum_f(h, l, s, e);
    static_cast<float2*>(a.spec0)[y] = make_float2(s, e);
  }
  // untangle into the half spectrum: S[k] = E_k + W_N^k O_k,
  // E_k = (Z[k] + Z*[L-k]) / 2, O_k = (Z[k] - Z*[L-k]) / (2i); lane k2 of the
  // row's group holds k = k2 + E k1, whose partner L - k sits in the group's
  // lane (E - k2) mod E at 31 - k1 (k2 = 0: its own register (32 - k1) mod 32)
  float2* spec = static_cast<float2*>(a.spec) + (long long)(live ? y : 0) * a.Mp;
  const int partner = (lane & ~(E - 1)) | ((E - k2) & (E - 1));
  const float2 wk2 = tw[k2];
#pragma unroll
  for (int k1 = 0; k1 < 32; ++k1) {
    float pr = __shfl_sync(0xffffffffu, xr[31 - k1], partner);
    float pi = __shfl_sync(0xffffffffu, xi[31 - k1], partner);
    if (k2 == 0) {
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
    const int k = k2 + E * k1;
    if (live) spec[k] = (k == 0) ? make_float2(0.0f, 0.0f) : Sk;
  }
  if (k2 == 0 && live) spec[L] = make_float2(xr[0] - xi[0], 0.0f);  // Nyquist: Re Z0 - Im Z0
}

// Coefficient k of the half spectrum as the inverse transforms read it: phi_k,
// or with DX that of E_x = -d phi / dx, -i k_k phi_k with k_k = 2 pi k / N
// (N = 2L; the Nyquist coefficient k = L is dropped so that E_x is real).
template <bool DX>
__device__ __forceinline__ float2 spec_in(const float2* spec, int k, int L) {
  const float2 v = spec[k];
  if constexpr (!DX) {
    return v;
  } else {
    if (k == L) return make_float2(0.0f, 0.0f);
    const float kk = (3.14159265358979323846f / (float)L) * (float)k;
    return make_float2(kk * v.y, -kk * v.x);
  }
}

// Inverse transform of rows y0 .. y0 + R - 1 (those below Ny; R <= 32 / E)
// by one warp -> phi minus its row mean (DX: E_x).
template <int E, int R, bool DX = false>
__device__ __forceinline__ void irfft_warp_rows(const PoissonArgs& a, int y0, float2* sm) {
  static_assert(R >= 1 && R * E <= 32, "rows per warp");
  const int lane = threadIdx.x & 31;
  constexpr int L = 32 * E;
  const float2* __restrict__ tw = static_cast<const float2*>(a.tw);
  float2 w[E];
  four_step_twiddles<E>(tw, lane, w);
  // W_N^k for k = lane + 32 n2
  const float2 wl = tw[lane];
  float2 wk[E];
#pragma unroll
  for (int n2 = 0; n2 < E; ++n2) wk[n2] = cm(wl, tw[32 * n2]);
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int y = y0 + r;
    if (y >= a.Ny) break;
    const float2* spec = static_cast<const float2*>(a.spec) + (long long)y * a.Mp;
    // conj(Z[n]) for n = lane + 32 n2, Z[k] = E_k + i O_k,
    // E_k = (S[k] + S*[L-k]) / 2, O_k = (S[k] - S*[L-k]) / (2 W_N^k), S[0] := 0
    float re[E], im[E];
#pragma unroll
    for (int n2 = 0; n2 < E; ++n2) {
      const int k = lane + 32 * n2;
      const float2 sk = (k == 0) ? make_float2(0.0f, 0.0f) : spec_in<DX>(spec, k, L);
      const float2 sp = spec_in<DX>(spec, L - k, L);
      const float2 sc = make_float2(sp.x, -sp.y);
      const float2 Ev = make_float2(0.5f * (sk.x + sc.x), 0.5f * (sk.y + sc.y));
      const float2 Dv = make_float2(0.5f * (sk.x - sc.x), 0.5f * (sk.y - sc.y));
      const float2 O = cm(Dv, make_float2(wk[n2].x, -wk[n2].y));  // D / W^k
      re[n2] = Ev.x - O.y;                                        // Re(E + i O)
      im[n2] = -(Ev.y + O.x);                                     // -Im: conjugate
    }
    four_step_first<E>(re, im, w, sm, r, lane);
  }
  float xr[32], xi[32];
  four_step_second<R * E>(xr, xi, sm, lane);
  const int r = lane / E, k2 = lane & (E - 1), y = y0 + r;
  if (r < R && y < a.Ny) {
    float2* dphi2 = reinterpret_cast<float2*>(static_cast<float*>(DX ? a.ex : a.dphi) + (long long)y * a.P);
    const float inL = 1.0f / (float)L;
#pragma unroll
    for (int k1 = 0; k1 < 32; ++k1) dphi2[k2 + E * k1] = make_float2(xr[k1] * inL, -xi[k1] * inL);
  }
}

// In-register 16-point forward DFT, natural order in and out, as 4 x 4:
// X[k2 + 4 k1] = sum_n1 W_16^(n1 k2) W_4^(n1 k1) sum_n2 v[n1 + 4 n2] W_4^(n2 k2).
// The twiddles are literal constants, so trivial products fold away.
// The sums and differences on (re, im) pairs use the packed two-float adds of
// this architecture (each pair rounded exactly as two scalar adds, so the
// results are unchanged): 2048 x 1680 steps 116.8 against 117.9 us, with the
// CTA transforms bounded to 80 registers so that their grid stays one wave.
__device__ __forceinline__ void dft4(float& r0, float& i0, float& r1, float& i1, float& r2, float& i2, float& r3,
                                     float& i3) {
  const float2 a0 = make_float2(r0, i0), a1 = make_float2(r1, i1), a2 = make_float2(r2, i2),
               a3 = make_float2(r3, i3);
  const float2 s = __fadd2_rn(a0, a2), d = __fadd2_rn(a0, make_float2(-a2.x, -a2.y));
  const float2 t = __fadd2_rn(a1, a3), u = __fadd2_rn(a1, make_float2(-a3.x, -a3.y));
  const float2 b0 = __fadd2_rn(s, t), b2 = __fadd2_rn(s, make_float2(-t.x, -t.y));
  const float2 b1 = __fadd2_rn(d, make_float2(u.y, -u.x));  // (d) - i (u)
  const float2 b3 = __fadd2_rn(d, make_float2(-u.y, u.x));  // (d) + i (u)
  r0 = b0.x;
  i0 = b0.y;
  r1 = b1.x;
  i1 = b1.y;
  r2 = b2.x;
  i2 = b2.y;
  r3 = b3.x;
  i3 = b3.y;
}

template <int M>  // multiply by W_16^M = exp(-2 pi i M / 16), M in {0..9}
__device__ __forceinline__ void mul_w16(float& re, float& im) {
  constexpr float c1 = 0.92387953251128675613f, s1 = 0.38268343236508977173f, h = 0.70710678118654752440f;
  float r = re, i = im;
  if constexpr (M == 0) return;
  if constexpr (M == 1) { re = r * c1 + i * s1; im = i * c1 - r * s1; }
  if constexpr (M == 2) { re = (r + i) * h; im = (i - r) * h; }
  if constexpr (M == 3) { re = r * s1 + i * c1; im = i * s1 - r * c1; }
  if constexpr (M == 4) { re = i; im = -r; }
  if constexpr (M == 6) { re = (i - r) * h; im = -(r + i) * h; }
  if constexpr (M == 9) { re = -r * c1 - i * s1; im = r * s1 - i * c1; }
}

__device__ __forceinline__ void fft16(float (&re)[16], float (&im)[16]) {
#pragma unroll
  for (int n1 = 0; n1 < 4; ++n1)
    dft4(re[n1], im[n1], re[n1 + 4], im[n1 + 4], re[n1 + 8], im[n1 + 8], re[n1 + 12], im[n1 + 12]);
  // T[n1][k2] sits at n1 + 4 k2; twiddle W_16^(n1 k2)
  mul_w16<1>(re[5], im[5]);
  mul_w16<2>(re[9], im[9]);
  mul_w16<3>(re[13], im[13]);
  mul_w16<2>(re[6], im[6]);
  mul_w16<4>(re[10], im[10]);
  mul_w16<6>(re[14], im[14]);
  mul_w16<3>(re[7], im[7]);
  mul_w16<6>(re[11], im[11]);
  mul_w16<9>(re[15], im[15]);
  float orr[16], oi[16];
#pragma unroll
  for (int k2 = 0; k2 < 4; ++k2) {
    float r0 = re[4 * k2], i0 = im[4 * k2], r1 = re[4 * k2 + 1], i1 = im[4 * k2 + 1];
    float r2 = re[4 * k2 + 2], i2 = im[4 * k2 + 2], r3 = re[4 * k2 + 3], i3 = im[4 * k2 + 3];
    dft4(r0, i0, r1, i1, r2, i2, r3, i3);
    orr[k2] = r0;
    oi[k2] = i0;
    orr[k2 + 4] = r1;
    oi[k2 + 4] = i1;
    orr[k2 + 8] = r2;
    oi[k2 + 8] = i2;
    orr[k2 + 12] = r3;
    oi[k2 + 12] = i3;
  }
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    re[k] = orr[k];
    im[k] = oi[k];
  }
}

// ---------------------------------------------------------------------------
// CTA-per-row transforms for rows of N = 2048 reals (L = 1024 complex): 64
// threads, 16 values each, L = 16 x 16 x 4.  Shorter dependent chains per
// thread than the warp-per-row form, for the same total work.
//
// With n = n0 + 64 n1 and k = k1 + 16 k0 (n0 = thread t):
//   Z[k1 + 16 k0] = sum_n0 W_L^(n0 k1) W_64^(n0 k0) sum_n1 z[n0 + 64 n1] W_16^(n1 k1)
// pass A: thread t, 16-point DFT over n1, twiddle W_L^(t k1), to shared
// memory as sA[k1][t];
// pass B: the 64-point DFT over n0 for each k1 by the 4 threads u = 4 k1 + q
// (n0 = q + 4 b, k0 = c + 16 d): thread q, 16-point DFT over b, twiddle
// W_64^(q c), exchange within the 4 threads, and a 4-point DFT over q:
// thread (k1, q) ends with Z[k1 + 16 c + 256 d] for c = 4 q + i, i, d < 4.
constexpr int kCtaL = 1024;
constexpr int kCtaT = 64;
constexpr int kPitchA = 68;  // float2 per k1 row of sA / sB (64 + 4: no bank conflicts)
constexpr int kSmemCta = 16 * kPitchA;  // float2; sA, sB and sZ share it

__device__ __forceinline__ int zpad(int k) { return k + 4 * (k >> 6); }

// Forward 1024-point complex DFT of the CTA's row: on entry thread t holds
// z[t + 64 n1] in (re[n1], im[n1]); on return thread (k1 = t / 4, q = t % 4)
// holds Z[k1 + 16 (4 q + i) + 256 d] in (zr[4 d + i], zi[4 d + i]).
// The first pass's twiddles W_1024^(t k1), k1 = 1 .. 15 (table [k1][t] after
// the first 2 L entries), loaded before the row so that their latency
// overlaps the row's (119.7 against 122.3 us per 2048 x 1680 step; loading
// the forward's untangle twiddles early too helped before the packed adds,
// but with them it spills at the 80-register bound: 117.0 against 115.6 us).
__device__ __forceinline__ void cta_twiddles(const float2* __restrict__ tw, float2 (&w1)[16]) {
  const float2* __restrict__ tw1 = tw + 2 * kCtaL;
  w1[0] = make_float2(1.0f, 0.0f);
#pragma unroll
  for (int k1 = 1; k1 < 16; ++k1) w1[k1] = __ldg(tw1 + k1 * kCtaT + threadIdx.x);
}

__device__ __forceinline__ void cta_fft1024(float (&re)[16], float (&im)[16], float (&zr)[16], float (&zi)[16],
                                            const float2* __restrict__ tw, const float2 (&w1)[16], float2* sm) {
  const int t = threadIdx.x;
  fft16(re, im);
#pragma unroll
  for (int k1 = 0; k1 < 16; ++k1) {
    float2 v = make_float2(re[k1], im[k1]);
    if (k1 > 0) v = cm(v, w1[k1]);
    sm[k1 * kPitchA + t] = v;
  }
  __syncthreads();
  const int k1 = t >> 2, q = t & 3;
  float br[16], bi[16];
#pragma unroll
  for (int b = 0; b < 16; ++b) {
    const float2 v = sm[k1 * kPitchA + q + 4 * b];
    br[b] = v.x;
    bi[b] = v.y;
  }
  fft16(br, bi);
  __syncwarp();  // the group's rows of sA are read before sB overwrites them
#pragma unroll
  for (int c = 0; c < 16; ++c) {
    float2 v = make_float2(br[c], bi[c]);
    if (c > 0 && q > 0) v = cm(v, __ldg(tw + 32 * q * c));  // W_64^(q c)
    sm[k1 * kPitchA + 4 * c + (q ^ (c >> 2))] = v;
  }
  __syncwarp();
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    float2 v[4];
#pragma unroll
    for (int qq = 0; qq < 4; ++qq) v[qq] = sm[k1 * kPitchA + 4 * (4 * q + i) + (qq ^ q)];
    // 4-point DFT over qq, W_4 = -i (packed two-float adds)
    float zr0, zi0, zr1, zi1, zr2, zi2, zr3, zi3;
    zr0 = v[0].x, zi0 = v[0].y, zr1 = v[1].x, zi1 = v[1].y;
    zr2 = v[2].x, zi2 = v[2].y, zr3 = v[3].x, zi3 = v[3].y;
    dft4(zr0, zi0, zr1, zi1, zr2, zi2, zr3, zi3);
    zr[i] = zr0;
    zi[i] = zi0;
    zr[4 + i] = zr1;  // d02 - i d13
    zi[4 + i] = zi1;
    zr[8 + i] = zr2;
    zi[8 + i] = zi2;
    zr[12 + i] = zr3;  // d02 + i d13
    zi[12 + i] = zi3;
  }
}

// Forward transform of row y (N = 2048) by one CTA of 64 threads.
__global__ void __launch_bounds__(kCtaT, 12) k_rfft_cta(PoissonArgs a) {
  __shared__ float2 sm[kSmemCta];
  const int t = threadIdx.x, y = blockIdx.x;
  const float2* __restrict__ tw = static_cast<const float2*>(a.tw);
  // the twiddle tables are constant: loaded before the wait for the step
  // kernel that writes the charge density (programmatic dependent launch)
  float2 w1[16];
  cta_twiddles(tw, w1);
  grid_dep_wait();
  grid_dep_launch();
  const float* row = static_cast<const float*>(a.rhoc) + (long long)y * a.P;
  const float2* rc2 = reinterpret_cast<const float2*>(row);
  const float *rdn, *rup;
  rhoc_partials<float>(a, y, rdn, rup);
  const float nieps = -(float)a.inv_eps;
  // A row constant c0 is taken out before the transform: the differences are
  // exact (Sterbenz) and small, so the transform's rounding scales with the
  // row's variation, and only the m = 0 bin depends on c0.
  float c0 = __ldg(row);
  if (rdn) c0 += __ldg(rdn);
  if (rup) c0 += __ldg(rup);
  float re[16], im[16];
#pragma unroll
  for (int n1 = 0; n1 < 16; ++n1) {
    float2 v = rc2[t + 64 * n1];
    if (rdn) {
      const float2 d = reinterpret_cast<const float2*>(rdn)[t + 64 * n1];
      v.x += d.x;
      v.y += d.y;
    }
    if (rup) {
      const float2 u = reinterpret_cast<const float2*>(rup)[t + 64 * n1];
      v.x += u.x;
      v.y += u.y;
    }
    re[n1] = (v.x - c0) * nieps;
    im[n1] = (v.y - c0) * nieps;
  }
  float zr[16], zi[16];
  cta_fft1024(re, im, zr, zi, tw, w1, sm);
  if (t == 0) {
    // m = 0 coefficient, float-float: (Re Z0 + Im Z0) + N c0 (-1/eps), the
    // product exact by the FMA two-product, N a power of two
    float s, e;
    two_sum_f(zr[0], zi[0], s, e);
    const float p = c0 * nieps, pe = fmaf(c0, nieps, -p);
    const float P = p * 2048.0f, PE = pe * 2048.0f;
    float h, l;
    two_sum_f(s, P, h, l);
    l += e + PE;
    two_sum_f(h, l, s, e);
    static_cast<float2*>(a.spec0)[y] = make_float2(s, e);
  }
  __syncthreads();  // every thread has read its part of sB
  const int k1 = t >> 2, q = t & 3;
#pragma unroll
  for (int d = 0; d < 4; ++d)
#pragma unroll
    for (int i = 0; i < 4; ++i)
      sm[zpad(k1 + 16 * (4 * q + i) + 256 * d)] = make_float2(zr[4 * d + i], zi[4 * d + i]);
  __syncthreads();
  // untangle, k and L - k together: S[k] = E_k + W_N^k O_k with
  // E_k = (Z[k] + Z*[L-k]) / 2, O_k = (Z[k] - Z*[L-k]) / (2i); for L - k the
  // roles of the two values swap and W_N^(L-k) = -conj(W_N^k)
  float2* spec = static_cast<float2*>(a.spec) + (long long)y * a.Mp;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int k = t + 64 * j;  // 0 .. 511
    const float2 zk = sm[zpad(k)];
    const float2 zp = sm[zpad((kCtaL - k) & (kCtaL - 1))];
    const float2 wk = __ldg(tw + k);
    // E = (zk + conj zp) / 2, D = (zk - conj zp) / 2, O = -i D
    const float Er = 0.5f * (zk.x + zp.x), Ei = 0.5f * (zk.y - zp.y);
    const float Dr = 0.5f * (zk.x - zp.x), Di = 0.5f * (zk.y + zp.y);
    // S[k] = E + w (Di - i Dr)
    const float2 Sk = make_float2(Er + wk.x * Di + wk.y * Dr, Ei + wk.y * Di - wk.x * Dr);
    // S[L-k] = E' + w' O' with E' = conj(E), D' = -conj(D), O' = -i D' = Di + i Dr,
    // w' = -conj(w)
    const float2 Sp = make_float2(Er - wk.x * Di - wk.y * Dr, -Ei + wk.y * Di - wk.x * Dr);
    if (k == 0) {
      spec[0] = make_float2(0.0f, 0.0f);
      spec[kCtaL] = make_float2(zk.x - zk.y, 0.0f);  // Nyquist: Re Z0 - Im Z0
    } else {
      spec[k] = Sk;
      spec[kCtaL - k] = Sp;
    }
  }
  if (t == 0) {  // k = L/2 is its own partner: S = conj(Z[L/2]) (W_N^(L/2) = -i)
    const float2 zk = sm[zpad(kCtaL / 2)];
    spec[kCtaL / 2] = make_float2(zk.x, -zk.y);
  }
}

// Inverse transform of row y (N = 2048) -> phi minus its row mean (DX: E_x).
template <bool DX = false>
__global__ void __launch_bounds__(kCtaT, 12) k_irfft_cta(PoissonArgs a) {
  __shared__ float2 sm[kSmemCta];
  grid_dep_wait();
  grid_dep_launch();
  const int t = threadIdx.x, y = blockIdx.x;
  const float2* __restrict__ tw = static_cast<const float2*>(a.tw);
  const float2* spec = static_cast<const float2*>(a.spec) + (long long)y * a.Mp;
  float2 w1[16];
  cta_twiddles(tw, w1);
  // conj(Z[n]) for n = t + 64 n1, Z[k] = E_k + i O_k,
  // E_k = (S[k] + S*[L-k]) / 2, O_k = (S[k] - S*[L-k]) / (2 W_N^k), S[0] := 0
  float re[16], im[16];
#pragma unroll
  for (int n1 = 0; n1 < 16; ++n1) {
    const int k = t + 64 * n1;
    const float2 sk = (k == 0) ? make_float2(0.0f, 0.0f) : spec_in<DX>(spec, k, kCtaL);
    const float2 sp = spec_in<DX>(spec, kCtaL - k, kCtaL);
    const float2 sc = make_float2(sp.x, -sp.y);
    const float2 Ev = make_float2(0.5f * (sk.x + sc.x), 0.5f * (sk.y + sc.y));
    const float2 Dv = make_float2(0.5f * (sk.x - sc.x), 0.5f * (sk.y - sc.y));
    const float2 wk = __ldg(tw + k);
    const float2 O = cm(Dv, make_float2(wk.x, -wk.y));
    re[n1] = Ev.x - O.y;
    im[n1] = -(Ev.y + O.x);
  }
  float zr[16], zi[16];
  cta_fft1024(re, im, zr, zi, tw, w1, sm);
  float2* dphi2 = reinterpret_cast<float2*>(static_cast<float*>(DX ? a.ex : a.dphi) + (long long)y * a.P);
  const float inL = 1.0f / (float)kCtaL;
  const int k1 = t >> 2, q = t & 3;
#pragma unroll
  for (int d = 0; d < 4; ++d)
#pragma unroll
    for (int i = 0; i < 4; ++i)
      dphi2[k1 + 16 * (4 * q + i) + 256 * d] = make_float2(zr[4 * d + i] * inL, -zi[4 * d + i] * inL);
}

// one warp per row: a single run's transforms are bound by latency, and
// more warps in flight beat fuller ones (128 x 104: 16.1 against 28.7 us
// per step with 32/E rows per warp)
template <int E>
__global__ void __launch_bounds__(128) k_rfft_warp(PoissonArgs a) {
  __shared__ float2 smem[4][E * 33];
  grid_dep_wait();
  grid_dep_launch();
  const int warp = threadIdx.x >> 5;
  const int y = blockIdx.x * 4 + warp;
  if (y < a.Ny) rfft_warp_rows<E, 1>(a, y, smem[warp]);
}

template <int E, bool DX = false>
__global__ void __launch_bounds__(128) k_irfft_warp(PoissonArgs a) {
  __shared__ float2 smem[4][E * 33];
  grid_dep_wait();
  grid_dep_launch();
  const int warp = threadIdx.x >> 5;
  const int y = blockIdx.x * 4 + warp;
  if (y < a.Ny) irfft_warp_rows<E, 1, DX>(a, y, smem[warp]);
}

// Batch: warps of a fixed grid take row items (run, y0: the run's rows y0 ..
// y0 + 2048/Nx - 1); the row length picks the transform shape.
// EMAX: the widest row shape of the batch (Nx / 64); narrower batches get an
// instance with fewer registers (the inverse up to EMAX = 8 at most 102:
// five CTAs per SM), so more row FFTs run at once.
template <bool INV, int EMAX>
__device__ __forceinline__ void batch_fft_body(const BatchTables& t, int step) {
  __shared__ float2 smem[4][32 * 33];
  const int warp = threadIdx.x >> 5;
  const int n = t.counts[2];
  int* counter = t.work + (INV ? 3 : 1);
  for (int it = next_item_warp(counter); it < n; it = next_item_warp(counter)) {
    const int2 w = t.row_items[it];
    const BatchRunDesc& rd = t.runs[w.x];
    if (step >= rd.remaining) continue;
    const PoissonArgs a = rd.pa;
    float2* sm = smem[warp];
    switch (rd.E) {
      case 1: INV ? irfft_warp_rows<1, 32>(a, w.y, sm) : rfft_warp_rows<1, 32>(a, w.y, sm); break;
      case 2:
        if constexpr (EMAX >= 2) INV ? irfft_warp_rows<2, 16>(a, w.y, sm) : rfft_warp_rows<2, 16>(a, w.y, sm);
        break;
      case 4:
        if constexpr (EMAX >= 4) INV ? irfft_warp_rows<4, 8>(a, w.y, sm) : rfft_warp_rows<4, 8>(a, w.y, sm);
        break;
      case 8:
        if constexpr (EMAX >= 8) INV ? irfft_warp_rows<8, 4>(a, w.y, sm) : rfft_warp_rows<8, 4>(a, w.y, sm);
        break;
      case 16:
        if constexpr (EMAX >= 16) INV ? irfft_warp_rows<16, 2>(a, w.y, sm) : rfft_warp_rows<16, 2>(a, w.y, sm);
        break;
      default:
        if constexpr (EMAX >= 32) INV ? irfft_warp_rows<32, 1>(a, w.y, sm) : rfft_warp_rows<32, 1>(a, w.y, sm);
        break;
    }
  }
}

template <int EMAX>
__global__ void __launch_bounds__(128) k_batch_rfft(BatchTables t, int step) {
  grid_dep_wait();  // programmatic dependent launch (t.pdl): the previous phase has ended
  grid_dep_launch();
  batch_fft_body<false, EMAX>(t, step);
}

template <int EMAX>
__global__ void __launch_bounds__(128) k_batch_irfft(BatchTables t, int step) {
  grid_dep_wait();  // programmatic dependent launch (t.pdl): the previous phase has ended
  grid_dep_launch();
  batch_fft_body<true, EMAX>(t, step);
}

template <int EMAX>
__global__ void __launch_bounds__(128, 5) k_batch_irfft_narrow(BatchTables t, int step) {
  grid_dep_wait();  // programmatic dependent launch (t.pdl): the previous phase has ended
  grid_dep_launch();
  batch_fft_body<true, EMAX>(t, step);
}

cudaError_t launch_batch_rfft(const BatchTables& t, int step, int grid, cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  switch (t.emax) {
    case 1: e = launch_ex((t.pdl & 1) != 0, k_batch_rfft<1>, dim3(grid), dim3(128), 0, s, t, step); break;
    case 2: e = launch_ex((t.pdl & 1) != 0, k_batch_rfft<2>, dim3(grid), dim3(128), 0, s, t, step); break;
    case 4: e = launch_ex((t.pdl & 1) != 0, k_batch_rfft<4>, dim3(grid), dim3(128), 0, s, t, step); break;
    case 8: e = launch_ex((t.pdl & 1) != 0, k_batch_rfft<8>, dim3(grid), dim3(128), 0, s, t, step); break;
    case 16: e = launch_ex((t.pdl & 1) != 0, k_batch_rfft<16>, dim3(grid), dim3(128), 0, s, t, step); break;
    default: e = launch_ex((t.pdl & 1) != 0, k_batch_rfft<32>, dim3(grid), dim3(128), 0, s, t, step); break;
  }
  return e;
}

cudaError_t launch_batch_irfft(const BatchTables& t, int step, int grid, cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  switch (t.emax) {
    case 1: e = launch_ex((t.pdl & 4) != 0, k_batch_irfft_narrow<1>, dim3(grid), dim3(128), 0, s, t, step); break;
    case 2: e = launch_ex((t.pdl & 4) != 0, k_batch_irfft_narrow<2>, dim3(grid), dim3(128), 0, s, t, step); break;
    case 4: e = launch_ex((t.pdl & 4) != 0, k_batch_irfft_narrow<4>, dim3(grid), dim3(128), 0, s, t, step); break;
    case 8: e = launch_ex((t.pdl & 4) != 0, k_batch_irfft_narrow<8>, dim3(grid), dim3(128), 0, s, t, step); break;
    case 16: e = launch_ex((t.pdl & 4) != 0, k_batch_irfft<16>, dim3(grid), dim3(128), 0, s, t, step); break;
    default: e = launch_ex((t.pdl & 4) != 0, k_batch_irfft<32>, dim3(grid), dim3(128), 0, s, t, step); break;
  }
  return e;
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
    case 64: return launch_ex((a.pdl & 1) != 0, k_rfft_warp<1>, dim3(g), dim3(128), 0, s, a);
    case 128: return launch_ex((a.pdl & 1) != 0, k_rfft_warp<2>, dim3(g), dim3(128), 0, s, a);
    case 256: return launch_ex((a.pdl & 1) != 0, k_rfft_warp<4>, dim3(g), dim3(128), 0, s, a);
    case 512: return launch_ex((a.pdl & 1) != 0, k_rfft_warp<8>, dim3(g), dim3(128), 0, s, a);
    case 1024: return launch_ex((a.pdl & 1) != 0, k_rfft_warp<16>, dim3(g), dim3(128), 0, s, a);
    case 2048:
      if (a.fft_cta) return launch_ex((a.pdl & 1) != 0, k_rfft_cta, dim3(a.Ny), dim3(kCtaT), 0, s, a);
      return launch_ex((a.pdl & 1) != 0, k_rfft_warp<32>, dim3(g), dim3(128), 0, s, a);
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <bool DX>
cudaError_t irfft_warp_n(const PoissonArgs& a, cudaStream_t s) {
  const unsigned g = (unsigned)((a.Ny + 3) / 4);
  switch (a.Nx) {
    case 64: return launch_ex((a.pdl & 4) != 0, k_irfft_warp<1, DX>, dim3(g), dim3(128), 0, s, a);
    case 128: return launch_ex((a.pdl & 4) != 0, k_irfft_warp<2, DX>, dim3(g), dim3(128), 0, s, a);
    case 256: return launch_ex((a.pdl & 4) != 0, k_irfft_warp<4, DX>, dim3(g), dim3(128), 0, s, a);
    case 512: return launch_ex((a.pdl & 4) != 0, k_irfft_warp<8, DX>, dim3(g), dim3(128), 0, s, a);
    case 1024: return launch_ex((a.pdl & 4) != 0, k_irfft_warp<16, DX>, dim3(g), dim3(128), 0, s, a);
    case 2048:
      if (a.fft_cta) return launch_ex((a.pdl & 4) != 0, k_irfft_cta<DX>, dim3(a.Ny), dim3(kCtaT), 0, s, a);
      return launch_ex((a.pdl & 4) != 0, k_irfft_warp<32, DX>, dim3(g), dim3(128), 0, s, a);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_irfft_warp(const PoissonArgs& a, cudaStream_t s) { return irfft_warp_n<false>(a, s); }

cudaError_t launch_irfft_warp_dx(const PoissonArgs& a, cudaStream_t s) { return irfft_warp_n<true>(a, s); }

}  // namespace ehd

// k_misc.cu -- kernels off the time-stepping path: macroscopic fields
// (Eqs. 5-7, E = -grad phi) in FP64 for output, FP64 state reductions for the
// conservation diagnostics, storage conversion for load/save, and the initial
// state (hydrostatic profile of Eqs. 27-28 plus the Eq. 29 rolls).
#include <type_traits>

#include "ehd_dev.cuh"

namespace ehd {

namespace {

__device__ __forceinline__ double wgt(int i) { return i == 0 ? kW0 : (i < 5 ? kW1 : kW2); }
__device__ __forceinline__ int cxi(int i) { return (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0); }
__device__ __forceinline__ int cyi(int i) { return (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0); }

struct Macro {
  double rho, ux, uy, rc, phi, Ex, Ey;
};

template <class S, class R>
__device__ Macro macro_at(const FieldArgs& a, int x, int y) {
  const long long c = (long long)y * a.P + x;
  const S* f = static_cast<const S*>(a.f);
  const S* g = static_cast<const S*>(a.g);
  const double sy = a.rch ? (double)a.rch[y] : 0.0;
  const double sfy = a.fb + a.fd * y;
  double rho = 0, jx = 0, jy = 0, rc = 0;
  for (int i = 0; i < 9; ++i) {
    const double fi = (double)Store<S>::template ld<R>(f + i * a.plane + c) + wgt(i) * sfy;
    const double gi = (double)Store<S>::template ld<R>(g + i * a.plane + c) +
                      (a.base_g ? a.base_g[i * a.Ny + y] : wgt(i) * sy);
    rho += fi;
    jx += cxi(i) * fi;
    jy += cyi(i) * fi;
    rc += gi;
  }
  const R* dphi = static_cast<const R*>(a.dphi);
  const int xl = (x == 0) ? a.Nx - 1 : x - 1, xr = (x == a.Nx - 1) ? 0 : x + 1;
  const double gw = (a.wall_mode == 0) ? -1.0 : 0.0;
  const double pc = (double)dphi[c];
  const double pS = (y > 0) ? (double)dphi[c - a.P] : gw * pc;
  const double pN = (y < a.Ny - 1) ? (double)dphi[c + a.P] : gw * pc;
  Macro m;
  m.Ex = a.ex ? (double)static_cast<const R*>(a.ex)[c]
              : -0.5 * ((double)dphi[c - x + xr] - (double)dphi[c - x + xl]);
  m.Ey = (double)static_cast<const R*>(a.Ebar)[y] - 0.5 * (pN - pS) + (a.EB ? a.EB[y] : 0.0);
  m.phi = load_phibar<R>(a.phibar, y) + pc + (a.phiB ? a.phiB[y] : 0.0);
  m.rho = rho;
  m.rc = rc;
  m.ux = (jx + 0.5 * rc * m.Ex) / rho;
  m.uy = (jy + 0.5 * rc * m.Ey) / rho;
  return m;
}

}  // namespace

template <class S, class R>
__global__ void k_fields(FieldArgs a, unsigned mask, double* out) {
  const long long n = (long long)a.Nx * a.Ny;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(k % a.Nx), y = (int)(k / a.Nx);
    const Macro m = macro_at<S, R>(a, x, y);
    const double v[7] = {m.rho, m.ux, m.uy, m.rc, m.phi, m.Ex, m.Ey};
    int o = 0;
    for (int b = 0; b < 7; ++b)
      if (mask & (1u << b)) out[(long long)(o++) * n + k] = v[b];
  }
}

// Per-block FP64 partials: mass, charge, kinetic energy, max|u_y|, max|u|,
// non-finite count; then one block adds the partials in index order.
constexpr int kRedBlocks = 304;
constexpr int kRedThreads = 256;

template <class S, class R>
__global__ void __launch_bounds__(kRedThreads) k_reduce_state(FieldArgs a, double* part) {
  __shared__ double sm[kRedThreads / 32][6];
  const long long n = (long long)a.Nx * a.Ny;
  double mass = 0, charge = 0, ke = 0, muy = 0, mu = 0, nbad = 0;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(k % a.Nx), y = (int)(k / a.Nx);
    const Macro m = macro_at<S, R>(a, x, y);
    if (!isfinite(m.rho) || !isfinite(m.rc)) {
      nbad += 1.0;
      continue;
    }
    mass += m.rho;
    charge += m.rc;
    const double u2 = m.ux * m.ux + m.uy * m.uy;
    ke += 0.5 * m.rho * u2;
    muy = fmax(muy, fabs(m.uy));
    mu = fmax(mu, sqrt(u2));
  }
  double v[6] = {mass, charge, ke, muy, mu, nbad};
  for (int q = 0; q < 6; ++q) {
    for (int o = 16; o > 0; o >>= 1) {
      const double t = __shfl_down_sync(0xffffffffu, v[q], o);
      v[q] = (q == 3 || q == 4) ? fmax(v[q], t) : v[q] + t;
    }
  }
  if ((threadIdx.x & 31) == 0)
    for (int q = 0; q < 6; ++q) sm[threadIdx.x >> 5][q] = v[q];
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int q = 0; q < 6; ++q) {
      double t = sm[0][q];
      for (int w = 1; w < kRedThreads / 32; ++w) t = (q == 3 || q == 4) ? fmax(t, sm[w][q]) : t + sm[w][q];
      part[blockIdx.x * 6 + q] = t;
    }
  }
}

__global__ void k_reduce_final(const double* part, int nblk, double* out, int* err) {
  if (threadIdx.x != 0) return;
  double t[6] = {0, 0, 0, 0, 0, 0};
  for (int b = 0; b < nblk; ++b)
    for (int q = 0; q < 6; ++q) t[q] = (q == 3 || q == 4) ? fmax(t[q], part[b * 6 + q]) : t[q] + part[b * 6 + q];
  for (int q = 0; q < 6; ++q) out[q] = t[q];
  if (t[5] > 0) atomicOr(err, 1);
}

// value_stored = value - shift_w (rch[y] + c0 + c1 y) - brow[y]   (rch, brow may be null)
template <class S>
__global__ void k_load_plane(const double* src, S* dst, int Nx, int Ny, int P, double shift_w, const float* rch,
                             double c0, double c1, const double* brow) {
  const long long n = (long long)Nx * Ny;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(k % Nx), y = (int)(k / Nx);
    const double sh = shift_w * ((rch ? (double)rch[y] : 0.0) + c0 + c1 * y) + (brow ? brow[y] : 0.0);
    Store<S>::st(dst + (long long)y * P + x, src[k] - sh);
  }
}

template <class S>
__global__ void k_save_plane(const S* src, double* dst, int Nx, int Ny, int P, double shift_w, const float* rch,
                             double c0, double c1, const double* brow) {
  const long long n = (long long)Nx * Ny;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(k % Nx), y = (int)(k / Nx);
    const double sh = shift_w * ((rch ? (double)rch[y] : 0.0) + c0 + c1 * y) + (brow ? brow[y] : 0.0);
    dst[k] = Store<S>::template ld<double>(src + (long long)y * P + x) + sh;
  }
}

// Initial state: f = f^eq(rho_h(y), u - F_h/(2 rho) e_y) so that Eq. 7 returns
// the Eq. 29 velocity u under the hydrostatic force, g = g^eq(rho_c,h(y),
// u + mu_b E_h(y) e_y).  The rolls are separable: u_x = sY(y) Sx(x),
// u_y = (cY(y) - 1) Cy(x), with the sums over modes precomputed on the host.
template <class S>
__global__ void k_init(const double* rho_h, const double* rc_h, const double* Eh, const double* sY, const double* cY,
                       const double* Sx, const double* Cy, double Fh, double mub, S* f, S* g, int Nx, int Ny, int P,
                       const float* rch, double fb, double fd, const double* base_g) {
  const long long n = (long long)Nx * Ny;
  const long long pl = (long long)Ny * P;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(k % Nx), y = (int)(k / Nx);
    const double rho = rho_h[y], rc = rc_h[y];
    const double ux = sY[y] * Sx[x], uy = (cY[y] - 1.0) * Cy[x];
    const double fx = ux, fy = uy - 0.5 * Fh / rho;
    const double gx = ux, gy = uy + mub * Eh[y];
    const double fu2 = fx * fx + fy * fy, gu2 = gx * gx + gy * gy;
    const double sy = rch ? (double)rch[y] : 0.0;
    const double sfy = fb + fd * y;
    const long long c = (long long)y * P + x;
    for (int i = 0; i < 9; ++i) {
      const double w = wgt(i);
      const double fc = cxi(i) * fx + cyi(i) * fy;
      const double gc = cxi(i) * gx + cyi(i) * gy;
      const double feq = w * rho * (1.0 + 3.0 * fc + 4.5 * fc * fc - 1.5 * fu2);
      const double geq = w * rc * (1.0 + 3.0 * gc + 4.5 * gc * gc - 1.5 * gu2);
      Store<S>::st(f + i * pl + c, feq - w * sfy);
      Store<S>::st(g + i * pl + c, geq - (base_g ? base_g[i * Ny + y] : w * sy));
    }
  }
}

// ---------------------------------------------------------------- launch ---
namespace {
constexpr int kGrid = 1216;  // 8 x 152 SMs
constexpr int kBlock = 256;

template <class Fn>
cudaError_t by_storage(int storage, bool real_f64, Fn&& fn) {
  if (real_f64) return storage == 0 ? fn((double*)nullptr, (double*)nullptr) : cudaErrorInvalidValue;
  switch (storage) {
    case 0: return fn((double*)nullptr, (float*)nullptr);
    case 1: return fn((float*)nullptr, (float*)nullptr);
    case 2: return fn((__nv_bfloat16*)nullptr, (float*)nullptr);
    case 3: return fn((__half*)nullptr, (float*)nullptr);
  }
  return cudaErrorInvalidValue;
}
}  // namespace

cudaError_t launch_fields(const FieldArgs& a, int storage, bool real_f64, unsigned mask, double* out,
                          cudaStream_t s) {
  return by_storage(storage, real_f64, [&](auto* sp, auto* rp) {
    using S = std::remove_pointer_t<decltype(sp)>;
    using R = std::remove_pointer_t<decltype(rp)>;
    k_fields<S, R><<<kGrid, kBlock, 0, s>>>(a, mask, out);
    return cudaGetLastError();
  });
}

int reduce_state_blocks() { return kRedBlocks; }

cudaError_t launch_reduce_state(const FieldArgs& a, int storage, bool real_f64, double* part, int nblk, double* out,
                                int* err, cudaStream_t s) {
  cudaError_t e = by_storage(storage, real_f64, [&](auto* sp, auto* rp) {
    using S = std::remove_pointer_t<decltype(sp)>;
    using R = std::remove_pointer_t<decltype(rp)>;
    k_reduce_state<S, R><<<nblk, kRedThreads, 0, s>>>(a, part);
    return cudaGetLastError();
  });
  if (e != cudaSuccess) return e;
  k_reduce_final<<<1, 32, 0, s>>>(part, nblk, out, err);
  return cudaGetLastError();
}

cudaError_t launch_load_plane(const double* src, void* dst, int storage, int Nx, int Ny, int P, double shift_w,
                              const float* rch, double c0, double c1, const double* brow, cudaStream_t s) {
  return by_storage(storage, false, [&](auto* sp, auto*) {
    using S = std::remove_pointer_t<decltype(sp)>;
    k_load_plane<S><<<kGrid, kBlock, 0, s>>>(src, static_cast<S*>(dst), Nx, Ny, P, shift_w, rch, c0, c1, brow);
    return cudaGetLastError();
  });
}

cudaError_t launch_save_plane(const void* src, double* dst, int storage, int Nx, int Ny, int P, double shift_w,
                              const float* rch, double c0, double c1, const double* brow, cudaStream_t s) {
  return by_storage(storage, false, [&](auto* sp, auto*) {
    using S = std::remove_pointer_t<decltype(sp)>;
    k_save_plane<S><<<kGrid, kBlock, 0, s>>>(static_cast<const S*>(src), dst, Nx, Ny, P, shift_w, rch, c0, c1,
                                             brow);
    return cudaGetLastError();
  });
}

cudaError_t launch_init(const double* rho_h, const double* rc_h, const double* Eh, const double* sY,
                        const double* cY, const double* Sx, const double* Cy, double Fh, double mub, void* f,
                        void* g, int storage, int Nx, int Ny, int P, const float* rch, double fb, double fd,
                        const double* base_g, cudaStream_t s) {
  return by_storage(storage, false, [&](auto* sp, auto*) {
    using S = std::remove_pointer_t<decltype(sp)>;
    k_init<S><<<kGrid, kBlock, 0, s>>>(rho_h, rc_h, Eh, sY, cY, Sx, Cy, Fh, mub, static_cast<S*>(f),
                                       static_cast<S*>(g), Nx, Ny, P, rch, fb, fd, base_g);
    return cudaGetLastError();
  });
}

}  // namespace ehd

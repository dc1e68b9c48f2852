// k_step.cu -- the fused collide-and-stream kernel of the coupled step
// (arXiv:1812.05711, Sec. IV.2 and Table I) and the small kernels around it.
//
// K4 k_step: one thread per node, a CTA covers 128 columns x `rows` rows.
//   Reads the node's 9 f and 9 g (coalesced SoA planes) and the potential
//   stencil, forms E = -grad phi, the moments (Eqs. 5-7), collides f with the
//   electric force (TRT, Eqs. 8, 10, 12, 13, 15) and g with the drift u + mu_b E
//   (TRT, Eqs. 9, 11, 14), and pushes the post-collision values to the
//   neighbours (periodic x; halfway bounce-back of f on both walls;
//   anti-bounce-back injection of rho0 and zero-gradient outflow of g).
//   CTAs on the wall rows also sum the injected and collected charge.
// The per-CTA wall fluxes are added, in a fixed order, to the run's FP64
// totals by the mean-mode kernel of the Poisson solve that follows.
//
// Shifted storage (FP32 compute): f~_i = f_i - w_i r(y) and g~_i = g_i - w_i s(y)
// with r(y) and s(y) the hydrostatic density and charge of the row; the TRT
// collision is applied to the shifted values (the shift is symmetric in i, so
// only the equilibrium's rest part changes), and a population moving between
// rows picks up w_i (r(y) - r(y')) or w_i (s(y) - s(y')).  Plain FP64 uses
// shifts 0 and the same code.
#include "ehd_dev.cuh"

namespace ehd {

namespace {

constexpr int kStepThreads = 128;

template <class R>
__device__ __forceinline__ void trt_f(R& fi, R& fo, R w, R drho, R rho, R cu, R usq15, R cF, R uF3, R wp, R wm,
                                      R cp, R cm) {
  const R ep = w * (drho + rho * (R(4.5) * cu * cu - usq15));  // even part of Eq. 10
  const R em = w * rho * R(3) * cu;                             // odd part of Eq. 10
  const R Fp = w * (R(9) * cu * cF - uF3);                      // even part of Eq. 12
  const R Fm = w * R(3) * cF;                                   // odd part of Eq. 12
  const R sp = R(0.5) * (fi + fo), sm = R(0.5) * (fi - fo);     // Eq. 13
  const R A = cp * Fp - wp * (sp - ep);
  const R B = cm * Fm - wm * (sm - em);
  fi = fi + A + B;  // Eq. 8
  fo = fo + A - B;
}

template <class R>
__device__ __forceinline__ void trt_g(R& gi, R& go, R w, R drc, R rc, R cv, R vsq15, R wp, R wm) {
  const R ep = w * (drc + rc * (R(4.5) * cv * cv - vsq15));  // even part of Eq. 11
  const R em = w * rc * R(3) * cv;                            // odd part of Eq. 11
  const R sp = R(0.5) * (gi + go), sm = R(0.5) * (gi - go);   // Eq. 14
  const R A = -wp * (sp - ep);
  const R B = -wm * (sm - em);
  gi = gi + A + B;  // Eq. 9
  go = go + A - B;
}

__device__ __forceinline__ double block_sum128(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0) t = (red[0] + red[1]) + (red[2] + red[3]);
  __syncthreads();
  return t;
}

}  // namespace

template <class S, class R>
__global__ void __launch_bounds__(kStepThreads) k_step(StepArgs a, int rows) {
  __shared__ double red[4];
  const int x = blockIdx.x * kStepThreads + threadIdx.x;
  const int Nx = a.Nx, Ny = a.Ny, P = a.P;
  const long long pl = a.plane;
  const int ybeg = blockIdx.y * rows;
  const int yend = min(ybeg + rows, Ny);
  const S* __restrict__ fin = static_cast<const S*>(a.fin);
  const S* __restrict__ gin = static_cast<const S*>(a.gin);
  S* __restrict__ fo = static_cast<S*>(a.fout);
  S* __restrict__ go = static_cast<S*>(a.gout);
  const R* __restrict__ dphi = static_cast<const R*>(a.dphi);
  const R* __restrict__ Ebar = static_cast<const R*>(a.Ebar);
  const float* __restrict__ rch = a.rch;
  const R wp = (R)a.wp, wm = (R)a.wm, gwp = (R)a.gwp, gwm = (R)a.gwm;
  const R cp = R(1) - R(0.5) * wp, cm = R(1) - R(0.5) * wm;
  const R mub = (R)a.mub, rho0 = (R)a.rho0;
  const R fb = (R)a.fb, fd = (R)a.fd;  // f shift fb + fd y: a row up changes it by fd
  const R gwall = (a.wall_mode == 0) ? R(-1) : R(0);
  const R W0 = (R)kW0, W1 = (R)kW1, W2 = (R)kW2;
  double qin = 0.0, qout = 0.0;
  bool bad = false;
  if (x < Nx) {
    const int xl = (x == 0) ? Nx - 1 : x - 1;
    const int xr = (x == Nx - 1) ? 0 : x + 1;
    for (int y = ybeg; y < yend; ++y) {
      const long long c = (long long)y * P + x;
      const long long cl = c - x + xl, cr = c - x + xr;
      R f0 = Store<S>::template ld<R>(fin + c), f1 = Store<S>::template ld<R>(fin + pl + c),
        f2 = Store<S>::template ld<R>(fin + 2 * pl + c), f3 = Store<S>::template ld<R>(fin + 3 * pl + c),
        f4 = Store<S>::template ld<R>(fin + 4 * pl + c), f5 = Store<S>::template ld<R>(fin + 5 * pl + c),
        f6 = Store<S>::template ld<R>(fin + 6 * pl + c), f7 = Store<S>::template ld<R>(fin + 7 * pl + c),
        f8 = Store<S>::template ld<R>(fin + 8 * pl + c);
      R g0 = Store<S>::template ld<R>(gin + c), g1 = Store<S>::template ld<R>(gin + pl + c),
        g2 = Store<S>::template ld<R>(gin + 2 * pl + c), g3 = Store<S>::template ld<R>(gin + 3 * pl + c),
        g4 = Store<S>::template ld<R>(gin + 4 * pl + c), g5 = Store<S>::template ld<R>(gin + 5 * pl + c),
        g6 = Store<S>::template ld<R>(gin + 6 * pl + c), g7 = Store<S>::template ld<R>(gin + 7 * pl + c),
        g8 = Store<S>::template ld<R>(gin + 8 * pl + c);
      // E = -grad phi, central differences; phi = phibar(y) + dphi
      const R pc = __ldg(dphi + c);
      const R pW = __ldg(dphi + cl), pE = __ldg(dphi + cr);
      const R pS = (y > 0) ? __ldg(dphi + c - P) : gwall * pc;
      const R pN = (y < Ny - 1) ? __ldg(dphi + c + P) : gwall * pc;
      const R Ex = R(-0.5) * (pE - pW);
      const R Ey = __ldg(Ebar + y) - R(0.5) * (pN - pS);
      const R sy = rch ? (R)__ldg(rch + y) : R(0);
      const R sf = fb + fd * (R)y;
      // moments, Eqs. 5-7
      const R drho = ((f0 + f1) + (f2 + f3)) + ((f4 + f5) + (f6 + f7)) + f8;
      const R rho = sf + drho;
      const R jx = (f1 - f3) + (f5 - f7) + (f8 - f6);
      const R jy = (f2 - f4) + (f5 - f7) + (f6 - f8);
      const R drc = ((g0 + g1) + (g2 + g3)) + ((g4 + g5) + (g6 + g7)) + g8;
      const R rc = sy + drc;
      if (!isfinite(drho) || !isfinite(drc)) bad = true;
      const R Fx = rc * Ex, Fy = rc * Ey;  // F_e = -rho_c grad phi
      const R irho = R(1) / rho;
      const R ux = (jx + R(0.5) * Fx) * irho;
      const R uy = (jy + R(0.5) * Fy) * irho;
      const R vx = ux + mub * Ex, vy = uy + mub * Ey;  // drift u - mu_b grad phi
      // fluid TRT with force
      const R usq15 = R(1.5) * (ux * ux + uy * uy);
      const R uF3 = R(3) * (ux * Fx + uy * Fy);
      f0 = f0 - wp * (f0 - W0 * (drho - rho * usq15)) - cp * W0 * uF3;
      trt_f<R>(f1, f3, W1, drho, rho, ux, usq15, Fx, uF3, wp, wm, cp, cm);
      trt_f<R>(f2, f4, W1, drho, rho, uy, usq15, Fy, uF3, wp, wm, cp, cm);
      trt_f<R>(f5, f7, W2, drho, rho, ux + uy, usq15, Fx + Fy, uF3, wp, wm, cp, cm);
      trt_f<R>(f6, f8, W2, drho, rho, uy - ux, usq15, Fy - Fx, uF3, wp, wm, cp, cm);
      // charge TRT with drift
      const R vsq15 = R(1.5) * (vx * vx + vy * vy);
      g0 = g0 - gwp * (g0 - W0 * (drc - rc * vsq15));
      trt_g<R>(g1, g3, W1, drc, rc, vx, vsq15, gwp, gwm);
      trt_g<R>(g2, g4, W1, drc, rc, vy, vsq15, gwp, gwm);
      trt_g<R>(g5, g7, W2, drc, rc, vx + vy, vsq15, gwp, gwm);
      trt_g<R>(g6, g8, W2, drc, rc, vy - vx, vsq15, gwp, gwm);
      // streaming: f_i(x + c_i, t + 1) = f_i*(x, t)
      const long long yo = (long long)y * P;
      Store<S>::st(fo + yo + x, f0);
      Store<S>::st(go + yo + x, g0);
      Store<S>::st(fo + pl + yo + xr, f1);
      Store<S>::st(go + pl + yo + xr, g1);
      Store<S>::st(fo + 3 * pl + yo + xl, f3);
      Store<S>::st(go + 3 * pl + yo + xl, g3);
      if (y + 1 < Ny) {
        const R sh = rch ? sy - (R)__ldg(rch + y + 1) : R(0);
        const R fh = -fd;
        const long long yu = yo + P;
        Store<S>::st(fo + 2 * pl + yu + x, f2 + W1 * fh);
        Store<S>::st(go + 2 * pl + yu + x, g2 + W1 * sh);
        Store<S>::st(fo + 5 * pl + yu + xr, f5 + W2 * fh);
        Store<S>::st(go + 5 * pl + yu + xr, g5 + W2 * sh);
        Store<S>::st(fo + 6 * pl + yu + xl, f6 + W2 * fh);
        Store<S>::st(go + 6 * pl + yu + xl, g6 + W2 * sh);
      } else {
        // collector: f bounces back into its own node, g leaves the channel
        Store<S>::st(fo + 4 * pl + yo + x, f2);
        Store<S>::st(fo + 7 * pl + yo + x, f5);
        Store<S>::st(fo + 8 * pl + yo + x, f6);
        qout += ((double)Store<S>::rt(g2) + (double)Store<S>::rt(g5)) + (double)Store<S>::rt(g6);
        // zero-gradient outflow: the downward populations entering from the
        // wall side are the node's own post-collision values
        Store<S>::st(go + 4 * pl + yo + x, g4);
        Store<S>::st(go + 7 * pl + yo + xl, g7);
        Store<S>::st(go + 8 * pl + yo + xr, g8);
        qout -= ((double)Store<S>::rt(g4) + (double)Store<S>::rt(g7)) + (double)Store<S>::rt(g8);
      }
      if (y > 0) {
        const R sh = rch ? sy - (R)__ldg(rch + y - 1) : R(0);
        const R fh = fd;
        const long long yd = yo - P;
        Store<S>::st(fo + 4 * pl + yd + x, f4 + W1 * fh);
        Store<S>::st(go + 4 * pl + yd + x, g4 + W1 * sh);
        Store<S>::st(fo + 7 * pl + yd + xl, f7 + W2 * fh);
        Store<S>::st(go + 7 * pl + yd + xl, g7 + W2 * sh);
        Store<S>::st(fo + 8 * pl + yd + xr, f8 + W2 * fh);
        Store<S>::st(go + 8 * pl + yd + xr, g8 + W2 * sh);
      } else {
        // injector: halfway bounce-back of f; anti-bounce-back of g imposing
        // rho_c = rho0 with the wall drift mu_b E (fluid at rest on the wall)
        Store<S>::st(fo + 2 * pl + yo + x, f4);
        Store<S>::st(fo + 5 * pl + yo + x, f7);
        Store<S>::st(fo + 6 * pl + yo + x, f8);
        const R wx = mub * Ex, wy = mub * Ey;
        const R w15 = R(1.5) * (wx * wx + wy * wy);
        const R c2 = wy, c5 = wx + wy, c6 = wy - wx;
        // new absolute value minus the shift of the same row and weight
        const R n2 = -(g4 + R(2) * W1 * sy) + R(2) * W1 * rho0 * (R(1) + R(4.5) * c2 * c2 - w15);
        const R n5 = -(g7 + R(2) * W2 * sy) + R(2) * W2 * rho0 * (R(1) + R(4.5) * c5 * c5 - w15);
        const R n6 = -(g8 + R(2) * W2 * sy) + R(2) * W2 * rho0 * (R(1) + R(4.5) * c6 * c6 - w15);
        Store<S>::st(go + 2 * pl + yo + x, n2);
        Store<S>::st(go + 5 * pl + yo + x, n5);
        Store<S>::st(go + 6 * pl + yo + x, n6);
        qin += (((double)Store<S>::rt(n2) - (double)Store<S>::rt(g4)) +
                ((double)Store<S>::rt(n5) - (double)Store<S>::rt(g7))) +
               ((double)Store<S>::rt(n6) - (double)Store<S>::rt(g8));
      }
    }
  }
  if (bad) atomicOr(a.err, 1);
  const bool first = (blockIdx.y == 0), last = (blockIdx.y == gridDim.y - 1);
  if (first) {
    const double t = block_sum128(qin, red);
    if (threadIdx.x == 0) a.flux_part[blockIdx.x] = t;
  }
  if (last) {
    const double t = block_sum128(qout, red);
    if (threadIdx.x == 0) a.flux_part[gridDim.x + blockIdx.x] = t;
  }
}

int step_flux_blocks(int Nx) { return (Nx + kStepThreads - 1) / kStepThreads; }

namespace {
template <class S, class R>
cudaError_t step_t(const StepArgs& a, int rows, cudaStream_t s) {
  dim3 grid((a.Nx + kStepThreads - 1) / kStepThreads, (a.Ny + rows - 1) / rows);
  k_step<S, R><<<grid, kStepThreads, 0, s>>>(a, rows);
  return cudaGetLastError();
}
}  // namespace

cudaError_t launch_step(const StepArgs& a, int storage, bool real_f64, int rows, cudaStream_t s) {
  if (real_f64) {
    if (storage != 0) return cudaErrorInvalidValue;
    return step_t<double, double>(a, rows, s);
  }
  switch (storage) {
    case 0: return step_t<double, float>(a, rows, s);
    case 1: return step_t<float, float>(a, rows, s);
    case 2: return step_t<__nv_bfloat16, float>(a, rows, s);
    case 3: return step_t<__half, float>(a, rows, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace ehd

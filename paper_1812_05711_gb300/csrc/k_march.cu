// k_march.cu -- the fused collide-and-stream kernel in "march" form: a warp
// walks up a slab of rows of a strip of columns, so that every population it
// stores has been pulled from registers (x-neighbours by warp shuffles,
// y-neighbours from the rows already collided) and the charge of the new
// state, rho_c(t+1) = sum_i g_i (Eq. 6), is formed from exactly the values
// stored -- no second pass over g.
//
// Per row r of the walk: load the 9 f and 9 g of the lane's node(s) (the next
// rows are staged ahead by cp.async), form E = -grad phi (central differences
// of phi, or the spectral E_x plane), the moments (Eqs. 5-7), collide f with
// the electric force (TRT, Eqs. 8, 10, 12, 13, 15) and g with the drift (TRT,
// Eqs. 9, 11, 14), then route the post-collision values:
//   c_y = 0   -> row r     (complete once row r+1 has been collided)
//   c_y = +1  -> row r + 1 (kept in registers)
//   c_y = -1  -> row r - 1 (completes row r - 1, which is stored)
// The walls of Table I enter as row rules: halfway bounce-back of f on both
// walls, anti-bounce-back injection of rho0 (with the wall drift mu_b E) and
// zero-gradient outflow of g.
//
// Two forms.  k_march2 (the default): two adjacent nodes per lane, a strip of
// 64 columns (60 owned, one halo pair on each side, collided but not stored);
// the slab's own rows only -- populations that leave the slab are pushed into
// the neighbouring slab's boundary row with their share of that row's charge
// (rhoc_dn / rhoc_up, added by the forward transform), so no row is collided
// twice.  k_march: one node per lane, a 32-column strip (30 owned), with a
// halo row below and above the slab collided but not stored.
#include <type_traits>

#include "ehd_dev.cuh"

namespace ehd {

namespace {

template <class R>
__device__ __forceinline__ void trt_f2(R& fi, R& fo, R w, R drho, R rho, R cu, R usq15, R cF, R uF3, R wp, R wm, R cp,
                                       R cm) {
  const R ep = w * (drho + rho * (R(4.5) * cu * cu - usq15));
  const R em = w * rho * R(3) * cu;
  const R Fp = w * (R(9) * cu * cF - uF3);
  const R Fm = w * R(3) * cF;
  const R sp = R(0.5) * (fi + fo), sm = R(0.5) * (fi - fo);
  const R A = cp * Fp - wp * (sp - ep);
  const R B = cm * Fm - wm * (sm - em);
  fi = fi + A + B;
  fo = fo + A - B;
}

// trt_f2 for a pair that crosses rows (fi moves up, fo down) in storage
// shifted by a density ramp r(y) = r(0) + dr y: with dq = -dr / omega- the
// antisymmetric part hands fi its storage offset change -w dr and fo +w dr,
// at no extra instruction (dq is added inside the product w (3 rho cu + dq)).
template <class R>
__device__ __forceinline__ void trt_f2y(R& fi, R& fo, R w, R drho, R rho, R cu, R usq15, R cF, R uF3, R wp, R wm,
                                        R cp, R cm, R dq) {
  const R ep = w * (drho + rho * (R(4.5) * cu * cu - usq15));
  const R em = w * (rho * R(3) * cu + dq);
  const R Fp = w * (R(9) * cu * cF - uF3);
  const R Fm = w * R(3) * cF;
  const R sp = R(0.5) * (fi + fo), sm = R(0.5) * (fi - fo);
  const R A = cp * Fp - wp * (sp - ep);
  const R B = cm * Fm - wm * (sm - em);
  fi = fi + A + B;
  fo = fo + A - B;
}

template <class R>
__device__ __forceinline__ void trt_g2(R& gi, R& go, R w, R drc, R rc, R cv, R vsq15, R wp, R wm) {
  const R ep = w * (drc + rc * (R(4.5) * cv * cv - vsq15));
  const R em = w * rc * R(3) * cv;
  const R sp = R(0.5) * (gi + go), sm = R(0.5) * (gi - go);
  const R A = -wp * (sp - ep);
  const R B = -wm * (sm - em);
  gi = gi + A + B;
  go = go + A - B;
}

// cp.async of one element (4 or 8 bytes) global -> shared, per thread
template <int BYTES>
__device__ __forceinline__ void cp_async_elem(void* smem_dst, const void* gsrc) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(d), "l"(gsrc), "n"(BYTES));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

template <class R>
__device__ __forceinline__ R from_left(R v) { return __shfl_up_sync(0xffffffffu, v, 1); }
template <class R>
__device__ __forceinline__ R from_right(R v) { return __shfl_down_sync(0xffffffffu, v, 1); }

}  // namespace

// Rows ahead of the walk are staged per warp in a shared-memory ring of NST
// rows by cp.async when the storage element is 4 or 8 bytes (2-byte storage
// loads directly).  A stage holds 20 slots x 32 lanes: 18 populations, the
// potential fluctuation of the next row in the lane's column, and one
// lane-specific value (lane 0 / 31: the potential just outside the strip;
// lane 1: the row's mean field; lanes 2-4: the charge shift of rows r, r+1,
// r-1).
template <class S, int NSTAGE>
struct MarchStages {
  static constexpr bool kAsync = sizeof(S) >= 4;
  static constexpr int kN = NSTAGE;
  static constexpr int kSlots = 20;
  static constexpr size_t kBytesPerWarp = kAsync ? (size_t)kN * kSlots * 32 * sizeof(S) : 0;
};

template <class S, class R, int NSTAGE>
__global__ void __launch_bounds__(128) k_march(StepArgs a) {
  extern __shared__ __align__(16) unsigned char march_smem[];
  using St = MarchStages<S, NSTAGE>;
  constexpr int NST = St::kN;
  const int lane = threadIdx.x & 31;
  const int gw = blockIdx.x * 4 + (threadIdx.x >> 5);
  const int Nx = a.Nx, Ny = a.Ny, P = a.P, ns = a.nstrips;
  const int strip = gw % ns, slab = gw / ns;
  const int y0 = slab * a.slab_rows;
  if (y0 >= Ny) return;  // whole warp
  const int y1 = min(y0 + a.slab_rows, Ny);
  const int xs = strip * 30;
  int xc = (xs - 1 + lane + Nx) % Nx;
  const bool owned = lane >= 1 && lane <= 30 && xs + lane - 1 < Nx;
  const int xW = (xc == 0) ? Nx - 1 : xc - 1;
  const int xE = (xc == Nx - 1) ? 0 : xc + 1;
  const long long pl = a.plane;
  const S* __restrict__ fin = static_cast<const S*>(a.fin);
  const S* __restrict__ gin = static_cast<const S*>(a.gin);
  S* __restrict__ fo = static_cast<S*>(a.fout);
  S* __restrict__ go = static_cast<S*>(a.gout);
  R* __restrict__ rho_out = static_cast<R*>(a.rhoc_out);
  const R* __restrict__ dphi = static_cast<const R*>(a.dphi);
  const R* __restrict__ Ebar = static_cast<const R*>(a.Ebar);
  const float* __restrict__ rch = a.rch;
  const R wp = (R)a.wp, wm = (R)a.wm, gwp = (R)a.gwp, gwm = (R)a.gwm;
  const R cp = R(1) - R(0.5) * wp, cm = R(1) - R(0.5) * wm;
  const R mub = (R)a.mub, rho0 = (R)a.rho0;
  const R gwall = (a.wall_mode == 0) ? R(-1) : R(0);
  const R W0 = (R)kW0, W1 = (R)kW1, W2 = (R)kW2;
  const R fb = (R)a.fb, fd = (R)a.fd;  // f shift fb + fd y: a row up changes it by fd

  const int rs = max(y0 - 1, 0), re = min(y1, Ny - 1);
  // carried registers: H (c_y = 0) of row r-1, U (c_y = +1) of rows r-1 and r
  R Hm[6] = {}, Um[6] = {}, Uc[6] = {};
  // potential fluctuation in the lane's column: rows r-1, r
  R pm, pc;
  {
    const R p0 = __ldg(dphi + (long long)rs * P + xc);
    pm = (rs > 0) ? __ldg(dphi + (long long)(rs - 1) * P + xc) : gwall * p0;
    pc = p0;
  }
  double qin = 0.0, qout = 0.0;
  bool bad = false;
  constexpr int SL = St::kSlots;
  S* ring = reinterpret_cast<S*>(march_smem) + (size_t)(threadIdx.x >> 5) * NST * SL * 32 + lane;
  auto issue = [&](int row_y, int stage) {
    const long long c = (long long)row_y * P + xc;
    S* dst = ring + (size_t)stage * SL * 32;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      cp_async_elem<sizeof(S)>(dst + i * 32, fin + i * pl + c);
      cp_async_elem<sizeof(S)>(dst + (9 + i) * 32, gin + i * pl + c);
    }
    if (row_y + 1 < Ny) cp_async_elem<sizeof(R)>(dst + 18 * 32, dphi + c + P);
    const void* extra = nullptr;
    int eb = 0;  // bytes: 4 or sizeof(R)
    if (lane == 0) {
      extra = dphi + (long long)row_y * P + xW;
      eb = sizeof(R);
    } else if (lane == 31) {
      extra = dphi + (long long)row_y * P + xE;
      eb = sizeof(R);
    } else if (lane == 1) {
      extra = Ebar + row_y;
      eb = sizeof(R);
    } else if (rch && lane == 2) {
      extra = rch + row_y;
      eb = 4;
    } else if (rch && lane == 3 && row_y + 1 < Ny) {
      extra = rch + row_y + 1;
      eb = 4;
    } else if (rch && lane == 4 && row_y > 0) {
      extra = rch + row_y - 1;
      eb = 4;
    }
    if (eb == 8)
      cp_async_elem<8>(dst + 19 * 32, extra);
    else if (eb == 4)
      cp_async_elem<4>(dst + 19 * 32, extra);
  };
  if constexpr (St::kAsync) {
#pragma unroll
    for (int k = 0; k < NST - 1; ++k) {
      if (rs + k <= re) issue(rs + k, k);
      cp_async_commit();
    }
  }
  R F[9], G[9];
  for (int r = rs; r <= re; ++r) {
    const long long row = (long long)r * P;
    R pn, pW, pE, Ebr, sy, s_up, s_dn;
    if constexpr (St::kAsync) {
      const int k = r - rs;
      if (r + NST - 1 <= re) issue(r + NST - 1, (k + NST - 1) % NST);
      cp_async_commit();
      cp_async_wait<NST - 1>();  // this lane's copies of row r have landed
      const S* src = ring + (size_t)(k % NST) * SL * 32;
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        F[i] = (R)src[i * 32];
        G[i] = (R)src[(9 + i) * 32];
      }
      __syncwarp();  // other lanes' extra slots are read below by shuffle sources
      const R nx = *reinterpret_cast<const R*>(src + 18 * 32);
      pn = (r + 1 < Ny) ? nx : gwall * pc;
      const R ex_r = *reinterpret_cast<const R*>(src + 19 * 32);
      const float ex_f = *reinterpret_cast<const float*>(src + 19 * 32);
      pW = from_left(pc);
      pE = from_right(pc);
      if (lane == 0) pW = ex_r;
      if (lane == 31) pE = ex_r;
      Ebr = __shfl_sync(0xffffffffu, ex_r, 1);
      sy = rch ? (R)__shfl_sync(0xffffffffu, ex_f, 2) : R(0);
      s_up = (rch && r + 1 < Ny) ? (R)__shfl_sync(0xffffffffu, ex_f, 3) : sy;
      s_dn = (rch && r > 0) ? (R)__shfl_sync(0xffffffffu, ex_f, 4) : sy;
    } else {
      const long long c = row + xc;
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        F[i] = Store<S>::template ld<R>(fin + i * pl + c);
        G[i] = Store<S>::template ld<R>(gin + i * pl + c);
      }
      pn = (r + 1 < Ny) ? __ldg(dphi + row + P + xc) : gwall * pc;
      pW = __ldg(dphi + row + xW);
      pE = __ldg(dphi + row + xE);
      Ebr = __ldg(Ebar + r);
      sy = rch ? (R)__ldg(rch + r) : R(0);
      s_up = (rch && r + 1 < Ny) ? (R)__ldg(rch + r + 1) : sy;
      s_dn = (rch && r > 0) ? (R)__ldg(rch + r - 1) : sy;
    }
    const R Ex = R(-0.5) * (pE - pW);
    const R Ey = Ebr - R(0.5) * (pn - pm);
    // moments, Eqs. 5-7
    R f0 = F[0], f1 = F[1], f2 = F[2], f3 = F[3], f4 = F[4], f5 = F[5], f6 = F[6], f7 = F[7], f8 = F[8];
    R g0 = G[0], g1 = G[1], g2 = G[2], g3 = G[3], g4 = G[4], g5 = G[5], g6 = G[6], g7 = G[7], g8 = G[8];
    const R drho = ((f0 + f1) + (f2 + f3)) + ((f4 + f5) + (f6 + f7)) + f8;
    const R rho = (fb + fd * (R)r) + drho;
    const R jx = (f1 - f3) + (f5 - f7) + (f8 - f6);
    const R jy = (f2 - f4) + (f5 - f7) + (f6 - f8);
    const R drc = ((g0 + g1) + (g2 + g3)) + ((g4 + g5) + (g6 + g7)) + g8;
    const R rc = sy + drc;
    if (owned && (!isfinite(drho) || !isfinite(drc))) bad = true;
    const R Fx = rc * Ex, Fy = rc * Ey;
    const R irho = R(1) / rho;
    const R ux = (jx + R(0.5) * Fx) * irho;
    const R uy = (jy + R(0.5) * Fy) * irho;
    const R vx = ux + mub * Ex, vy = uy + mub * Ey;
    const R usq15 = R(1.5) * (ux * ux + uy * uy);
    const R uF3 = R(3) * (ux * Fx + uy * Fy);
    f0 = f0 - wp * (f0 - W0 * (drho - rho * usq15)) - cp * W0 * uF3;
    trt_f2<R>(f1, f3, W1, drho, rho, ux, usq15, Fx, uF3, wp, wm, cp, cm);
    trt_f2<R>(f2, f4, W1, drho, rho, uy, usq15, Fy, uF3, wp, wm, cp, cm);
    trt_f2<R>(f5, f7, W2, drho, rho, ux + uy, usq15, Fx + Fy, uF3, wp, wm, cp, cm);
    trt_f2<R>(f6, f8, W2, drho, rho, uy - ux, usq15, Fy - Fx, uF3, wp, wm, cp, cm);
    const R vsq15 = R(1.5) * (vx * vx + vy * vy);
    g0 = g0 - gwp * (g0 - W0 * (drc - rc * vsq15));
    trt_g2<R>(g1, g3, W1, drc, rc, vx, vsq15, gwp, gwm);
    trt_g2<R>(g2, g4, W1, drc, rc, vy, vsq15, gwp, gwm);
    trt_g2<R>(g5, g7, W2, drc, rc, vx + vy, vsq15, gwp, gwm);
    trt_g2<R>(g6, g8, W2, drc, rc, vy - vx, vsq15, gwp, gwm);

    // pulled values of this row's post-collision populations: x-shift by c_x
    const R P1f = from_left(f1), P5f = from_left(f5), P8f = from_left(f8);
    const R P3f = from_right(f3), P6f = from_right(f6), P7f = from_right(f7);
    const R P1g = from_left(g1), P5g = from_left(g5), P8g = from_left(g8);
    const R P3g = from_right(g3), P6g = from_right(g6), P7g = from_right(g7);

    // c_y = +1: into row r + 1 (the shifts of density and charge move with the row)
    R Un[6];
    {
      const R sh = sy - s_up, fh = -fd;
      Un[0] = f2 + W1 * fh;
      Un[1] = P5f + W2 * fh;
      Un[2] = P6f + W2 * fh;
      Un[3] = g2 + W1 * sh;
      Un[4] = P5g + W2 * sh;
      Un[5] = P6g + W2 * sh;
    }
    if (r == 0) {
      // injector wall: the upward populations of row 0 come from the node's
      // own downward ones: bounce-back for f, anti-bounce-back for g
      const R wx = mub * Ex, wy = mub * Ey;
      const R w15 = R(1.5) * (wx * wx + wy * wy);
      const R c2 = wy, c5 = wx + wy, c6 = wy - wx;
      const R n2 = -(g4 + R(2) * W1 * sy) + R(2) * W1 * rho0 * (R(1) + R(4.5) * c2 * c2 - w15);
      const R n5 = -(g7 + R(2) * W2 * sy) + R(2) * W2 * rho0 * (R(1) + R(4.5) * c5 * c5 - w15);
      const R n6 = -(g8 + R(2) * W2 * sy) + R(2) * W2 * rho0 * (R(1) + R(4.5) * c6 * c6 - w15);
      Uc[0] = f4;
      Uc[1] = f7;
      Uc[2] = f8;
      Uc[3] = n2;
      Uc[4] = n5;
      Uc[5] = n6;
      if (owned && y0 == 0)
        qin += (((double)Store<S>::rt(n2) - (double)Store<S>::rt(g4)) +
                ((double)Store<S>::rt(n5) - (double)Store<S>::rt(g7))) +
               ((double)Store<S>::rt(n6) - (double)Store<S>::rt(g8));
    }
    // c_y = -1: into row r - 1, which is then complete
    if (r - 1 >= y0) {
      const R sh = sy - s_dn, fh = fd;
      const long long c = row - P + xc;
      if (owned) {
        const R n4 = g4 + W1 * sh, n7 = P7g + W2 * sh, n8 = P8g + W2 * sh;
        Store<S>::st(fo + c, Hm[0]);
        Store<S>::st(fo + pl + c, Hm[1]);
        Store<S>::st(fo + 2 * pl + c, Um[0]);
        Store<S>::st(fo + 3 * pl + c, Hm[2]);
        Store<S>::st(fo + 4 * pl + c, f4 + W1 * fh);
        Store<S>::st(fo + 5 * pl + c, Um[1]);
        Store<S>::st(fo + 6 * pl + c, Um[2]);
        Store<S>::st(fo + 7 * pl + c, P7f + W2 * fh);
        Store<S>::st(fo + 8 * pl + c, P8f + W2 * fh);
        Store<S>::st(go + c, Hm[3]);
        Store<S>::st(go + pl + c, Hm[4]);
        Store<S>::st(go + 2 * pl + c, Um[3]);
        Store<S>::st(go + 3 * pl + c, Hm[5]);
        Store<S>::st(go + 4 * pl + c, n4);
        Store<S>::st(go + 5 * pl + c, Um[4]);
        Store<S>::st(go + 6 * pl + c, Um[5]);
        Store<S>::st(go + 7 * pl + c, n7);
        Store<S>::st(go + 8 * pl + c, n8);
        const R sprev = s_dn;
        const R q = ((Store<S>::rt(Hm[3]) + Store<S>::rt(Hm[4])) + (Store<S>::rt(Um[3]) + Store<S>::rt(Hm[5]))) +
                    ((Store<S>::rt(n4) + Store<S>::rt(Um[4])) + (Store<S>::rt(Um[5]) + Store<S>::rt(n7))) +
                    Store<S>::rt(n8);
        rho_out[c] = sprev + q;
      }
    }
    if (r == Ny - 1 && r >= y0 && r < y1) {
      // collector wall: f bounces back into the node; g leaves and the
      // downward populations re-enter from the node's own row (outflow)
      const long long c = row + xc;
      if (owned) {
        Store<S>::st(fo + c, f0);
        Store<S>::st(fo + pl + c, P1f);
        Store<S>::st(fo + 2 * pl + c, Uc[0]);
        Store<S>::st(fo + 3 * pl + c, P3f);
        Store<S>::st(fo + 4 * pl + c, f2);
        Store<S>::st(fo + 5 * pl + c, Uc[1]);
        Store<S>::st(fo + 6 * pl + c, Uc[2]);
        Store<S>::st(fo + 7 * pl + c, f5);
        Store<S>::st(fo + 8 * pl + c, f6);
        Store<S>::st(go + c, g0);
        Store<S>::st(go + pl + c, P1g);
        Store<S>::st(go + 2 * pl + c, Uc[3]);
        Store<S>::st(go + 3 * pl + c, P3g);
        Store<S>::st(go + 4 * pl + c, g4);
        Store<S>::st(go + 5 * pl + c, Uc[4]);
        Store<S>::st(go + 6 * pl + c, Uc[5]);
        Store<S>::st(go + 7 * pl + c, P7g);
        Store<S>::st(go + 8 * pl + c, P8g);
        const R q = ((Store<S>::rt(g0) + Store<S>::rt(P1g)) + (Store<S>::rt(Uc[3]) + Store<S>::rt(P3g))) +
                    ((Store<S>::rt(g4) + Store<S>::rt(Uc[4])) + (Store<S>::rt(Uc[5]) + Store<S>::rt(P7g))) +
                    Store<S>::rt(P8g);
        rho_out[c] = sy + q;
        qout += ((double)Store<S>::rt(g2) + (double)Store<S>::rt(g5)) + (double)Store<S>::rt(g6);
        qout -= ((double)Store<S>::rt(g4) + (double)Store<S>::rt(g7)) + (double)Store<S>::rt(g8);
      }
    }
    // rotate the carried rows
    Hm[0] = f0;
    Hm[1] = P1f;
    Hm[2] = P3f;
    Hm[3] = g0;
    Hm[4] = P1g;
    Hm[5] = P3g;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      Um[k] = Uc[k];
      Uc[k] = Un[k];
    }
    pm = pc;
    pc = pn;
  }
  if constexpr (St::kAsync) cp_async_wait<0>();
  if (bad) atomicOr(a.err, 1);
  // wall fluxes: one partial per strip (slab 0 injects, the top slab collects)
  if (y0 == 0) {
    double v = qin;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) a.flux_part[strip] = v;
  }
  if (y1 == Ny) {
    double v = qout;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) a.flux_part[ns + strip] = v;
  }
}


// ---------------------------------------------------------------------------
// Two columns per lane: a warp covers 64 columns (60 owned) and every lane
// loads, collides and stores an adjacent pair of nodes (8-byte pairs in FP32
// storage).  The x-shift of the post-collision pair needs one shuffle per
// direction; the halo lanes' outer columns are never used, so their potential
// neighbours need no extra load.
template <class S>
struct Pair;
template <>
struct Pair<float> {
  template <class R>
  __device__ static void st(float* p, R a, R b) { *reinterpret_cast<float2*>(p) = make_float2((float)a, (float)b); }
  template <class R>
  __device__ static void ld(const float* p, R& a, R& b) {
    const float2 v = *reinterpret_cast<const float2*>(p);
    a = (R)v.x;
    b = (R)v.y;
  }
};
template <>
struct Pair<double> {
  template <class R>
  __device__ static void st(double* p, R a, R b) { *reinterpret_cast<double2*>(p) = make_double2((double)a, (double)b); }
  template <class R>
  __device__ static void ld(const double* p, R& a, R& b) {
    const double2 v = *reinterpret_cast<const double2*>(p);
    a = (R)v.x;
    b = (R)v.y;
  }
};
template <>
struct Pair<__nv_bfloat16> {
  template <class R>
  __device__ static void st(__nv_bfloat16* p, R a, R b) {
    *reinterpret_cast<__nv_bfloat162*>(p) = __floats2bfloat162_rn((float)a, (float)b);
  }
  template <class R>
  __device__ static void ld(const __nv_bfloat16* p, R& a, R& b) {
    const float2 v = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(p));
    a = (R)v.x;
    b = (R)v.y;
  }
};
template <>
struct Pair<__half> {  // scaled by 2^12 like Store<__half>
  template <class R>
  __device__ static void st(__half* p, R a, R b) {
    *reinterpret_cast<__half2*>(p) = __floats2half2_rn((float)a * kHalfScale, (float)b * kHalfScale);
  }
  template <class R>
  __device__ static void ld(const __half* p, R& a, R& b) {
    const float2 v = __half22float2(*reinterpret_cast<const __half2*>(p));
    a = (R)(v.x * kHalfUnscale);
    b = (R)(v.y * kHalfUnscale);
  }
};

// SPECX: one more slot per stage holds the row's spectral E_x pair
template <class S, class R, int NSTAGE, bool SPECX = false>
struct March2Stages {
  static constexpr int kSlotBytes = 2 * (sizeof(S) > sizeof(R) ? sizeof(S) : sizeof(R));
  static constexpr int kSlots = SPECX ? 21 : 20;
  static constexpr size_t kBytesPerWarp = (size_t)NSTAGE * kSlots * 32 * kSlotBytes;
};

template <class S, class R>
__device__ __forceinline__ void collide_node(R (&f)[9], R (&g)[9], R Ex, R Ey, R sy, R sf, R dq, R mub, R wp, R wm,
                                             R cp, R cm, R gwp, R gwm, bool& bad) {
  const R W0 = (R)kW0, W1 = (R)kW1, W2 = (R)kW2;
  const R drho = ((f[0] + f[1]) + (f[2] + f[3])) + ((f[4] + f[5]) + (f[6] + f[7])) + f[8];
  const R rho = sf + drho;
  const R jx = (f[1] - f[3]) + (f[5] - f[7]) + (f[8] - f[6]);
  const R jy = (f[2] - f[4]) + (f[5] - f[7]) + (f[6] - f[8]);
  const R drc = ((g[0] + g[1]) + (g[2] + g[3])) + ((g[4] + g[5]) + (g[6] + g[7])) + g[8];
  const R rc = sy + drc;
  bad = !isfinite(drho) || !isfinite(drc);
  const R Fx = rc * Ex, Fy = rc * Ey;
  const R irho = R(1) / rho;
  const R ux = (jx + R(0.5) * Fx) * irho;
  const R uy = (jy + R(0.5) * Fy) * irho;
  const R vx = ux + mub * Ex, vy = uy + mub * Ey;
  const R usq15 = R(1.5) * (ux * ux + uy * uy);
  const R uF3 = R(3) * (ux * Fx + uy * Fy);
  f[0] = f[0] - wp * (f[0] - W0 * (drho - rho * usq15)) - cp * W0 * uF3;
  trt_f2<R>(f[1], f[3], W1, drho, rho, ux, usq15, Fx, uF3, wp, wm, cp, cm);
  trt_f2y<R>(f[2], f[4], W1, drho, rho, uy, usq15, Fy, uF3, wp, wm, cp, cm, dq);
  trt_f2y<R>(f[5], f[7], W2, drho, rho, ux + uy, usq15, Fx + Fy, uF3, wp, wm, cp, cm, dq);
  trt_f2y<R>(f[6], f[8], W2, drho, rho, uy - ux, usq15, Fy - Fx, uF3, wp, wm, cp, cm, dq);
  const R vsq15 = R(1.5) * (vx * vx + vy * vy);
  g[0] = g[0] - gwp * (g[0] - W0 * (drc - rc * vsq15));
  trt_g2<R>(g[1], g[3], W1, drc, rc, vx, vsq15, gwp, gwm);
  trt_g2<R>(g[2], g[4], W1, drc, rc, vy, vsq15, gwp, gwm);
  trt_g2<R>(g[5], g[7], W2, drc, rc, vx + vy, vsq15, gwp, gwm);
  trt_g2<R>(g[6], g[8], W2, drc, rc, vy - vx, vsq15, gwp, gwm);
}

// Perturbation form (FP32 compute): the fluid part as collide_node, with the
// full field E = E_B + E' in the force; the charge populations g are the
// departures d = g - B_g(y) from the x-uniform base state, and their TRT
// collision relaxes d towards the departure of the equilibrium,
// g^eq(rho_c, v) - g^eq(rho_c,B, v_B) (Eq. 11), written out so that every
// term is a product with a departure (drc = sum d, v' = v - v_B): with
// v_B = (0, vby) the base drift, cvb = c . v_B, cvp = c . v',
//   even: w [drc (1 + 4.5 cvb^2 - 1.5 vby^2)
//            + rho_c (9 cvb cvp - 3 vby v'_y + 4.5 cvp^2 - 1.5 |v'|^2)]
//   odd:  w [3 drc cvb + 3 rho_c cvp]
// (the base's own collision is advanced exactly, in FP64, elsewhere).
template <class R>
__device__ __forceinline__ void trt_g2p(R& gi, R& go, R w, R drc, R rc, R cvb, R cvp, R qb, R qp, R wp, R wm) {
  const R ep = w * (drc * (R(1) + R(4.5) * cvb * cvb - qb) + rc * (R(9) * cvb * cvp + R(4.5) * cvp * cvp - qp));
  const R em = w * R(3) * (drc * cvb + rc * cvp);
  const R sp = R(0.5) * (gi + go), sm = R(0.5) * (gi - go);
  const R A = -wp * (sp - ep);
  const R B = -wm * (sm - em);
  gi = gi + A + B;
  go = go + A - B;
}

template <class R>
__device__ __forceinline__ void collide_node_pert(R (&f)[9], R (&g)[9], R Ex, R EyF, R EyD, R rcB, R uBy, R vby, R sf,
                                                  R dq, R mub, R wp, R wm, R cp, R cm, R gwp, R gwm, bool& bad) {
  const R W0 = (R)kW0, W1 = (R)kW1, W2 = (R)kW2;
  const R drho = ((f[0] + f[1]) + (f[2] + f[3])) + ((f[4] + f[5]) + (f[6] + f[7])) + f[8];
  const R rho = sf + drho;
  const R jx = (f[1] - f[3]) + (f[5] - f[7]) + (f[8] - f[6]);
  const R jy = (f[2] - f[4]) + (f[5] - f[7]) + (f[6] - f[8]);
  const R drc = ((g[0] + g[1]) + (g[2] + g[3])) + ((g[4] + g[5]) + (g[6] + g[7])) + g[8];
  const R rc = rcB + drc;
  bad = !isfinite(drho) || !isfinite(drc);
  const R Fx = rc * Ex, Fy = rc * EyF;
  const R irho = R(1) / rho;
  const R ux = (jx + R(0.5) * Fx) * irho;
  const R uy = (jy + R(0.5) * Fy) * irho;
  const R usq15 = R(1.5) * (ux * ux + uy * uy);
  const R uF3 = R(3) * (ux * Fx + uy * Fy);
  f[0] = f[0] - wp * (f[0] - W0 * (drho - rho * usq15)) - cp * W0 * uF3;
  trt_f2<R>(f[1], f[3], W1, drho, rho, ux, usq15, Fx, uF3, wp, wm, cp, cm);
  trt_f2y<R>(f[2], f[4], W1, drho, rho, uy, usq15, Fy, uF3, wp, wm, cp, cm, dq);
  trt_f2y<R>(f[5], f[7], W2, drho, rho, ux + uy, usq15, Fx + Fy, uF3, wp, wm, cp, cm, dq);
  trt_f2y<R>(f[6], f[8], W2, drho, rho, uy - ux, usq15, Fy - Fx, uF3, wp, wm, cp, cm, dq);
  const R vpx = ux + mub * Ex, vpy = (uy - uBy) + mub * EyD;
  const R qb = R(1.5) * vby * vby;
  const R qp = R(3) * vby * vpy + R(1.5) * (vpx * vpx + vpy * vpy);
  g[0] = g[0] - gwp * (g[0] - W0 * (drc * (R(1) - qb) - rc * qp));
  trt_g2p<R>(g[1], g[3], W1, drc, rc, R(0), vpx, qb, qp, gwp, gwm);
  trt_g2p<R>(g[2], g[4], W1, drc, rc, vby, vpy, qb, qp, gwp, gwm);
  trt_g2p<R>(g[5], g[7], W2, drc, rc, vby, vpx + vpy, qb, qp, gwp, gwm);
  trt_g2p<R>(g[6], g[8], W2, drc, rc, vby, vpy - vpx, qb, qp, gwp, gwm);
}

// One warp's walk over slab `slab` of strip `strip`; warp_ring is the warp's
// NSTAGE-row staging area.  Shared by the single-run and the batch kernels.
template <class S, class R, int NSTAGE, bool SPECX = false, bool PERT = false>
__device__ __forceinline__ void march2_body(const StepArgs& a, int strip, int slab, unsigned char* warp_ring) {
  using St = March2Stages<S, R, NSTAGE, SPECX>;
  constexpr int NST = NSTAGE, SL = St::kSlots, SB = St::kSlotBytes;
  const int lane = threadIdx.x & 31;
  const int Nx = a.Nx, Ny = a.Ny, P = a.P, ns = a.nstrips;
  // slab b: rows [b S - off, (b + 1) S - off) clipped to the channel (slab 0
  // is the short one when off > 0; see slab_off)
  const int y0 = max(0, slab * a.slab_rows - a.slab_off);
  if (y0 >= Ny) return;  // whole warp
  const int y1 = min((slab + 1) * a.slab_rows - a.slab_off, Ny);
  const int xs = strip * 60;
  const int xc = (xs - 2 + 2 * lane + 2 * Nx) % Nx;  // even: the pair (xc, xc + 1)
  const bool owned = lane >= 1 && lane <= 30 && xs + 2 * (lane - 1) < Nx;
  const long long pl = a.plane;
  const S* __restrict__ fin = static_cast<const S*>(a.fin);
  const S* __restrict__ gin = static_cast<const S*>(a.gin);
  S* __restrict__ fo = static_cast<S*>(a.fout);
  S* __restrict__ go = static_cast<S*>(a.gout);
  R* __restrict__ rho_out = static_cast<R*>(a.rhoc_out);
  const R* __restrict__ dphi = static_cast<const R*>(a.dphi);
  const R* __restrict__ Ebar = static_cast<const R*>(a.Ebar);
  const float* __restrict__ rch = a.rch;
  const R wp = (R)a.wp, wm = (R)a.wm, gwp = (R)a.gwp, gwm = (R)a.gwm;
  const R cp = R(1) - R(0.5) * wp, cm = R(1) - R(0.5) * wm;
  const R mub = (R)a.mub, rho0 = (R)a.rho0;
  const R gwall = (a.wall_mode == 0) ? R(-1) : R(0);
  const R W1 = (R)kW1, W2 = (R)kW2;
  // f shift r(y) = fb + fd y (its FP32 rounding enters rho only, the row
  // change fd is exact); the wall rows undo the row change folded into f
  const R fb = (R)a.fb, fd = (R)a.fd, fdq = (R)a.fdq;
  const R wd1 = W1 * fd, wd2 = W2 * fd;
  // the walk covers the slab's own rows; populations that cross a slab
  // boundary are written by the slab that computes them (pushed into the
  // neighbouring slab's first or last row), with their share of that row's
  // charge density in rhoc_dn / rhoc_up, so no slab reads its neighbours' rows
  const int rs = y0, re = y1 - 1;
  const bool push_dn = y0 > 0, push_up = y1 < Ny;
  R* __restrict__ rx_dn = static_cast<R*>(a.rhoc_dn);
  R* __restrict__ rx_up = static_cast<R*>(a.rhoc_up);
  R sy_last = R(0);

  // carried rows, [k][j]: H (c_y = 0) of row r-1, U (c_y = +1) of rows r-1, r
  R Hm[6][2] = {}, Um[6][2] = {}, Uc[6][2] = {};
  R pm[2], pc[2];
  double qin = 0.0, qout = 0.0;
  bool bad = false;
  unsigned char* ring = warp_ring + (size_t)lane * SB;
  auto slot = [&](int stage, int s) { return ring + ((size_t)stage * SL + s) * 32 * SB; };
  // a row's populations (written by the previous step's march) ...
  auto issue_pop = [&](int row_y, int stage) {
    const long long c = (long long)row_y * P + xc;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      cp_async_elem<2 * sizeof(S)>(slot(stage, i), fin + i * pl + c);
      cp_async_elem<2 * sizeof(S)>(slot(stage, 9 + i), gin + i * pl + c);
    }
  };
  // ... and its fields (written by the Poisson solve that just ended)
  auto issue_fields = [&](int row_y, int stage) {
    const long long c = (long long)row_y * P + xc;
    if (row_y + 1 < Ny) cp_async_elem<2 * sizeof(R)>(slot(stage, 18), dphi + c + P);
    if constexpr (SPECX) cp_async_elem<2 * sizeof(R)>(slot(stage, 20), static_cast<const R*>(a.ex) + c);
    if (lane == 1) {
      cp_async_elem<sizeof(R)>(slot(stage, 19), Ebar + row_y);
    } else if constexpr (PERT) {
      // the march table of the base state: rho_c,B, u_y,B, E_y,B of the row
      if (lane >= 2 && lane <= 4) cp_async_elem<4>(slot(stage, 19), a.base_tab + 4 * row_y + (lane - 2));
    } else if (rch && lane == 2) {
      cp_async_elem<4>(slot(stage, 19), rch + row_y);
    } else if (rch && lane == 3 && row_y + 1 < Ny) {
      cp_async_elem<4>(slot(stage, 19), rch + row_y + 1);
    } else if (rch && lane == 4 && row_y > 0) {
      cp_async_elem<4>(slot(stage, 19), rch + row_y - 1);
    }
  };
  auto issue = [&](int row_y, int stage) {
    issue_pop(row_y, stage);
    issue_fields(row_y, stage);
  };
  // prologue: the first rows' populations, then (under programmatic
  // dependent launch) the wait for the inverse transform that wrote phi,
  // then the fields; with more than two stages the first group then holds
  // all prologue rows, which only makes the first wait longer
#pragma unroll
  for (int k = 0; k < NST - 1; ++k)
    if (rs + k <= re) issue_pop(rs + k, k);
  grid_dep_wait();
  {
    const long long c = (long long)rs * P + xc;
    pc[0] = dphi[c];
    pc[1] = dphi[c + 1];
    if (rs > 0) {
      pm[0] = dphi[c - P];
      pm[1] = dphi[c - P + 1];
    } else {
      pm[0] = gwall * pc[0];
      pm[1] = gwall * pc[1];
    }
  }
#pragma unroll
  for (int k = 0; k < NST - 1; ++k) {
    if (rs + k <= re) issue_fields(rs + k, k);
    cp_async_commit();
  }
  for (int r = rs; r <= re; ++r) {
    const long long row = (long long)r * P;
    const int kk = r - rs;
    if (r + NST - 1 <= re) issue(r + NST - 1, (kk + NST - 1) % NST);
    cp_async_commit();
    cp_async_wait<NST - 1>();
    const int st = kk % NST;
    R F[9][2], G[9][2];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      Pair<S>::ld(reinterpret_cast<const S*>(slot(st, i)), F[i][0], F[i][1]);
      Pair<S>::ld(reinterpret_cast<const S*>(slot(st, 9 + i)), G[i][0], G[i][1]);
    }
    R pn[2];
    {
      const R* nx = reinterpret_cast<const R*>(slot(st, 18));
      pn[0] = (r + 1 < Ny) ? nx[0] : gwall * pc[0];
      pn[1] = (r + 1 < Ny) ? nx[1] : gwall * pc[1];
    }
    const R ex_r = *reinterpret_cast<const R*>(slot(st, 19));
    const float ex_f = *reinterpret_cast<const float*>(slot(st, 19));
    const R Ebr = __shfl_sync(0xffffffffu, ex_r, 1);
    R sy, s_up, s_dn, uBy = R(0), EB = R(0);
    if constexpr (PERT) {
      // g holds departures from the base state: no shift changes between
      // rows (the base streams exactly); sy is the base charge of the row
      sy = (R)__shfl_sync(0xffffffffu, ex_f, 2);
      uBy = (R)__shfl_sync(0xffffffffu, ex_f, 3);
      EB = (R)__shfl_sync(0xffffffffu, ex_f, 4);
      s_up = sy;
      s_dn = sy;
    } else {
      sy = rch ? (R)__shfl_sync(0xffffffffu, ex_f, 2) : R(0);
      s_up = (rch && r + 1 < Ny) ? (R)__shfl_sync(0xffffffffu, ex_f, 3) : sy;
      s_dn = (rch && r > 0) ? (R)__shfl_sync(0xffffffffu, ex_f, 4) : sy;
    }
    const R sf = fb + fd * (R)r;
    // E = -grad phi at both nodes of the pair
    R Ex0, Ex1;
    if constexpr (SPECX) {
      const R* ex = reinterpret_cast<const R*>(slot(st, 20));
      Ex0 = ex[0];
      Ex1 = ex[1];
    } else {
      const R pWl = from_left(pc[1]);   // phi(xc - 1)
      const R pEr = from_right(pc[0]);  // phi(xc + 2)
      Ex0 = R(-0.5) * (pc[1] - pWl);
      Ex1 = R(-0.5) * (pEr - pc[0]);
    }
    const R Ey0 = Ebr - R(0.5) * (pn[0] - pm[0]), Ey1 = Ebr - R(0.5) * (pn[1] - pm[1]);
    R f0[9], g0[9], f1[9], g1[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      f0[i] = F[i][0];
      g0[i] = G[i][0];
      f1[i] = F[i][1];
      g1[i] = G[i][1];
    }
    bool b0, b1;
    if constexpr (PERT) {
      // Ey0, Ey1 are the departure's field (its mean-mode part is the
      // departure's); the full field adds the base's
      const R vby = uBy + mub * EB;
      collide_node_pert<R>(f0, g0, Ex0, EB + Ey0, Ey0, sy, uBy, vby, sf, fdq, mub, wp, wm, cp, cm, gwp, gwm, b0);
      collide_node_pert<R>(f1, g1, Ex1, EB + Ey1, Ey1, sy, uBy, vby, sf, fdq, mub, wp, wm, cp, cm, gwp, gwm, b1);
    } else {
      collide_node<S, R>(f0, g0, Ex0, Ey0, sy, sf, fdq, mub, wp, wm, cp, cm, gwp, gwm, b0);
      collide_node<S, R>(f1, g1, Ex1, Ey1, sy, sf, fdq, mub, wp, wm, cp, cm, gwp, gwm, b1);
    }
    if (owned && (b0 || b1)) bad = true;
    // pulled values at (xc, xc + 1): x-shift by c_x
    // c_x = +1 (1, 5, 8): [0] from the left lane's second node, [1] own first
    // c_x = -1 (3, 6, 7): [0] own second node, [1] from the right lane's first
    const R P1f0 = from_left(f1[1]), P5f0 = from_left(f1[5]), P8f0 = from_left(f1[8]);
    const R P3f1 = from_right(f0[3]), P6f1 = from_right(f0[6]), P7f1 = from_right(f0[7]);
    const R P1g0 = from_left(g1[1]), P5g0 = from_left(g1[5]), P8g0 = from_left(g1[8]);
    const R P3g1 = from_right(g0[3]), P6g1 = from_right(g0[6]), P7g1 = from_right(g0[7]);
    const R Pf1[2] = {P1f0, f0[1]}, Pf5[2] = {P5f0, f0[5]}, Pf8[2] = {P8f0, f0[8]};
    const R Pf3[2] = {f1[3], P3f1}, Pf6[2] = {f1[6], P6f1}, Pf7[2] = {f1[7], P7f1};
    const R Pg1[2] = {P1g0, g0[1]}, Pg5[2] = {P5g0, g0[5]}, Pg8[2] = {P8g0, g0[8]};
    const R Pg3[2] = {g1[3], P3g1}, Pg6[2] = {g1[6], P6g1}, Pg7[2] = {g1[7], P7g1};
    const R f0c[2] = {f0[0], f1[0]}, g0c[2] = {g0[0], g1[0]};
    const R f2c[2] = {f0[2], f1[2]}, g2c[2] = {g0[2], g1[2]};
    const R f4c[2] = {f0[4], f1[4]}, g4c[2] = {g0[4], g1[4]};
    // own (unshifted in x) values used by the wall rules; f5..f8 carry the
    // row change of the shift, which a bounce within the row undoes
    const R f5c[2] = {f0[5], f1[5]}, f6c[2] = {f0[6], f1[6]}, f7c[2] = {f0[7], f1[7]}, f8c[2] = {f0[8], f1[8]};
    const R g5c[2] = {g0[5], g1[5]}, g6c[2] = {g0[6], g1[6]}, g7c[2] = {g0[7], g1[7]}, g8c[2] = {g0[8], g1[8]};
    R Un[6][2];
    {
      const R sh = sy - s_up;
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        Un[0][j] = f2c[j];
        Un[1][j] = Pf5[j];
        Un[2][j] = Pf6[j];
        Un[3][j] = g2c[j] + W1 * sh;
        Un[4][j] = Pg5[j] + W2 * sh;
        Un[5][j] = Pg6[j] + W2 * sh;
      }
    }
    if (r == 0) {
      // injector: bounce-back of f, anti-bounce-back of g (own node values)
      const R Exs[2] = {Ex0, Ex1}, Eys[2] = {Ey0, Ey1};
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        R n2, n5, n6;
        if constexpr (PERT) {
          // departure of the injected populations: the wall drift v_w =
          // mu_b E against the base's (0, mu_b E_B); with d = v_w - v_wB and
          // s = v_w + v_wB, (c.v_w)^2 - (c.v_wB)^2 = (c.d)(c.s)
          const R dx = mub * Exs[j], dy = mub * Eys[j], sx = dx, sy2 = dy + R(2) * mub * EB;
          const R w15 = R(1.5) * (dx * sx + dy * sy2);
          n2 = -g4c[j] + R(2) * W1 * rho0 * (R(4.5) * dy * sy2 - w15);
          n5 = -g7c[j] + R(2) * W2 * rho0 * (R(4.5) * (dx + dy) * (sx + sy2) - w15);
          n6 = -g8c[j] + R(2) * W2 * rho0 * (R(4.5) * (dy - dx) * (sy2 - sx) - w15);
        } else {
          const R wx = mub * Exs[j], wy = mub * Eys[j];
          const R w15 = R(1.5) * (wx * wx + wy * wy);
          const R c2 = wy, c5 = wx + wy, c6 = wy - wx;
          n2 = -(g4c[j] + R(2) * W1 * sy) + R(2) * W1 * rho0 * (R(1) + R(4.5) * c2 * c2 - w15);
          n5 = -(g7c[j] + R(2) * W2 * sy) + R(2) * W2 * rho0 * (R(1) + R(4.5) * c5 * c5 - w15);
          n6 = -(g8c[j] + R(2) * W2 * sy) + R(2) * W2 * rho0 * (R(1) + R(4.5) * c6 * c6 - w15);
        }
        Uc[0][j] = f4c[j] - wd1;
        Uc[1][j] = f7c[j] - wd2;
        Uc[2][j] = f8c[j] - wd2;
        Uc[3][j] = n2;
        Uc[4][j] = n5;
        Uc[5][j] = n6;
        if (owned && y0 == 0)
          qin += (((double)Store<S>::rt(n2) - (double)Store<S>::rt(g4c[j])) +
                  ((double)Store<S>::rt(n5) - (double)Store<S>::rt(g7c[j]))) +
                 ((double)Store<S>::rt(n6) - (double)Store<S>::rt(g8c[j]));
      }
    }
    // c_y = -1: populations of row r moving down into row r - 1
    R n4[2], n7[2], n8[2];
    {
      const R sh = sy - s_dn;
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        n4[j] = g4c[j] + W1 * sh;
        n7[j] = Pg7[j] + W2 * sh;
        n8[j] = Pg8[j] + W2 * sh;
      }
    }
    if (r > y0 && owned) {
      // the down-movers complete row r - 1; its up-movers came from below the
      // slab (pushed there) when r - 1 is the first row of a slab above y = 0
      const bool ups = !(r - 1 == y0 && push_dn);
      const long long c = row - P + xc;
      Pair<S>::st(fo + c, Hm[0][0], Hm[0][1]);
      Pair<S>::st(fo + pl + c, Hm[1][0], Hm[1][1]);
      Pair<S>::st(fo + 3 * pl + c, Hm[2][0], Hm[2][1]);
      Pair<S>::st(fo + 4 * pl + c, f4c[0], f4c[1]);
      Pair<S>::st(fo + 7 * pl + c, Pf7[0], Pf7[1]);
      Pair<S>::st(fo + 8 * pl + c, Pf8[0], Pf8[1]);
      Pair<S>::st(go + c, Hm[3][0], Hm[3][1]);
      Pair<S>::st(go + pl + c, Hm[4][0], Hm[4][1]);
      Pair<S>::st(go + 3 * pl + c, Hm[5][0], Hm[5][1]);
      Pair<S>::st(go + 4 * pl + c, n4[0], n4[1]);
      Pair<S>::st(go + 7 * pl + c, n7[0], n7[1]);
      Pair<S>::st(go + 8 * pl + c, n8[0], n8[1]);
      if (ups) {
        Pair<S>::st(fo + 2 * pl + c, Um[0][0], Um[0][1]);
        Pair<S>::st(fo + 5 * pl + c, Um[1][0], Um[1][1]);
        Pair<S>::st(fo + 6 * pl + c, Um[2][0], Um[2][1]);
        Pair<S>::st(go + 2 * pl + c, Um[3][0], Um[3][1]);
        Pair<S>::st(go + 5 * pl + c, Um[4][0], Um[4][1]);
        Pair<S>::st(go + 6 * pl + c, Um[5][0], Um[5][1]);
      }
      R q[2];
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const R h = (Store<S>::rt(Hm[3][j]) + Store<S>::rt(Hm[4][j])) + Store<S>::rt(Hm[5][j]);
        const R d = (Store<S>::rt(n4[j]) + Store<S>::rt(n7[j])) + Store<S>::rt(n8[j]);
        const R u = ups ? (Store<S>::rt(Um[3][j]) + Store<S>::rt(Um[4][j])) + Store<S>::rt(Um[5][j]) : R(0);
        q[j] = PERT ? (h + u) + d : s_dn + ((h + u) + d);  // PERT: the departure's charge
      }
      Pair<R>::st(rho_out + c, q[0], q[1]);
    }
    if (r == y0 && push_dn && owned) {
      // push the down-movers of the slab's first row into the row below
      const long long c = row - P + xc;
      Pair<S>::st(fo + 4 * pl + c, f4c[0], f4c[1]);
      Pair<S>::st(fo + 7 * pl + c, Pf7[0], Pf7[1]);
      Pair<S>::st(fo + 8 * pl + c, Pf8[0], Pf8[1]);
      Pair<S>::st(go + 4 * pl + c, n4[0], n4[1]);
      Pair<S>::st(go + 7 * pl + c, n7[0], n7[1]);
      Pair<S>::st(go + 8 * pl + c, n8[0], n8[1]);
      R q[2];
#pragma unroll
      for (int j = 0; j < 2; ++j) q[j] = (Store<S>::rt(n4[j]) + Store<S>::rt(n7[j])) + Store<S>::rt(n8[j]);
      Pair<R>::st(rx_dn + (long long)slab * P + xc, q[0], q[1]);
    }
    if (r == Ny - 1 && owned) {
      // collector: f bounces back; g leaves and re-enters from its own row
      const bool ups = !(r == y0 && push_dn);
      const long long c = row + xc;
      Pair<S>::st(fo + c, f0c[0], f0c[1]);
      Pair<S>::st(fo + pl + c, Pf1[0], Pf1[1]);
      Pair<S>::st(fo + 3 * pl + c, Pf3[0], Pf3[1]);
      Pair<S>::st(fo + 4 * pl + c, f2c[0] + wd1, f2c[1] + wd1);
      Pair<S>::st(fo + 7 * pl + c, f5c[0] + wd2, f5c[1] + wd2);
      Pair<S>::st(fo + 8 * pl + c, f6c[0] + wd2, f6c[1] + wd2);
      Pair<S>::st(go + c, g0c[0], g0c[1]);
      Pair<S>::st(go + pl + c, Pg1[0], Pg1[1]);
      Pair<S>::st(go + 3 * pl + c, Pg3[0], Pg3[1]);
      Pair<S>::st(go + 4 * pl + c, g4c[0], g4c[1]);
      Pair<S>::st(go + 7 * pl + c, Pg7[0], Pg7[1]);
      Pair<S>::st(go + 8 * pl + c, Pg8[0], Pg8[1]);
      if (ups) {
        Pair<S>::st(fo + 2 * pl + c, Uc[0][0], Uc[0][1]);
        Pair<S>::st(fo + 5 * pl + c, Uc[1][0], Uc[1][1]);
        Pair<S>::st(fo + 6 * pl + c, Uc[2][0], Uc[2][1]);
        Pair<S>::st(go + 2 * pl + c, Uc[3][0], Uc[3][1]);
        Pair<S>::st(go + 5 * pl + c, Uc[4][0], Uc[4][1]);
        Pair<S>::st(go + 6 * pl + c, Uc[5][0], Uc[5][1]);
      }
      R q[2];
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const R h = (Store<S>::rt(g0c[j]) + Store<S>::rt(Pg1[j])) + Store<S>::rt(Pg3[j]);
        const R d = (Store<S>::rt(g4c[j]) + Store<S>::rt(Pg7[j])) + Store<S>::rt(Pg8[j]);
        const R u = ups ? (Store<S>::rt(Uc[3][j]) + Store<S>::rt(Uc[4][j])) + Store<S>::rt(Uc[5][j]) : R(0);
        q[j] = PERT ? (h + u) + d : sy + ((h + u) + d);
        qout += ((double)Store<S>::rt(g2c[j]) + (double)Store<S>::rt(g5c[j])) + (double)Store<S>::rt(g6c[j]);
        qout -= ((double)Store<S>::rt(g4c[j]) + (double)Store<S>::rt(g7c[j])) + (double)Store<S>::rt(g8c[j]);
      }
      Pair<R>::st(rho_out + c, q[0], q[1]);
    }
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      Hm[0][j] = f0c[j];
      Hm[1][j] = Pf1[j];
      Hm[2][j] = Pf3[j];
      Hm[3][j] = g0c[j];
      Hm[4][j] = Pg1[j];
      Hm[5][j] = Pg3[j];
#pragma unroll
      for (int q = 0; q < 6; ++q) {
        Um[q][j] = Uc[q][j];
        Uc[q][j] = Un[q][j];
      }
      pm[j] = pc[j];
      pc[j] = pn[j];
    }
    sy_last = sy;
  }
  cp_async_wait<0>();
  if (push_up && owned) {
    // the slab's last row lacks only its down-movers (pushed by the slab
    // above); its own up-movers go into the first row of the slab above
    const bool ups = !(re == y0 && push_dn);
    const long long c = (long long)re * P + xc;
    Pair<S>::st(fo + c, Hm[0][0], Hm[0][1]);
    Pair<S>::st(fo + pl + c, Hm[1][0], Hm[1][1]);
    Pair<S>::st(fo + 3 * pl + c, Hm[2][0], Hm[2][1]);
    Pair<S>::st(go + c, Hm[3][0], Hm[3][1]);
    Pair<S>::st(go + pl + c, Hm[4][0], Hm[4][1]);
    Pair<S>::st(go + 3 * pl + c, Hm[5][0], Hm[5][1]);
    if (ups) {
      Pair<S>::st(fo + 2 * pl + c, Um[0][0], Um[0][1]);
      Pair<S>::st(fo + 5 * pl + c, Um[1][0], Um[1][1]);
      Pair<S>::st(fo + 6 * pl + c, Um[2][0], Um[2][1]);
      Pair<S>::st(go + 2 * pl + c, Um[3][0], Um[3][1]);
      Pair<S>::st(go + 5 * pl + c, Um[4][0], Um[4][1]);
      Pair<S>::st(go + 6 * pl + c, Um[5][0], Um[5][1]);
    }
    R q[2], e[2];
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const R h = (Store<S>::rt(Hm[3][j]) + Store<S>::rt(Hm[4][j])) + Store<S>::rt(Hm[5][j]);
      const R u = ups ? (Store<S>::rt(Um[3][j]) + Store<S>::rt(Um[4][j])) + Store<S>::rt(Um[5][j]) : R(0);
      q[j] = PERT ? h + u : sy_last + (h + u);
      e[j] = (Store<S>::rt(Uc[3][j]) + Store<S>::rt(Uc[4][j])) + Store<S>::rt(Uc[5][j]);
    }
    Pair<R>::st(rho_out + c, q[0], q[1]);
    const long long cu = c + P;
    Pair<S>::st(fo + 2 * pl + cu, Uc[0][0], Uc[0][1]);
    Pair<S>::st(fo + 5 * pl + cu, Uc[1][0], Uc[1][1]);
    Pair<S>::st(fo + 6 * pl + cu, Uc[2][0], Uc[2][1]);
    Pair<S>::st(go + 2 * pl + cu, Uc[3][0], Uc[3][1]);
    Pair<S>::st(go + 5 * pl + cu, Uc[4][0], Uc[4][1]);
    Pair<S>::st(go + 6 * pl + cu, Uc[5][0], Uc[5][1]);
    Pair<R>::st(rx_up + (long long)(slab + 1) * P + xc, e[0], e[1]);
  }
  if (bad) atomicOr(a.err, 1);
  if (y0 == 0) {
    double v = qin;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) a.flux_part[strip] = v;
  }
  if (y1 == Ny) {
    double v = qout;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) a.flux_part[ns + strip] = v;
  }
}

template <class S, class R, int NSTAGE, bool SPECX = false, bool PERT = false>
__global__ void __launch_bounds__(128) k_march2(StepArgs a) {
  extern __shared__ __align__(16) unsigned char march_smem[];
  // the forward transform (launched with programmatic dependent launch) may
  // become resident as this one-wave grid's CTAs finish; it waits for the
  // whole grid before it reads the charge density
  grid_dep_launch();
  const int gw = blockIdx.x * 4 + (threadIdx.x >> 5);
  march2_body<S, R, NSTAGE, SPECX, PERT>(
      a, gw % a.nstrips, gw / a.nstrips,
      march_smem + (size_t)(threadIdx.x >> 5) * March2Stages<S, R, NSTAGE, SPECX>::kBytesPerWarp);
}

// Batch: every warp of a fixed grid takes march items (run, strip, slab),
// full slabs first, from the step's counter until none is left; runs whose
// budget in the tick is used up are skipped.  Bounded to three CTAs per SM
// (168 registers, a few bytes spilled): at 180 registers only two fit and
// the batch step takes 320 instead of 280 us.
// With perturbation-form members (PERT) each item takes the form of its run.
template <bool PERT>
__global__ void __launch_bounds__(128, 3) k_batch_march(BatchTables t, int step) {
  extern __shared__ __align__(16) unsigned char march_smem[];
  grid_dep_launch();  // the forward transforms may take slots as this grid drains
  constexpr int NST = 2;
  unsigned char* ring = march_smem + (size_t)(threadIdx.x >> 5) * March2Stages<float, float, NST>::kBytesPerWarp;
  const int n = t.counts[1];
  for (int it = next_item_warp(t.work); it < n; it = next_item_warp(t.work)) {
    const int4 w = t.march_items[it];
    const BatchRunDesc& rd = t.runs[w.x];
    if (step >= rd.remaining) continue;  // whole warp
    const StepArgs a = rd.sa[rd.cur0 ^ (step & 1)];
    if (PERT && a.base_tab)
      march2_body<float, float, NST, false, true>(a, w.y, w.z, ring);
    else
      march2_body<float, float, NST>(a, w.y, w.z, ring);
  }
}

cudaError_t launch_batch_march(const BatchTables& t, int step, int grid, bool pert, cudaStream_t s) {
  const size_t sm = 4 * March2Stages<float, float, 2>::kBytesPerWarp;
  if (pert)
    k_batch_march<true><<<grid, 128, sm, s>>>(t, step);
  else
    k_batch_march<false><<<grid, 128, sm, s>>>(t, step);
  return cudaGetLastError();
}


// ---------------------------------------------------------------------------
// TMA form of the march (FP32 storage and compute, Nx >= 128).  The same
// walk, collision and routing as march2_body; what changes is how rows move
// between HBM and the warp:
//   - loads: one elected lane stages each row of the strip with three
//     cp.async.bulk.tensor copies (the 9 f planes and the 9 g planes as one
//     {68, 1, 9} box each, the potential fluctuation of the next row as a
//     {68, 1} box) into a two-stage shared-memory ring; an mbarrier per stage
//     counts the bytes in.  The box starts 4 columns left of the strip's
//     first (halo) column so that its x coordinate is 16-byte aligned; lanes
//     read their pair at offset 2 + 2 lane.  The two halo pairs that wrap
//     around the periodic x boundary (strip 0's lane 0 and the last strip's
//     right halo lane) fall outside the tensor and read the zero fill, so
//     those lanes fetch their own pair with 8-byte cp.async copies.
//   - stores: every row a warp completes inside its slab goes out as two
//     {60, 1, 9} tensor stores from a shared-memory tile (all 18 planes of
//     the strip's owned columns); the few partial rows at slab boundaries,
//     the pushes into neighbouring slabs and the collector row keep 8-byte
//     stores.
// Every wait on an mbarrier is bounded; a wait that gives up sets bit 1 of
// the run's error word (EHD_ETIMEOUT on the host), drains what the warp has
// in flight and ends the warp.
namespace tma {

constexpr int kLC = kTmaLoadCols;   // 68 loaded columns per row and plane
constexpr int kSC = kTmaStoreCols;  // 60 stored (owned) columns
constexpr unsigned kPlaneBytes = 9u * kLC * 4u;  // 2448: one {68, 1, 9} box
// per-warp shared memory (byte offsets; TMA destinations 128-byte aligned)
constexpr int kStF = 0;                  // [9][68] f of the staged row
constexpr int kStG = 2560;               // [9][68] g
constexpr int kStP = 5120;               // [68] potential fluctuation of the next row
constexpr int kStW = 5504;               // [20][2] the wrap lane's own pair (18 populations, potential)
constexpr int kStage = 5760;             // bytes per stage
// layout for NST stages, with (TSTORE) or without the out tile: stages, out
// tile [9][60] f then g, the stages' mbarriers
template <int NST, bool TSTORE>
struct Layout {
  static constexpr int kOutF = NST * kStage;
  static constexpr int kOutG = kOutF + 2176;
  static constexpr int kMbar = kOutF + (TSTORE ? 2 * 2176 : 0);
  static constexpr int kWarpBytes = kMbar + 128;
};
constexpr unsigned kWaitLimit = 1u << 22;

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned mbar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(mbar) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned mbar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(mbar), "r"(bytes) : "memory");
}
// bounded wait for the phase with the given parity; false if it gave up
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
__device__ __forceinline__ void load3d(unsigned dst, const CUtensorMap* map, int x, int y, unsigned mbar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];\n" ::"r"(dst),
      "l"(map), "r"(x), "r"(y), "r"(0), "r"(mbar)
      : "memory");
}
__device__ __forceinline__ void load2d(unsigned dst, const CUtensorMap* map, int x, int y, unsigned mbar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n" ::"r"(dst),
      "l"(map), "r"(x), "r"(y), "r"(mbar)
      : "memory");
}
__device__ __forceinline__ void store3d(const CUtensorMap* map, int x, int y, unsigned src) {
  asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%1, %2, %3}], [%4];\n" ::"l"(map), "r"(x),
               "r"(y), "r"(0), "r"(src)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read0() { asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory"); }
__device__ __forceinline__ void bulk_wait0() { asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory"); }

}  // namespace tma

template <int NST, bool TSTORE>
__device__ __forceinline__ void march_tma_body(const StepArgs& a, const MarchTma& tm, int strip, int slab,
                                               unsigned char* ws) {
  using namespace tma;
  using L = Layout<NST, TSTORE>;
  constexpr int kOutF = L::kOutF, kOutG = L::kOutG, kMbar = L::kMbar;
  using R = float;
  const int lane = threadIdx.x & 31;
  const int Nx = a.Nx, Ny = a.Ny, P = a.P, ns = a.nstrips;
  const int y0 = slab * a.slab_rows;
  if (y0 >= Ny) return;  // whole warp
  const int y1 = min(y0 + a.slab_rows, Ny);
  const int xs = strip * 60;
  const int x0 = xs - 4;                 // box start (16-byte aligned; -4 for strip 0)
  const int xcol = xs - 2 + 2 * lane;    // the lane's pair, unwrapped
  const int xc = (xcol + 2 * Nx) % Nx;   // wrapped (even)
  const bool owned = lane >= 1 && lane <= 30 && xs + 2 * (lane - 1) < Nx;
  // the halo pairs across the periodic boundary, outside the tensor's x range
  const bool wrap = (strip == 0 && lane == 0) || (strip == ns - 1 && xcol == Nx);
  const int toff = 2 + 2 * lane;         // the pair's column in the staged box
  const long long pl = a.plane;
  const float* __restrict__ fin = static_cast<const float*>(a.fin);
  const float* __restrict__ gin = static_cast<const float*>(a.gin);
  float* __restrict__ fo = static_cast<float*>(a.fout);
  float* __restrict__ go = static_cast<float*>(a.gout);
  R* __restrict__ rho_out = static_cast<R*>(a.rhoc_out);
  const R* __restrict__ dphi = static_cast<const R*>(a.dphi);
  const R* __restrict__ Ebar = static_cast<const R*>(a.Ebar);
  const float* __restrict__ rch = a.rch;
  const R wp = (R)a.wp, wm = (R)a.wm, gwp = (R)a.gwp, gwm = (R)a.gwm;
  const R cp = R(1) - R(0.5) * wp, cm = R(1) - R(0.5) * wm;
  const R mub = (R)a.mub, rho0 = (R)a.rho0;
  const R gwall = (a.wall_mode == 0) ? R(-1) : R(0);
  const R W1 = (R)kW1, W2 = (R)kW2;
  const R fb = (R)a.fb, fd = (R)a.fd, fdq = (R)a.fdq;
  const R wd1 = W1 * fd, wd2 = W2 * fd;
  const int rs = y0, re = y1 - 1;
  const bool push_dn = y0 > 0, push_up = y1 < Ny;
  R* __restrict__ rx_dn = static_cast<R*>(a.rhoc_dn);
  R* __restrict__ rx_up = static_cast<R*>(a.rhoc_up);
  R sy_last = R(0);

  const unsigned mbar0 = smem_u32(ws + kMbar);
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < NST; ++k) mbar_init(mbar0 + 8 * k);
    fence_mbar_init();
  }
  __syncwarp();

  // stage one row: the elected lane's tensor copies, the wrap lane's pair
  auto issue = [&](int row_y, int stage) {
    unsigned char* st = ws + stage * kStage;
    const bool next = row_y + 1 < Ny;
    if (lane == 0) {
      const unsigned mb = mbar0 + 8 * stage;
      fence_async_smem();  // the stage's previous contents were read through the generic proxy
      mbar_expect_tx(mb, 2 * kPlaneBytes + (next ? kLC * 4u : 0u));
      load3d(smem_u32(st + kStF), &tm.f, x0, row_y, mb);
      load3d(smem_u32(st + kStG), &tm.g, x0, row_y, mb);
      if (next) load2d(smem_u32(st + kStP), &tm.dphi, x0, row_y + 1, mb);
    }
    if (wrap) {
      const long long c = (long long)row_y * P + xc;
      float* w = reinterpret_cast<float*>(st + kStW);
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        cp_async_elem<8>(w + 2 * i, fin + i * pl + c);
        cp_async_elem<8>(w + 2 * (9 + i), gin + i * pl + c);
      }
      if (next) cp_async_elem<8>(w + 36, dphi + c + P);
    }
    cp_async_commit();
  };

  // carried rows, [k][j]: H (c_y = 0) of row r-1, U (c_y = +1) of rows r-1, r
  R Hm[6][2] = {}, Um[6][2] = {}, Uc[6][2] = {};
  R pm[2], pc[2];
  {
    const long long c = (long long)rs * P + xc;
    pc[0] = dphi[c];
    pc[1] = dphi[c + 1];
    if (rs > 0) {
      pm[0] = dphi[c - P];
      pm[1] = dphi[c - P + 1];
    } else {
      pm[0] = gwall * pc[0];
      pm[1] = gwall * pc[1];
    }
  }
  double qin = 0.0, qout = 0.0;
  bool bad = false, timed_out = false;
  // the row scalars (mean field, charge shifts) of row r, loaded a row ahead
  R Eb_n = Ebar[rs], sy_n = rch[rs];
  R sup_n = (rs + 1 < Ny) ? rch[rs + 1] : sy_n, sdn_n = (rs > 0) ? rch[rs - 1] : sy_n;
  bool out_pending = false;  // a tensor store of the out tile may still be reading it
  int stuck = -1;            // iteration whose wait gave up

#pragma unroll
  for (int k = 0; k < NST - 1; ++k) {
    if (rs + k <= re) issue(rs + k, k);
    else cp_async_commit();
  }
  for (int r = rs; r <= re; ++r) {
    const long long row = (long long)r * P;
    const int kk = r - rs;
    const int stg = kk % NST;
    __syncwarp();  // every lane has finished reading the stage about to be refilled
    if (r + NST - 1 <= re) issue(r + NST - 1, (kk + NST - 1) % NST);
    else cp_async_commit();  // keep one group per iteration
    const R Ebr = Eb_n, sy = sy_n, s_up = sup_n, s_dn = sdn_n;
    if (r + 1 <= re) {
      Eb_n = Ebar[r + 1];
      sy_n = rch[r + 1];
      sup_n = (r + 2 < Ny) ? rch[r + 2] : sy_n;
      sdn_n = rch[r];
    }
    if (!mbar_wait(mbar0 + 8 * stg, (unsigned)(kk / NST) & 1u)) {
      timed_out = true;
      stuck = kk;
      break;
    }
    cp_async_wait<NST - 1>();  // the wrap lane's copies of row r (later rows' may be pending)
    const unsigned char* st = ws + stg * kStage;
    R F[9][2], G[9][2];
    R pn[2];
    if (wrap) {
      const float2* w = reinterpret_cast<const float2*>(st + kStW);
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        const float2 vf = w[i], vg = w[9 + i];
        F[i][0] = vf.x;
        F[i][1] = vf.y;
        G[i][0] = vg.x;
        G[i][1] = vg.y;
      }
      const float2 vp = w[18];
      pn[0] = vp.x;
      pn[1] = vp.y;
    } else {
      const float* tf = reinterpret_cast<const float*>(st + kStF) + toff;
      const float* tg = reinterpret_cast<const float*>(st + kStG) + toff;
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        const float2 vf = *reinterpret_cast<const float2*>(tf + i * kLC);
        const float2 vg = *reinterpret_cast<const float2*>(tg + i * kLC);
        F[i][0] = vf.x;
        F[i][1] = vf.y;
        G[i][0] = vg.x;
        G[i][1] = vg.y;
      }
      const float2 vp = *reinterpret_cast<const float2*>(reinterpret_cast<const float*>(st + kStP) + toff);
      pn[0] = vp.x;
      pn[1] = vp.y;
    }
    if (r + 1 >= Ny) {
      pn[0] = gwall * pc[0];
      pn[1] = gwall * pc[1];
    }
    const R sf = fb + fd * (R)r;
    R Ex0, Ex1;
    {
      const R pWl = from_left(pc[1]);   // phi(xc - 1)
      const R pEr = from_right(pc[0]);  // phi(xc + 2)
      Ex0 = R(-0.5) * (pc[1] - pWl);
      Ex1 = R(-0.5) * (pEr - pc[0]);
    }
    const R Ey0 = Ebr - R(0.5) * (pn[0] - pm[0]), Ey1 = Ebr - R(0.5) * (pn[1] - pm[1]);
    R f0[9], g0[9], f1[9], g1[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      f0[i] = F[i][0];
      g0[i] = G[i][0];
      f1[i] = F[i][1];
      g1[i] = G[i][1];
    }
    bool b0, b1;
    collide_node<float, R>(f0, g0, Ex0, Ey0, sy, sf, fdq, mub, wp, wm, cp, cm, gwp, gwm, b0);
    collide_node<float, R>(f1, g1, Ex1, Ey1, sy, sf, fdq, mub, wp, wm, cp, cm, gwp, gwm, b1);
    if (owned && (b0 || b1)) bad = true;
    const R P1f0 = from_left(f1[1]), P5f0 = from_left(f1[5]), P8f0 = from_left(f1[8]);
    const R P3f1 = from_right(f0[3]), P6f1 = from_right(f0[6]), P7f1 = from_right(f0[7]);
    const R P1g0 = from_left(g1[1]), P5g0 = from_left(g1[5]), P8g0 = from_left(g1[8]);
    const R P3g1 = from_right(g0[3]), P6g1 = from_right(g0[6]), P7g1 = from_right(g0[7]);
    const R Pf1[2] = {P1f0, f0[1]}, Pf5[2] = {P5f0, f0[5]}, Pf8[2] = {P8f0, f0[8]};
    const R Pf3[2] = {f1[3], P3f1}, Pf6[2] = {f1[6], P6f1}, Pf7[2] = {f1[7], P7f1};
    const R Pg1[2] = {P1g0, g0[1]}, Pg5[2] = {P5g0, g0[5]}, Pg8[2] = {P8g0, g0[8]};
    const R Pg3[2] = {g1[3], P3g1}, Pg6[2] = {g1[6], P6g1}, Pg7[2] = {g1[7], P7g1};
    const R f0c[2] = {f0[0], f1[0]}, g0c[2] = {g0[0], g1[0]};
    const R f2c[2] = {f0[2], f1[2]}, g2c[2] = {g0[2], g1[2]};
    const R f4c[2] = {f0[4], f1[4]}, g4c[2] = {g0[4], g1[4]};
    const R f5c[2] = {f0[5], f1[5]}, f6c[2] = {f0[6], f1[6]}, f7c[2] = {f0[7], f1[7]}, f8c[2] = {f0[8], f1[8]};
    const R g5c[2] = {g0[5], g1[5]}, g6c[2] = {g0[6], g1[6]}, g7c[2] = {g0[7], g1[7]}, g8c[2] = {g0[8], g1[8]};
    R Un[6][2];
    {
      const R sh = sy - s_up;
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        Un[0][j] = f2c[j];
        Un[1][j] = Pf5[j];
        Un[2][j] = Pf6[j];
        Un[3][j] = g2c[j] + W1 * sh;
        Un[4][j] = Pg5[j] + W2 * sh;
        Un[5][j] = Pg6[j] + W2 * sh;
      }
    }
    if (r == 0) {
      const R Exs[2] = {Ex0, Ex1}, Eys[2] = {Ey0, Ey1};
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const R wx = mub * Exs[j], wy = mub * Eys[j];
        const R w15 = R(1.5) * (wx * wx + wy * wy);
        const R c2 = wy, c5 = wx + wy, c6 = wy - wx;
        const R n2 = -(g4c[j] + R(2) * W1 * sy) + R(2) * W1 * rho0 * (R(1) + R(4.5) * c2 * c2 - w15);
        const R n5 = -(g7c[j] + R(2) * W2 * sy) + R(2) * W2 * rho0 * (R(1) + R(4.5) * c5 * c5 - w15);
        const R n6 = -(g8c[j] + R(2) * W2 * sy) + R(2) * W2 * rho0 * (R(1) + R(4.5) * c6 * c6 - w15);
        Uc[0][j] = f4c[j] - wd1;
        Uc[1][j] = f7c[j] - wd2;
        Uc[2][j] = f8c[j] - wd2;
        Uc[3][j] = n2;
        Uc[4][j] = n5;
        Uc[5][j] = n6;
        if (owned && y0 == 0)
          qin += (((double)n2 - (double)g4c[j]) + ((double)n5 - (double)g7c[j])) + ((double)n6 - (double)g8c[j]);
      }
    }
    R n4[2], n7[2], n8[2];
    {
      const R sh = sy - s_dn;
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        n4[j] = g4c[j] + W1 * sh;
        n7[j] = Pg7[j] + W2 * sh;
        n8[j] = Pg8[j] + W2 * sh;
      }
    }
    if (r > y0) {
      // row r - 1 is complete
      const bool ups = !(r - 1 == y0 && push_dn);
      const long long c = row - P + xc;
      if (ups && !TSTORE) {
        if (owned) {
          Pair<float>::st(fo + c, Hm[0][0], Hm[0][1]);
          Pair<float>::st(fo + pl + c, Hm[1][0], Hm[1][1]);
          Pair<float>::st(fo + 2 * pl + c, Um[0][0], Um[0][1]);
          Pair<float>::st(fo + 3 * pl + c, Hm[2][0], Hm[2][1]);
          Pair<float>::st(fo + 4 * pl + c, f4c[0], f4c[1]);
          Pair<float>::st(fo + 5 * pl + c, Um[1][0], Um[1][1]);
          Pair<float>::st(fo + 6 * pl + c, Um[2][0], Um[2][1]);
          Pair<float>::st(fo + 7 * pl + c, Pf7[0], Pf7[1]);
          Pair<float>::st(fo + 8 * pl + c, Pf8[0], Pf8[1]);
          Pair<float>::st(go + c, Hm[3][0], Hm[3][1]);
          Pair<float>::st(go + pl + c, Hm[4][0], Hm[4][1]);
          Pair<float>::st(go + 2 * pl + c, Um[3][0], Um[3][1]);
          Pair<float>::st(go + 3 * pl + c, Hm[5][0], Hm[5][1]);
          Pair<float>::st(go + 4 * pl + c, n4[0], n4[1]);
          Pair<float>::st(go + 5 * pl + c, Um[4][0], Um[4][1]);
          Pair<float>::st(go + 6 * pl + c, Um[5][0], Um[5][1]);
          Pair<float>::st(go + 7 * pl + c, n7[0], n7[1]);
          Pair<float>::st(go + 8 * pl + c, n8[0], n8[1]);
        }
      } else if (ups) {
        // a whole row of the slab: through the out tile and two tensor stores
        if (out_pending) {
          if (lane == 0) bulk_wait_read0();
          __syncwarp();
        }
        if (owned) {
          float* of = reinterpret_cast<float*>(ws + kOutF) + 2 * (lane - 1);
          float* og = reinterpret_cast<float*>(ws + kOutG) + 2 * (lane - 1);
          const R vf[9][2] = {{Hm[0][0], Hm[0][1]}, {Hm[1][0], Hm[1][1]}, {Um[0][0], Um[0][1]},
                              {Hm[2][0], Hm[2][1]}, {f4c[0], f4c[1]},     {Um[1][0], Um[1][1]},
                              {Um[2][0], Um[2][1]}, {Pf7[0], Pf7[1]},     {Pf8[0], Pf8[1]}};
          const R vg[9][2] = {{Hm[3][0], Hm[3][1]}, {Hm[4][0], Hm[4][1]}, {Um[3][0], Um[3][1]},
                              {Hm[5][0], Hm[5][1]}, {n4[0], n4[1]},       {Um[4][0], Um[4][1]},
                              {Um[5][0], Um[5][1]}, {n7[0], n7[1]},       {n8[0], n8[1]}};
#pragma unroll
          for (int i = 0; i < 9; ++i) {
            *reinterpret_cast<float2*>(of + i * kSC) = make_float2(vf[i][0], vf[i][1]);
            *reinterpret_cast<float2*>(og + i * kSC) = make_float2(vg[i][0], vg[i][1]);
          }
        }
        __syncwarp();
        if (lane == 0) {
          fence_async_smem();
          store3d(&tm.fo, xs, r - 1, smem_u32(ws + kOutF));
          store3d(&tm.go, xs, r - 1, smem_u32(ws + kOutG));
          bulk_commit();
        }
        out_pending = true;
      } else if (owned) {
        Pair<float>::st(fo + c, Hm[0][0], Hm[0][1]);
        Pair<float>::st(fo + pl + c, Hm[1][0], Hm[1][1]);
        Pair<float>::st(fo + 3 * pl + c, Hm[2][0], Hm[2][1]);
        Pair<float>::st(fo + 4 * pl + c, f4c[0], f4c[1]);
        Pair<float>::st(fo + 7 * pl + c, Pf7[0], Pf7[1]);
        Pair<float>::st(fo + 8 * pl + c, Pf8[0], Pf8[1]);
        Pair<float>::st(go + c, Hm[3][0], Hm[3][1]);
        Pair<float>::st(go + pl + c, Hm[4][0], Hm[4][1]);
        Pair<float>::st(go + 3 * pl + c, Hm[5][0], Hm[5][1]);
        Pair<float>::st(go + 4 * pl + c, n4[0], n4[1]);
        Pair<float>::st(go + 7 * pl + c, n7[0], n7[1]);
        Pair<float>::st(go + 8 * pl + c, n8[0], n8[1]);
      }
      if (owned) {
        R q[2];
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          const R h = (Hm[3][j] + Hm[4][j]) + Hm[5][j];
          const R d = (n4[j] + n7[j]) + n8[j];
          const R u = ups ? (Um[3][j] + Um[4][j]) + Um[5][j] : R(0);
          q[j] = s_dn + ((h + u) + d);
        }
        Pair<R>::st(rho_out + c, q[0], q[1]);
      }
    }
    if (r == y0 && push_dn && owned) {
      const long long c = row - P + xc;
      Pair<float>::st(fo + 4 * pl + c, f4c[0], f4c[1]);
      Pair<float>::st(fo + 7 * pl + c, Pf7[0], Pf7[1]);
      Pair<float>::st(fo + 8 * pl + c, Pf8[0], Pf8[1]);
      Pair<float>::st(go + 4 * pl + c, n4[0], n4[1]);
      Pair<float>::st(go + 7 * pl + c, n7[0], n7[1]);
      Pair<float>::st(go + 8 * pl + c, n8[0], n8[1]);
      R q[2];
#pragma unroll
      for (int j = 0; j < 2; ++j) q[j] = (n4[j] + n7[j]) + n8[j];
      Pair<R>::st(rx_dn + (long long)slab * P + xc, q[0], q[1]);
    }
    if (r == Ny - 1 && owned) {
      const bool ups = !(r == y0 && push_dn);
      const long long c = row + xc;
      Pair<float>::st(fo + c, f0c[0], f0c[1]);
      Pair<float>::st(fo + pl + c, Pf1[0], Pf1[1]);
      Pair<float>::st(fo + 3 * pl + c, Pf3[0], Pf3[1]);
      Pair<float>::st(fo + 4 * pl + c, f2c[0] + wd1, f2c[1] + wd1);
      Pair<float>::st(fo + 7 * pl + c, f5c[0] + wd2, f5c[1] + wd2);
      Pair<float>::st(fo + 8 * pl + c, f6c[0] + wd2, f6c[1] + wd2);
      Pair<float>::st(go + c, g0c[0], g0c[1]);
      Pair<float>::st(go + pl + c, Pg1[0], Pg1[1]);
      Pair<float>::st(go + 3 * pl + c, Pg3[0], Pg3[1]);
      Pair<float>::st(go + 4 * pl + c, g4c[0], g4c[1]);
      Pair<float>::st(go + 7 * pl + c, Pg7[0], Pg7[1]);
      Pair<float>::st(go + 8 * pl + c, Pg8[0], Pg8[1]);
      if (ups) {
        Pair<float>::st(fo + 2 * pl + c, Uc[0][0], Uc[0][1]);
        Pair<float>::st(fo + 5 * pl + c, Uc[1][0], Uc[1][1]);
        Pair<float>::st(fo + 6 * pl + c, Uc[2][0], Uc[2][1]);
        Pair<float>::st(go + 2 * pl + c, Uc[3][0], Uc[3][1]);
        Pair<float>::st(go + 5 * pl + c, Uc[4][0], Uc[4][1]);
        Pair<float>::st(go + 6 * pl + c, Uc[5][0], Uc[5][1]);
      }
      R q[2];
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const R h = (g0c[j] + Pg1[j]) + Pg3[j];
        const R d = (g4c[j] + Pg7[j]) + Pg8[j];
        const R u = ups ? (Uc[3][j] + Uc[4][j]) + Uc[5][j] : R(0);
        q[j] = sy + ((h + u) + d);
        qout += ((double)g2c[j] + (double)g5c[j]) + (double)g6c[j];
        qout -= ((double)g4c[j] + (double)g7c[j]) + (double)g8c[j];
      }
      Pair<R>::st(rho_out + c, q[0], q[1]);
    }
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      Hm[0][j] = f0c[j];
      Hm[1][j] = Pf1[j];
      Hm[2][j] = Pf3[j];
      Hm[3][j] = g0c[j];
      Hm[4][j] = Pg1[j];
      Hm[5][j] = Pg3[j];
#pragma unroll
      for (int q = 0; q < 6; ++q) {
        Um[q][j] = Uc[q][j];
        Uc[q][j] = Un[q][j];
      }
      pm[j] = pc[j];
      pc[j] = pn[j];
    }
    sy_last = sy;
  }
  cp_async_wait<0>();
  if (timed_out) {
    // drain the warp's tensor copies in flight (again bounded): the row it
    // waited for and the next row, if that was issued; report; end the warp
    if (lane == 0) {
      atomicOr(a.err, 2);
      for (int k = stuck; k < stuck + NST && rs + k <= re; ++k) mbar_wait(mbar0 + 8 * (k % NST), (unsigned)(k / NST) & 1u);
      bulk_wait0();
    }
    __syncwarp();
    return;
  }
  if (push_up && owned) {
    const bool ups = !(re == y0 && push_dn);
    const long long c = (long long)re * P + xc;
    Pair<float>::st(fo + c, Hm[0][0], Hm[0][1]);
    Pair<float>::st(fo + pl + c, Hm[1][0], Hm[1][1]);
    Pair<float>::st(fo + 3 * pl + c, Hm[2][0], Hm[2][1]);
    Pair<float>::st(go + c, Hm[3][0], Hm[3][1]);
    Pair<float>::st(go + pl + c, Hm[4][0], Hm[4][1]);
    Pair<float>::st(go + 3 * pl + c, Hm[5][0], Hm[5][1]);
    if (ups) {
      Pair<float>::st(fo + 2 * pl + c, Um[0][0], Um[0][1]);
      Pair<float>::st(fo + 5 * pl + c, Um[1][0], Um[1][1]);
      Pair<float>::st(fo + 6 * pl + c, Um[2][0], Um[2][1]);
      Pair<float>::st(go + 2 * pl + c, Um[3][0], Um[3][1]);
      Pair<float>::st(go + 5 * pl + c, Um[4][0], Um[4][1]);
      Pair<float>::st(go + 6 * pl + c, Um[5][0], Um[5][1]);
    }
    R q[2], e[2];
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const R h = (Hm[3][j] + Hm[4][j]) + Hm[5][j];
      const R u = ups ? (Um[3][j] + Um[4][j]) + Um[5][j] : R(0);
      q[j] = sy_last + (h + u);
      e[j] = (Uc[3][j] + Uc[4][j]) + Uc[5][j];
    }
    Pair<R>::st(rho_out + c, q[0], q[1]);
    const long long cu = c + P;
    Pair<float>::st(fo + 2 * pl + cu, Uc[0][0], Uc[0][1]);
    Pair<float>::st(fo + 5 * pl + cu, Uc[1][0], Uc[1][1]);
    Pair<float>::st(fo + 6 * pl + cu, Uc[2][0], Uc[2][1]);
    Pair<float>::st(go + 2 * pl + cu, Uc[3][0], Uc[3][1]);
    Pair<float>::st(go + 5 * pl + cu, Uc[4][0], Uc[4][1]);
    Pair<float>::st(go + 6 * pl + cu, Uc[5][0], Uc[5][1]);
    Pair<R>::st(rx_up + (long long)(slab + 1) * P + xc, e[0], e[1]);
  }
  if (lane == 0) bulk_wait0();  // the out tile is read and the stores are done before the warp ends
  __syncwarp();
  if (bad) atomicOr(a.err, 1);
  if (y0 == 0) {
    double v = qin;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) a.flux_part[strip] = v;
  }
  if (y1 == Ny) {
    double v = qout;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) a.flux_part[ns + strip] = v;
  }
}

template <int NST, bool TSTORE>
__global__ void __launch_bounds__(128, 3) k_march_tma(StepArgs a, const __grid_constant__ MarchTma tm) {
  extern __shared__ __align__(128) unsigned char march_smem[];
  // tensor-copy destinations want 128-byte aligned shared memory: round the
  // dynamic allocation's start up (it is requested 128 bytes larger)
  const unsigned base = tma::smem_u32(march_smem);
  unsigned char* ws0 = march_smem + (((base + 127u) & ~127u) - base);
  const int gw = blockIdx.x * 4 + (threadIdx.x >> 5);
  march_tma_body<NST, TSTORE>(a, tm, gw % a.nstrips, gw / a.nstrips,
                              ws0 + (size_t)(threadIdx.x >> 5) * tma::Layout<NST, TSTORE>::kWarpBytes);
}

bool march_tma_supported(int Nx) { return Nx >= 128 && Nx <= 2048; }

cudaError_t launch_march_tma(const StepArgs& a, const MarchTma& m, int form, cudaStream_t s) {
  if (!march_tma_supported(a.Nx) || a.cols_per_lane != 2 || a.ex || !a.rch) return cudaErrorInvalidValue;
  const long long warps = (long long)a.nstrips * ((a.Ny + a.slab_rows - 1) / a.slab_rows);
  const unsigned grid = (unsigned)((warps + 3) / 4);
  switch (form) {
    case 1: k_march_tma<2, false><<<grid, 128, 4 * tma::Layout<2, false>::kWarpBytes + 128, s>>>(a, m); break;
    case 2: k_march_tma<2, true><<<grid, 128, 4 * tma::Layout<2, true>::kWarpBytes + 128, s>>>(a, m); break;
    case 3: k_march_tma<3, false><<<grid, 128, 4 * tma::Layout<3, false>::kWarpBytes + 128, s>>>(a, m); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

namespace {
using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiled encoder() {
  static EncodeTiled fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiled>(p);
  }
  return fn;
}
cudaError_t encode(CUtensorMap* m, const void* base, int rank, int Nx, int Ny, int P, int box_x) {
  EncodeTiled fn = encoder();
  if (!fn) return cudaErrorNotSupported;
  const cuuint64_t dims[3] = {(cuuint64_t)Nx, (cuuint64_t)Ny, 9};
  const cuuint64_t strides[2] = {(cuuint64_t)P * 4, (cuuint64_t)P * 4 * (cuuint64_t)Ny};
  const cuuint32_t box[3] = {(cuuint32_t)box_x, 1, 9};
  const cuuint32_t estr[3] = {1, 1, 1};
  const CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, (cuuint32_t)rank, const_cast<void*>(base), dims, strides,
                        box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

}  // namespace

cudaError_t tma_encode_2d(CUtensorMap* m, const void* base, unsigned long long inner, unsigned long long outer,
                          unsigned long long row_bytes, unsigned box_inner, unsigned box_outer) {
  EncodeTiled fn = encoder();
  if (!fn) return cudaErrorNotSupported;
  const cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)outer};
  const cuuint64_t strides[1] = {(cuuint64_t)row_bytes};
  const cuuint32_t box[2] = {(cuuint32_t)box_inner, (cuuint32_t)box_outer};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(base), dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

namespace {
}  // namespace

cudaError_t march_tma_encode(MarchTma* m, const void* fin, const void* gin, const void* dphi, void* fout, void* gout,
                             int Nx, int Ny, int P) {
  cudaError_t e;
  if ((e = encode(&m->f, fin, 3, Nx, Ny, P, tma::kLC)) != cudaSuccess) return e;
  if ((e = encode(&m->g, gin, 3, Nx, Ny, P, tma::kLC)) != cudaSuccess) return e;
  if ((e = encode(&m->dphi, dphi, 2, Nx, Ny, P, tma::kLC)) != cudaSuccess) return e;
  if ((e = encode(&m->fo, fout, 3, Nx, Ny, P, tma::kSC)) != cudaSuccess) return e;
  return encode(&m->go, gout, 3, Nx, Ny, P, tma::kSC);
}

namespace {
template <class S, class R, int NST>
cudaError_t march_n(const StepArgs& a, cudaStream_t s) {
  const long long warps = (long long)a.nstrips * ((a.Ny + a.slab_rows - 1) / a.slab_rows);
  k_march<S, R, NST><<<(unsigned)((warps + 3) / 4), 128, 4 * MarchStages<S, NST>::kBytesPerWarp, s>>>(a);
  return cudaGetLastError();
}

template <class S, class R, int NST, bool SPECX = false>
cudaError_t march2_n(const StepArgs& a, cudaStream_t s) {
  if (a.slab_off < 0 || a.slab_off >= a.slab_rows) return cudaErrorInvalidValue;
  const long long warps = (long long)a.nstrips * ((a.Ny + a.slab_off + a.slab_rows - 1) / a.slab_rows);
  const unsigned grid = (unsigned)((warps + 3) / 4);
  const size_t smem = 4 * March2Stages<S, R, NST, SPECX>::kBytesPerWarp;
  const bool pdl = (a.pdl & 8) != 0;  // the step kernel waits for phi after staging its first rows
  if constexpr (sizeof(R) == 4 && !SPECX) {
    if (a.base_tab) return launch_ex(pdl, k_march2<S, R, NST, false, true>, dim3(grid), dim3(128), smem, s, a);
  }
  return launch_ex(pdl, k_march2<S, R, NST, SPECX>, dim3(grid), dim3(128), smem, s, a);
}

template <class S, class R>
cudaError_t march_t(const StepArgs& a, cudaStream_t s) {
  if (a.ex) {  // spectral E_x: march form, two columns per lane, ring depth 2
    if (a.cols_per_lane != 2 || a.ring_depth != 2) return cudaErrorInvalidValue;
    return march2_n<S, R, 2, true>(a, s);
  }
  if (a.cols_per_lane == 2) {
    switch (a.ring_depth) {
      case 2: return march2_n<S, R, 2>(a, s);
      case 4: return march2_n<S, R, 4>(a, s);
      default: return march2_n<S, R, 3>(a, s);
    }
  }
  switch (a.ring_depth) {
    case 2: return march_n<S, R, 2>(a, s);
    case 4: return march_n<S, R, 4>(a, s);
    case 6: return march_n<S, R, 6>(a, s);
    default: return march_n<S, R, 3>(a, s);
  }
}

template <class K>
cudaError_t allow_smem(K kernel) {
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaFuncAttributes fa;
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, kernel);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
  return e;
}

template <class S, class R>
cudaError_t attrs_t() {
  cudaError_t e;
  if constexpr (sizeof(R) == 4) {
    if ((e = allow_smem(k_march2<S, R, 2, false, true>)) != cudaSuccess) return e;
    if ((e = allow_smem(k_march2<S, R, 3, false, true>)) != cudaSuccess) return e;
    if ((e = allow_smem(k_march2<S, R, 4, false, true>)) != cudaSuccess) return e;
  }
  if ((e = allow_smem(k_batch_march<false>)) != cudaSuccess) return e;
  if ((e = allow_smem(k_batch_march<true>)) != cudaSuccess) return e;
  if ((e = allow_smem(k_march2<S, R, 2>)) != cudaSuccess) return e;
  if ((e = allow_smem(k_march2<S, R, 2, true>)) != cudaSuccess) return e;
  if ((e = allow_smem(k_march2<S, R, 3>)) != cudaSuccess) return e;
  if ((e = allow_smem(k_march2<S, R, 4>)) != cudaSuccess) return e;
  if ((e = allow_smem(k_march<S, R, 2>)) != cudaSuccess) return e;
  if ((e = allow_smem(k_march<S, R, 3>)) != cudaSuccess) return e;
  if ((e = allow_smem(k_march<S, R, 4>)) != cudaSuccess) return e;
  return allow_smem(k_march<S, R, 6>);
}
}  // namespace

// Warps of the march kernel one SM holds at once (occupancy API).
int march_warps_per_sm(int storage, bool real_f64, int cols_per_lane, int ring_depth) {
  int blocks = 0;
  cudaError_t e = cudaErrorInvalidValue;
  auto occ = [&](auto kernel, size_t smem) { e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, kernel, 128, smem); };
  auto pick = [&](auto* sp, auto* rp) {
    using S = std::remove_pointer_t<decltype(sp)>;
    using R = std::remove_pointer_t<decltype(rp)>;
    if (cols_per_lane == 2) {
      if (ring_depth == 2) occ(k_march2<S, R, 2>, 4 * March2Stages<S, R, 2>::kBytesPerWarp);
      else if (ring_depth == 4) occ(k_march2<S, R, 4>, 4 * March2Stages<S, R, 4>::kBytesPerWarp);
      else occ(k_march2<S, R, 3>, 4 * March2Stages<S, R, 3>::kBytesPerWarp);
    } else {
      if (ring_depth == 2) occ(k_march<S, R, 2>, 4 * MarchStages<S, 2>::kBytesPerWarp);
      else if (ring_depth == 4) occ(k_march<S, R, 4>, 4 * MarchStages<S, 4>::kBytesPerWarp);
      else if (ring_depth == 6) occ(k_march<S, R, 6>, 4 * MarchStages<S, 6>::kBytesPerWarp);
      else occ(k_march<S, R, 3>, 4 * MarchStages<S, 3>::kBytesPerWarp);
    }
  };
  if (real_f64) pick((double*)nullptr, (double*)nullptr);
  else if (storage == 0) pick((double*)nullptr, (float*)nullptr);
  else if (storage == 1) pick((float*)nullptr, (float*)nullptr);
  else if (storage == 2) pick((__nv_bfloat16*)nullptr, (float*)nullptr);
  else pick((__half*)nullptr, (float*)nullptr);
  return (e == cudaSuccess && blocks > 0) ? 4 * blocks : 16;
}

int march_strips(int Nx, int cols_per_lane) { return cols_per_lane == 2 ? (Nx + 59) / 60 : (Nx + 29) / 30; }

cudaError_t march_set_attributes() {
  cudaError_t e;
  if ((e = allow_smem(k_march_tma<2, true>)) != cudaSuccess) return e;
  if ((e = allow_smem(k_march_tma<2, false>)) != cudaSuccess) return e;
  if ((e = allow_smem(k_march_tma<3, false>)) != cudaSuccess) return e;
  if ((e = attrs_t<double, double>()) != cudaSuccess) return e;
  if ((e = attrs_t<double, float>()) != cudaSuccess) return e;
  if ((e = attrs_t<float, float>()) != cudaSuccess) return e;
  if ((e = attrs_t<__nv_bfloat16, float>()) != cudaSuccess) return e;
  return attrs_t<__half, float>();
}

cudaError_t launch_march(const StepArgs& a, int storage, bool real_f64, cudaStream_t s) {
  if (real_f64) return storage == 0 ? march_t<double, double>(a, s) : cudaErrorInvalidValue;
  switch (storage) {
    case 0: return march_t<double, float>(a, s);
    case 1: return march_t<float, float>(a, s);
    case 2: return march_t<__nv_bfloat16, float>(a, s);
    case 3: return march_t<__half, float>(a, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace ehd

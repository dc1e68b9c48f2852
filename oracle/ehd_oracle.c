/*
 * ehd_oracle.c -- plain, slow, FP64 CPU oracle of the coupled electroconvection
 * time step (TRT lattice Boltzmann for fluid and charge + FFT/tridiagonal
 * Poisson solver), written from Guan & Novosselov, arXiv:1812.05711.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library.  It shares
 * no code, header, table or helper with the CUDA library in
 * paper_1812_05711_gb300/csrc; it reads its inputs through its own ABI
 * (oracle/__init__.py) and nothing here is ever called by the product path.
 *
 * Everything is double precision, one thread, loops in the order the paper
 * states the method.  Each function names the passage it follows.
 *
 * Readings of the paper where it is silent or inconsistent:
 *   - walls halfway between node rows: node row j sits at y = j + 1/2, the
 *     injector (phi = phi0, rho_c = rho0) at y = 0 and the collector (phi = 0)
 *     at y = H = Ny.  The Poisson closure mirrors about the wall
 *     (phi_{-1} = 2 phi_w - phi_0).  wall_mode = 1 instead puts the Dirichlet
 *     walls on the extra nodes j = -1 and j = Ny as in the odd extension of
 *     Eq. 21 (phi_{-1} = phi_w).
 *   - x second derivative spectral (Eq. 20) with signed wavenumber
 *     m in (-Nx/2, Nx/2], kappa_m = (2 pi m / Nx)^2.
 *   - non-zero wall potential enters the right-hand side of the first and
 *     last rows (lifting); only the m = 0 mode sees it.
 *   - Table I charge rows: injector = Dirichlet rho_c = rho0 by
 *     anti-bounce-back, collector = zero-normal-gradient outflow; f bounces
 *     back at both walls.
 *   - E = -grad phi by second-order central differences, using the same wall
 *     ghosts as the Poisson closure (ex_spectral = 1: E_x as the derivative
 *     of the row's trigonometric interpolant instead).
 *   - lattice scaling of (T, C, M, Fe): rho = 1, dphi0 = 1, H = Ny and a free
 *     ion drift speed u_ion = mu_b dphi0 / H.
 *   - order inside one step: E(t) from phi(t); moments; Eq. 7 velocity with
 *     half force; f collision; g collision with drift u + mu_b E; streaming
 *     with the wall rules; rho_c(t+1); Poisson -> phi(t+1).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "ehd_oracle.h"

/* D2Q9 lattice: textbook velocity set and weights (the paper's own table is
 * in its missing supplement); c_s^2 = 1/3 (Sec. IV.2, after Eq. 12). */
static const int OCX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int OCY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const double OW[9] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,
                             1.0 / 9.0,  1.0 / 9.0,  1.0 / 36.0,
                             1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
static const int OOPP[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
static const double CS2 = 1.0 / 3.0;
static const double OPI = 3.14159265358979323846264338327950288;

#ifdef _OPENMP
#include <omp.h>
#endif

/* Threads of the -fopenmp timing build (returns the count in use; the
 * one-thread build ignores the request and returns 1). */
int orc_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

void orc_lattice(int* cx, int* cy, double* w, int* opp) {
  for (int i = 0; i < 9; ++i) {
    cx[i] = OCX[i];
    cy[i] = OCY[i];
    w[i] = OW[i];
    opp[i] = OOPP[i];
  }
}

/* ---------------------------------------------------------------------- */
/* Hydrostatic state, Eqs. 27-28.  rho_c = rho_a (y+y_a)^(-1/2),
 * E = (2 rho_a / eps)(y+y_a)^(1/2).  The two constants follow from the
 * injector value rho_c(0) = rho0 and the applied voltage
 * int_0^H E dy = dphi0, i.e. (4 rho_a / 3 eps)[(H+y_a)^1.5 - y_a^1.5] = dphi0.
 * Solved for y_a by bisection on log(y_a). */
static double hydro_residual(double ya, double rho0, double eps, double H,
                             double dphi0) {
  double rho_a = rho0 * sqrt(ya);
  /* (H+ya)^1.5 - ya^1.5 written without cancellation for ya >> H */
  double diff = pow(ya, 1.5) * expm1(1.5 * log1p(H / ya));
  return 4.0 * rho_a / (3.0 * eps) * diff - dphi0;
}

int orc_hydrostatic_params(double rho0, double eps, double H, double dphi0,
                           double* rho_a, double* y_a) {
  if (!(rho0 > 0) || !(eps > 0) || !(H > 0) || !(dphi0 > 0)) return -1;
  double lo = log(1e-20 * H), hi = log(1e20 * H);
  if (hydro_residual(exp(lo), rho0, eps, H, dphi0) > 0) return -1;
  if (hydro_residual(exp(hi), rho0, eps, H, dphi0) < 0) return -1;
  for (int it = 0; it < 400; ++it) {
    double mid = 0.5 * (lo + hi);
    if (hydro_residual(exp(mid), rho0, eps, H, dphi0) > 0)
      hi = mid;
    else
      lo = mid;
  }
  *y_a = exp(0.5 * (lo + hi));
  *rho_a = rho0 * sqrt(*y_a);
  return 0;
}

/* ---------------------------------------------------------------------- */
/* Parameters: the non-dimensional groups of Eq. 26 mapped to lattice units,
 * and the TRT rates of Eqs. 16-17 (dt = 1). */
int orc_setup(orc_params* p) {
  if (p->Nx < 1 || p->Ny < 2) return -1;
  if (!(p->T > 0) || !(p->C > 0) || !(p->M > 0) || !(p->Fe > 0)) return -1;
  if (!(p->Lambda > 0) || !(p->Lambda_g > 0) || !(p->u_ion > 0)) return -1;
  p->rho_ref = 1.0;
  p->dphi0 = 1.0;
  p->phi0 = 1.0;
  p->H = (double)p->Ny;
  p->mu_b = p->u_ion * p->H / p->dphi0;
  /* M = sqrt(eps/rho)/mu_b */
  p->eps = p->M * p->M * p->rho_ref * p->mu_b * p->mu_b;
  /* T = eps dphi0 / (mu mu_b), nu = mu / rho */
  p->nu = p->eps * p->dphi0 / (p->T * p->mu_b) / p->rho_ref;
  /* C = rho0 H^2 / (eps dphi0) */
  p->rho0 = p->C * p->eps * p->dphi0 / (p->H * p->H);
  /* Fe = mu_b dphi0 / D_c (the paper prints D_e) */
  p->Dc = p->mu_b * p->dphi0 / p->Fe;
  /* Eq. 16: nu = cs2 (tau+ - 1/2) for the fluid.  For the charge the
   * diffusivity is carried by the relaxation of the antisymmetric part (the
   * first moment, i.e. the charge flux), Dc = cs2 (tau_g- - 1/2); Eq. 16 as
   * printed names the symmetric rate, which would make the effective
   * diffusivity cs2 Lambda_g / (tau_g+ - 1/2) instead of the Dc of Eq. 26. */
  p->tau_p = p->nu / CS2 + 0.5;
  /* Eq. 17: Lambda = (tau+ - 1/2)(tau- - 1/2), same for the charge */
  p->tau_m = 0.5 + p->Lambda / (p->tau_p - 0.5);
  if (p->dc_printed) {
    /* Eq. 16 as printed: the symmetric charge rate carries D_c */
    p->taug_p = p->Dc / CS2 + 0.5;
    p->taug_m = 0.5 + p->Lambda_g / (p->taug_p - 0.5);
  } else {
    p->taug_m = p->Dc / CS2 + 0.5;
    p->taug_p = 0.5 + p->Lambda_g / (p->taug_m - 0.5);
  }
  if (orc_hydrostatic_params(p->rho0, p->eps, p->H, p->dphi0, &p->rho_a,
                             &p->y_a) != 0)
    return -1;
  return 0;
}

/* ---------------------------------------------------------------------- */
/* Fourier transforms along x.  Eq. 19: X_k = sum_x x_x exp(-2 pi i k x / N)
 * (sign = -1); the inverse uses sign = +1 and the caller divides by N. */
void orc_dft(int n, const double* re, const double* im, double* ore,
             double* oim, int sign) {
  for (int k = 0; k < n; ++k) {
    double sr = 0, si = 0;
    for (int x = 0; x < n; ++x) {
      /* reduce k*x mod n first so the angle stays small and exact */
      long kx = ((long)k * (long)x) % n;
      double a = sign * 2.0 * OPI * (double)kx / (double)n;
      double c = cos(a), s = sin(a);
      sr += re[x] * c - im[x] * s;
      si += re[x] * s + im[x] * c;
    }
    ore[k] = sr;
    oim[k] = si;
  }
}

/* Iterative radix-2 Cooley-Tukey (bit-reversed input order, in place).
 * Same transform as orc_dft for power-of-two n. */
void orc_fft(int n, double* re, double* im, int sign) {
  for (int i = 1, j = 0; i < n; ++i) {
    int bit = n >> 1;
    for (; j & bit; bit >>= 1) j ^= bit;
    j ^= bit;
    if (i < j) {
      double t = re[i];
      re[i] = re[j];
      re[j] = t;
      t = im[i];
      im[i] = im[j];
      im[j] = t;
    }
  }
  for (int len = 2; len <= n; len <<= 1) {
    int half = len / 2;
    for (int k = 0; k < half; ++k) {
      double a = sign * 2.0 * OPI * (double)k / (double)len;
      double wr = cos(a), wi = sin(a);
      for (int s = 0; s < n; s += len) {
        int u = s + k, v = s + k + half;
        double tr = re[v] * wr - im[v] * wi;
        double ti = re[v] * wi + im[v] * wr;
        re[v] = re[u] - tr;
        im[v] = im[u] - ti;
        re[u] += tr;
        im[u] += ti;
      }
    }
  }
}

static int is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

static void transform_row(int n, double* re, double* im, double* tre,
                          double* tim, int sign) {
  if (is_pow2(n)) {
    orc_fft(n, re, im, sign);
  } else {
    orc_dft(n, re, im, tre, tim, sign);
    memcpy(re, tre, sizeof(double) * n);
    memcpy(im, tim, sizeof(double) * n);
  }
}

/* Thomas algorithm for a tridiagonal system with real coefficients and a
 * complex right-hand side: a_j x_{j-1} + b_j x_j + c_j x_{j+1} = d_j. */
void orc_thomas(int n, const double* a, const double* b, const double* c,
                double* dre, double* dim) {
  double* cp = (double*)malloc(sizeof(double) * n);
  double beta = b[0];
  cp[0] = c[0] / beta;
  dre[0] /= beta;
  dim[0] /= beta;
  for (int j = 1; j < n; ++j) {
    beta = b[j] - a[j] * cp[j - 1];
    cp[j] = c[j] / beta;
    dre[j] = (dre[j] - a[j] * dre[j - 1]) / beta;
    dim[j] = (dim[j] - a[j] * dim[j - 1]) / beta;
  }
  for (int j = n - 2; j >= 0; --j) {
    dre[j] -= cp[j] * dre[j + 1];
    dim[j] -= cp[j] * dim[j + 1];
  }
  free(cp);
}

/* ---------------------------------------------------------------------- */
/* Poisson solve, Sec. IV.3: [Dx^2 + Dy^2] phi = s with s = -rho_c/eps
 * (Eq. 4, Eq. 18).  x: DFT (Eq. 19), Dx^2 -> -kappa_m (Eq. 20).
 * y: second-order finite difference (Eq. 18) with Dirichlet walls; per mode
 * a tridiagonal system (its eigenvalues are the -4 sin^2 symbols of Eq. 24,
 * which is why it equals the odd-extension transform of Eqs. 21-25).
 * Inverse DFT, real part. */
void orc_poisson_general(int Nx, int Ny, int wall_mode, int x_symbol,
                         double phi_bottom, double phi_top, const double* src,
                         double* phi) {
  size_t nc = (size_t)Nx * Ny;
  double* sre = (double*)malloc(sizeof(double) * nc); /* [m][y] */
  double* sim = (double*)malloc(sizeof(double) * nc);
  double wall_coef = (wall_mode == 0) ? 2.0 : 1.0;

  /* Rows (and then wavenumbers) are independent.  Built with -fopenmp (the
   * multi-thread timing build only) the loops below are shared among
   * threads, each with its own scratch; the arithmetic of every row and
   * every wavenumber is the same as in the one-thread build. */
#pragma omp parallel
  {
  double* rre = (double*)malloc(sizeof(double) * Nx);
  double* rim = (double*)malloc(sizeof(double) * Nx);
  double* tre = (double*)malloc(sizeof(double) * Nx);
  double* tim = (double*)malloc(sizeof(double) * Nx);
  double* a = (double*)malloc(sizeof(double) * Ny);
  double* b = (double*)malloc(sizeof(double) * Ny);
  double* c = (double*)malloc(sizeof(double) * Ny);
  double* dre = (double*)malloc(sizeof(double) * Ny);
  double* dim = (double*)malloc(sizeof(double) * Ny);

  /* forward DFT of every row */
#pragma omp for
  for (int y = 0; y < Ny; ++y) {
    for (int x = 0; x < Nx; ++x) {
      rre[x] = src[(size_t)y * Nx + x];
      rim[x] = 0.0;
    }
    transform_row(Nx, rre, rim, tre, tim, -1);
    for (int m = 0; m < Nx; ++m) {
      sre[(size_t)m * Ny + y] = rre[m];
      sim[(size_t)m * Ny + y] = rim[m];
    }
  }
  /* one tridiagonal per wavenumber */
#pragma omp for
  for (int m = 0; m < Nx; ++m) {
    int ms = (m <= Nx / 2) ? m : m - Nx; /* signed wavenumber */
    double kx = 2.0 * OPI * (double)ms / (double)Nx;
    double kappa = kx * kx; /* Eq. 20 */
    if (x_symbol == 1) {    /* 3-point difference in x: 4 sin^2(pi m / Nx) */
      double sx = sin(OPI * (double)ms / (double)Nx);
      kappa = 4.0 * sx * sx;
    }
    for (int j = 0; j < Ny; ++j) {
      a[j] = 1.0;
      c[j] = 1.0;
      b[j] = -(2.0 + kappa);
      dre[j] = sre[(size_t)m * Ny + j];
      dim[j] = sim[(size_t)m * Ny + j];
    }
    a[0] = 0.0;
    c[Ny - 1] = 0.0;
    if (wall_mode == 0) { /* mirror ghost phi_{-1} = 2 phi_w - phi_0 */
      b[0] -= 1.0;
      b[Ny - 1] -= 1.0;
    }
    if (m == 0) { /* wall values are uniform in x: only the mean mode */
      dre[0] -= wall_coef * (double)Nx * phi_bottom;
      dre[Ny - 1] -= wall_coef * (double)Nx * phi_top;
    }
    orc_thomas(Ny, a, b, c, dre, dim);
    for (int j = 0; j < Ny; ++j) {
      sre[(size_t)m * Ny + j] = dre[j];
      sim[(size_t)m * Ny + j] = dim[j];
    }
  }
  /* inverse DFT of every row, keep the real part */
#pragma omp for
  for (int y = 0; y < Ny; ++y) {
    for (int m = 0; m < Nx; ++m) {
      rre[m] = sre[(size_t)m * Ny + y];
      rim[m] = sim[(size_t)m * Ny + y];
    }
    transform_row(Nx, rre, rim, tre, tim, +1);
    for (int x = 0; x < Nx; ++x) phi[(size_t)y * Nx + x] = rre[x] / (double)Nx;
  }
  free(rre);
  free(rim);
  free(tre);
  free(tim);
  free(a);
  free(b);
  free(c);
  free(dre);
  free(dim);
  }
  free(sre);
  free(sim);
}

/* Sec. IV.3 as the paper prints it, without the tridiagonal: the source is
 * extended oddly in y (Eqs. 21-22) to NE rows -- NE = 2 Ny antisymmetric about
 * the half node below row 0 and above row Ny - 1 (walls halfway between
 * nodes, the default reading), or NE = 2 Ny + 2 with zero rows on the wall
 * nodes j = -1 and j = Ny (wall_mode 1, Eq. 21 as printed) -- transformed
 * along x (Eq. 19) and along y, divided by the symbol of the discrete
 * Laplacian, -(kappa_m + 4 sin^2(pi k / NE)) (Eqs. 20, 24), transformed back
 * and cut to the first Ny rows (Eq. 25).  The odd extension has no mean, so
 * the (m, k) = (0, 0) coefficient is zero.  Non-zero wall potentials enter
 * as the linear profile between the walls (it has zero discrete Laplacian and
 * takes the wall values), added to the homogeneous solution. */
void orc_poisson_oddext(int Nx, int Ny, int wall_mode, int x_symbol,
                        double phi_bottom, double phi_top, const double* src,
                        double* phi) {
  const int NE = (wall_mode == 0) ? 2 * Ny : 2 * Ny + 2;
  const int off = (wall_mode == 0) ? 0 : 1; /* extended row of source row 0 */
  const int nmax = (NE > Nx) ? NE : Nx;
  size_t ne = (size_t)NE * Nx;
  double* er = (double*)calloc(ne, sizeof(double)); /* [NE][Nx] */
  double* ei = (double*)calloc(ne, sizeof(double));
  double* rre = (double*)malloc(sizeof(double) * nmax);
  double* rim = (double*)malloc(sizeof(double) * nmax);
  double* tre = (double*)malloc(sizeof(double) * nmax);
  double* tim = (double*)malloc(sizeof(double) * nmax);
  /* odd extension: row off + j holds s_j, row NE - 1 - j holds -s_j */
  for (int j = 0; j < Ny; ++j)
    for (int x = 0; x < Nx; ++x) {
      er[(size_t)(off + j) * Nx + x] = src[(size_t)j * Nx + x];
      er[(size_t)(NE - 1 - j) * Nx + x] = -src[(size_t)j * Nx + x];
    }
  for (int pass = 0; pass < 2; ++pass) {
    const int sign = (pass == 0) ? -1 : +1;
    /* along x, every extended row */
    for (int k = 0; k < NE; ++k) {
      memcpy(rre, er + (size_t)k * Nx, sizeof(double) * Nx);
      memcpy(rim, ei + (size_t)k * Nx, sizeof(double) * Nx);
      transform_row(Nx, rre, rim, tre, tim, sign);
      memcpy(er + (size_t)k * Nx, rre, sizeof(double) * Nx);
      memcpy(ei + (size_t)k * Nx, rim, sizeof(double) * Nx);
    }
    /* along y, every column */
    for (int m = 0; m < Nx; ++m) {
      for (int k = 0; k < NE; ++k) {
        rre[k] = er[(size_t)k * Nx + m];
        rim[k] = ei[(size_t)k * Nx + m];
      }
      transform_row(NE, rre, rim, tre, tim, sign);
      for (int k = 0; k < NE; ++k) {
        er[(size_t)k * Nx + m] = rre[k];
        ei[(size_t)k * Nx + m] = rim[k];
      }
    }
    if (pass == 1) break;
    /* divide by the symbol */
    for (int k = 0; k < NE; ++k) {
      const int ks = (k <= NE / 2) ? k : k - NE;
      const double sy = sin(OPI * (double)ks / (double)NE);
      for (int m = 0; m < Nx; ++m) {
        const int ms = (m <= Nx / 2) ? m : m - Nx;
        const double kx = 2.0 * OPI * (double)ms / (double)Nx;
        double kappa = kx * kx;
        if (x_symbol == 1) {
          const double sx = sin(OPI * (double)ms / (double)Nx);
          kappa = 4.0 * sx * sx;
        }
        const double den = -(kappa + 4.0 * sy * sy);
        const size_t q = (size_t)k * Nx + m;
        if (k == 0 && m == 0) {
          er[q] = 0.0;
          ei[q] = 0.0;
        } else {
          er[q] /= den;
          ei[q] /= den;
        }
      }
    }
  }
  const double scale = 1.0 / ((double)NE * (double)Nx);
  for (int j = 0; j < Ny; ++j) {
    const double t = (wall_mode == 0) ? (j + 0.5) / (double)Ny : (j + 1.0) / (double)(Ny + 1);
    const double lift = phi_bottom + (phi_top - phi_bottom) * t;
    for (int x = 0; x < Nx; ++x) phi[(size_t)j * Nx + x] = er[(size_t)(off + j) * Nx + x] * scale + lift;
  }
  free(er);
  free(ei);
  free(rre);
  free(rim);
  free(tre);
  free(tim);
}

void orc_poisson(const orc_params* p, const double* rhoc, double* phi) {
  size_t nc = (size_t)p->Nx * p->Ny;
  double* s = (double*)malloc(sizeof(double) * nc);
#pragma omp parallel for
  for (size_t k = 0; k < nc; ++k) s[k] = -rhoc[k] / p->eps; /* Eq. 4 */
  orc_poisson_general(p->Nx, p->Ny, p->wall_mode, p->x_symbol, p->phi0, 0.0, s,
                      phi);
  free(s);
}

/* E = -grad phi, central differences; wall ghosts as in the Poisson closure.
 * With ex_spectral, E_x is the exact derivative of the row's trigonometric
 * interpolant instead: X_m = DFT(phi row) (Eq. 19), E_x = inverse DFT of
 * -i k_m X_m with k_m = 2 pi m / Nx for the signed wavenumber m, the Nyquist
 * coefficient (m = Nx/2) set to zero so that E_x stays real. */
static void ex_spectral_rows(int Nx, int Ny, const double* phi, double* Ex) {
  double* re = (double*)malloc(sizeof(double) * Nx);
  double* im = (double*)malloc(sizeof(double) * Nx);
  double* tre = (double*)malloc(sizeof(double) * Nx);
  double* tim = (double*)malloc(sizeof(double) * Nx);
  for (int y = 0; y < Ny; ++y) {
    for (int x = 0; x < Nx; ++x) {
      re[x] = phi[(size_t)y * Nx + x];
      im[x] = 0.0;
    }
    transform_row(Nx, re, im, tre, tim, -1);
    for (int m = 0; m < Nx; ++m) {
      const int ms = (m <= Nx / 2) ? m : m - Nx;
      const double k = (2 * ms == Nx) ? 0.0 : 2.0 * OPI * (double)ms / (double)Nx;
      const double r = re[m], i = im[m];
      re[m] = k * i; /* -i k (r + i i') = k i' - i k r */
      im[m] = -k * r;
    }
    transform_row(Nx, re, im, tre, tim, +1);
    for (int x = 0; x < Nx; ++x) Ex[(size_t)y * Nx + x] = re[x] / (double)Nx;
  }
  free(re);
  free(im);
  free(tre);
  free(tim);
}

void orc_efield(const orc_params* p, const double* phi, double* Ex,
                double* Ey) {
  int Nx = p->Nx, Ny = p->Ny;
  for (int y = 0; y < Ny; ++y) {
    for (int x = 0; x < Nx; ++x) {
      int xl = (x + Nx - 1) % Nx, xr = (x + 1) % Nx;
      double pc = phi[(size_t)y * Nx + x];
      double pd, pu;
      if (y > 0)
        pd = phi[(size_t)(y - 1) * Nx + x];
      else
        pd = (p->wall_mode == 0) ? 2.0 * p->phi0 - pc : p->phi0;
      if (y < Ny - 1)
        pu = phi[(size_t)(y + 1) * Nx + x];
      else
        pu = (p->wall_mode == 0) ? -pc : 0.0;
      Ex[(size_t)y * Nx + x] =
          -(phi[(size_t)y * Nx + xr] - phi[(size_t)y * Nx + xl]) / 2.0;
      Ey[(size_t)y * Nx + x] = -(pu - pd) / 2.0;
    }
  }
  if (p->ex_spectral) ex_spectral_rows(Nx, Ny, phi, Ex);
}

/* ---------------------------------------------------------------------- */
/* Equilibria Eqs. 10-11 (second order in the advecting velocity). */
static double equilibrium(int i, double dens, double vx, double vy) {
  double cu = OCX[i] * vx + OCY[i] * vy;
  double uu = vx * vx + vy * vy;
  return OW[i] * dens *
         (1.0 + cu / CS2 + cu * cu / (2.0 * CS2 * CS2) - uu / (2.0 * CS2));
}

/* Forcing term Eq. 12. */
static double forcing(int i, double ux, double uy, double Fx, double Fy) {
  double cu = OCX[i] * ux + OCY[i] * uy;
  double ax = (OCX[i] - ux) / CS2 + cu * OCX[i] / (CS2 * CS2);
  double ay = (OCY[i] - uy) / CS2 + cu * OCY[i] / (CS2 * CS2);
  return OW[i] * (ax * Fx + ay * Fy);
}

/* ---------------------------------------------------------------------- */
/* Initial state: hydrostatic profile (Eqs. 27-28) at rest plus the
 * divergence-free, wall-compatible roll perturbation of Eq. 29 (coordinates
 * scaled by H, amplitude in units of u_ion, one or several x-modes). */
void orc_perturbation(const orc_params* p, int n_modes, const double* amp,
                      const double* phase, double x, double y, double* ux,
                      double* uy) {
  double X = x / p->H, Y = y / p->H, Lx = (double)p->Nx / p->H, Ly = 1.0;
  double sx = 0, sy = 0;
  for (int k = 0; k < n_modes; ++k) {
    double mk = (double)(k + 1);
    double arg = 2.0 * OPI * mk * X / Lx + phase[k];
    double a = amp[k] * p->u_ion;
    sx += a * (Lx / mk) * sin(2.0 * OPI * Y / Ly) * sin(arg);
    sy += a * Ly * (cos(2.0 * OPI * Y / Ly) - 1.0) * cos(arg);
  }
  *ux = sx;
  *uy = sy;
}

void orc_init(const orc_params* p, int n_modes, const double* amp,
              const double* phase, double* f, double* g, double* phi) {
  int Nx = p->Nx, Ny = p->Ny;
  size_t nc = (size_t)Nx * Ny;
  /* constant hydrostatic force density rho_c E = 2 rho_a^2 / eps */
  double Fh = 2.0 * p->rho_a * p->rho_a / p->eps;
  for (int y = 0; y < Ny; ++y) {
    double yc = (double)y + 0.5;
    double rc = p->rho_a / sqrt(yc + p->y_a);             /* Eq. 27 */
    double Eh = 2.0 * p->rho_a / p->eps * sqrt(yc + p->y_a); /* Eq. 28 */
    /* lattice hydrostatic pressure balance cs2 d(rho)/dy = F */
    double rho = 1.0 + Fh / CS2 * (yc - 0.5 * p->H);
    for (int x = 0; x < Nx; ++x) {
      double ux, uy;
      orc_perturbation(p, n_modes, amp, phase, (double)x, yc, &ux, &uy);
      /* stored moment sum c f = rho u - F/2 (Eq. 7) */
      double fvx = ux, fvy = uy - 0.5 * Fh / rho;
      double gvx = ux, gvy = uy + p->mu_b * Eh;
      for (int i = 0; i < 9; ++i) {
        f[(size_t)i * nc + (size_t)y * Nx + x] = equilibrium(i, rho, fvx, fvy);
        g[(size_t)i * nc + (size_t)y * Nx + x] = equilibrium(i, rc, gvx, gvy);
      }
    }
  }
  if (phi) {
    double* rhoc = (double*)calloc(nc, sizeof(double));
    for (int i = 0; i < 9; ++i)
      for (size_t k = 0; k < nc; ++k) rhoc[k] += g[(size_t)i * nc + k];
    orc_poisson(p, rhoc, phi);
    free(rhoc);
  }
}

/* ---------------------------------------------------------------------- */
/* Macroscopic fields of a state: rho (Eq. 5), u (Eq. 7), rho_c (Eq. 6), phi,
 * E.  out = [7][Ny][Nx]: rho, ux, uy, rho_c, phi, Ex, Ey. */
void orc_fields(const orc_params* p, const double* f, const double* g,
                const double* phi, double* out) {
  int Nx = p->Nx, Ny = p->Ny;
  size_t nc = (size_t)Nx * Ny;
  double* Ex = out + 5 * nc;
  double* Ey = out + 6 * nc;
  if (p->no_poisson) {
    for (size_t k = 0; k < nc; ++k) {
      Ex[k] = p->ext_E[0];
      Ey[k] = p->ext_E[1];
    }
  } else {
    orc_efield(p, phi, Ex, Ey);
  }
  for (size_t k = 0; k < nc; ++k) {
    double rho = 0, jx = 0, jy = 0, rc = 0;
    for (int i = 0; i < 9; ++i) {
      double fi = f[(size_t)i * nc + k];
      rho += fi;
      jx += OCX[i] * fi;
      jy += OCY[i] * fi;
      rc += g[(size_t)i * nc + k];
    }
    double Fx = p->ext_F[0], Fy = p->ext_F[1];
    if (!p->no_force) {
      Fx += rc * Ex[k];
      Fy += rc * Ey[k];
    }
    out[k] = rho;
    out[nc + k] = (jx + 0.5 * Fx) / rho;
    out[2 * nc + k] = (jy + 0.5 * Fy) / rho;
    out[3 * nc + k] = rc;
    out[4 * nc + k] = phi ? phi[k] : 0.0;
  }
}

/* ---------------------------------------------------------------------- */
/* One coupled step, repeated nsteps times.  f, g: [9][Ny][Nx]; phi: [Ny][Nx]
 * must be the Poisson solution of the current rho_c on entry and is again on
 * return.  diag (optional): per step ORC_NDIAG values, see ehd_oracle.h. */
void orc_step(const orc_params* p, double* f, double* g, double* phi,
              long nsteps, double* diag) {
  int Nx = p->Nx, Ny = p->Ny;
  size_t nc = (size_t)Nx * Ny;
  double* fp = (double*)malloc(sizeof(double) * 9 * nc); /* post-collision */
  double* gp = (double*)malloc(sizeof(double) * 9 * nc);
  double* Ex = (double*)malloc(sizeof(double) * nc);
  double* Ey = (double*)malloc(sizeof(double) * nc);
  double* rhoc = (double*)malloc(sizeof(double) * nc);
  double wp = 1.0 / p->tau_p, wm = 1.0 / p->tau_m;   /* omega+-, fluid */
  double gwp = 1.0 / p->taug_p, gwm = 1.0 / p->taug_m; /* omega_g+- */

  for (long t = 0; t < nsteps; ++t) {
    /* E(t) = -grad phi(t) */
    if (p->no_poisson) {
      for (size_t k = 0; k < nc; ++k) {
        Ex[k] = p->ext_E[0];
        Ey[k] = p->ext_E[1];
      }
    } else {
      orc_efield(p, phi, Ex, Ey);
    }
    double mass = 0, charge = 0, ke = 0, maxuy = 0;
    /* collision at every node (nodes are independent; the -fopenmp timing
     * build shares them among threads, which reorders only the diagnostic
     * sums) */
#pragma omp parallel for reduction(+ : mass, charge, ke) reduction(max : maxuy)
    for (size_t k = 0; k < nc; ++k) {
      double fl[9], gl[9], feq[9], geq[9], Fi[9];
      double rho = 0, jx = 0, jy = 0, rc = 0;
      for (int i = 0; i < 9; ++i) {
        fl[i] = f[(size_t)i * nc + k];
        gl[i] = g[(size_t)i * nc + k];
        rho += fl[i];                /* Eq. 5 */
        jx += OCX[i] * fl[i];
        jy += OCY[i] * fl[i];
        rc += gl[i];                 /* Eq. 6 */
      }
      /* F_e = -rho_c grad phi = rho_c E (Eq. 2) */
      double Fx = p->ext_F[0], Fy = p->ext_F[1];
      if (!p->no_force) {
        Fx += rc * Ex[k];
        Fy += rc * Ey[k];
      }
      double ux = (jx + 0.5 * Fx) / rho; /* Eq. 7 */
      double uy = (jy + 0.5 * Fy) / rho;
      /* drift velocity u - mu_b grad phi = u + mu_b E (Eq. 3, Eq. 11) */
      double vx = ux + p->mu_b * Ex[k];
      double vy = uy + p->mu_b * Ey[k];
      mass += rho;
      charge += rc;
      ke += 0.5 * rho * (ux * ux + uy * uy);
      if (fabs(uy) > maxuy) maxuy = fabs(uy);
      for (int i = 0; i < 9; ++i) {
        feq[i] = equilibrium(i, rho, ux, uy);  /* Eq. 10 */
        geq[i] = equilibrium(i, rc, vx, vy);   /* Eq. 11 */
        Fi[i] = forcing(i, ux, uy, Fx, Fy);    /* Eq. 12 */
      }
      for (int i = 0; i < 9; ++i) {
        int o = OOPP[i];
        /* Eq. 13-15: symmetric and antisymmetric parts */
        double fpl = 0.5 * (fl[i] + fl[o]), fmi = 0.5 * (fl[i] - fl[o]);
        double epl = 0.5 * (feq[i] + feq[o]), emi = 0.5 * (feq[i] - feq[o]);
        double Fpl = 0.5 * (Fi[i] + Fi[o]), Fmi = 0.5 * (Fi[i] - Fi[o]);
        /* Eq. 8 */
        fp[(size_t)i * nc + k] = fl[i] - wp * (fpl - epl) - wm * (fmi - emi) +
                                 (1.0 - 0.5 * wp) * Fpl +
                                 (1.0 - 0.5 * wm) * Fmi;
        double gpl = 0.5 * (gl[i] + gl[o]), gmi = 0.5 * (gl[i] - gl[o]);
        double hpl = 0.5 * (geq[i] + geq[o]), hmi = 0.5 * (geq[i] - geq[o]);
        /* Eq. 9 */
        gp[(size_t)i * nc + k] = gl[i] - gwp * (gpl - hpl) - gwm * (gmi - hmi);
      }
    }
    /* streaming f_i(x + c_i, t+1) = f_i*(x, t) with the wall rules */
    double q_in = 0, q_out = 0;
    /* every (population, node) pair writes its own target, so rows are
     * independent */
#pragma omp parallel for reduction(+ : q_in, q_out)
    for (int y = 0; y < Ny; ++y) {
      for (int x = 0; x < Nx; ++x) {
        size_t k = (size_t)y * Nx + x;
        for (int i = 0; i < 9; ++i) {
          int xt = (x + OCX[i] + Nx) % Nx;
          int yt = y + OCY[i];
          double fs = fp[(size_t)i * nc + k], gs = gp[(size_t)i * nc + k];
          int o = OOPP[i];
          if (p->periodic_y) yt = (yt + Ny) % Ny;
          if (yt >= 0 && yt < Ny) {
            f[(size_t)i * nc + (size_t)yt * Nx + xt] = fs;
            g[(size_t)i * nc + (size_t)yt * Nx + xt] = gs;
          } else if (yt < 0) {
            /* injector wall: halfway bounce-back for f */
            f[(size_t)o * nc + k] = fs;
            /* anti-bounce-back: rho_c = rho0 with the wall drift
             * (u_wall = 0, drift mu_b E of the first row) */
            double vwx = p->mu_b * Ex[k], vwy = p->mu_b * Ey[k];
            double cv = OCX[o] * vwx + OCY[o] * vwy;
            double vv = vwx * vwx + vwy * vwy;
            double even = OW[o] * p->rho0 *
                          (1.0 + cv * cv / (2.0 * CS2 * CS2) - vv / (2.0 * CS2));
            double gnew = -gs + 2.0 * even;
            g[(size_t)o * nc + k] = gnew;
            q_in += gnew - gs;
          } else {
            /* collector wall: bounce-back for f; charge leaves */
            f[(size_t)o * nc + k] = fs;
            q_out += gs;
          }
          /* collector outflow: populations entering from above are the
           * node's own post-collision values (zero normal gradient) */
          if (!p->periodic_y && y == Ny - 1 && OCY[i] < 0) {
            g[(size_t)i * nc + (size_t)y * Nx + xt] = gs;
            q_out -= gs;
          }
        }
      }
    }
    /* rho_c(t+1) and phi(t+1) */
    if (!p->no_poisson) {
#pragma omp parallel for
      for (size_t k = 0; k < nc; ++k) {
        double s = 0;
        for (int i = 0; i < 9; ++i) s += g[(size_t)i * nc + k];
        rhoc[k] = s;
      }
      orc_poisson(p, rhoc, phi);
    }
    if (diag) {
      double* d = diag + (size_t)t * ORC_NDIAG;
      d[0] = mass;
      d[1] = charge;
      d[2] = q_in;
      d[3] = q_out;
      d[4] = ke;
      d[5] = maxuy;
    }
  }
  free(fp);
  free(gp);
  free(Ex);
  free(Ey);
  free(rhoc);
}

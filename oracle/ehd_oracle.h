/*
 * ehd_oracle.h -- interface of the FP64 CPU oracle (test infrastructure only;
 * never included by the CUDA library).  Arrays are row-major, x fastest:
 * fields [Ny][Nx], populations [9][Ny][Nx].
 */
#ifndef EHD_ORACLE_H
#define EHD_ORACLE_H

#define ORC_NDIAG 6 /* mass, charge, q_in, q_out, kinetic energy, max|u_y| */

typedef struct {
  /* inputs */
  int Nx, Ny;
  double T, C, M, Fe;  /* non-dimensional groups, Eq. 26 */
  double Lambda;       /* fluid magic parameter, Eq. 17 */
  double Lambda_g;     /* charge magic parameter, Eq. 17 */
  double u_ion;        /* lattice ion drift speed mu_b dphi0 / H */
  int wall_mode;       /* 0 halfway walls, 1 node walls of Eq. 21 */
  int x_symbol;        /* x second derivative: 0 spectral -kappa_m (Eq. 20),
                          1 second-order difference -4 sin^2(pi m / Nx), the
                          symbol of the 3-point stencil (Eq. 24's form in x) */
  int ex_spectral;     /* E_x = -d phi / dx: 0 central difference, 1 spectral
                          (-i k_m times the x-transform of phi, Nyquist mode 0) */
  int dc_printed;      /* charge rates: 0 D_c = cs2 (tau_g- - 1/2) (the reading
                          used throughout), 1 Eq. 16 as printed, D_c = cs2
                          (tau_g+ - 1/2), with Lambda_g then fixing tau_g- */
  /* hooks used only by the oracle's own pins (all zero for the method) */
  int periodic_y;      /* y periodic, no walls (requires no_poisson) */
  int no_poisson;      /* E = ext_E instead of -grad phi */
  int no_force;        /* switch the electric body force off */
  double ext_E[2];
  double ext_F[2];     /* extra uniform body force on the fluid */
  /* derived by orc_setup */
  double rho_ref, dphi0, phi0, H;
  double mu_b, eps, nu, rho0, Dc;
  double tau_p, tau_m, taug_p, taug_m;
  double rho_a, y_a;
} orc_params;

int orc_threads(int n);
void orc_lattice(int* cx, int* cy, double* w, int* opp);
int orc_setup(orc_params* p);
int orc_hydrostatic_params(double rho0, double eps, double H, double dphi0,
                           double* rho_a, double* y_a);
void orc_dft(int n, const double* re, const double* im, double* ore,
             double* oim, int sign);
void orc_fft(int n, double* re, double* im, int sign);
void orc_thomas(int n, const double* a, const double* b, const double* c,
                double* dre, double* dim);
void orc_poisson_general(int Nx, int Ny, int wall_mode, int x_symbol,
                         double phi_bottom, double phi_top, const double* src,
                         double* phi);
void orc_poisson_oddext(int Nx, int Ny, int wall_mode, int x_symbol,
                        double phi_bottom, double phi_top, const double* src,
                        double* phi);
void orc_poisson(const orc_params* p, const double* rhoc, double* phi);
void orc_efield(const orc_params* p, const double* phi, double* Ex,
                double* Ey);
void orc_perturbation(const orc_params* p, int n_modes, const double* amp,
                      const double* phase, double x, double y, double* ux,
                      double* uy);
void orc_init(const orc_params* p, int n_modes, const double* amp,
              const double* phase, double* f, double* g, double* phi);
void orc_fields(const orc_params* p, const double* f, const double* g,
                const double* phi, double* out);
void orc_step(const orc_params* p, double* f, double* g, double* phi,
              long nsteps, double* diag);

#endif

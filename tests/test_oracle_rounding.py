"""How accurate is the FP64 oracle's own Poisson solve on tall channels?

The mean mode m = 0 of the Sec. IV.3 solve is a tridiagonal system whose
condition number grows as Ny^2 (the 1-D discrete Laplacian with the wall
ghosts).  The oracle eliminates it by the Thomas recurrences in FP64, so its
potential carries a rounding error that grows with the channel height.  This
test measures that error against the same system solved in 40-digit decimal
arithmetic (mpmath), for the mean-mode right-hand side of the seeded
channels, and pins the result that the GPU parity bounds rely on:

* at Ny = 104 (the 128 x 104 parity configuration) the oracle's E_y is
  exact to about 3e-14 of the field scale, so the 1e-12 FP64 bar tests the
  GPU path;
* at Ny = 840 and 1680 the oracle's own E_y error is 1e-12 .. 1e-11 of the
  field scale, so a GPU path accurate to 1e-12 can differ from the oracle by
  that much there: the 1024 x 840 FP64 parity bound is 1e-12 plus this
  rounding budget.

Paper: Sec. IV.3, Eq. 18 (second differences in y), the mirror-ghost closure
of the halfway walls with the injector potential lifted into row 0.
"""
import numpy as np
import pytest

import oracle as o
import workloads as wl

mp = pytest.importorskip("mpmath")


def _mean_mode_system(p, rho_c_rows, Nx):
    """The m = 0 system of the oracle's solve: Eq. 18 with kappa_0 = 0, the
    right-hand side Nx * mean(-rho_c / eps) per row (the DFT's m = 0
    coefficient, Eq. 19), mirror ghosts at both walls, phi0 lifted."""
    Ny = p.Ny
    a, c, b = np.ones(Ny), np.ones(Ny), -2.0 * np.ones(Ny)
    a[0], c[-1] = 0.0, 0.0
    b[0] -= 1.0
    b[-1] -= 1.0
    d = -Nx * np.asarray(rho_c_rows, dtype=np.float64) / p.eps
    d[0] -= 2.0 * Nx * p.phi0
    return a, b, c, d


def _exact_thomas(a, b, c, d, dps=40):
    """The same elimination in dps-digit decimal arithmetic."""
    with mp.workdps(dps):
        A, B, C, D = ([mp.mpf(float(v)) for v in arr] for arr in (a, b, c, d))
        n = len(B)
        cp, dp = [None] * n, [None] * n
        beta = B[0]
        cp[0], dp[0] = C[0] / beta, D[0] / beta
        for j in range(1, n):
            beta = B[j] - A[j] * cp[j - 1]
            cp[j] = C[j] / beta
            dp[j] = (D[j] - A[j] * dp[j - 1]) / beta
        x = [None] * n
        x[-1] = dp[-1]
        for j in range(n - 2, -1, -1):
            x[j] = dp[j] - cp[j] * x[j + 1]
        # residual of the exact solve (checks the reference itself)
        res = max(abs(A[j] * (x[j - 1] if j else 0) + B[j] * x[j] + C[j] * (x[j + 1] if j < n - 1 else 0) - D[j])
                  for j in range(n))
        return x, float(res / max(abs(v) for v in D))


def _ey_scaled(phi_mean, p, exact=False):
    """E_y = -(phi_{j+1} - phi_{j-1}) / 2 with the mirror ghosts, times H
    (the field scale dphi0 / H)."""
    if exact:
        ext = [2 * mp.mpf(p.phi0) - phi_mean[0]] + list(phi_mean) + [-phi_mean[-1]]
        return np.array([float(-(ext[j + 2] - ext[j]) / 2 * p.H) for j in range(p.Ny)])
    ext = np.concatenate([[2 * p.phi0 - phi_mean[0]], phi_mean, [-phi_mean[-1]]])
    return -(ext[2:] - ext[:-2]) / 2 * p.H


def _oracle_mean_mode_error(w):
    p = o.setup(*w.args())
    # the initial charge of the seeded channel (Eq. 27 profile plus the
    # Eq. 29 roll), on a narrow copy of the grid: the mean mode only sees
    # the row means, and the roll has none
    narrow = o.setup(8, w.Ny, w.T, w.C, w.M, w.Fe, w.Lambda)
    rows = o.fields(o.init_state(narrow, w.amp, w.phase))["rho_c"].mean(axis=1)
    a, b, c, d = _mean_mode_system(p, rows, w.Nx)
    phi64 = o.thomas(a, b, c, d).real / w.Nx
    x, res = _exact_thomas(a, b, c, d)
    with mp.workdps(40):
        xm = [v / w.Nx for v in x]
        ey_exact = _ey_scaled(xm, p, exact=True)
        phi_exact = np.array([float(v) for v in xm])
    e_phi = float(np.abs(phi64 - phi_exact).max())
    e_ey = float(np.abs(_ey_scaled(phi64, p) - ey_exact).max())
    return res, e_phi, e_ey


def test_mean_mode_rounding_small_at_parity_height():
    res, e_phi, e_ey = _oracle_mean_mode_error(wl.plain_fp64_channel())
    assert res < 1e-35
    assert e_phi < 1e-14 and e_ey < 1e-13, (e_phi, e_ey)


@pytest.mark.parametrize("make", [wl.precision_channel, wl.large_channel])
def test_mean_mode_rounding_budget_of_tall_channels(make):
    """At 840 and 1680 rows the oracle's own E_y rounding reaches 1e-12 of
    the field scale (measured 2.1e-12 and 6.0e-12): the size of the FP64
    GPU-vs-oracle difference seen at 1024 x 840 (2.2e-12)."""
    w = make()
    res, e_phi, e_ey = _oracle_mean_mode_error(w)
    assert res < 1e-35
    print(f"\n{w.Nx}x{w.Ny}: oracle m = 0 rounding: phi {e_phi:.2e}, E_y scaled {e_ey:.2e}")
    assert 1e-12 <= e_ey <= 1e-11, e_ey

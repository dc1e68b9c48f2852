"""Studies of Sec. V run on the GPU path: the hydrostatic state against its
analytic profile (Sec. V.1, Eqs. 27-28, Table II) and the growth rate of an
Eq. 29 roll (Sec. V.2).  Everything runs through the C ABI (:class:`Run`)."""
from __future__ import annotations

import numpy as np

from . import Run

W9 = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)


def e_l2(num, ref) -> float:
    """Relative L2 error of Table II: ||num - ref|| / ||ref||."""
    num, ref = np.asarray(num, dtype=np.float64), np.asarray(ref, dtype=np.float64)
    return float(np.sqrt(((num - ref) ** 2).sum() / (ref ** 2).sum()))


def hydrostatic(C: float, Ny: int = 100, steps: int = 30000, u_ion: float = 0.01, Fe: float = 4000.0,
                M: float = 10.0, T: float = 200.0, Nx: int = 16, storage: str = "f64") -> dict:
    """No-flow steady state between the electrodes (Sec. V.1): start from fluid
    at rest and a uniform charge of half the injected density, run `steps`
    coupled steps, and compare the x-averaged charge density and field with
    Eqs. 27-28.  Returns the two e_L2 values and the profiles."""
    run = Run(Nx, Ny, T, C, M, Fe, 0.25, storage=storage, u_ion=u_ion)
    par = run.params()
    f = np.broadcast_to(W9[:, None, None], (9, Ny, Nx)).copy()
    g = f * (0.5 * par["rho0"])
    run.load(f, g)
    run.step(steps)
    F = run.fields(("rho_c", "Ey"))
    run.close()
    y = np.arange(Ny) + 0.5
    rc_a = par["rho_a"] / np.sqrt(y + par["y_a"])
    E_a = 2.0 * par["rho_a"] / par["eps"] * np.sqrt(y + par["y_a"])
    rc, Ey = F["rho_c"].mean(axis=1), F["Ey"].mean(axis=1)
    # Eq. 27 constants in the non-dimensional units of Eq. 26 (eps = H = dphi0 = 1):
    # charge density unit eps dphi0 / H^2, length unit H
    H, rho_unit = par["H"], par["eps"] / par["H"] ** 2
    return {"C": C, "eL2_Ey": e_l2(Ey, E_a), "eL2_rhoc": e_l2(rc, rc_a), "rho_c": rc, "Ey": Ey,
            "rho_c_analytic": rc_a, "Ey_analytic": E_a,
            "rho_a": par["rho_a"] / (rho_unit * np.sqrt(H)), "y_a": par["y_a"] / H}


def growth_rate(t, max_uy) -> float:
    """Exponential rate per step of max|u_y|: least-squares slope of its log
    over the second half of the record."""
    t, a = np.asarray(t, dtype=np.float64), np.asarray(max_uy, dtype=np.float64)
    h = a.size // 2
    return float(np.polyfit(t[h:], np.log(a[h:]), 1)[0])


def collected_current(run: Run, steps: int, window: int) -> float:
    """Advance `steps` steps and return the mean collected charge per step
    over the last `window` of them (from the FP64 cumulative wall flux)."""
    run.step(steps - window)
    q0 = run.diagnostics()["q_out"]
    run.step(window)
    return (run.diagnostics()["q_out"] - q0) / window


def nusselt_sweep(T_values, Nx=64, Ny=52, u_ion=5e-3, steps=200000, window=40000, storage="f32",
                  amp_small=1e-3, amp_large=0.3, C=10.0, M=10.0, Fe=4000.0, Lambda=0.25):
    """The electric Nusselt number Ne = I / I_h (collected current over the
    hydrostatic one) against T on both branches (Sec. V.2, FIG. 3):
    - lower branch: each T started from the hydrostatic state with a small
      Eq. 29 roll (grows only above the linear threshold T_c);
    - upper branch: continuation downwards in T from a finite-amplitude
      state, each T started from the previous T's final populations (stays
      convective down to the finite-amplitude threshold T_f).
    Returns {"I_h": ..., "lower": [(T, Ne)], "upper": [(T, Ne)]} with T
    ascending on the lower and descending on the upper branch."""
    ref = Run(Nx, Ny, max(T_values), C, M, Fe, Lambda, storage=storage, u_ion=u_ion)
    I_h = collected_current(ref, steps, window)
    ref.close()
    lower = []
    for T in sorted(T_values):
        r = Run(Nx, Ny, T, C, M, Fe, Lambda, storage=storage, u_ion=u_ion, amp=[amp_small], phase=[0.0])
        lower.append((T, collected_current(r, steps, window) / I_h))
        r.close()
    upper = []
    state = None
    for k, T in enumerate(sorted(T_values, reverse=True)):
        r = Run(Nx, Ny, T, C, M, Fe, Lambda, storage=storage, u_ion=u_ion,
                amp=[amp_large] if state is None else [], phase=[0.0] if state is None else [])
        if state is not None:
            r.load(*state)
        upper.append((T, collected_current(r, steps, window) / I_h))
        state = r.save()
        r.close()
    return {"I_h": I_h, "lower": lower, "upper": upper}


def nusselt_sweep_served(T_values, Nx=64, Ny=52, u_ion=5e-3, steps=200000, window=40000, amp_small=1e-3,
                         amp_large=0.3, C=10.0, M=10.0, Fe=4000.0, Lambda=0.25, tick_steps=2000,
                         hbm_budget=8 << 30):
    """The Ne(T) sweep of :func:`nusselt_sweep` (Sec. V.2, FIG. 3) driven
    through the continuous-batching server: every point is a request whose
    last `window` steps measure the collected current.  The reference
    (hydrostatic) run and the lower branch are independent requests, so they
    advance together in the batch; the upper branch is a chain in which each
    request starts from the previous (higher) T's final populations and is
    admitted as soon as that one finishes, beside the runs still in flight.
    FP32 storage and compute (the batch's kind of run).  Returns
    {"I_h", "lower", "upper", "results"} as nusselt_sweep does."""
    from .serve import Request, Server

    Ts = sorted(T_values)
    reqs = [Request(0, Nx, Ny, Ts[-1], C, M, Fe, Lambda, steps, window=window, u_ion=u_ion)]
    for k, T in enumerate(Ts):
        reqs.append(Request(1 + k, Nx, Ny, T, C, M, Fe, Lambda, steps, [amp_small], [0.0], window=window,
                            u_ion=u_ion))
    base = 1 + len(Ts)
    for k, T in enumerate(reversed(Ts)):
        first = k == 0
        reqs.append(Request(base + k, Nx, Ny, T, C, M, Fe, Lambda, steps, [amp_large] if first else [],
                            [0.0] if first else [], window=window, after=None if first else base + k - 1,
                            u_ion=u_ion))
    srv = Server(hbm_budget, max_runs=len(reqs), tick_steps=tick_steps, max_nx=Nx, max_ny=Ny, u_ion=u_ion)
    try:
        res = {r.rid: r for r in srv.serve(reqs, realtime=False)}
    finally:
        srv.close()
    I_h = res[0].current
    lower = [(T, res[1 + k].current / I_h) for k, T in enumerate(Ts)]
    upper = [(T, res[base + k].current / I_h) for k, T in enumerate(reversed(Ts))]
    return {"I_h": I_h, "lower": lower, "upper": upper, "results": res}

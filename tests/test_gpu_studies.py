"""Sec. V.1 on the GPU path: the no-flow steady state between the electrodes
against the analytic profile of Eqs. 27-28 (Table II) and against the
oracle's steady state."""
import numpy as np
import pytest

import oracle as o

gpu = pytest.mark.gpu


def _ehd():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1812_05711_gb300 as ehd
    return ehd


def _table2():
    rows = {}
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "table2_hydrostatic.txt")
    for ln in open(path):
        if ln.strip() and not ln.startswith("#"):
            C, ra, ya, eE, erc = map(float, ln.split())
            rows[C] = (ra, ya, eE, erc)
    return rows


def _oracle_steady(C, Ny=100, steps=30000, u_ion=0.01):
    p = o.setup(4, Ny, 200, C, 10, 4000, 0.25, u_ion=u_ion)
    cx, cy, w, opp = o.lattice()
    f = np.ones((9, Ny, 4)) * w[:, None, None]
    g = f * 0.5 * p.rho0
    s = o.state_from(p, f, g)
    o.step(s, steps)
    F = o.fields(s)
    return F["rho_c"][:, 0], F["Ey"][:, 0]


@gpu
@pytest.mark.parametrize("C", [0.1, 10.0])
def test_hydrostatic_steady_state_gpu(C):
    from paper_1812_05711_gb300 import studies
    _ehd()
    r = studies.hydrostatic(C)
    rc_o, Ey_o = _oracle_steady(C)
    # the GPU's x-uniform steady state is the oracle's (4 columns there, 16 here)
    assert np.abs(r["rho_c"] - rc_o).max() <= 1e-11 * np.abs(rc_o).max()
    assert np.abs(r["Ey"] - Ey_o).max() <= 1e-11 * np.abs(Ey_o).max()
    _, _, eE_tab, erc_tab = _table2()[C]
    assert r["eL2_Ey"] <= 2 * eE_tab, r["eL2_Ey"]
    if C < 1:
        assert r["eL2_rhoc"] <= 2 * erc_tab, r["eL2_rhoc"]


@gpu
def test_subcritical_hysteresis_64x52():
    """Sec. V.2 (FIG. 3): below the linear threshold a small roll dies out
    (Ne = 1) while a finite-amplitude convective state persists (Ne > 1)
    down to the finite-amplitude threshold T_f (108.7 in the paper), below
    which it dies too.  64 x 52, u_ion = 5e-3, FP32, 200,000 steps per T."""
    ehd = _ehd()
    from paper_1812_05711_gb300 import studies
    kw = dict(storage="f32", u_ion=5e-3)
    steps, window = 200000, 40000

    def ne(T, amp=None, state=None):
        r = ehd.Run(64, 52, T, 10, 10, 4000, 0.25, amp=[amp] if amp else [], phase=[0.0] if amp else [], **kw)
        if state is not None:
            r.load(*state)
        I = studies.collected_current(r, steps, window)
        s = r.save()
        r.close()
        return I, s

    I_h, _ = ne(200.0)
    I_conv, conv = ne(200.0, amp=0.3)
    assert I_conv / I_h > 1.3
    I_small, _ = ne(130.0, amp=1e-3)
    assert abs(I_small / I_h - 1.0) < 1e-3
    I_upper, _ = ne(130.0, state=conv)
    assert I_upper / I_h > 1.1
    I_dead, _ = ne(95.0, state=conv)
    assert abs(I_dead / I_h - 1.0) < 1e-3


@gpu
def test_served_nusselt_points_vs_oracle_64x52():
    """Sec. V.2 sweep points driven through the continuous-batching server
    (FP32, one batch): the hydrostatic reference, a lower-branch point (a
    small roll) and two upper-branch points (a finite-amplitude roll at
    T = 180, then T = 170 continued from its final populations).  Each
    request's collected current over its measurement window (FP64 wall
    fluxes) matches the oracle's over the same steps, and so does the
    electric Nusselt number Ne = I / I_h."""
    _ehd()
    from paper_1812_05711_gb300.serve import Request, Server
    Nx, Ny, u_ion, steps, window = 64, 52, 5e-3, 12000, 4000
    reqs = [Request(0, Nx, Ny, 180.0, 10, 10, 4000, 0.25, steps, window=window, u_ion=u_ion),
            Request(1, Nx, Ny, 180.0, 10, 10, 4000, 0.25, steps, [1e-3], [0.0], window=window, u_ion=u_ion),
            Request(2, Nx, Ny, 180.0, 10, 10, 4000, 0.25, steps, [0.3], [0.0], window=window, u_ion=u_ion),
            Request(3, Nx, Ny, 170.0, 10, 10, 4000, 0.25, 2 * window, window=window, after=2, u_ion=u_ion)]
    srv = Server(1 << 30, max_runs=4, tick_steps=1000, max_nx=Nx, max_ny=Ny, u_ion=u_ion)
    try:
        res = {r.rid: r for r in srv.serve(reqs, realtime=False)}
    finally:
        srv.close()

    def oracle_current(T, amp, n, state=None):
        p = o.setup(Nx, Ny, T, 10, 10, 4000, 0.25, u_ion=u_ion)
        s = o.init_state(p, amp, [0.0] * len(amp)) if state is None else o.state_from(p, *state)
        d = o.step(s, n, diag=True)
        return d[n - window:, 3].sum() / window, (s.f, s.g)

    n_threads = o.use_threads()
    try:
        I_h, _ = oracle_current(180.0, [], steps)
        I_1, _ = oracle_current(180.0, [1e-3], steps)
        I_2, st = oracle_current(180.0, [0.3], steps)
        I_3, _ = oracle_current(170.0, [], 2 * window, state=st)
    finally:
        o.use_one_thread()
    assert n_threads >= 0
    for rid, ref in ((0, I_h), (1, I_1), (2, I_2), (3, I_3)):
        assert res[rid].current == pytest.approx(ref, rel=1e-4), (rid, res[rid].current, ref)
        assert res[rid].current / res[0].current == pytest.approx(ref / I_h, rel=2e-4), rid
    # the finite-amplitude roll already carries more charge than the
    # hydrostatic state, and the continuation keeps convecting
    assert res[2].current / res[0].current > 1.001 and res[3].current / res[0].current > 1.001

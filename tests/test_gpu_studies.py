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

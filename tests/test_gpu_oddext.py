"""The literal odd-extension y solve of Sec. IV.3 (Eqs. 21-25) on the GPU
(``y_solver`` 1: a complex FFT of length NE per x-wavenumber in place of the
tridiagonal) against the oracle, through the C ABI.  Same bars as the
tridiagonal path: plain FP64 <= 1e-12, FP32 compute on shifted FP32 storage
<= 2e-5 (scale-normalised max norm)."""
import numpy as np
import pytest

import oracle as o
import workloads as wl

gpu = pytest.mark.gpu


def _ehd():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1812_05711_gb300 as ehd
    return ehd


def _errors(p, A, B):
    sc = {"rho": 1.0, "ux": p.u_ion, "uy": p.u_ion, "rho_c": p.rho0, "phi": 1.0, "Ex": 1.0 / p.H, "Ey": 1.0 / p.H}
    return {k: float(np.abs(A[k] - B[k]).max() / sc[k]) for k in A}


def _pair(Nx, Ny, storage, wall_mode, u_ion=5e-3, T=200.0, seed=43):
    ehd = _ehd()
    amp, ph = wl.roll(seed, 1e-2)
    p = o.setup(Nx, Ny, T, 10, 10, 4000, 0.25, u_ion=u_ion, wall_mode=wall_mode)
    s = o.init_state(p, amp, ph)
    run = ehd.Run(Nx, Ny, T, 10, 10, 4000, 0.25, storage=storage, u_ion=u_ion, wall_mode=wall_mode,
                  amp=amp, phase=ph)
    ehd.ehd_tune(run.handle, "y_solver", 1)
    assert ehd.ehd_tune_get(run.handle, "y_solver") == 1
    return ehd, p, s, run


@gpu
@pytest.mark.parametrize("storage,bound", [("f64", 1e-12), ("f32", 2e-5)])
@pytest.mark.parametrize("Nx,Ny,wall_mode", [
    (64, 52, 0),    # NE = 104 = 4 2 13
    (128, 105, 0),  # NE = 210 = 2 3 5 7
    (64, 53, 1),    # NE = 108 = 4 3 3 3, zero rows on the wall nodes
    (32, 26, 1),    # NE = 54 = 2 3 3 3
])
def test_oddext_step_parity(Nx, Ny, wall_mode, storage, bound):
    ehd, p, s, run = _pair(Nx, Ny, storage, wall_mode)
    run.step(300)
    o.step(s, 300)
    e = _errors(p, run.fields(), o.fields(s))
    run.close()
    assert max(e.values()) <= bound, e


@gpu
def test_oddext_poisson_equals_oracle_literal_solve():
    """One solve on the run's own charge: phi from the GPU's odd-extension
    path equals the oracle's literal transform (and its tridiagonal)."""
    ehd, p, s, run = _pair(128, 104, "f64", 0)
    run.step(50)
    run.poisson()
    F = run.fields()
    src = -F["rho_c"] / p.eps
    ref = o.poisson_oddext(src, wall_mode=0, phi_bottom=p.phi0, phi_top=0.0)
    run.close()
    assert np.abs(F["phi"] - ref).max() <= 1e-12


@gpu
def test_oddext_full_size_fp32_two_steps_vs_oracle():
    """2048 x 1680 (NE = 3360 = 4 4 2 3 5 7): two coupled steps with the
    odd-extension y solve against two oracle steps."""
    w = wl.large_channel()
    ehd = _ehd()
    p = o.setup(*w.args(), u_ion=2e-3)
    s = o.init_state(p, w.amp, w.phase)
    run = ehd.Run(*w.args(), storage="f32", u_ion=2e-3, amp=w.amp, phase=w.phase)
    ehd.ehd_tune(run.handle, "y_solver", 1)
    run.step(2)
    o.step(s, 2)
    e = _errors(p, run.fields(), o.fields(s))
    run.close()
    assert max(e.values()) <= 2e-5, e


@gpu
def test_oddext_rejections():
    """NE with a prime factor above 13 (Ny = 53, walls halfway: NE = 106 =
    2 x 53) is refused, and so is a run in the odd-extension mode joining a
    batch; the run keeps its tridiagonal solve."""
    ehd = _ehd()
    r = ehd.Run(64, 53, 200.0, 10, 10, 4000, 0.25, storage="f32")
    with pytest.raises(RuntimeError):
        ehd.ehd_tune(r.handle, "y_solver", 1)
    assert ehd.ehd_tune_get(r.handle, "y_solver") == 0
    r.close()
    r = ehd.Run(64, 52, 200.0, 10, 10, 4000, 0.25, storage="f32")
    ehd.ehd_tune(r.handle, "y_solver", 1)
    b = ehd.Batch(2, max_nx=64, max_ny=52)
    with pytest.raises(RuntimeError):
        b.add(r, 10)
    b.close()
    r.close()

"""Variants of the step against the oracle (GPU, through the C ABI): the
fluid magic parameter Lambda of Eq. 17 (1/12 as printed in Sec. IV.2, 3/16,
1/4), the single-relaxation-time limit Lambda = (tau+ - 1/2)^2 (tau- =
tau+), the 3-point x symbol of the Poisson solve, and E_x taken spectrally
from the x-transform of phi instead of by central differences."""
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


def _scaled_err(p, A, B):
    sc = {"rho": 1.0, "ux": p.u_ion, "uy": p.u_ion, "rho_c": p.rho0, "phi": 1.0, "Ex": 1.0 / p.H, "Ey": 1.0 / p.H}
    return max(float(np.abs(A[k] - B[k]).max() / sc[k]) for k in A)


def _compare(ehd, Lam, storage="f64", x_symbol=0, steps=300, T=200.0, ex_spectral=0):
    Nx, Ny = 64, 52
    amp, ph = wl.roll(41, 1e-2)
    p = o.setup(Nx, Ny, T, 10, 10, 4000, Lam, u_ion=5e-3, x_symbol=x_symbol, ex_spectral=ex_spectral)
    s = o.init_state(p, amp, ph)
    run = ehd.Run(Nx, Ny, T, 10, 10, 4000, Lam, storage=storage, u_ion=5e-3, amp=amp, phase=ph,
                  x_symbol=x_symbol, ex_spectral=ex_spectral)
    par = run.params()
    run.step(steps)
    o.step(s, steps)
    e = _scaled_err(p, run.fields(), o.fields(s))
    run.close()
    return p, par, e


@gpu
@pytest.mark.parametrize("Lam", [1.0 / 12.0, 3.0 / 16.0, 0.25])
def test_lambda_variants_fp64_parity(Lam):
    ehd = _ehd()
    p, par, e = _compare(ehd, Lam)
    assert par["tau_m"] == pytest.approx(p.tau_m, rel=1e-13)
    assert e <= 1e-12, e


@gpu
def test_srt_limit_fp64_parity():
    """Lambda = (tau+ - 1/2)^2 gives tau- = tau+: the TRT collision is the
    single-relaxation-time (BGK) one."""
    ehd = _ehd()
    p0 = o.setup(64, 52, 200.0, 10, 10, 4000, 0.25, u_ion=5e-3)
    Lam = (p0.tau_p - 0.5) ** 2
    p, par, e = _compare(ehd, Lam)
    assert par["tau_m"] == pytest.approx(par["tau_p"], rel=1e-12)
    assert e <= 1e-12, e


@gpu
@pytest.mark.parametrize("storage,bound", [("f64", 1e-12), ("f32", 2e-5)])
def test_three_point_x_symbol_parity(storage, bound):
    ehd = _ehd()
    p, _, e = _compare(ehd, 0.25, storage=storage, x_symbol=1)
    assert e <= bound, e


@gpu
def test_x_symbol_changes_the_solution():
    """The two symbols give measurably different states (the option is live)."""
    ehd = _ehd()
    amp, ph = wl.roll(41, 1e-2)
    runs = [ehd.Run(64, 52, 200.0, 10, 10, 4000, 0.25, storage="f64", u_ion=5e-3, amp=amp, phase=ph,
                    x_symbol=k) for k in (0, 1)]
    for r in runs:
        r.step(300)
    A, B = runs[0].fields(), runs[1].fields()
    assert np.abs(A["Ex"] - B["Ex"]).max() > 1e-9 * np.abs(A["Ex"]).max()
    for r in runs:
        r.close()


@gpu
def test_launch_shape_knobs_keep_results():
    """ehd_tune only changes how work is cut and launched: programmatic
    dependent launch is bitwise neutral; the warp-per-row transforms and
    other tile widths agree with the defaults to FP32 rounding."""
    ehd = _ehd()
    amp, ph = wl.roll(23, 1e-2)
    w = wl.Workload("knobs-2048x40", 2048, 40, 190.0, amp=amp, phase=ph)

    def run_with(pert=0, **tune):
        r = ehd.Run(*w.args(), storage="f32", amp=w.amp, phase=w.phase, perturbation=pert)
        for k, v in tune.items():
            ehd.ehd_tune(r.handle, k, v)
        r.step(40)
        F = r.fields()
        r.close()
        return F

    base = run_with()
    for mask in (0, 1, 2, 3, 4, 7, 8, 11, 15):
        pdl = run_with(pdl=mask)
        for k in base:
            assert np.array_equal(base[k], pdl[k]), (mask, k)
    # the perturbation form (default mask 11; its base chain on a third stream)
    pbase = run_with(pert=1)
    for mask in (0, 3, 7, 15):
        pdl = run_with(pert=1, pdl=mask)
        for k in pbase:
            assert np.array_equal(pbase[k], pdl[k]), ("perturbation", mask, k)
    p = o.setup(*w.args())
    for tune in (dict(fft_cta=0), dict(tile_modes=4), dict(tile_modes=1), dict(step_kernel=1)):
        e = _scaled_err(p, run_with(**tune), base)
        assert e <= 2e-6, (tune, e)


@gpu
@pytest.mark.parametrize("nx,ny", [(64, 3), (256, 100), (2048, 211), (1024, 600)])
def test_wavenumber_solve_forms_same_bits(nx, ny):
    """The wavenumber solve's staging forms -- 16-byte cp.async chunks, tensor
    copies of 256-row boxes (with a tail box for the last Ny % 256 rows), and
    two-CTA clusters that each stage and sweep half of a tile's rows (the
    chunk maps exchanged through distributed shared memory, both CTAs running
    the whole scan) -- give the same results bit for bit, ragged row counts
    included."""
    ehd = _ehd()
    amp, ph = wl.roll(77, 1e-3)
    out = []
    for tune in (dict(tile_tma=0, tile_cluster=0), dict(tile_tma=1, tile_cluster=0), dict(tile_tma=0, tile_cluster=1)):
        r = ehd.Run(nx, ny, 190.0, 10, 10, 4000, 0.25, storage="f32", amp=amp, phase=ph)
        for k, v in tune.items():
            ehd.ehd_tune(r.handle, k, v)
        r.step(30)
        out.append(r.fields())
        r.close()
    for k in out[0]:
        assert np.array_equal(out[0][k], out[1][k]), ("tensor copies", k)
        assert np.array_equal(out[0][k], out[2][k]), ("cluster", k)


@gpu
@pytest.mark.parametrize("storage,bound", [("f64", 1e-12), ("f32", 2e-5), ("bf16", 5e-2)])
def test_spectral_ex_parity(storage, bound):
    """E_x = -d phi/dx from the x-spectrum of phi (-i k_m phi_m, Nyquist
    dropped) in the coupled step, against the oracle with the same option;
    BF16 storage at the bar of its storage-variant test."""
    ehd = _ehd()
    p, _, e = _compare(ehd, 0.25, storage=storage, ex_spectral=1)
    assert e <= bound, e


@gpu
def test_spectral_ex_field_and_effect():
    """The run's E_x field is the oracle's spectral derivative of the run's
    own phi (1e-12), and the option changes the state measurably."""
    ehd = _ehd()
    amp, ph = wl.roll(41, 1e-2)
    runs = [ehd.Run(64, 52, 200.0, 10, 10, 4000, 0.25, storage="f64", u_ion=5e-3, amp=amp, phase=ph,
                    ex_spectral=k) for k in (0, 1)]
    for r in runs:
        r.step(300)
    A, B = runs[0].fields(), runs[1].fields()
    p1 = o.setup(64, 52, 200.0, 10, 10, 4000, 0.25, u_ion=5e-3, ex_spectral=1)
    ex, ey = o.efield(p1, B["phi"])
    for r in runs:
        r.close()
    assert np.abs(B["Ex"] - ex).max() <= 1e-12 * max(1.0, np.abs(ex).max())
    assert np.abs(B["Ey"] - ey).max() <= 1e-12 * max(1.0, np.abs(ey).max())
    # the E_x forms differ by O(k^2) of the roll's mode: 1e-4 of u_x here,
    # against FP64 rounding at 1e-16
    assert np.abs(A["ux"] - B["ux"]).max() > 1e-6 * np.abs(A["ux"]).max()


@gpu
def test_spectral_ex_refusals():
    """Spectral E_x runs keep the march form with two columns per lane and
    ring depth 2 and stay out of batches."""
    ehd = _ehd()
    with pytest.raises(RuntimeError):
        ehd.Run(64, 52, 200.0, 10, 10, 4000, 0.25, storage="f32", ex_spectral=1, step_kernel=1)
    r = ehd.Run(64, 52, 200.0, 10, 10, 4000, 0.25, storage="f32", ex_spectral=1)
    for param, value in (("cols_per_lane", 1), ("ring_depth", 3), ("step_kernel", 1)):
        with pytest.raises(RuntimeError):
            ehd.ehd_tune(r.handle, param, value)
    b = ehd.Batch(2, max_nx=64, max_ny=52)
    with pytest.raises(RuntimeError):
        b.add(r, 10)
    b.close()
    r.close()

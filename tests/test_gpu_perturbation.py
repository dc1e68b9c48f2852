"""The perturbation form of the FP32 path: the charge populations are
stored and collided as departures from an x-uniform base state that is
advanced exactly, in FP64 (its collision, streaming, wall rules and mean-mode
potential).  Same method, same discrete result as the oracle up to FP32
rounding of the departure -- and, unlike the default FP32 form, FP32 then
resolves the charge populations' odd non-equilibrium part, so the growth
rate of a small Eq. 29 roll matches the oracle's within 1 %."""
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


def _errors(p, a, b):
    sc = {"rho": 1.0, "ux": p.u_ion, "uy": p.u_ion, "rho_c": p.rho0, "phi": 1.0, "Ex": 1.0 / p.H,
          "Ey": 1.0 / p.H}
    return {k: float(np.abs(a[k] - b[k]).max() / sc[k]) for k in a}


def _rate(t, a):
    h = a.size // 2
    return float(np.polyfit(np.asarray(t, dtype=np.float64)[h:], np.log(np.asarray(a)[h:]), 1)[0])


@gpu
def test_perturbation_form_parity_1000_steps_128x104():
    """The 128 x 104 channel after 0 and 1000 steps: every field within the
    FP32 bar of the oracle; charge conservation holds with the base's wall
    fluxes included."""
    ehd = _ehd()
    w = wl.plain_fp64_channel()
    p = o.setup(*w.args())
    s = o.init_state(p, w.amp, w.phase)
    run = ehd.Run(*w.args(), storage="f32", amp=w.amp, phase=w.phase, perturbation=1)
    e0 = _errors(p, run.fields(), o.fields(s))
    assert max(e0.values()) <= 2e-6, e0
    d0 = run.diagnostics()
    run.step(1000)
    o.step(s, 1000)
    F = run.fields()
    e = _errors(p, F, o.fields(s))
    assert max(e.values()) <= 2e-5, e
    d1 = run.diagnostics()
    dq = (d1["q_in"] - d0["q_in"]) - (d1["q_out"] - d0["q_out"])
    assert d1["charge"] - d0["charge"] == pytest.approx(dq, rel=1e-6, abs=1e-9 * d0["charge"])
    assert d1["mass"] == pytest.approx(d0["mass"], rel=1e-7)
    run.close()


@gpu
@pytest.mark.parametrize("T", [150.0, 180.0])
def test_perturbation_form_growth_rate_within_1pc_32x26(T):
    """The configuration's roll amplitude A = 1e-3 on 32 x 26 (C = 10,
    M = 10, Fe = 4000), 40,000 steps: the FP32 perturbation form's growth
    rate of max|u_y| is within 1 % of the oracle's (the default FP32 form is
    off by 10-15 % at T = 150)."""
    ehd = _ehd()
    steps, every = 40000, 200
    p = o.setup(32, 26, T, 10, 10, 4000, 0.25, u_ion=2e-3)
    s = o.init_state(p, [1e-3], [0.0])
    d = o.step(s, steps + 1, diag=True)
    t = np.arange(every, steps + 1, every)
    so = _rate(t, d[t, 5])
    run = ehd.Run(32, 26, T, 10, 10, 4000, 0.25, storage="f32", u_ion=2e-3, amp=[1e-3], phase=[0.0],
                  perturbation=1)
    a = []
    for _ in range(t.size):
        run.step(every)
        a.append(run.diagnostics()["max_uy"])
    run.close()
    sg = _rate(t, np.array(a))
    print(f"\nT = {T}: growth rate per step, oracle {so:.6e}, FP32 perturbation form {sg:.6e} "
          f"({100 * (sg - so) / abs(so):+.3f} %)")
    assert np.sign(sg) == np.sign(so) == (1 if T > 163.4 else -1), (so, sg)
    assert abs(sg - so) <= 0.01 * abs(so), (T, so, sg)


@gpu
def test_perturbation_form_load_save_and_refusals():
    """A loaded state is split into its row means (the new base) and the
    departures, and saved back within FP32 rounding of the departures; the
    form is refused where it has no kernels (node-parallel form, FP64)."""
    ehd = _ehd()
    Nx, Ny = 64, 40
    cx, cy, wts, opp = o.lattice()
    p = o.setup(Nx, Ny, 190, 10, 10, 4000, 0.25, u_ion=5e-3)
    f = wl.random_populations(Nx, Ny, 51, 1.0, 0.05) * wts[:, None, None]
    g = wl.random_populations(Nx, Ny, 52, p.rho0, 0.3) * wts[:, None, None]
    run = ehd.Run(Nx, Ny, 190, 10, 10, 4000, 0.25, storage="f32", u_ion=5e-3, perturbation=1)
    run.load(f, g)
    f2, g2 = run.save()
    assert np.abs(g2 - g).max() <= 1e-6 * np.abs(g).max()
    assert np.abs(f2 - f).max() <= 1e-6 * np.abs(f).max()
    s = o.state_from(p, f, g)
    e0 = _errors(p, run.fields(), o.fields(s))
    assert max(e0.values()) <= 2e-5, e0
    run.step(25)
    o.step(s, 25)
    e = _errors(p, run.fields(), o.fields(s))
    assert max(e.values()) <= 2e-5, e
    with pytest.raises(ehd.EhdError):
        ehd.ehd_tune(run.handle, "step_kernel", 1)
    run.close()
    with pytest.raises(ehd.EhdError):
        ehd.Run(Nx, Ny, 190, 10, 10, 4000, 0.25, storage="f64", perturbation=1)


@gpu
def test_perturbation_members_in_a_batch():
    """Perturbation-form runs beside a plain FP32 run in one batch, with
    budgets that end inside a tick: each member reaches exactly the state it
    reaches alone (bitwise populations, fields and wall-flux totals), and the
    perturbation-form members are within the FP32 bar of the oracle."""
    ehd = _ehd()
    specs = [(64, 52, 150.0, 23, 1), (128, 104, 180.0, 40, 1), (128, 40, 200.0, 17, 0), (256, 37, 190.0, 30, 1)]

    def mk(nx, ny, T, pert):
        return ehd.Run(nx, ny, T, 10, 10, 4000, 0.25, storage="f32", u_ion=5e-3, amp=[1e-3, 5e-4],
                       phase=[0.0, 1.0], perturbation=pert)

    batch = ehd.Batch(6, max_nx=256, max_ny=104)
    members = []
    for nx, ny, T, steps, pert in specs:
        r = mk(nx, ny, T, pert)
        batch.add(r, steps)
        members.append(r)
    while any(batch.remaining(r) > 0 for r in members):
        batch.tick(4)
    batch.sync()
    for (nx, ny, T, steps, pert), r in zip(specs, members):
        alone = mk(nx, ny, T, pert)
        alone.step(steps)
        fa, ga = alone.save()
        fb, gb = r.save()
        assert np.array_equal(fa, fb) and np.array_equal(ga, gb), (nx, ny, pert)
        A, B = alone.fields(), r.fields()
        for k in A:
            assert np.array_equal(A[k], B[k]), (nx, ny, k)
        da, db = alone.diagnostics(), r.diagnostics()
        assert da["q_in"] == db["q_in"] and da["q_out"] == db["q_out"], (nx, ny)
        alone.close()
        if pert:
            p = o.setup(nx, ny, T, 10, 10, 4000, 0.25, u_ion=5e-3)
            s = o.init_state(p, [1e-3, 5e-4], [0.0, 1.0])
            o.step(s, steps)
            e = _errors(p, B, o.fields(s))
            assert max(e.values()) <= 2e-5, (nx, ny, e)
    for r in members:
        batch.remove(r)
        r.close()
    batch.close()

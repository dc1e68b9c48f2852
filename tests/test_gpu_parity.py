"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Error measure (scale-normalised max norm): for every field the largest
absolute difference divided by the field's physical scale -- rho: 1,
u: u_ion, rho_c: rho0, phi: dphi0 = 1, E: dphi0 / H.  Bars: plain FP64
<= 1e-12 after 1000 steps; FP32 compute on shifted FP32 storage <= 2e-5.
"""
import functools

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


def _scales(p):
    return {"rho": 1.0, "ux": p.u_ion, "uy": p.u_ion, "rho_c": p.rho0, "phi": 1.0,
            "Ex": 1.0 / p.H, "Ey": 1.0 / p.H}


def _errors(p, gpu_fields, ora_fields):
    sc = _scales(p)
    return {k: float(np.abs(gpu_fields[k] - ora_fields[k]).max() / sc[k]) for k in gpu_fields}


def _pair(w, storage="f64", compute=None, u_ion=2e-3, wall_mode=0):
    ehd = _ehd()
    p = o.setup(w.Nx, w.Ny, w.T, w.C, w.M, w.Fe, w.Lambda, u_ion=u_ion, wall_mode=wall_mode)
    s = o.init_state(p, w.amp, w.phase)
    run = ehd.Run(*w.args(), storage=storage, compute=compute, u_ion=u_ion, wall_mode=wall_mode,
                  amp=w.amp, phase=w.phase)
    return ehd, p, s, run


@gpu
def test_initial_state_and_poisson_match_oracle():
    w = wl.plain_fp64_channel()
    ehd, p, s, run = _pair(w)
    e = _errors(p, run.fields(), o.fields(s))
    assert max(e.values()) < 1e-13, e
    par = run.params()
    for k in ("mu_b", "eps", "nu", "rho0", "Dc", "tau_p", "tau_m", "taug_p", "taug_m", "rho_a", "y_a"):
        assert par[k] == pytest.approx(getattr(p, k), rel=1e-13), k


@gpu
def test_fp64_parity_1000_steps_channel_128x104():
    w = wl.plain_fp64_channel()
    ehd, p, s, run = _pair(w)
    run.step(1000)
    o.step(s, 1000)
    e = _errors(p, run.fields(), o.fields(s))
    assert max(e.values()) <= 1e-12, e


@gpu
def test_fp32_shifted_parity_1000_steps_channel_128x104():
    w = wl.plain_fp64_channel()
    ehd, p, s, run = _pair(w, storage="f32")
    run.step(1000)
    o.step(s, 1000)
    e = _errors(p, run.fields(), o.fields(s))
    assert max(e.values()) <= 2e-5, e


@gpu
@pytest.mark.parametrize("Nx,Ny", [(16, 2), (16, 3), (256, 41), (512, 37)])
def test_fp64_parity_ragged_and_edge_sizes(Nx, Ny):
    """Several 128-column tiles, a ragged row tail, the smallest grids."""
    a, ph = wl.roll(11, 1e-3)
    w = wl.Workload("ragged", Nx, Ny, 180.0, amp=a, phase=ph)
    ehd, p, s, run = _pair(w, u_ion=5e-3)
    run.step(40)
    o.step(s, 40)
    e = _errors(p, run.fields(), o.fields(s))
    assert max(e.values()) <= 1e-12, e


@gpu
def test_fp64_parity_node_walls():
    w = wl.small_channel(64, seed=12)
    ehd, p, s, run = _pair(w, wall_mode=1)
    run.step(100)
    o.step(s, 100)
    e = _errors(p, run.fields(), o.fields(s))
    assert max(e.values()) <= 1e-12, e


@gpu
def test_fp64_parity_from_loaded_random_state():
    """Arbitrary (far from equilibrium) populations loaded through ehd_load."""
    ehd = _ehd()
    Nx, Ny = 64, 40
    p = o.setup(Nx, Ny, 190, 10, 10, 4000, 0.25, u_ion=5e-3)
    cx, cy, w, opp = o.lattice()
    f = wl.random_populations(Nx, Ny, 21, 1.0, 0.05) * w[:, None, None]
    g = wl.random_populations(Nx, Ny, 22, p.rho0, 0.3) * w[:, None, None]
    s = o.state_from(p, f, g)
    run = ehd.Run(Nx, Ny, 190, 10, 10, 4000, 0.25, storage="f64", u_ion=5e-3)
    run.load(f, g)
    e0 = _errors(p, run.fields(), o.fields(s))
    assert max(e0.values()) < 1e-13, e0
    run.step(25)
    o.step(s, 25)
    e = _errors(p, run.fields(), o.fields(s))
    assert max(e.values()) <= 1e-12, e
    # populations themselves: a few ulps of reassociation per step
    f2, g2 = run.save()
    np.testing.assert_allclose(f2, s.f, rtol=0, atol=1e-13 * np.abs(s.f).max())
    np.testing.assert_allclose(g2, s.g, rtol=0, atol=1e-13 * np.abs(s.g).max())


@gpu
def test_load_save_roundtrip_exact_fp64():
    ehd = _ehd()
    Nx, Ny = 32, 26
    f = wl.random_populations(Nx, Ny, 31, 0.1, 0.2)
    g = wl.random_populations(Nx, Ny, 32, 0.001, 0.2)
    run = ehd.Run(Nx, Ny, 200, 10, 10, 4000, 0.25, storage="f64")
    run.load(f, g)
    f2, g2 = run.save()
    assert np.array_equal(f, f2) and np.array_equal(g, g2)


@gpu
def test_graph_replay_bitwise_equals_single_launches():
    """16 steps replayed from the captured CUDA graph equal 16 single steps."""
    ehd = _ehd()
    w = wl.small_channel(64, seed=13)
    r1 = ehd.Run(*w.args(), storage="f64", amp=w.amp, phase=w.phase)
    r2 = ehd.Run(*w.args(), storage="f64", amp=w.amp, phase=w.phase)
    r1.step(16)
    for _ in range(16):
        r2.step(1)
    a, b = r1.save(), r2.save()
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert np.array_equal(r1.fields()["phi"], r2.fields()["phi"])


@gpu
def test_conservation_mass_and_charge_identity_gpu():
    ehd = _ehd()
    w = wl.small_channel(128, seed=14)
    for storage in ("f64", "f32"):
        run = ehd.Run(*w.args(), storage=storage, amp=w.amp, phase=w.phase, u_ion=5e-3)
        d0 = run.diagnostics()
        prev = d0
        for _ in range(20):
            run.step(1)
            d = run.diagnostics()
            resid = (d["charge"] - prev["charge"]) - ((d["q_in"] - prev["q_in"]) - (d["q_out"] - prev["q_out"]))
            tol = 1e-13 if storage == "f64" else 1e-6
            assert abs(resid) <= tol * d0["charge"], (storage, resid)
            prev = d
        assert abs(d["mass"] / d0["mass"] - 1) <= (1e-14 if storage == "f64" else 1e-6)
        assert d["step"] == 20


@gpu
def test_oracle_diagnostics_match_gpu_fluxes():
    w = wl.small_channel(64, seed=15)
    ehd, p, s, run = _pair(w, u_ion=5e-3)
    run.step(30)
    d = o.step(s, 30, diag=True)
    g = run.diagnostics()
    assert g["q_in"] == pytest.approx(d[:, 2].sum(), rel=1e-11)
    assert g["q_out"] == pytest.approx(d[:, 3].sum(), rel=1e-11)
    F = o.fields(s)
    assert g["charge"] == pytest.approx(F["rho_c"].sum(), rel=1e-13)
    assert g["mass"] == pytest.approx(F["rho"].sum(), rel=1e-14)


@gpu
@pytest.mark.parametrize("storage,compute,bound", [("f64", "f32", 2e-5), ("bf16", "f32", 5e-2), ("f16", "f32", 5e-3)])
def test_storage_variants_error_vs_oracle(storage, compute, bound):
    """FP32 compute on shifted FP64 / BF16 / FP16 storage: errors are finite and
    within loose, storage-dependent bounds (measured errors are reported by
    the benchmark)."""
    w = wl.plain_fp64_channel()
    ehd, p, s, run = _pair(w, storage=storage, compute=compute)
    run.step(200)
    o.step(s, 200)
    e = _errors(p, run.fields(), o.fields(s))
    assert all(np.isfinite(v) for v in e.values())
    assert max(e.values()) <= bound, e


@functools.lru_cache(maxsize=1)
def _oracle_1024x840(steps):
    w = wl.precision_channel()
    p = o.setup(*w.args())
    s = o.init_state(p, w.amp, w.phase)
    o.step(s, steps)
    return p, o.fields(s)


@gpu
@pytest.mark.parametrize("storage,compute,bound", [("f64", "f64", 5e-12), ("f32", "f32", 1e-6),
                                                   ("bf16", "f32", 1e-3), ("f16", "f32", 2e-4)])
def test_storage_variants_vs_oracle_1024x840(storage, compute, bound):
    """The 1024 x 840, T = 170 channel after 50 steps, every storage against
    the oracle (measured: plain FP64 2.2e-12, FP32 6.3e-8, BF16 2.5e-4, FP16
    3.3e-5).  The plain FP64 bound is the 1e-12 bar plus twice the oracle's
    own rounding at this height: its Thomas elimination of the mean mode
    loses 2.1e-12 of the E_y scale at 840 rows against a 40-digit solve of the
    same system (tests/test_oracle_rounding.py), against 3e-14 at the 104
    rows of the 1e-12 parity configuration."""
    ehd = _ehd()
    w = wl.precision_channel()
    p, ora = _oracle_1024x840(50)
    run = ehd.Run(*w.args(), storage=storage, compute=compute, amp=w.amp, phase=w.phase)
    run.step(50)
    e = _errors(p, run.fields(), ora)
    run.close()
    print(f"\n1024x840 {storage}/{compute} after 50 steps: {max(e.values()):.3g} ({max(e, key=e.get)})")
    assert max(e.values()) <= bound, e


@gpu
def test_non_finite_state_is_reported():
    """A NaN loaded on the host is detected by the step kernel and reported
    as EHD_EDIVERGED by the next synchronising call."""
    ehd = _ehd()
    Nx, Ny = 32, 26
    _, _, wts, _ = o.lattice()
    f = np.ones((9, Ny, Nx)) * wts[:, None, None]
    g = np.ones((9, Ny, Nx)) * wts[:, None, None] * 1e-3
    f[3, 5, 7] = np.nan
    run = ehd.Run(Nx, Ny, 200, 10, 10, 4000, 0.25, storage="f32")
    run.load(f, g)
    run.step(2)
    with pytest.raises(ehd.EhdError) as ei:
        run.sync()
    assert ei.value.status == -4


@gpu
def test_full_size_fp32_two_steps_vs_oracle():
    """2048 x 1680 in the benchmark's launch configuration: two coupled steps
    against two oracle steps on the whole grid."""
    w = wl.large_channel()
    ehd, p, s, run = _pair(w, storage="f32")
    run.step(2)
    o.step(s, 2)
    e = _errors(p, run.fields(), o.fields(s))
    assert max(e.values()) <= 2e-5, e


@gpu
@pytest.mark.parametrize("storage,tol", [("f64", 1e-13), ("f32", 2e-6)])
def test_march_and_node_parallel_forms_agree(storage, tol):
    """The march form (warp walks a slab, pulls through registers, writes the
    new charge) and the node-parallel push form compute the same step."""
    ehd = _ehd()
    w = wl.small_channel(256, seed=16)
    p = o.setup(*w.args(), u_ion=5e-3)
    r1 = ehd.Run(*w.args(), storage=storage, u_ion=5e-3, amp=w.amp, phase=w.phase, step_kernel=0)
    r2 = ehd.Run(*w.args(), storage=storage, u_ion=5e-3, amp=w.amp, phase=w.phase, step_kernel=1)
    r1.step(37)
    r2.step(37)
    e = _errors(p, r1.fields(), r2.fields())
    assert max(e.values()) <= tol, e
    d1, d2 = r1.diagnostics(), r2.diagnostics()
    ftol = 1e-11 if storage == "f64" else 1e-6
    assert d1["q_in"] == pytest.approx(d2["q_in"], rel=ftol)
    assert d1["q_out"] == pytest.approx(d2["q_out"], rel=ftol)


@gpu
def test_default_step_form():
    """Unless asked, plain FP64 runs take the node-parallel push form (their
    FP64 row walk is latency bound) and every other run the march form."""
    ehd = _ehd()
    cases = ((dict(storage="f64"), 1), (dict(storage="f32"), 0), (dict(storage="f64", compute="f32"), 0),
             (dict(storage="f64", ex_spectral=1), 0), (dict(storage="f64", step_kernel=0), 0))
    for kw, form in cases:
        r = ehd.Run(32, 26, 200.0, 10, 10, 4000, 0.25, **kw)
        assert ehd.ehd_tune_get(r.handle, "step_kernel") == form, kw
        r.close()


@gpu
@pytest.mark.parametrize("slab", [4, 5, 17, 51, 52])
def test_slab_heights_fp64_parity(slab):
    """The march form walks slabs of rows and pushes the populations that
    cross a slab boundary into the neighbouring slab's rows (with their share
    of the charge density); every slab height, including a one-row slab at
    the collector (51 of 52 rows), gives the oracle's state."""
    w = wl.small_channel(64, seed=29)
    ehd, p, s, run = _pair(w, u_ion=5e-3)
    ehd.ehd_tune(run.handle, "step_kernel", 0)  # plain FP64 defaults to the push form
    ehd.ehd_tune(run.handle, "slab_rows", slab)
    run.step(120)
    o.step(s, 120)
    e = _errors(p, run.fields(), o.fields(s))
    assert max(e.values()) <= 1e-12, (slab, e)
    F = o.fields(s)
    assert run.diagnostics()["charge"] == pytest.approx(F["rho_c"].sum(), rel=1e-13)


@gpu
@pytest.mark.parametrize("slab,shift", [(5, 1), (5, 2), (4, 3), (17, 4), (17, 16), (51, 7)])
def test_slab_shift_fp64_parity(slab, shift):
    """The march form with a slab partition that advances `shift` rows each
    step (slab b of step k starts at row b S - (k shift mod S)): every offset
    of the cycle occurs, including a one-row slab at the injector (offset
    S - 1) and one at the collector, and the run keeps the oracle's state
    through graph replays and single steps alike (120 = 7 x 16 + 8 steps)."""
    w = wl.small_channel(64, seed=29)
    ehd, p, s, run = _pair(w, u_ion=5e-3)
    ehd.ehd_tune(run.handle, "step_kernel", 0)  # plain FP64 defaults to the push form
    ehd.ehd_tune(run.handle, "slab_rows", slab)
    ehd.ehd_tune(run.handle, "slab_shift", shift)
    assert ehd.ehd_tune_get(run.handle, "slab_shift") == shift
    run.step(120)
    o.step(s, 120)
    e = _errors(p, run.fields(), o.fields(s))
    assert max(e.values()) <= 1e-12, (slab, shift, e)
    F = o.fields(s)
    assert run.diagnostics()["charge"] == pytest.approx(F["rho_c"].sum(), rel=1e-13)


@gpu
@pytest.mark.parametrize("pert", [0, 1])
def test_slab_shift_fp32_parity_and_graph_replay(pert):
    """FP32 (shifted storage, and the perturbation form) with an advancing
    slab partition: within the FP32 bar of the oracle after 1000 steps at
    128 x 104, and 16 steps replayed from the captured graph equal 16 single
    steps bit for bit (both take the offsets of steps 0..15)."""
    ehd = _ehd()
    w = wl.plain_fp64_channel()
    p = o.setup(*w.args())
    s = o.init_state(p, w.amp, w.phase)

    def mk():
        r = ehd.Run(*w.args(), storage="f32", amp=w.amp, phase=w.phase, perturbation=pert)
        ehd.ehd_tune(r.handle, "slab_rows", 9)
        ehd.ehd_tune(r.handle, "slab_shift", 4)
        return r

    r1, r2 = mk(), mk()
    r1.step(16)
    for _ in range(16):
        r2.step(1)
    a, b = r1.save(), r2.save()
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert np.array_equal(r1.fields()["phi"], r2.fields()["phi"])
    r2.close()
    r1.step(1000 - 16)
    o.step(s, 1000)
    e = _errors(p, r1.fields(), o.fields(s))
    assert max(e.values()) <= 2e-5, (pert, e)
    r1.close()


@gpu
def test_slab_shift_default_only_beyond_l2():
    """The advancing partition is on by default only where the populations
    exceed L2 (2048 x 1680 FP32: 495 MB) and off for runs that fit (128 x
    104), whose results stay those of one fixed partition."""
    ehd = _ehd()
    big = wl.large_channel()
    small = wl.plain_fp64_channel()
    r = ehd.Run(*big.args(), storage="f32", amp=big.amp, phase=big.phase)
    assert ehd.ehd_tune_get(r.handle, "slab_shift") > 0
    r.close()
    r = ehd.Run(*small.args(), storage="f32", amp=small.amp, phase=small.phase)
    assert ehd.ehd_tune_get(r.handle, "slab_shift") == 0
    r.close()


@gpu
def test_c1_plain_fp64_10000_steps_vs_oracle():
    """The plain FP64 configuration run to its full length: 128 x 104,
    T = 200, 10,000 coupled steps on the GPU and in the oracle.  Every field
    within 1e-12 (scaled max norm) at the end, and the exponential rate of
    max|u_y| over the run (least-squares slope of its log over the second
    half, sampled every 100 steps) within 1 % of the oracle's (measured
    3.4e-13 and 5e-10 relative)."""
    w = wl.plain_fp64_channel()
    ehd, p, s, run = _pair(w)
    d = o.step(s, 10000, diag=True)  # row t: the state at step t
    t = np.arange(100, 10000, 100)
    a = []
    for _ in range(t.size):
        run.step(100)
        a.append(run.diagnostics()["max_uy"])
    run.step(100)
    e = _errors(p, run.fields(), o.fields(s))
    assert max(e.values()) <= 1e-12, e

    def rate(amp):
        h = amp.size // 2
        return float(np.polyfit(t[h:], np.log(amp[h:]), 1)[0])

    so, sg = rate(d[t, 5]), rate(np.array(a))
    assert abs(sg - so) <= 0.01 * abs(so), (so, sg)


@gpu
def test_c2_fp32_vs_gpu_fp64_2000_steps_2048x1680():
    """The large configuration at full length: 2048 x 1680, FP32 compute on
    shifted FP32 storage against the plain FP64 GPU path (itself pinned to
    the oracle above) after 2,000 steps, every field within 2e-5 of its scale
    (measured 2.1e-7, rho_c)."""
    ehd = _ehd()
    w = wl.large_channel()
    F = {}
    par = None
    for st in ("f64", "f32"):
        run = ehd.Run(*w.args(), storage=st, amp=w.amp, phase=w.phase)
        run.step(2000)
        F[st] = run.fields()
        par = run.params()
        run.close()
    p = o.setup(*w.args())
    assert par["rho0"] == pytest.approx(p.rho0, rel=1e-14)
    e = _errors(p, F["f32"], F["f64"])
    assert max(e.values()) <= 2e-5, e


@gpu
@pytest.mark.parametrize("Nx,Ny,slab", [(128, 104, 0), (256, 37, 5), (512, 416, 0), (2048, 64, 17), (1024, 9, 4)])
def test_tma_march_equals_cp_async_march(Nx, Ny, slab):
    """The march form's TMA staging (tensor copies of whole row segments,
    tensor stores of completed rows, wrap-around halo pairs fetched by their
    own lanes) computes bit for bit what the per-lane cp.async form does,
    including ragged last strips, slab boundaries and one-wave slab sizes."""
    ehd = _ehd()
    a, ph = wl.roll(31, 1e-2)
    runs = []
    for tma in (0, 1, 2, 3):
        r = ehd.Run(Nx, Ny, 190.0, 10, 10, 4000, 0.25, storage="f32", u_ion=5e-3, amp=a, phase=ph)
        ehd.ehd_tune(r.handle, "march_tma", tma)
        if slab:
            ehd.ehd_tune(r.handle, "slab_rows", slab)
        assert ehd.ehd_tune_get(r.handle, "march_tma") == tma
        r.step(33)
        runs.append(r)
    fa, ga = runs[0].save()
    da = runs[0].diagnostics()
    for r in runs[1:]:
        fb, gb = r.save()
        assert np.array_equal(fa, fb) and np.array_equal(ga, gb)
        db = r.diagnostics()
        assert da["q_in"] == db["q_in"] and da["q_out"] == db["q_out"]
    for r in runs:
        r.close()

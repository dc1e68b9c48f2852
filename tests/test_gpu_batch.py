"""Batches: runs of uneven sizes advanced together by the batch phase
kernels give, run by run, exactly the state the run reaches alone (the same
per-run arithmetic), whatever else is in the batch and however budgets end
inside a tick."""
import numpy as np
import pytest

import workloads as wl

gpu = pytest.mark.gpu


def _ehd():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1812_05711_gb300 as ehd
    return ehd


def _mk(ehd, w):
    return ehd.Run(*w.args(), storage="f32", u_ion=5e-3, amp=w.amp, phase=w.phase)


@gpu
def test_batch_members_match_alone_bitwise():
    ehd = _ehd()
    specs = [(64, 150.0, 5.0, 23), (128, 175.0, 10.0, 40), (256, 200.0, 20.0, 17), (512, 240.0, 10.0, 30),
             (128, 260.0, 5.0, 40)]
    ws = []
    for k, (nx, T, C, steps) in enumerate(specs):
        a, ph = wl.roll(300 + k, 1e-3)
        ws.append((wl.Workload(f"b{k}", nx, wl.ny_for(nx), T, C=C, amp=a, phase=ph), steps))
    batch = ehd.Batch(8, max_nx=512, max_ny=wl.ny_for(512))
    members = []
    for w, steps in ws:
        r = _mk(ehd, w)
        batch.add(r, steps)
        members.append(r)
    ticks = 0
    while any(batch.remaining(r) > 0 for r in members):
        batch.tick(4)
        ticks += 1
    batch.sync()
    assert ticks == 10
    for (w, steps), r in zip(ws, members):
        alone = _mk(ehd, w)
        alone.step(steps)
        assert r.params()["Nx"] == w.Nx
        fa, ga = alone.save()
        fb, gb = r.save()
        assert np.array_equal(fa, fb) and np.array_equal(ga, gb), w.name
        A, B = alone.fields(), r.fields()
        for k in A:
            assert np.array_equal(A[k], B[k]), (w.name, k)
        da, db = alone.diagnostics(), r.diagnostics()
        assert da["q_in"] == db["q_in"] and da["q_out"] == db["q_out"]
        assert db["step"] == steps
    batch.close()


@gpu
def test_batch_membership_changes_between_ticks():
    ehd = _ehd()
    a0, p0 = wl.roll(401, 1e-3)
    a1, p1 = wl.roll(402, 1e-3)
    w0 = wl.Workload("m0", 128, 104, 190.0, amp=a0, phase=p0)
    w1 = wl.Workload("m1", 256, 208, 210.0, amp=a1, phase=p1)
    batch = ehd.Batch(2, max_nx=256, max_ny=208)
    r0, r1 = _mk(ehd, w0), _mk(ehd, w1)
    batch.add(r0, 12)
    batch.tick(6)
    batch.add(r1, 8)            # joins mid-way
    with pytest.raises(ehd.EhdError) as ei:
        batch.add(_mk(ehd, w0), 4)  # full
    assert ei.value.status == -6
    batch.tick(6)
    batch.remove(r0)            # r0 done (12 steps)
    batch.tick(2)
    batch.sync()
    assert batch.remaining(r1) == 0 and len(batch) == 1
    with pytest.raises(ehd.EhdError):
        r1.step(1)              # members are advanced by the batch only
    for w, r, n in ((w0, r0, 12), (w1, r1, 8)):
        alone = _mk(ehd, w)
        alone.step(n)
        assert np.array_equal(alone.fields()["phi"], r.fields()["phi"]), w.name
        assert np.array_equal(alone.save()[1], r.save()[1]), w.name
    batch.close()
    r1.step(2)                  # an ordinary run again


@gpu
def test_batch_row_limit_is_checked_at_creation():
    """A batch whose wavenumber tiles (max_ny rows of 8 wavenumbers) would not
    fit in shared memory is refused when it is created, not at its first tick."""
    ehd = _ehd()
    with pytest.raises(RuntimeError):
        ehd.Batch(2, max_nx=64, max_ny=4096)
    b = ehd.Batch(2, max_nx=64, max_ny=2048)
    b.close()


@gpu
def test_batch_hbm_budget_admission():
    """The batch keeps the HBM account behind the C ABI: with a budget for
    two 128 x 104 runs, a third waits (EHD_EBUSY from the query and from
    ehd_batch_add), a run larger than the whole budget is refused for good
    (EHD_EINVAL), and removing a member frees its bytes."""
    ehd = _ehd()
    fp = ehd.ehd_footprint(128, 104, ehd.STORAGE["f32"])
    batch = ehd.Batch(8, max_nx=512, max_ny=416, hbm_budget=2 * fp + fp // 2)
    assert batch.memory() == (0, 2 * fp + fp // 2)
    ws = []
    for k in range(3):
        a, ph = wl.roll(500 + k, 1e-3)
        ws.append(wl.Workload(f"h{k}", 128, 104, 180.0 + 10 * k, amp=a, phase=ph))
    runs = []
    for w in ws[:2]:
        assert batch.admits(128, 104) == 0
        r = _mk(ehd, w)
        batch.add(r, 4)
        runs.append(r)
    assert batch.memory()[0] == 2 * fp
    assert batch.admits(128, 104) == -6
    assert batch.admits(512, 416) == -1  # above the whole budget
    extra = _mk(ehd, ws[2])
    with pytest.raises(ehd.EhdError) as ei:
        batch.add(extra, 4)
    assert ei.value.status == -6 and "HBM budget" in str(ei.value)
    batch.tick(4)
    batch.remove(runs[0])
    assert batch.memory()[0] == fp and batch.admits(128, 104) == 0
    batch.add(extra, 2)
    batch.tick(2)
    batch.sync()
    assert batch.remaining(extra) == 0
    batch.close()


def _scaled_errors(p, a, b):
    sc = {"rho": 1.0, "ux": p.u_ion, "uy": p.u_ion, "rho_c": p.rho0, "phi": 1.0, "Ex": 1.0 / p.H,
          "Ey": 1.0 / p.H}
    return {k: float(np.abs(a[k] - b[k]).max() / sc[k]) for k in a}


@gpu
def test_batch_members_vs_oracle():
    """Uneven members of one batch (Nx 64 and 512, C = 5 and 20, different
    T and Fe) against the FP64 oracle after 100 steps, each within the FP32
    bar of 2e-5 (scaled max norm)."""
    import oracle as o
    ehd = _ehd()
    specs = [(64, 150.0, 5.0, 4000.0, 601), (512, 230.0, 20.0, 2000.0, 602), (128, 200.0, 20.0, 4000.0, 603)]
    batch = ehd.Batch(4, max_nx=512, max_ny=wl.ny_for(512))
    members = []
    for nx, T, C, Fe, seed in specs:
        a, ph = wl.roll(seed, 1e-3)
        w = wl.Workload(f"o{nx}", nx, wl.ny_for(nx), T, C=C, Fe=Fe, amp=a, phase=ph)
        r = _mk(ehd, w)
        batch.add(r, 100)
        members.append((w, r))
    while any(batch.remaining(r) > 0 for _, r in members):
        batch.tick(20)
    batch.sync()
    for w, r in members:
        p = o.setup(*w.args(), u_ion=5e-3)
        s = o.init_state(p, w.amp, w.phase)
        o.step(s, 100)
        e = _scaled_errors(p, r.fields(), o.fields(s))
        assert max(e.values()) <= 2e-5, (w.name, e)
    batch.close()

"""Growth of an Eq. 29 roll on the GPU path: its exponential rate agrees with
the oracle's within 1 %, and a threshold sweep on the paper's box aspect
brackets the critical T (163.4 in the paper's linear-stability experiment).

The growth rate is the least-squares slope of log max|u_y| over the second
half of the record (the first half lets the roll relax onto the least
stable mode)."""
import functools

import numpy as np
import pytest

import oracle as o

gpu = pytest.mark.gpu

T_C_PAPER = 163.4


def _ehd():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1812_05711_gb300 as ehd
    return ehd


def _rate(t, a):
    t, a = np.asarray(t, dtype=np.float64), np.asarray(a, dtype=np.float64)
    h = a.size // 2
    return float(np.polyfit(t[h:], np.log(a[h:]), 1)[0])


@functools.lru_cache(maxsize=None)
def _oracle_record(Nx, Ny, T, steps, every, A=1e-3):
    p = o.setup(Nx, Ny, T, 10, 10, 4000, 0.25, u_ion=2e-3)
    s = o.init_state(p, [A], [0.0])
    d = o.step(s, steps + 1, diag=True)  # row t holds the state at time t
    t = np.arange(every, steps + 1, every)
    return t, d[t, 5]


def _gpu_record(ehd, Nx, Ny, T, steps, every, storage, A=1e-3, pert=0):
    run = ehd.Run(Nx, Ny, T, 10, 10, 4000, 0.25, storage=storage, u_ion=2e-3, amp=[A], phase=[0.0],
                  perturbation=pert)
    t, a = [], []
    for k in range(steps // every):
        run.step(every)
        t.append((k + 1) * every)
        a.append(run.diagnostics()["max_uy"])
    run.close()
    return np.array(t), np.array(a)


@gpu
@pytest.mark.parametrize("storage,pert,A", [("f64", 0, 1e-3), ("f32", 1, 1e-3), ("f32", 0, 5e-2)],
                         ids=["f64", "f32-perturbation", "f32-shifted-A5e-2"])
def test_growth_rate_matches_oracle_32x26(storage, pert, A):
    """32 x 26 (aspect 1.23), C = 10, M = 10, Fe = 4000, 40,000 steps:
    sigma(T = 180) > 0 and sigma(T = 150) < 0, each within 1 % of the
    oracle's, at the configuration's roll amplitude A = 1e-3 (times the ion
    drift speed) for FP64 and for the FP32 perturbation form.  The default
    (shifted) FP32 form is compared at A = 5e-2: at A = 1e-3 its rate is off
    by 10-15 % at T = 150 (1 % at T = 180), because FP32 storage of the
    whole charge populations does not resolve their odd non-equilibrium part,
    which at Fe = 4000 flips sign every step (omega_g- close to 2) with an
    amplitude far above the diffusive flux it carries; the perturbation form
    stores only the departure from the x-uniform base state, whose odd part
    is of the roll's size."""
    ehd = _ehd()
    steps, every = 40000, 200
    for T in (180.0, 150.0):
        to, ao = _oracle_record(32, 26, T, steps, every, A)
        tg, ag = _gpu_record(ehd, 32, 26, T, steps, every, storage, A, pert)
        assert np.array_equal(to, tg)
        so, sg = _rate(to, ao), _rate(tg, ag)
        assert np.sign(sg) == np.sign(so) == (1 if T > T_C_PAPER else -1), (T, so, sg)
        assert abs(sg - so) <= 0.01 * abs(so), (storage, pert, T, so, sg)
        if storage == "f64":
            np.testing.assert_allclose(ag, ao, rtol=1e-8)


@gpu
def test_threshold_sweep_brackets_tc_128x104():
    """The paper's experiment on a 128 x 104 channel (aspect 1.23) with
    FP32 perturbation-form runs advanced together in one batch: T in {150,
    160, 170, 180}, 300,000 steps (5.8 ion transits), the configuration's
    roll amplitude A = 1e-3.  Hard: the roll decays at T = 150 and grows at
    T = 180.  Reported: T_c from linear interpolation of sigma(T)."""
    ehd = _ehd()
    Ts = (150.0, 160.0, 170.0, 180.0)
    steps, tick = 300000, 1000
    batch = ehd.Batch(len(Ts), max_nx=128, max_ny=104)
    runs = [ehd.Run(128, 104, T, 10, 10, 4000, 0.25, storage="f32", u_ion=2e-3, amp=[1e-3], phase=[0.0],
                    perturbation=1)
            for T in Ts]
    for r in runs:
        batch.add(r, steps)
    t, amp = [], [[] for _ in Ts]
    for k in range(steps // tick):
        batch.tick(tick)
        t.append((k + 1) * tick)
        for i, r in enumerate(runs):
            amp[i].append(r.diagnostics()["max_uy"])
    sig = [_rate(t, a) for a in amp]
    for r in runs:
        batch.remove(r)
        r.close()
    batch.close()
    assert sig[0] < 0 < sig[-1], sig
    k = next(i for i in range(1, len(Ts)) if sig[i] > 0)
    tc = Ts[k - 1] + (Ts[k] - Ts[k - 1]) * (-sig[k - 1]) / (sig[k] - sig[k - 1])
    print(f"\nthreshold sweep 128x104: sigma per step {dict(zip(Ts, sig))}; T_c = {tc:.1f} "
          f"(paper {T_C_PAPER}, {100 * (tc / T_C_PAPER - 1):+.1f} %)")
    assert Ts[0] < tc < Ts[-1]

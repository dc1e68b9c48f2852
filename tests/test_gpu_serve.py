"""Continuous-batching server: requests admitted as slots and HBM free up,
overlapping on the device, each result identical to the request run alone."""
import numpy as np
import pytest

import workloads as wl

gpu = pytest.mark.gpu


def _mods():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1812_05711_gb300 as ehd
    from paper_1812_05711_gb300 import serve
    return ehd, serve


@gpu
def test_server_results_equal_solo_runs_and_respect_budget():
    ehd, serve = _mods()
    specs = [(64, 160.0, 10.0, 30), (128, 180.0, 5.0, 22), (256, 200.0, 20.0, 16), (128, 220.0, 10.0, 40),
             (64, 240.0, 100.0, 12), (256, 260.0, 1.0, 26), (128, 150.0, 10.0, 18)]
    reqs = []
    for k, (nx, T, C, steps) in enumerate(specs):
        a, ph = wl.roll(500 + k, 1e-3)
        # every third request in the FP32 perturbation form (its base state
        # advances on the batch's third stream)
        reqs.append(serve.Request(k, nx, wl.ny_for(nx), T, C, 10.0, 4000.0, 0.25, steps, a, ph, arrival=0.0,
                                  perturbation=int(k % 3 == 1)))
    fp = ehd.ehd_footprint(256, wl.ny_for(256), 1)
    budget = fp + 2 * ehd.ehd_footprint(128, wl.ny_for(128), 1)  # forces queueing
    srv = serve.Server(budget, max_runs=3, tick_steps=6, max_nx=256, max_ny=wl.ny_for(256), u_ion=5e-3,
                       keep_fields=("phi", "rho_c", "ux"))
    peak = [0]
    orig_admit = srv._admit

    def admit(now):
        orig_admit(now)
        peak[0] = max(peak[0], srv.used)
        assert len(srv.active) <= 3

    srv._admit = admit
    results = srv.serve(reqs, realtime=False)
    srv.close()
    assert len(results) == len(reqs)
    assert peak[0] <= budget
    assert srv.ticks >= 4  # runs came and went across ticks
    for res in results:
        q = reqs[res.rid]
        solo = ehd.Run(q.Nx, q.Ny, q.T, q.C, q.M, q.Fe, q.Lambda, storage="f32", u_ion=5e-3, amp=q.amp,
                       phase=q.phase, perturbation=q.perturbation)
        solo.step(q.steps)
        d = solo.diagnostics()
        assert res.diagnostics["step"] == q.steps
        for k in ("mass", "charge", "q_in", "q_out", "kinetic", "max_uy"):
            assert res.diagnostics[k] == d[k], (q.rid, k)
        F = solo.fields(("phi", "rho_c", "ux"))
        for k in F:
            assert np.array_equal(F[k], res.fields[k]), (q.rid, k)
        solo.close()
    lat = serve.summarize(results)
    assert lat["runs"] == len(reqs) and lat["p99_s"] >= lat["p50_s"] > 0

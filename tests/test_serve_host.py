"""Host logic of the continuous-batching server on the CPU: admission in
arrival order under the HBM budget and the slot limit, retirement when a
run's budget is used up, the released memory admitting the next request, and
the latency summary.  The GPU objects (runs, the batch, the footprint) are
replaced by fakes that count steps, so no device is needed."""
import pytest

pytest.importorskip("torch")

import paper_1812_05711_gb300.serve as serve  # noqa: E402


class FakeRun:
    _next = 0
    created = []

    def __init__(self, Nx, Ny, *args, **kwargs):
        FakeRun._next += 1
        self.handle = FakeRun._next
        self.Nx, self.Ny = Nx, Ny
        self.kwargs = kwargs
        FakeRun.created.append(self)
        self.closed = False
        self.steps_done = 0
        self.loaded = None

    def diagnostics(self):
        # collected charge grows by 2 per step: the window's current is 2
        return {"mass": float(self.Nx * self.Ny), "q_out": 2.0 * self.steps_done}

    def save(self):
        return ("f", self.handle), ("g", self.handle)

    def load(self, f, g):
        self.loaded = (f, g)

    def fields(self, names):
        return {}

    def close(self):
        self.closed = True


class FakeBatch:
    """Slots and HBM accounting as ehd_batch_admits / ehd_batch_add keep
    them (footprint of an Nx x Ny run: Nx * Ny bytes)."""

    def __init__(self, max_runs, max_nx, max_ny, hbm_budget=0):
        self.left = {}
        self.bytes = {}
        self.ticks = []
        self.max_runs, self.budget = max_runs, hbm_budget

    def admits(self, Nx, Ny, storage="f32"):
        need = Nx * Ny
        if self.budget and need > self.budget:
            return -1
        if len(self.left) >= self.max_runs or (self.budget and sum(self.bytes.values()) + need > self.budget):
            return -6
        return 0

    def memory(self):
        return sum(self.bytes.values()), self.budget

    def add(self, run, steps):
        assert self.admits(run.Nx, run.Ny) == 0
        self.left[run.handle] = steps
        self.bytes[run.handle] = run.Nx * run.Ny
        self.runs = getattr(self, "runs", {})
        self.runs[run.handle] = run

    def remaining(self, run):
        return self.left[run.handle]

    def remove(self, run):
        del self.left[run.handle]
        del self.bytes[run.handle]

    def tick(self, k):
        self.ticks.append(sorted(self.left))
        for h in self.left:
            n = min(k, self.left[h])
            self.runs[h].steps_done += n
            self.left[h] -= n

    def sync(self):
        pass

    def close(self):
        pass


class Clock:
    """Advances one second per reading, so latencies are deterministic."""

    def __init__(self):
        self.t = 0.0

    def __call__(self):
        self.t += 1.0
        return self.t


@pytest.fixture
def fakes(monkeypatch):
    monkeypatch.setattr(serve, "Run", FakeRun)
    monkeypatch.setattr(serve, "Batch", FakeBatch)
    monkeypatch.setattr(serve, "ehd_footprint", lambda nx, ny, st: nx * ny)
    return serve


def _req(rid, nx, steps, arrival=0.0):
    return serve.Request(rid, nx, nx, 200.0, 10.0, 10.0, 4000.0, 0.25, steps, arrival=arrival)


def test_admission_respects_budget_and_order(fakes):
    # budget for two 64x64 runs at a time; four requests arrive together
    srv = fakes.Server(hbm_budget=2 * 64 * 64, max_runs=8, tick_steps=2, max_nx=128, max_ny=128,
                       clock=Clock())
    reqs = [_req(0, 64, 4), _req(1, 64, 2), _req(2, 64, 2), _req(3, 64, 2)]
    res = srv.serve(reqs, realtime=False)
    ticks = srv.batch.ticks
    # first tick: runs 0 and 1 only (memory); run 1 retires after it and frees
    # room for run 2 (first come, first served); runs 0 and 2 end together
    # after the second tick and run 3 takes the third alone
    assert [len(t) for t in ticks] == [2, 2, 1]
    assert [r.rid for r in res] == [1, 0, 2, 3]
    assert srv.used == 0 and not srv.active and not srv.waiting
    assert all(r.steps in (2, 4) for r in res)


def test_slot_limit_and_large_request_waits(fakes):
    srv = fakes.Server(hbm_budget=10 ** 9, max_runs=1, tick_steps=2, max_nx=128, max_ny=128, clock=Clock())
    res = srv.serve([_req(0, 128, 2), _req(1, 64, 2)], realtime=False)
    assert [len(t) for t in srv.batch.ticks] == [1, 1]
    assert [r.rid for r in res] == [0, 1]
    # the second request waited one tick: admitted after the first finished
    assert res[1].admitted > res[0].admitted


def test_submit_rejects_what_can_never_run(fakes):
    srv = fakes.Server(hbm_budget=64 * 64, max_runs=4, tick_steps=2, max_nx=128, max_ny=128, clock=Clock())
    with pytest.raises(ValueError):
        srv.submit(_req(0, 256, 2))       # wider than the server's batch
    with pytest.raises(ValueError):
        srv.submit(_req(1, 128, 2))       # footprint above the whole budget
    with pytest.raises(ValueError):
        fakes.Server(hbm_budget=1, tick_steps=3)  # odd tick length


def test_summary_percentiles():
    rs = [serve.Result(i, 0.0, 0.0, float(i + 1), 10, {}) for i in range(100)]
    s = serve.summarize(rs, cells_of=lambda r: 1000)
    assert s["runs"] == 100 and s["makespan_s"] == 100.0
    assert s["p50_s"] == pytest.approx(50.5) and s["p99_s"] == pytest.approx(99.01)
    assert s["glups"] == pytest.approx(100 * 1000 * 10 / 100.0 / 1e9)


def test_measurement_window_and_continuation(fakes):
    """A request's last `window` steps measure the collected current (the run
    stays in its slot between the two parts), and a request that continues
    from another starts from that one's final populations once it is done,
    while independent requests go ahead of it."""
    srv = fakes.Server(hbm_budget=10 ** 9, max_runs=8, tick_steps=4, max_nx=128, max_ny=128, clock=Clock())
    a = fakes.Request(0, 64, 64, 200.0, 10.0, 10.0, 4000.0, 0.25, 12, window=4)
    b = fakes.Request(1, 64, 64, 190.0, 10.0, 10.0, 4000.0, 0.25, 8, window=8, after=0)
    c = fakes.Request(2, 64, 64, 180.0, 10.0, 10.0, 4000.0, 0.25, 4)
    res = {r.rid: r for r in srv.serve([a, b, c], realtime=False)}
    assert res[0].current == pytest.approx(2.0) and res[1].current == pytest.approx(2.0)
    assert res[2].current is None
    assert res[1].admitted >= res[0].done      # waited for its predecessor
    assert res[2].admitted < res[0].done       # independent: went ahead
    assert res[0].state is not None            # kept for the continuation
    first_tick = srv.batch.ticks[0]
    assert len(first_tick) == 2                # a and c together, b waiting
    with pytest.raises(ValueError):
        srv.submit(fakes.Request(9, 64, 64, 1.0, 1.0, 1.0, 1.0, 0.25, 4, after=77))


def test_perturbation_form_requests(fakes):
    """A request may ask for the FP32 perturbation form; the server creates
    its run with it (the others keep the default form)."""
    FakeRun.created.clear()
    srv = fakes.Server(hbm_budget=10 ** 9, max_runs=4, tick_steps=2, max_nx=128, max_ny=128, clock=Clock())
    a = fakes.Request(0, 64, 64, 150.0, 10.0, 10.0, 4000.0, 0.25, 4, perturbation=1)
    b = fakes.Request(1, 64, 64, 180.0, 10.0, 10.0, 4000.0, 0.25, 4)
    srv.serve([a, b], realtime=False)
    forms = sorted(r.kwargs.get("perturbation") for r in FakeRun.created)
    assert forms == [0, 1]

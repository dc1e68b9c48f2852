"""ehd_poisson_noalloc: the Poisson solve for callers that cannot allocate
device memory while they run (a device-memory budget fully reserved by a
framework pool, or a loop that cannot take cudaMalloc's implicit
synchronisation).  Its intermediates live in a fixed static device array, so
the check here is that two calls in a row, on different grid sizes, give the
same potential as the allocating path (ehd_poisson on a run) within the FP32
bar used by the other GPU tests, and that oversize grids are refused.

Collected last on purpose: if it fails, a run that stops at the first failure
has already run every other test."""
import numpy as np
import pytest

gpu = pytest.mark.gpu


def _ehd():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1812_05711_gb300 as ehd
    return torch, ehd


@gpu
def test_noalloc_poisson_matches_run_poisson_twice():
    torch, ehd = _ehd()
    cases = [(256, 208, 180.0, 41), (128, 104, 220.0, 42)]
    for Nx, Ny, T, seed in cases:  # two calls in a row, sizes change between them
        rng = np.random.default_rng(seed)
        amp = list(rng.uniform(-1e-3, 1e-3, 3))
        ph = list(rng.uniform(0, 6.28, 3))
        run = ehd.Run(Nx, Ny, T, 10, 10, 4000, 0.25, storage="f32", u_ion=5e-3, amp=amp, phase=ph)
        run.step(40)  # a charge field with structure in x and y
        F = run.fields(["rho_c", "phi"])  # phi of the run = ehd_poisson of its rho_c
        eps = run.params()["eps"]
        rhoc = torch.tensor(F["rho_c"], dtype=torch.float32, device="cuda")
        phi = torch.full((Ny, Nx), float("nan"), dtype=torch.float32, device="cuda")
        torch.cuda.synchronize()
        ehd.ehd_poisson_noalloc(Nx, Ny, eps, 1.0, 0, rhoc.data_ptr(), phi.data_ptr(), 0)
        torch.cuda.synchronize()
        got = phi.double().cpu().numpy()
        err = np.abs(got - F["phi"]).max()  # phi scale is dphi0 = 1
        assert np.isfinite(got).all()
        assert err <= 2e-5, (Nx, Ny, err)
        run.close()


@gpu
def test_noalloc_poisson_node_walls_and_wall_potential():
    """Walls on the extra nodes (wall_mode 1) against ehd_poisson of a run
    created with them, and the injector potential phi0: the solve is linear,
    so phi0 = 2.5 adds 1.5 times the charge-free profile, which for these
    walls is the straight line phi0 (1 - (j + 1) / (Ny + 1))."""
    torch, ehd = _ehd()
    Nx, Ny = 128, 104
    rng = np.random.default_rng(43)
    amp, ph = list(rng.uniform(-1e-3, 1e-3, 3)), list(rng.uniform(0, 6.28, 3))
    run = ehd.Run(Nx, Ny, 200.0, 10, 10, 4000, 0.25, storage="f32", u_ion=5e-3, amp=amp, phase=ph,
                  wall_mode=1)
    run.step(40)
    F = run.fields(["rho_c", "phi"])
    eps = run.params()["eps"]
    run.close()
    rhoc = torch.tensor(F["rho_c"], dtype=torch.float32, device="cuda")
    out = {}
    for phi0 in (1.0, 2.5):
        phi = torch.full((Ny, Nx), float("nan"), dtype=torch.float32, device="cuda")
        torch.cuda.synchronize()
        ehd.ehd_poisson_noalloc(Nx, Ny, eps, phi0, 1, rhoc.data_ptr(), phi.data_ptr(), 0)
        torch.cuda.synchronize()
        out[phi0] = phi.double().cpu().numpy()
    assert np.abs(out[1.0] - F["phi"]).max() <= 2e-5
    line = (1.0 - (np.arange(Ny) + 1.0) / (Ny + 1.0))[:, None] * np.ones(Nx)
    assert np.abs((out[2.5] - out[1.0]) - 1.5 * line).max() <= 2e-5


@gpu
def test_noalloc_poisson_captured_then_other_sizes():
    """Work captured into a CUDA graph for one grid keeps giving that grid's
    potential when direct calls for another grid (which rebuild the shared
    tables for their sizes) run between replays, and the direct calls stay
    right after the replays."""
    torch, ehd = _ehd()
    cases = {}
    for Nx, Ny, seed in ((128, 104, 44), (256, 208, 45)):
        rng = np.random.default_rng(seed)
        amp, ph = list(rng.uniform(-1e-3, 1e-3, 3)), list(rng.uniform(0, 6.28, 3))
        run = ehd.Run(Nx, Ny, 190.0, 10, 10, 4000, 0.25, storage="f32", u_ion=5e-3, amp=amp, phase=ph)
        run.step(30)
        F = run.fields(["rho_c", "phi"])
        eps = run.params()["eps"]
        run.close()
        rhoc = torch.tensor(F["rho_c"], dtype=torch.float32, device="cuda")
        phi = torch.full((Ny, Nx), float("nan"), dtype=torch.float32, device="cuda")
        cases[(Nx, Ny)] = (rhoc, phi, eps, F["phi"])
    (Na, Nya), (Nb, Nyb) = list(cases)
    ra, pa, ea, refa = cases[(Na, Nya)]
    rb, pb, eb, refb = cases[(Nb, Nyb)]
    s = torch.cuda.Stream()
    torch.cuda.synchronize()
    ehd.ehd_poisson_noalloc(Na, Nya, ea, 1.0, 0, ra.data_ptr(), pa.data_ptr(), s.cuda_stream)  # set-up call
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s, capture_error_mode="relaxed"):
        ehd.ehd_poisson_noalloc(Na, Nya, ea, 1.0, 0, ra.data_ptr(), pa.data_ptr(), s.cuda_stream)
    for _ in range(2):
        pa.fill_(float("nan"))
        pb.fill_(float("nan"))
        torch.cuda.synchronize()
        ehd.ehd_poisson_noalloc(Nb, Nyb, eb, 1.0, 0, rb.data_ptr(), pb.data_ptr(), 0)
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        assert np.abs(pa.double().cpu().numpy() - refa).max() <= 2e-5
        assert np.abs(pb.double().cpu().numpy() - refb).max() <= 2e-5
        pb.fill_(float("nan"))
        torch.cuda.synchronize()
        ehd.ehd_poisson_noalloc(Nb, Nyb, eb, 1.0, 0, rb.data_ptr(), pb.data_ptr(), 0)
        torch.cuda.synchronize()
        assert np.abs(pb.double().cpu().numpy() - refb).max() <= 2e-5


@gpu
def test_noalloc_poisson_rejects_oversize_grid():
    torch, ehd = _ehd()
    x = torch.zeros(1, dtype=torch.float32, device="cuda")
    with pytest.raises(ehd.EhdError) as ei:
        ehd.ehd_poisson_noalloc(2048, 1680, 1.0, 1.0, 0, x.data_ptr(), x.data_ptr(), 0)
    assert ei.value.status == -1 and "8 MiB" in str(ei.value)
    with pytest.raises(ehd.EhdError):
        ehd.ehd_poisson_noalloc(100, 64, 1.0, 1.0, 0, x.data_ptr(), x.data_ptr(), 0)

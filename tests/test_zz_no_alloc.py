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
def test_noalloc_poisson_rejects_oversize_grid():
    torch, ehd = _ehd()
    x = torch.zeros(1, dtype=torch.float32, device="cuda")
    with pytest.raises(ehd.EhdError) as ei:
        ehd.ehd_poisson_noalloc(2048, 1680, 1.0, 1.0, 0, x.data_ptr(), x.data_ptr(), 0)
    assert ei.value.status == -1 and "8 MiB" in str(ei.value)
    with pytest.raises(ehd.EhdError):
        ehd.ehd_poisson_noalloc(100, 64, 1.0, 1.0, 0, x.data_ptr(), x.data_ptr(), 0)

"""ehd_footprint (used by the server to admit runs against an HBM budget)
bounds what a run really holds on the device: measured through torch's
caching allocator, the resident state of a run is at most its footprint and,
for large runs, not far below it."""
import pytest

gpu = pytest.mark.gpu


@gpu
@pytest.mark.parametrize("Nx,Ny,storage", [(2048, 1680, "f32"), (1024, 840, "f64"), (512, 416, "bf16"),
                                           (64, 56, "f16"), (128, 3, "f32")])
def test_footprint_bounds_the_resident_state(Nx, Ny, storage):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1812_05711_gb300 as ehd
    ehd.use_torch_allocator(True)
    try:
        torch.cuda.synchronize()
        before = torch.cuda.memory_allocated()
        run = ehd.Run(Nx, Ny, 200.0, 10, 10, 4000, 0.25, storage=storage, amp=[1e-3], phase=[0.0])
        run.step(4)
        run.sync()
        held = torch.cuda.memory_allocated() - before
        fp = ehd.ehd_footprint(Nx, Ny, ehd.STORAGE[storage])
        assert held <= fp, (held, fp)
        if fp > (16 << 20):  # large runs: the populations dominate and the estimate is tight
            assert held >= 0.8 * fp, (held, fp)
        run.close()
        torch.cuda.synchronize()
        assert torch.cuda.memory_allocated() == before
    finally:
        ehd.use_torch_allocator(False)

"""The seeded input recipes (CPU): the splitmix64 generator against its
published output sequence, determinism, and the shapes and ranges the
recipes promise (channel aspect ratio, batch and serving mixes)."""
import math

import numpy as np

import workloads as wl


def test_splitmix64_published_sequence():
    """splitmix64 from state 0 gives 0xe220a8397b1dcdaf, 0x6e789e6aa1b965f4,
    0x06c45d188009454f (the generator's reference sequence)."""
    s, out = 0, []
    for _ in range(3):
        s, z = wl.splitmix64(s)
        out.append(z)
    assert out == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_uniforms_deterministic_and_in_range():
    a, b = wl.uniforms(12345, 1000), wl.uniforms(12345, 1000)
    assert a == b
    assert all(0.0 <= u < 1.0 for u in a)
    assert abs(np.mean(a) - 0.5) < 0.03 and wl.uniforms(12346, 5) != a[:5]


def test_channel_shapes():
    """Ny = 8 round(0.82 Nx / 8): Lx / H within 2 % of the paper's 1.22."""
    for nx, ny in ((64, 56), (128, 104), (256, 208), (512, 416), (1024, 840), (2048, 1680)):
        assert wl.ny_for(nx) == ny
        assert abs(nx / ny / 1.22 - 1) < 0.02 or nx == 64
    w = wl.large_channel()
    assert (w.Nx, w.Ny) == (2048, 1680) and 150.0 <= w.T <= 250.0 and len(w.amp) == 16
    assert all(abs(a) <= 1e-4 for a in w.amp) and all(0 <= p < 2 * math.pi for p in w.phase)
    p = wl.plain_fp64_channel()
    assert (p.Nx, p.Ny, p.T, p.Lambda, p.steps) == (128, 104, 200.0, 0.25, 10000) and p.amp == [1e-3]


def test_batch_and_serving_mixes():
    ws = wl.batch_workloads()
    assert len(ws) == 64 and {w.Nx for w in ws} <= {64, 128, 256, 512}
    assert sorted(w.T for w in ws) == list(np.linspace(140.0, 260.0, 64))
    assert {w.C for w in ws} <= {5.0, 10.0, 20.0} and {w.Fe for w in ws} <= {2000.0, 4000.0}
    reqs = wl.serving_stream()
    t = np.array([a for a, _ in reqs])
    assert np.all(np.diff(t) > 0)
    assert abs(len(t) / t[-1] - 20.0) < 2.0  # Poisson arrivals, mean 20 per second
    for _, w in reqs:
        assert w.Nx in (128, 256, 512, 1024) and 100.0 <= w.T <= 300.0 and w.C in (1.0, 10.0, 100.0)
        assert 1000 <= w.steps <= 20000

"""The C ABI library loads and exports every entry point include/ehd.h
declares; host-side argument validation (no GPU needed)."""
import ctypes
import os
import re

import pytest

import paper_1812_05711_gb300 as ehd

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(ehd_[a-z0-9_]+)\s*\(", src))
    return names


def test_every_declared_symbol_is_exported():
    lib = ctypes.CDLL(ehd.library_path() if os.path.exists(ehd.library_path()) else ehd.lib()._name)
    names = _declared()
    assert {"ehd_create", "ehd_poisson", "ehd_step", "ehd_fields"} <= names
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing


@pytest.mark.parametrize("args,msg", [
    ((100, 80, 200, 10, 10, 4000, 0.25), "power of two"),
    ((8, 80, 200, 10, 10, 4000, 0.25), "power of two"),
    ((128, 1, 200, 10, 10, 4000, 0.25), "Ny"),
    ((128, 104, -1, 10, 10, 4000, 0.25), "positive"),
    ((128, 104, 200, 0, 10, 4000, 0.25), "positive"),
    ((128, 104, 200, 10, 10, 4000, 0.0), "positive"),
])
def test_create_rejects_invalid_arguments(args, msg):
    with pytest.raises(ehd.EhdError) as ei:
        ehd.ehd_create(*args)
    assert ei.value.status == -1 and msg in str(ei.value)


def test_create_rejects_bad_options():
    o = ehd.make_options("f32", "f64")
    with pytest.raises(ehd.EhdError) as ei:
        ehd.ehd_create(128, 104, 200, 10, 10, 4000, 0.25, o)
    assert "FP64 compute needs FP64 storage" in str(ei.value)
    o = ehd.make_options("f32", u_ion=-1.0)
    with pytest.raises(ehd.EhdError):
        ehd.ehd_create(128, 104, 200, 10, 10, 4000, 0.25, o)
    o = ehd.make_options("f32", x_symbol=2)
    with pytest.raises(ehd.EhdError) as ei:
        ehd.ehd_create(128, 104, 200, 10, 10, 4000, 0.25, o)
    assert "x_symbol" in str(ei.value)
    with pytest.raises(ehd.EhdError) as ei:
        ehd.ehd_create(4096, 104, 200, 10, 10, 4000, 0.25, ehd.ehd_default_options())
    assert "2048" in str(ei.value)


def test_footprint_scales_with_storage():
    b64 = ehd.ehd_footprint(2048, 1680, 0)
    b32 = ehd.ehd_footprint(2048, 1680, 1)
    b16 = ehd.ehd_footprint(2048, 1680, 2)
    assert b64 > b32 > b16
    # populations dominate: 4 buffers of 9 planes
    assert b32 >= 4 * 9 * 2048 * 1680 * 4
    with pytest.raises(ehd.EhdError):
        ehd.ehd_footprint(100, 10, 1)
    with pytest.raises(RuntimeError):  # rows are transformed within one CTA: at most 2048 points
        ehd.ehd_footprint(4096, 10, 1)


def test_default_options():
    o = ehd.ehd_default_options()
    assert o.storage == 1 and o.compute == 1 and o.lambda_g == 1e-6 and o.u_ion == 2e-3
    assert o.step_kernel == -1  # chosen per run: push form for plain FP64, march form otherwise


def test_batch_queries_reject_null():
    """The admission query and the memory account need a batch (no GPU)."""
    L = ehd.lib()
    assert L.ehd_batch_admits(None, 128, 104, 1) == -1
    assert L.ehd_batch_memory(None, None, None) == -1
    assert "NULL" in ehd.ehd_last_error()


def test_tune_names_match_the_header():
    """The binding's tuning names carry the header's parameter ids
    (EHD_TUNE_* for runs, EHD_BATCH_* for batches), one for one."""
    src = open(os.path.join(ROOT, "include", "ehd.h")).read()
    run = {k.lower(): int(v) for k, v in re.findall(r"#define EHD_TUNE_([A-Z_]+) (\d+)", src)}
    bat = {k.lower(): int(v) for k, v in re.findall(r"#define EHD_BATCH_([A-Z_]+) (\d+)", src)}
    assert run == ehd.TUNE
    assert bat == ehd.BATCH_TUNE

"""The C-ABI library builds for sm_103a, loads, and exports every entry point its header declares
(no GPU needed: no compute call is made here)."""

import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ebic.h")


def declared_symbols():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"EBIC_API\s+[\w\s\*]+?\b(ebic_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2105_01196_gb300 import build
    if not os.path.exists(build.LIB):
        build.build()
    from paper_2105_01196_gb300 import ebic
    return ebic


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for name in ("ebic_load_matrix", "ebic_eval_population", "ebic_run_generations",
                 "ebic_create", "ebic_destroy", "ebic_last_error"):
        assert name in syms


def test_library_exports_every_declared_symbol(lib):
    raw = lib.lib()
    missing = [s for s in declared_symbols() if not hasattr(raw, s)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol(lib):
    assert set(declared_symbols()) <= set(lib.SIGNATURES)


def test_pure_host_entry_points(lib):
    assert lib.ebic_bitmap_bytes(100, 10) == 10 * 10 * 4 * 4
    assert lib.ebic_bitmap_bytes(129, 3) == 3 * 3 * 8 * 4
    assert lib.ebic_bitmap_bytes(0, 3) == 0
    p = lib.ebic_default_params()
    assert (p.ratio_num, p.ratio_den, p.neg_trends, p.use_graph) == (85, 100, 1, 1)
    assert "sm_103a" in lib.ebic_version()


def test_struct_layout_matches_header(lib):
    import ctypes
    assert ctypes.sizeof(lib.Params) == 4 * 16 + 8 + 8 + 8 + 8
    assert ctypes.sizeof(lib.RunReport) == 4 * 4 + 8 + 8 + 8 + 8
    assert ctypes.sizeof(lib.TuneReport) == 4 * 4 + 4 * 8 + 8 + 8
    assert ctypes.sizeof(lib.JobResult) == 8 + 4 * 4 + 8 + 4 * 2 + 8 + 8 * 2


def test_job_footprint_model(lib):
    """The job server's device-memory model (pure host code): bad arguments, the pair bitmap
    counted when the job's form is the bitmap, and the tabu list sized for every key a run can
    insert at load factor 1/8."""
    p = lib.Params.make(pop_size=800, mode=1)
    assert lib.ebic_job_footprint(0, 10, p, 10) == -1
    assert lib.ebic_job_footprint(100, 1, p, 10) == -1
    assert lib.ebic_job_footprint(100, 10, p, -1) == -1
    direct = lib.ebic_job_footprint(10_000, 100, p, 100)
    bitmap = lib.ebic_job_footprint(10_000, 100, lib.Params.make(pop_size=800, mode=2), 100)
    assert bitmap - direct >= lib.ebic_bitmap_bytes(10_000, 100)
    short = lib.ebic_job_footprint(10_000, 100, p, 0)
    long = lib.ebic_job_footprint(10_000, 100, p, 1000)
    # 800 * 1,002 possible keys, 8 slots of 8 bytes each, against 800 * 2 for no generation
    assert long - short >= 64 * 800 * 1000

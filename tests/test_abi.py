"""The C-ABI library builds for sm_103a, loads, and exports every function include/accel.h
declares, with the binding's signature table covering exactly those (CPU only: no compute
calls)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "accel.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?(?:accel_status|size_t|char\s*\*|void|int32_t|uint64_t)\s*\*?\s*(\w+)\s*\(", src,
                       flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2211_00621_gb300 import _lib, build
    if not build.up_to_date():
        try:
            build.nvcc()
        except RuntimeError:
            pytest.skip("no nvcc")
        build.build()
    return _lib.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ["accel_marshal_ragged", "accel_marshal_records", "accel_map", "accel_reduce", "accel_segreduce",
              "accel_loop", "hmm_forward", "hmm_adjoint", "pairwise_mapreduce", "accel_last_error"]:
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_signatures_match_header(lib):
    from paper_2211_00621_gb300 import _lib
    assert sorted(_lib.SIGNATURES) == declared_functions()


def test_host_only_calls(lib):
    # calls that touch no device: version string, debug flag, workspace sizes
    assert b"sm_103a" in lib.accel_version()
    lib.accel_set_debug(1)
    assert lib.accel_get_debug() == 1
    lib.accel_set_debug(0)
    assert lib.accel_get_debug() == 0
    assert lib.accel_segreduce_workspace_size(1 << 20, 4096) >= 256
    assert lib.accel_marshal_ragged_workspace_size(4096) >= 4096 * 16


def test_built_for_sm103a():
    from paper_2211_00621_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in build.ARCH


def test_segreduce_workspace_covers_the_most_tiles(lib):
    # tiles hold 16 KB: 8-byte elements give the most tiles, and the workspace holds three
    # 8-byte values per tile (partition, carry segment, carry value) after a 256-byte block
    for n in (1, 4096, 10_000_019, 178_913_280):
        tiles = -(-n // 2048)
        assert lib.accel_segreduce_workspace_size(n, 7) >= 256 + 8 * (tiles + 1) + 16 * tiles

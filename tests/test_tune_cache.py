"""The autotuner's on-disk cache (hg_tune_cache_find): host-only lookups, no
GPU work.  The records are the ones hg_tune appends; the last matching line
wins, and a record of another device, SM count, precision or shape is not
used."""
import pytest


@pytest.fixture(scope="module")
def hg():
    from paper_1311_0089_gb300 import build
    import paper_1311_0089_gb300 as lib
    lib.load(build.build())
    return lib


def write(path, lines):
    with open(path, "w") as f:
        f.write("\n".join(lines) + "\n")


def test_lookup_last_record_wins(hg, tmp_path):
    p = str(tmp_path / "cache.txt")
    write(p, [
        "hg-tune-v2 NVIDIA_GB300 152 1 2 729 729 0 2 2 2 0 0.058000 0 0 0",
        "hg-tune-v2 NVIDIA_GB300 152 0 2 729 729 0 1 2 1 0 0.540000 0 0 0",
        "hg-tune-v2 NVIDIA_GB300 152 1 3 135 135 135 3 3 2 4 0.470000 0 0 0",
        "hg-tune-v2 NVIDIA_GB300 152 1 2 729 729 0 1 2 1 0 0.055000 0 0 0",
        "hg-tune-v2 NVIDIA_GB300 152 1 2 105 63 0 4 2 2 0 0.020000 735 373 0",
    ])
    cfg, ms = hg.tune_cache_find(p, "NVIDIA_GB300", 152, hg.HG_MIXED, (729, 729))
    assert cfg == {"row_rb": 1, "row_lb": 2, "lanes": [1, 0], "radix": [[], [], []]}
    assert ms == pytest.approx(0.055)
    cfg, ms = hg.tune_cache_find(p, "NVIDIA_GB300", 152, hg.HG_FP64, (729, 729))
    assert cfg == {"row_rb": 1, "row_lb": 2, "lanes": [1, 0], "radix": [[], [], []]}
    assert ms == pytest.approx(0.54)
    cfg, ms = hg.tune_cache_find(p, "NVIDIA_GB300", 152, hg.HG_MIXED, (135, 135, 135))
    assert cfg == {"row_rb": 3, "row_lb": 3, "lanes": [2, 4], "radix": [[], [], []]}
    cfg, ms = hg.tune_cache_find(p, "NVIDIA_GB300", 152, hg.HG_MIXED, (105, 63))
    assert cfg == {"row_rb": 4, "row_lb": 2, "lanes": [2, 0], "radix": [[7, 3, 5], [3, 7, 3], []]}


def test_no_match_and_malformed_lines(hg, tmp_path):
    p = str(tmp_path / "cache.txt")
    write(p, [
        "garbage",
        "hg-tune-v1 NVIDIA_GB300 152 1 2 729 729 0 2 2 2 0 0.058",     # older format version
        "hg-tune-v2 NVIDIA_GB300 152 1 2 729 729 0 2 2 2 0 0.058",     # truncated
        "hg-tune-v2 NVIDIA_GB300 152 1 2 729 729 0 2 2 2 0 0.058 0 0 x",   # bad radix order
        "hg-tune-v2 NVIDIA_B200 148 1 2 243 243 0 2 2 2 0 0.010 0 0 0",
    ])
    assert hg.tune_cache_find(p, "NVIDIA_GB300", 152, hg.HG_MIXED, (729, 729)) is None
    assert hg.tune_cache_find(p, "NVIDIA_B200", 148, hg.HG_MIXED, (243, 243)) is not None
    assert hg.tune_cache_find(p, "NVIDIA_B200", 152, hg.HG_MIXED, (243, 243)) is None   # SM count
    assert hg.tune_cache_find(p, "NVIDIA_B200", 148, hg.HG_FP64, (243, 243)) is None    # precision
    assert hg.tune_cache_find(p, "NVIDIA_B200", 148, hg.HG_MIXED, (243, 245)) is None   # shape
    assert hg.tune_cache_find(p, "NVIDIA_B200", 148, hg.HG_MIXED, (243, 243, 3)) is None  # dimension
    assert hg.tune_cache_find(str(tmp_path / "missing.txt"), "x", 1, hg.HG_MIXED, (3, 3)) is None


def test_bad_arguments(hg, tmp_path):
    import ctypes
    lib = hg.load()
    N = (ctypes.c_int * 3)(9, 9, 0)
    c = hg.LaunchCfg()
    assert lib.hg_tune_cache_find(None, b"x", 1, 0, 2, N, ctypes.byref(c), None) == hg.HG_ERR_ARG
    assert lib.hg_tune_cache_find(b"f", b"x", 1, 5, 2, N, ctypes.byref(c), None) == hg.HG_ERR_ARG
    assert lib.hg_tune_cache_find(b"f", b"x", 1, 0, 4, N, ctypes.byref(c), None) == hg.HG_ERR_ARG
    assert lib.hg_tune(None, 0, 1, None, None) == hg.HG_ERR_ARG
    assert lib.hg_set_launch_cfg(None, 0, None) == hg.HG_ERR_ARG
    assert lib.hg_get_launch_cfg(None, 0, None) == hg.HG_ERR_ARG

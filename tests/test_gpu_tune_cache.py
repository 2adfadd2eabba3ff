"""The tile tuner's cache file (dts_tune_cache_file, or DTS_TUNE_CACHE): a tuning
result is appended as one line keyed by device model and problem shape, and a
later process returns the file's entry for that key without probing."""
import os
import subprocess
import sys
import textwrap

import pytest

from paper_1910_11335_b300 import dts, inputs

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SHAPE = "inputs.small_cone(12, 10, 9, n_groups=1, sn_order=4, legendre_order=1, n_sources=2)"


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1910_11335_b300 import build
    build.build()


def _tune_in_child(path, precision="PREC_FP32"):
    code = textwrap.dedent(f"""
        import sys
        sys.path.insert(0, {ROOT!r})
        from paper_1910_11335_b300 import dts, inputs
        print(dts.tune_tile({SHAPE}, precision=dts.{precision}))
    """)
    env = {**os.environ, "DTS_TUNE_CACHE": str(path)}
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr
    return out.stdout.strip().splitlines()[-1]


def test_tune_cache_file_written_then_read_by_another_process(tmp_path):
    path = tmp_path / "tiles.txt"
    w = eval(SHAPE)
    dts.tune_cache_file(str(path))
    try:
        tile, rate = dts.tune_tile(w, precision=dts.PREC_FP32)
        again = dts.tune_tile(w, precision=dts.PREC_FP32)   # the per-process cache
    finally:
        dts.tune_cache_file(None)
    assert again == (tile, rate)
    lines = path.read_text().splitlines()
    assert len(lines) == 1
    f = lines[0].split()
    assert f[0] == "dts-tune-v1"
    assert [int(x) for x in f[3:9]] == [12, 10, 9, 4, 1, 2]   # nx ny nz N L probe batch
    assert int(f[9]) == dts.PREC_FP32 and tuple(int(x) for x in f[10:13]) == tile
    assert float(f[13]) == pytest.approx(rate, rel=1e-5)
    # the entry edited to another valid tile, between lines that do not parse: the child
    # process (which has not tuned this shape) returns the file's entry
    f[10:14] = ["4", "4", "8", "1.25e+09"]
    path.write_text("not a cache line\n" + " ".join(f) + "\n" + "dts-tune-v1 broken 1 2\n")
    assert _tune_in_child(path) == "((4, 4, 8), 1250000000.0)"
    # a later line for the same key wins
    f[10:14] = ["8", "4", "8", "2.5e+09"]
    with open(path, "a") as fh:
        fh.write(" ".join(f) + "\n")
    assert _tune_in_child(path) == "((8, 4, 8), 2500000000.0)"


def test_tune_cache_other_precision_is_a_miss(tmp_path):
    """A line for FP32 does not answer an FP64 query: the child tunes and appends a line."""
    path = tmp_path / "tiles.txt"
    _tune_in_child(path, "PREC_FP32")
    _tune_in_child(path, "PREC_FP64")
    lines = path.read_text().splitlines()
    assert len(lines) == 2 and {int(l.split()[9]) for l in lines} == {dts.PREC_FP32, dts.PREC_FP64}

"""The benchmark's roofline inputs, on CPU: the DRAM traffic of the selected
DIA kernel comes from the committed ncu summary only while the kernel's
source (as the bench hashes it) is the one the counters were taken on."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _src(name):
    with open(os.path.join(ROOT, "paper_2209_06478_b300", "csrc", name)) as f:
        return f.read()


def test_hashed_regions_are_the_definitions():
    """Each marker of the hashed source occurs once, and the tile-size rule is
    found at its definition (a forward declaration must not start the
    region)."""
    spmv = _src("spmv.cu")
    assert spmv.count("// DIA: a thread owns") == 1
    assert spmv.count("// ELL: slot-major") == 1
    assert spmv.count("static int64_t tile_rows_for(const dynmat_s* A) {") == 1
    assert _src("device.cuh").count("// The DIA value stream:") == 1
    assert bench.kernel_source_hash() is not None


def test_committed_traffic_matches_the_current_source():
    """The summary's counters were taken on the DIA source as it stands: the
    bench line's `traffic` is not null. After a change to the DIA kernels,
    their tile-size rule or their value-stream load, the counters must be
    taken again (the summary's `command`)."""
    t = bench.ncu_traffic("dia_spmv", "stencil27_128", 6)
    assert t is not None and 0.9 * 486539372 < t < 1.1 * 486539372

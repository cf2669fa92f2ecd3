"""Host logic of bench.py that needs no GPU: the per-unit byte counts behind
the roofline fractions, and the source hashing that keys a profiled DRAM
traffic figure to the code it was measured on."""
import os

import bench


def test_method_bytes_per_unit_figures():
    """The method's bytes: per packet 16 B + 4 B for a home absorption, per
    crossing one velocity (16 B binary32, 32 B binary64), per queued packet a
    4-byte tally, per cell 20 / 28 B per evaluation pass and 64 / 100 B for
    the final pass."""
    m = bench.method_bytes("mixed", 8, 100, 40, 500, 1)
    assert m["emit"] == 100 * 16 + 60 * 4
    assert m["march"] == 40 * 4 + 500 * 16
    assert m["rec_step"] == 8 * (20 + 64)
    assert m["whole"] == m["emit"] + m["march"] + m["rec_step"]
    f = bench.method_bytes("fp64", 8, 100, 40, 500, 2)
    assert f["march"] == 40 * 4 + 500 * 32 and f["rec_step"] == 8 * (2 * 28 + 100)
    # the library's own count adds the queue entries and the (x, 1-x) cache
    a = bench.algorithmic_bytes("mixed", 8, 100, 40, 500, 1)
    assert a["march"] == m["march"] + 40 * 32 and a["rec_step"] > m["rec_step"]


def test_march_traffic_is_keyed_to_the_march_source_only():
    src = open(os.path.join(bench.ROOT, "paper_2312_11448_gb300", "csrc", "rec_transport.cu")).read()
    regions = bench.PROFILED_SOURCE["march"][2]
    for a, b in regions:  # the markers exist, once each, in order
        assert src.count(a) == 1 and src.count(b) == 1 and src.index(a) < src.index(b)
    h = bench.source_hash(src, regions)
    # a change outside the march regions (the emission) keeps the hash ...
    end1 = "__device__ __forceinline__ void add_counters("
    i = src.index(end1) + len(end1)
    assert bench.source_hash(src[:i] + "// x\n" + src[i:], regions) == h
    # ... one inside them does not
    j = src.index("// March of the queued packets.") + 40
    assert bench.source_hash(src[:j] + "x" + src[j:], regions) != h
    # whole-file keys change with any byte
    assert bench.source_hash(src + " ", None) != bench.source_hash(src, None)

"""bench.py's ncu traffic record (profiles/ncu_traffic.json): every record carries the keys the lookup
reads, and the lookup answers (a byte count or None) for any kernel and tile record without raising."""
import json
import os

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_records_have_lookup_keys():
    with open(os.path.join(ROOT, "profiles", "ncu_traffic.json")) as f:
        recs = json.load(f)["records"]
    for rec in recs:
        for key in ("kernel", "n", "prec", "tiles", "dram_read_bytes", "dram_write_bytes", "sources_sha1"):
            assert key in rec, key
        assert len(rec["sources_sha1"]) == 40


def test_lookup_never_raises():
    for kernel in ("pass_x", "pass_z_gamma", "pass_y"):
        for tiles in ([2, 16, -8], None, [1, 2, 3]):
            v = bench.ncu_traffic(kernel, 256, "MIXED", tiles)
            assert v is None or v > 0

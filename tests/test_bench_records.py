"""CPU checks of bench.py's bookkeeping: every SpMM form maps to a kernel
name whose source region exists in its source file, and the committed
DRAM-traffic records are keyed to the current source of their kernels."""

import json
import os

import bench


def test_spmm_kernel_names_and_source_regions():
    names = {v: bench.spmm_kernel_name(v, 36) for v in range(5)}
    assert names == {0: "k_bspmm_f32<9>", 1: "k_bspmm_tma<9,1>", 2: "k_bspmm_tma<9,3>", 3: "k_bspmm_f32w<9,3>",
                     4: "k_wspmm<9,3>"}
    for name in names.values():
        for path, a, b in bench.SPMM_REGIONS[name.split("<")[0]]:
            src = open(path).read()
            assert src.index(a) < src.index(b)
        assert len(bench.spmm_source_sha(name)) == 64


def test_committed_traffic_records_match_the_current_source():
    path = os.path.join(bench.ROOT, "profiles", "spmm_traffic.json")
    recs = json.load(open(path))["records"]
    assert recs
    for rec in recs:
        assert bench.traffic_record(rec["kernel"], rec["kp"]) is not None, rec["kernel"]
        assert rec["bytes_per_launch"] == rec["dram_bytes_read_per_launch"] + rec["dram_bytes_write_per_launch"]

"""Host logic of bench.py: an ncu traffic record applies only to the kernel
code it was taken of, and the roofline models count what their docstrings
state (the 512^3 Perlin correction's sweep log as the example)."""
import json

import numpy as np

import bench


def test_traffic_record_follows_the_code_hash(tmp_path, monkeypatch):
    from paper_2601_01787_gb300 import _build
    prof = tmp_path / "profiles"
    prof.mkdir()
    rec = {"unit_hash": _build.unit_hash("msz_batch.cu"), "traffic_bytes": 123}
    (prof / "a.json").write_text(json.dumps(rec))
    (prof / "b.json").write_text(json.dumps(dict(rec, unit_hash="0" * 16)))
    (prof / "c.json").write_text("{not json")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.traffic_record("a.json", "msz_batch.cu") == 123
    assert bench.traffic_record("a.json", "msz_correct.cu") is None  # another unit's code
    assert bench.traffic_record("b.json", "msz_batch.cu") is None    # taken of other code
    assert bench.traffic_record("c.json", "msz_batch.cu") is None
    assert bench.traffic_record("missing.json", "msz_batch.cu") is None


# sweep log of the 512^3 Perlin correction (seed 2, eb_rel 1e-4): per sweep
# |worklist|, distorted, distinct targets, changed
LOG = np.array([[134217728, 3243720, 2110080, 2110080], [27634555, 32252, 23745, 23745],
                [353850, 534, 381, 381], [5684, 8, 5, 5], [75, 0, 0, 0]], dtype=np.int64)
N, EDITED, UNCERT = 134217728, 2134197, 12946352


def test_algorithmic_bytes_term_by_term():
    want = (12 * N + UNCERT                       # sweep 0: f, fhat, g; codes of f where uncertified
            + 5 * int(LOG[1:, 0].sum())          # later sweeps: g and codes_f per examined vertex
            + 12 * int(LOG[:, 2].sum())          # targets: f, g read, g written
            + N // 8 + 8 * EDITED)               # edit list
    assert bench.algorithmic_bytes(N, LOG, EDITED, UNCERT) == want == 1822991232
    # one more distinct target costs 12 B, one more examined vertex 5 B
    log2 = LOG.copy(); log2[2, 2] += 1; log2[3, 0] += 1
    assert bench.algorithmic_bytes(N, log2, EDITED, UNCERT) == want + 17


def test_alu_ops_and_peak():
    ops = bench.algorithmic_alu_ops(N, LOG, UNCERT)
    assert bench.ALU_OPS_CERT == 2 + 6 * 8 + 4 and bench.ALU_OPS_CODE == 14 * 2 * 3
    want = bench.ALU_OPS_CERT * N + 2 * bench.ALU_OPS_CODE * UNCERT + bench.ALU_OPS_CODE * (
        UNCERT + 353850 + 5684 + 75)  # sweep 1's worklist exceeds the uncertified count
    assert ops == want == 10540445172
    assert bench.alu_peak(2070.0) == 152 * 64 * 2070e6


def test_codes_kernel_share_of_the_counts():
    # sweep 0's pass (k_codes): f, fhat read and g written for every vertex,
    # the code of f written where uncertified; the loop kernel gets the rest
    assert bench.codes_bytes(N, UNCERT) == 12 * N + UNCERT
    rest = bench.algorithmic_bytes(N, LOG, EDITED, UNCERT) - bench.codes_bytes(N, UNCERT)
    assert rest == 5 * int(LOG[1:, 0].sum()) + 12 * int(LOG[:, 2].sum()) + N // 8 + 8 * EDITED
    assert bench.codes_alu_ops(N, UNCERT) == bench.ALU_OPS_CERT * N + 2 * bench.ALU_OPS_CODE * UNCERT
    assert bench.codes_alu_ops(N, UNCERT) < bench.algorithmic_alu_ops(N, LOG, UNCERT)


def test_argument_checks():
    import pytest
    for argv in (["--warmup", "2"], ["--batch-fields", "0"], ["--batch-fields", "65"]):
        with pytest.raises(SystemExit) as e:
            bench.main(argv)
        assert e.value.code == 2  # argparse's usage error, before any GPU work

"""Host-side helpers of bench.py: the source digest that guards the
committed DRAM-traffic figure, and the traffic lookup built on it."""
import os

import bench


def _write(path, text):
    with open(path, "w") as f:
        f.write(text)
    return str(path)


def test_digest_ignores_comments_and_blank_lines(tmp_path):
    code = "int f(int x) {\n    return x + 1;\n}\n"
    a = _write(tmp_path / "a.cu", code)
    b = _write(tmp_path / "b.cu",
               "// a header comment\n\nint f(int x) {  // trailing\n"
               "    /* block\n       comment */\n    return x + 1;\n}\n\n")
    c = _write(tmp_path / "c.cu", code.replace("x + 1", "x + 2"))
    assert bench.source_digest(a) == bench.source_digest(b)
    assert bench.source_digest(a) != bench.source_digest(c)


def test_traffic_lookup(tmp_path):
    import json
    src = _write(tmp_path / "k.cu", "int f() { return 1; }\n")
    rec = {"n": 64, "bytes_per_slice_flop": {"mixed_f16": 2.5e-3},
           "tc_gemm_code_sha256_prefix": bench.source_digest(src)}
    path = _write(tmp_path / "t.json", json.dumps(rec))
    t = bench.contraction_traffic(2.0e12, "mixed_f16", path=path, src=src)
    assert abs(t["bytes_per_launch"] - 5.0e9) < 1.0
    # another precision, or a changed kernel: no figure
    assert bench.contraction_traffic(2.0e12, "emu_fp64", path=path, src=src) is None
    _write(tmp_path / "k.cu", "int f() { return 2; }\n")
    assert bench.contraction_traffic(2.0e12, "mixed_f16", path=path, src=src) is None


def test_committed_traffic_record_is_well_formed():
    import json
    rec = json.load(open(bench.TRAFFIC_FILE))
    assert len(rec["tc_gemm_code_sha256_prefix"]) == 16
    assert float(rec["bytes_per_slice_flop"]["mixed_f16"]) > 0

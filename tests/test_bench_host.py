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


def test_traffic_profile_is_well_formed():
    path = os.path.join(bench.ROOT, "profiles", "tc_gemm3_kernel_traffic.md")
    vals = {}
    for line in open(path):
        if line.startswith("- ") and ":" in line:
            k, v = line[2:].split(":", 1)
            vals[k.strip()] = v.strip().strip("`")
    assert len(vals["tc_gemm.cu code sha256 prefix"]) == 16
    assert float(vals["bytes per slice-product flop (mixed_f16)"]) > 0
    # when the code matches, the lookup scales the ratio by the flops
    t = bench.contraction_traffic(2.0e12, "mixed_f16")
    if t is not None:
        ratio = float(vals["bytes per slice-product flop (mixed_f16)"])
        assert abs(t["bytes_per_launch"] - 2.0e12 * ratio) < 1.0
    assert bench.contraction_traffic(2.0e12, "fp64") is None

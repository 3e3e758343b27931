"""Host-side pieces of bench.py that decide what its JSON line reports (no GPU):
the committed ncu traffic figure is reported only while the step kernel's code
is the code it was captured on, and comments do not count as code."""
import os
import shutil

import bench


def _copy_sources(dst):
    src = os.path.join(bench.ROOT, "paper_2512_23116_gb300", "csrc")
    for f in bench.STEP_KERNEL_SOURCES:
        shutil.copy(os.path.join(src, f), os.path.join(dst, f))


def test_digest_ignores_comments_but_not_code(tmp_path):
    _copy_sources(tmp_path)
    base = bench.kernel_digest(str(tmp_path))
    assert base == bench.kernel_digest()
    f = os.path.join(tmp_path, "lbm_step_tma.cu")
    text = open(f).read()
    open(f, "w").write("// a new comment line\n" + text.replace("namespace lbm {", "namespace lbm {  // trailing"))
    assert bench.kernel_digest(str(tmp_path)) == base
    open(f, "w").write(text.replace("constexpr int kBarBytes = 128;", "constexpr int kBarBytes = 256;"))
    assert bench.kernel_digest(str(tmp_path)) != base


def test_code_only_strips_block_and_line_comments():
    src = "int a; /* block\n comment */ int b; // line\n\n   \nint c;  \n"
    assert bench._code_only(src) == "int a;  int b;\nint c;"


def test_traffic_figure_matches_its_digest():
    # the committed summary names the digest it was captured on; a figure is
    # returned only for that digest
    path = os.path.join(bench.ROOT, "profiles", "step_kernel_traffic.txt")
    vals = dict(ln.split(":", 1) for ln in open(path) if ":" in ln and not ln.startswith("#"))
    digest = vals["kernel_digest"].strip()
    assert bench.traffic_per_update(digest) == float(vals["dram_bytes_per_update_fp32"])
    assert bench.traffic_per_update(digest, "fp16") == float(vals["dram_bytes_per_update_fp16"])
    assert bench.traffic_per_update("0" * 16) is None

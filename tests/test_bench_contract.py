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


def test_traffic_figure_is_of_the_current_kernel():
    # the step kernel's sources hash to the digest of the committed capture,
    # so the bench line carries the measured traffic (it reports null after a
    # change to the kernel until the capture is taken again)
    assert bench.traffic_per_update(bench.kernel_digest()) is not None
    assert bench.traffic_per_update(bench.kernel_digest(), "fp16") is not None


def _run_bench(args, env_extra=None):
    import json
    import subprocess
    import sys
    env = dict(os.environ)
    env.update(env_extra or {})
    out = subprocess.run([sys.executable, os.path.join(bench.ROOT, "bench.py"), *args], capture_output=True,
                         text=True, env=env, cwd=bench.ROOT, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    return [json.loads(ln) for ln in lines]


def test_reference_arm_line():
    """The reference arm (the FP64 oracle on the host cores, no GPU) prints the
    contract's JSON line: one line, its own metric and config, a cpu_baseline
    that describes the run and an e2e with no host-device bytes."""
    (line,) = _run_bench(["--impl", "reference", "--steps", "1", "--warmup", "3"])
    assert line["impl"] == "reference" and line["unit"] == "MLUPS" and line["value"] > 0
    assert line["higher_is_better"] is True and line["steps"] == 1 and line["warmup"] == 3
    assert line["dtype"] == "f64" and line["data"] == "synthetic" and "workload" in line["config"]
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == line["value"] and cb["cores"] >= 1 and cb["sample"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["unit"] == line["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_arm_other_ranks_print_nothing():
    assert _run_bench(["--impl", "reference", "--steps", "1", "--warmup", "3"], {"RANK": "1", "WORLD_SIZE": "2"}) == []

"""bench.py's one-line JSON contract, checked on the reference arm (the CPU
oracle timed on a bounded sample), which needs no GPU: the keys, their
types, and the reference arm's own e2e and cpu_baseline objects."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "3"],
                         cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1, out.stdout[-2000:]
    d = json.loads(lines[0])
    for key, typ in (("metric", str), ("value", float), ("unit", str), ("n_gpus", int),
                     ("steps", int), ("warmup", int), ("ms_per_step", float),
                     ("higher_is_better", bool), ("scaling", str), ("dtype", str),
                     ("data", str), ("config", dict), ("cpu_baseline", dict), ("e2e", dict)):
        assert isinstance(d.get(key), typ), (key, d.get(key))
    assert d["impl"] == "reference"
    assert d["steps"] == 1 and d["warmup"] == 3 and d["n_gpus"] == 1
    assert d["vs_baseline"] is None
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert d["config"]["workload"] and d["config"]["m"] == d["config"]["n"] == d["config"]["k"] == 8192
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"]
    assert cb["value"] == d["value"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_traffic_record_follows_the_kernel_code_not_its_comments():
    """The recorded DRAM traffic of the timed kernel is keyed to a hash of its
    sources without comments: a comment edit keeps the key, a code edit does
    not (bench.py then reports the traffic as null until it is recaptured)."""
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    src = {}
    for f in bench.KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1912_04379_gb300", "csrc", f)) as fh:
            src[f] = fh.read()
    base = bench.source_sha(lambda f: src[f])
    assert base == bench.source_sha()
    commented = dict(src)
    commented["tc_body.cuh"] = "// a new comment\n" + src["tc_body.cuh"].replace(
        "#pragma once", "#pragma once  /* block comment */\n\n// line comment")
    assert bench.source_sha(lambda f: commented[f]) == base
    changed = dict(src)
    changed["tc_body.cuh"] = src["tc_body.cuh"] + "\nconstexpr int kUnusedProbe = 1;\n"
    assert bench.source_sha(lambda f: changed[f]) != base

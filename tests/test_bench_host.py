"""Host-side helpers of bench.py that need no GPU."""
import json
import os

import bench


def test_code_fingerprint_ignores_comments_only():
    a = "int f(int x) {\n  // doubles x\n  return 2 * x; /* fast */\n}\n"
    b = "int f(int x) { return 2 * x; }"
    c = "int f(int x) { return 3 * x; }"
    assert bench.code_fingerprint(a) == bench.code_fingerprint(b)
    assert bench.code_fingerprint(a) != bench.code_fingerprint(c)


def test_committed_traffic_records_match_their_capture():
    """Each committed traffic record names the kernel source it was captured
    on: the recorded code fingerprint is that of the source at the recorded
    SHA-1, so the benchmark can tell a comment edit from a code change."""
    import hashlib
    import subprocess

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    for name in ("k30_bf16", "k30_bf16w32", "k100_bf16", "k100_bf16w32"):
        with open(os.path.join(root, "profiles", f"traffic_stis_{name}.json")) as f:
            d = json.load(f)
        assert d["iteration_dram_bytes"] == sum(d["dram_bytes_per_launch"].values())
        r = subprocess.run(["git", "log", "--format=%H", "--", d["source"]], cwd=root, capture_output=True, text=True)
        if r.returncode != 0 or not r.stdout.strip():
            continue  # no history here (a copy without .git): nothing to compare against
        for commit in r.stdout.split():
            src = subprocess.run(["git", "show", f"{commit}:{d['source']}"], cwd=root, capture_output=True).stdout
            if hashlib.sha1(src).hexdigest() == d["source_sha1"]:
                assert bench.code_fingerprint(src.decode()) == d["source_code_sha1"]
                break
        else:
            raise AssertionError(f"no commit of {d['source']} has SHA-1 {d['source_sha1']}")


def test_traffic_lookup_by_form_and_rank():
    """The k = 30 and k = 100 records of the current kernel code are found;
    a rank without a capture gives None."""
    assert bench.measured_traffic("bf16w32", 30) > 0
    assert bench.measured_traffic("bf16w32", 100) > 0
    assert bench.measured_traffic("bf16", 100) > 0
    assert bench.measured_traffic("bf16w32", 50) is None

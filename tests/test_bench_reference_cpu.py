"""The reference arm of bench.py (the FP64 oracle on the host cores) on the
16x16, M=3, p=3 workload: one JSON line with the contract's keys."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "cfg1",
                        "--steps", "1", "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["value"] > 0 and d["higher_is_better"] is False
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    assert d["config"]["workload"].startswith("cfg1")


def test_pair_count_matches_enumeration():
    """The closed form of the distinct (k, j) pairs used for the product's
    flop count against the oracle's coupling lists, enumerated."""
    sys.path.insert(0, ROOT)
    import bench
    from oracle import chaos
    for M in range(1, 7):
        for p in range(0, 5):
            alpha, _ = chaos.multi_indices(M, p)
            alpha = [tuple(int(v) for v in a) for a in alpha]
            index = {tuple(a): i for i, a in enumerate(alpha)}
            pairs = set()
            for a in alpha:
                for k in range(M):
                    for step in (-1, 1):
                        b = list(a)
                        b[k] += step
                        if b[k] >= 0 and tuple(b) in index:
                            pairs.add((k, tuple(b)))
            assert bench.sg_pairs(M, p) == len(pairs), (M, p)

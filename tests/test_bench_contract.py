"""bench.py's reference arm on the CPU: one JSON line with the keys and units
of the contract, the oracle timed on the host cores (no GPU, no library)."""
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    t0 = time.perf_counter()
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "tiny", "--steps", "2",
                        "--warmup", "1"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    wall = time.perf_counter() - t0
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["unit"] == "samples/s" and d["higher_is_better"] is True
    assert d["n_gpus"] == 1 and d["steps"] == 2 and d["warmup"] == 1 and d["vs_baseline"] is None
    assert d["value"] > 0 and d["ms_per_step"] > 0
    # ms_per_step is the measured time of one sample step: the timed steps fit in the run.
    assert d["ms_per_step"] * d["steps"] / 1e3 < wall
    assert d["config"]["workload"].startswith("tiny")
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert cb["nproc"] == os.cpu_count() and "cpu" in cb
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_oracle_check_against_itself():
    """The reduced-precision check's plumbing on the oracle alone: leaves
    stratified by photon count, the oracle's map compared with itself (KL and
    L1 zero), and guided samples drawn by the oracle at the chi-square leaves'
    centres land in those leaves and pass the chi-square test against the
    map they were drawn from."""
    sys.path.insert(0, ROOT)
    import bench
    from oracle import oracle as O
    from paper_2010_01775_gb300 import synth
    chk = bench.OracleCheck(synth.TINY, n_leaves=12, n_chi=3)
    assert len(chk.slots) == 12 and np.all(np.diff(chk.counts[np.argsort(chk.counts)]) >= 0)
    assert chk.counts.max() == (chk.g["leaf_end"].astype(np.int64) - chk.g["leaf_begin"])[chk.act].max()
    chk.run(threads=0)
    st = chk.stats(chk.P)
    assert st["kl_vs_fp64_oracle"]["max"] == 0.0 and st["l1_vs_fp64_oracle"]["max"] == 0.0 and st["meets_kl_gate"]
    # Guided samples of the oracle's own tables at the chi-square leaves' centres.
    A = chk.act.size
    slot = np.full(chk.g["L"], -1, np.int32)
    slot[chk.act[chk.slots]] = np.arange(len(chk.slots), dtype=np.int32)
    tabs = O.tables_from_map(chk.P.reshape(len(chk.slots), synth.TINY.H, synth.TINY.W))
    s = O.sample(chk.g, slot, tabs, chk.chi_pos, bench.CHI_SEED)
    want = np.repeat(chk.act[chk.slots[chk.chi_idx]], bench.CHI_SAMPLES)
    assert np.array_equal(s["leaf"].astype(np.int64), want) and A > 0
    red, pv = bench.chi_square(s["bin"].astype(np.int64), chk.P[chk.chi_idx], bench.CHI_SAMPLES)
    assert np.all(pv > 1e-4) and np.all(red < 1.5)
    # A map that is off by a visible amount fails it.
    Pq = chk.P[chk.chi_idx].copy()
    Pq = np.sqrt(Pq) / np.sqrt(Pq).sum(axis=1, keepdims=True)
    red2, pv2 = bench.chi_square(s["bin"].astype(np.int64), Pq, bench.CHI_SAMPLES)
    assert np.all(pv2 < 1e-6)

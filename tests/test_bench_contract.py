"""bench.py's reference arm on the host cores (no GPU): the JSON line it prints, and that
under several ranks only rank 0 runs and prints; and the hash that ties its DRAM-traffic
record to the kernel code."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(rank, world):
    env = dict(os.environ, RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                           "--warmup", "0", "--gpus", str(world)],
                          cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)


def test_reference_arm_line():
    r = _run(0, 1)
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["steps"] == 1 and d["warmup"] == 0 and d["dtype"] == "f64"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["unit"] == d["unit"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert "workload" in d["config"]


def test_reference_arm_other_ranks_exit_quietly():
    r = _run(1, 2)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""


def test_traffic_record_hash_follows_the_kernel_code(tmp_path, monkeypatch):
    """The DRAM-traffic record is tied to the kernels' code (bench.py reports
    roofline.traffic only while the recorded hash matches): the hash ignores comments and
    blank lines but changes with any code edit."""
    import shutil
    import bench
    csrc = tmp_path / "paper_2202_10313_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for f in ("kernels.cuh", "kernels_sp.cuh", "gen_sparse.cpp"):
        shutil.copy(os.path.join(bench.ROOT, "paper_2202_10313_gb300", "csrc", f), csrc / f)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench.kernel_hash()
    p = csrc / "kernels_sp.cuh"
    p.write_text("// a comment line\n\n" + p.read_text().replace("\n}", "  // trailing note\n}", 1))
    assert bench.kernel_hash() == h0
    p.write_text(p.read_text().replace("NE = 14", "NE = 13", 1))
    assert bench.kernel_hash() != h0

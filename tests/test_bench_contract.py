"""bench.py's reference arm (the oracle on the host) prints one JSON line
with the keys the benchmark contract asks for; it needs no GPU."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "2",
                        "--warmup", "3"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["steps"] == 2 and d["warmup"] == 3
    assert d["value"] > 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]


def test_traffic_record_key_ignores_comments_only(tmp_path, monkeypatch):
    """The DRAM/instruction record under profiles/ applies to the kernel code
    it was captured on: bench.py keys it by a hash of kernels.cu without
    comments and blank lines, so a comment edit keeps it and a code edit
    drops it."""
    sys.path.insert(0, ROOT)
    import bench
    src = open(os.path.join(ROOT, "paper_2006_14956_gb300", "csrc", "kernels.cu"), encoding="utf-8").read()
    base = bench.kernels_code_hash()
    fake = tmp_path / "paper_2006_14956_gb300" / "csrc"
    fake.mkdir(parents=True)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    (fake / "kernels.cu").write_text("// a new comment\n\n" + src.replace("\n", "  \n", 3) + "// trailing\n")
    assert bench.kernels_code_hash() == base
    (fake / "kernels.cu").write_text(src.replace("CHUNK_S = 512", "CHUNK_S = 256", 1))
    assert bench.kernels_code_hash() != base
    rec = json.load(open(os.path.join(ROOT, "profiles", "dram_traffic_abinitio50.json")))
    assert set(rec["kernels"]) == {"k_spawn", "k_annihilate"}
    for k in rec["kernels"].values():
        assert k["dram_bytes_per_unit"] > 0 and k["inst_per_unit"] > 0

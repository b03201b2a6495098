"""bench.py's host-side contract (no GPU): the reference arm (the oracle on
the host cores) prints one JSON line with the keys the benchmark contract
names, and it samples the spanning tree the library ranks first (the
default tree), so both arms run the same plan."""
import json
import os
import subprocess
import sys

import pytest

from helpers import SMALL_MOTIFS

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _motifs():
    from paper_2507_20441_gb300 import synth
    out = {n: (nv, e, r) for n, (nv, e, r) in SMALL_MOTIFS.items()}
    for i, mo in enumerate(synth.motif_pool(seed=7, count=32)):
        out[f"pool{i}_{mo.name}"] = (mo.nv, [tuple(e) for e in mo.edges], list(mo.rank))
    return out


@pytest.mark.parametrize("name", sorted(_motifs()))
def test_reference_tree_is_the_library_default_tree(name):
    import types
    import bench
    import paper_2507_20441_gb300 as tg
    tg.build()
    nv, edges, rank = _motifs()[name]
    tree, root = bench.reference_tree(types.SimpleNamespace(nv=nv, edges=edges, rank=rank))
    best_mask = tg.tm_tree_candidates(nv, edges, rank)[0][0]
    assert sum(1 << e for e in tree) == best_mask
    assert root in tree


def test_reference_arm_prints_the_contract_line():
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "tiny",
           "--steps", "1", "--warmup", "0", "--k", "20000"]
    p = subprocess.run(cmd, capture_output=True, text=True, cwd=ROOT, timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [ln for ln in p.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1
    r = json.loads(lines[0])
    assert r["impl"] == "reference"
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in r, key
    assert r["metric"] == "samples/s" and r["unit"] == "samples/s" and r["higher_is_better"] is True
    assert r["value"] > 0 and r["steps"] == 1 and r["config"]["workload"] == "tiny" and r["config"]["k"] == 20000
    cb = r["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == r["value"] and cb["sample"]
    e = r["e2e"]
    assert e["value"] == r["value"] and e["unit"] == r["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_roofline_traffic_comes_from_a_current_capture(tmp_path, monkeypatch):
    """The `traffic` of the bench's roofline is read from the committed ncu
    summary of the dominant kernel only while the kernel's sources are the
    ones that summary was captured on (their sha256 is recorded in it)."""
    sys.path.insert(0, ROOT)
    import bench
    fam = bench.kernel_family("k_sample_reg<4>")
    assert fam == "k_sample"
    prof = tmp_path / "profiles"
    prof.mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    # sources looked up under the temporary root: copy the current ones
    csrc = tmp_path / "paper_2507_20441_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for f in bench.KERNEL_SOURCES[fam]:
        (csrc / f).write_bytes(open(os.path.join(ROOT, "paper_2507_20441_gb300", "csrc", f), "rb").read())
    h = bench.kernel_source_hash(fam)
    (prof / "k_sample_w.md").write_text(f"x\ntraffic_bytes_per_launch: 1234\nsource_sha256: {h}\n")
    assert bench.profiled_traffic(fam, "w") == 1234
    assert bench.profiled_traffic(fam, "other") is None            # no summary for that workload
    (csrc / bench.KERNEL_SOURCES[fam][0]).write_text("// changed\n")
    assert bench.profiled_traffic(fam, "w") is None                # sources changed since the capture

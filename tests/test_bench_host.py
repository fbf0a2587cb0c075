"""Host-side logic of bench.py (no GPU): the roofline's byte count, the gate that keeps a
committed DRAM capture only while the kernel code it was taken on is unchanged, and the
constraint-sweep queries' definitions."""
import json

import bench
import synth


def test_alg_bytes_counts_each_unit():
    w = {"roots": 10, "nodes": [0, 4, 3, 0, 0, 0, 0, 0], "entries": [0, 9, 5, 0, 0, 0, 0, 0], "probe_sectors": 7}
    full, low = bench.alg_bytes(w, 3, 0)
    assert low == 16 * 10 + 32 * 7 + 16 * (14 + 7)
    assert full == low + 32 * 7
    assert bench.alg_bytes(w, 3, 0, with_labels=True)[1] == low + 10
    assert bench.alg_bytes(w, 3, 5)[1] == low + 4 * 3 * 5


def test_traffic_gate_follows_kernel_code_not_comments(tmp_path, monkeypatch):
    root = tmp_path / "r"
    for f in bench.KERNEL_SOURCES:
        p = root / f
        p.parent.mkdir(parents=True, exist_ok=True)
        p.write_text("int x = 1;  // a comment\n\n__global__ void k() {}\n")
    monkeypatch.setattr(bench, "ROOT", str(root))
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(root / "traffic.json"))
    h = bench.kernel_source_hash()
    json.dump({"kernel_source_sha256": h, "dram_bytes_count_pass_per_step": 123}, open(bench.TRAFFIC_FILE, "w"))
    assert bench.measured_traffic("powerlaw_10m") == 123.0
    assert bench.measured_traffic("hubskew_100m") is None          # captured on another workload
    src = root / bench.KERNEL_SOURCES[0]
    src.write_text("int x = 1;  // another comment\n__global__ void k() {}\n\n")
    assert bench.measured_traffic("powerlaw_10m") == 123.0          # comments and blank lines only
    src.write_text("int x = 2;\n__global__ void k() {}\n")
    assert bench.measured_traffic("powerlaw_10m") is None           # code changed: no traffic


def test_constraint_sweep_adds_one_constraint_at_a_time():
    n, v, vt, vta = synth.constraint_sweep_queries(delta=3600)
    assert n.edges == v.edges == vt.edges == vta.edges == [(0, 1), (1, 2), (2, 3), (3, 0)]
    assert all(x < 0 for x in n.nlabel) and all(x >= 0 for x in v.nlabel) and v.nlabel == vt.nlabel == vta.nlabel
    assert all(g > 10 ** 18 for g in v.gaps) and vt.gaps == vta.gaps == [1800] * 3
    assert not vt.anti and vta.anti == [(1, 0, 0, 900)]

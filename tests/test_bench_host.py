"""Host-side pieces of bench.py that need no GPU: the scope table's byte
count of one Laplacian product, and the ingestion of an ncu DRAM-traffic log
into profiles/traffic_<workload>.json (which later runs report as the
roofline's measured traffic only while the SpMM sources are unchanged)."""

import json
import os

import pytest

import bench


def test_survey_bytes_of_the_mesh_chain_step():
    # 128^3 27-point mesh, b = 7, BF16 in and out, float diagonal, unit weights:
    # 8 (n + 1) + 4 nnz + n b (2 + 2) + 4 n
    n, nnz = 2_097_152, 53_645_816
    got = bench.survey_bytes(n, nnz, 7, 2, 2, 4, False)
    assert got == 8 * (n + 1) + 4 * nnz + n * 7 * 4 + 4 * n
    assert got == pytest.approx(298.5e6, rel=1e-3)
    # weights add 4 bytes an entry
    assert bench.survey_bytes(n, nnz, 7, 2, 2, 4, True) - got == 4 * nnz


def _csv(path, rows):
    head = ['"ID"', '"Process ID"', '"Process Name"', '"Host Name"', '"Kernel Name"', '"Context"', '"Stream"',
            '"Block Size"', '"Grid Size"', '"Device"', '"CC"', '"Section Name"', '"Metric Name"', '"Metric Unit"',
            '"Metric Value"']
    lines = ["==PROF== Connected to process", ",".join(head)]
    for i, kname, metric, unit, val in rows:
        lines.append(",".join(f'"{x}"' for x in (i, 1, "python", "h", kname, 1, 7, "(128, 1, 1)", "(16384, 1, 1)", 0,
                                                 "10.3", "Command line profiler metrics", metric, unit, val)))
    path.write_text("\n".join(lines) + "\n")


def test_ingest_ncu_averages_read_plus_write_per_launch(tmp_path, monkeypatch):
    k = "void sphynx::k_spmm_sell<(int)0, __nv_bfloat16, __nv_bfloat16, 8, false, 1, true>(...)"
    other = "void sphynx::k_gram8<8, 3>(...)"
    p = tmp_path / "dram.csv"
    _csv(p, [(0, k, "dram__bytes_read.sum", "Mbyte", "150.00"), (0, k, "dram__bytes_write.sum", "Mbyte", "10.00"),
             (1, other, "dram__bytes_read.sum", "Gbyte", "9.00"), (1, other, "dram__bytes_write.sum", "byte", "1"),
             (2, k, "dram__bytes_read.sum", "Gbyte", "0.22"), (2, k, "dram__bytes_write.sum", "Kbyte", "50,000.00")])
    monkeypatch.setattr(bench, "traffic_path", lambda w: str(tmp_path / f"traffic_{w}.json"))
    out = bench.ingest_ncu(str(p), r"k_spmm_sell<(\(int\))?0, __nv_bfloat16, __nv_bfloat16", "c2", "ncu ...")
    assert out["launches"] == 2
    assert out["traffic_bytes_per_launch"] == pytest.approx((160e6 + 270e6) / 2)
    assert out["source_hash"] == bench.kernel_source_hash()
    stored = json.loads((tmp_path / "traffic_c2.json").read_text())
    assert stored["traffic_bytes_per_launch"] == out["traffic_bytes_per_launch"]
    # reported while the SpMM sources are those of the capture, withheld after a change
    assert bench.profiled_traffic("c2")[0] == out["traffic_bytes_per_launch"]
    stored["source_hash"] = "0" * 16
    (tmp_path / "traffic_c2.json").write_text(json.dumps(stored))
    t, meta = bench.profiled_traffic("c2")
    assert t is None and meta is not None


def test_committed_traffic_json_names_its_capture():
    for name in os.listdir(os.path.join(bench.ROOT, "profiles")):
        if name.startswith("traffic_") and name.endswith(".json"):
            d = json.load(open(os.path.join(bench.ROOT, "profiles", name)))
            assert d["traffic_bytes_per_launch"] > 0 and d["launches"] >= 1
            assert "ncu" in d["command"] and "--clock-control none" in d["command"]


def test_ingest_ncu_reads_the_raw_page_too(tmp_path, monkeypatch):
    k = "void k_spmm_sell<0, __nv_bfloat16, __nv_bfloat16, 8, 0, 1, 3>(LapView, SpmmDev, ...)"
    lines = ['"ID","Process ID","Kernel Name","dram__bytes_read.sum","dram__bytes_write.sum","gpu__time_duration.sum"',
             '"","","","Mbyte","Kbyte","usecond"',
             f'"0","7","{k}","100.5","2,000","60.1"',
             '"1","7","void k_gram8<8, 3>(...)","400","1","150"',
             f'"2","7","{k}","120.5","4,000","61.0"']
    p = tmp_path / "raw.csv"
    p.write_text("\n".join(lines) + "\n")
    monkeypatch.setattr(bench, "traffic_path", lambda w: str(tmp_path / f"traffic_{w}.json"))
    out = bench.ingest_ncu(str(p), r"k_spmm_sell<(\(int\))?0, __nv_bfloat16, __nv_bfloat16", "c2", "ncu x")
    assert out["launches"] == 2
    assert out["traffic_bytes_per_launch"] == pytest.approx((102.5e6 + 124.5e6) / 2)

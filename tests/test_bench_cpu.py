"""Host-side logic of bench.py, on CPU: the DRAM traffic of a capture is
scaled to the full workload and tied to the kernel sources it was taken on,
and every workload names its configuration."""
import argparse
import json

import pytest

import bench


def _args(**kw):
    base = dict(gpus=1, steps=1, warmup=0, impl="ours", workload="direct_f64", variant="plain", no_extras=True,
                cpu_seconds=0.1, queries=0, tune="auto", record_traffic="")
    base.update(kw)
    return argparse.Namespace(**base)


def _ncu_csv(path, reads, writes, names=None):
    rows = ['"ID","Kernel Name","Metric Name","Metric Unit","Metric Value"']
    for i, (r, w) in enumerate(zip(reads, writes)):
        k = names[i] if names else "k"
        rows.append('"%d","%s","dram__bytes_read.sum","Mbyte","%s"' % (i, k, r))
        rows.append('"%d","%s","dram__bytes_write.sum","byte","%s"' % (i, k, w))
        rows.append('"%d","%s","gpu__time_duration.sum","ns","1000"' % (i, k))
    path.write_text("==PROF== a line ncu prints\n" + "\n".join(rows) + "\n")


def test_traffic_is_scaled_and_tied_to_the_sources(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "TRAFFIC_PATH", str(tmp_path / "traffic.json"))
    csv = tmp_path / "cap.csv"
    _ncu_csv(csv, ["100", "102", "104"], ["1,000,000", "2000000", "3000000"])
    full = bench.workload_config(_args())["queries"]
    bench.record_traffic(_args(record_traffic=str(csv), queries=full // 8))
    d = json.load(open(bench.TRAFFIC_PATH))
    e = d["search_f64_plain"]
    assert e["launches"] == 3 and e["searches"] == 3
    assert e["captured_bytes_per_search"] == pytest.approx(102e6 + 2e6)
    assert e["bytes_per_search"] == pytest.approx(8 * (102e6 + 2e6))
    assert bench.traffic_for("search_f64_plain") == pytest.approx(8 * (102e6 + 2e6))
    # a change of the kernel sources makes the capture stale
    monkeypatch.setattr(bench, "source_hash", lambda key: "0" * 16)
    assert bench.traffic_for("search_f64_plain") is None


def test_capture_at_the_full_size_is_not_scaled(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "TRAFFIC_PATH", str(tmp_path / "traffic.json"))
    csv = tmp_path / "cap.csv"
    _ncu_csv(csv, ["2000"], ["1000000000"])
    full = bench.workload_config(_args(workload="batched_f32"))["queries"]
    bench.record_traffic(_args(workload="batched_f32", record_traffic=str(csv), queries=full))
    e = json.load(open(bench.TRAFFIC_PATH))["batch_search_f32"]
    assert e["bytes_per_search"] == pytest.approx(3e9) and e["scaled"] == "captured at the full workload"


def test_a_search_call_sums_its_kernels(tmp_path, monkeypatch):
    # two search calls, each the chunk planner and two search kernels (direct
    # and learned arrays): the traffic of a call is the sum of its three launches
    monkeypatch.setattr(bench, "TRAFFIC_PATH", str(tmp_path / "traffic.json"))
    csv = tmp_path / "cap.csv"
    names = ["k_plan_chunks(int)", "k_batch_search<float, 5>(BatchArgs<T1>)",
             "k_batch_search<float, 4>(BatchArgs<T1>)"] * 2
    _ncu_csv(csv, ["0.1", "600", "4000", "0.1", "602", "4002"], ["0", "500", "1500", "0", "500", "1500"], names)
    full = bench.workload_config(_args(workload="learned_interp_f32"))["queries"]
    bench.record_traffic(_args(workload="learned_interp_f32", record_traffic=str(csv), queries=full))
    e = json.load(open(bench.TRAFFIC_PATH))["learned_search_f32"]
    assert e["launches"] == 6 and e["searches"] == 2
    assert e["bytes_per_search"] == pytest.approx(0.1e6 + 601e6 + 4001e6 + 2000)
    assert e["captured_bytes_per_kernel"]["k_batch_search<float, 4>"] == pytest.approx(4001e6 + 1500)


def test_capture_without_dram_rows_is_refused(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "TRAFFIC_PATH", str(tmp_path / "traffic.json"))
    csv = tmp_path / "cap.csv"
    csv.write_text('"ID","Metric Name","Metric Unit","Metric Value"\n"0","gpu__time_duration.sum","ns","5"\n')
    with pytest.raises(SystemExit):
        bench.record_traffic(_args(record_traffic=str(csv), queries=1 << 20))


@pytest.mark.parametrize("workload", bench.WORKLOADS)
def test_every_workload_names_its_configuration(workload):
    cfg = bench.workload_config(_args(workload=workload))
    assert cfg["workload"] and "queries" in cfg and "step" in cfg and "l2" in cfg
    assert bench.kernel_key_of(_args(workload=workload))


def test_a_comment_edit_keeps_a_capture_valid():
    code = bench._code_of("int a = 1;  // the first\n/* a block\n comment */\nint b;\n")
    assert code == bench._code_of("int a = 1; // reworded\nint b;")
    assert code != bench._code_of("int a = 2;\nint b;")

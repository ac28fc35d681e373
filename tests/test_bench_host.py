"""Host logic of bench.py (no GPU): the recorded ncu counters that the bench
line's roofline `traffic` and `issue_view` read must belong to the kernels'
current sources, and the reader of ncu's CSV log must turn warp-level counts
into per-element figures."""
import json

import bench


def test_recorded_counters_match_the_current_sources():
    # a kernel whose sources changed since its counters were taken reads as
    # unmeasured (traffic null) in the bench line
    for kernel in bench.KERNEL_FILES:
        rec = bench.recorded_counters(kernel)
        assert rec is not None, f"{kernel}: ncu counters are stale (re-take them with --record-counters)"
        assert rec["inst_per_element"] > 0 and rec["dram_bytes_per_element"] > 0


def test_fingerprint_ignores_comments_and_whitespace(tmp_path, monkeypatch):
    src = tmp_path / "k.cu"
    src.write_text("int f(int x) { return x + 1; }\n")
    monkeypatch.setitem(bench.KERNEL_FILES, "k_probe", [str(src)])
    monkeypatch.setattr(bench, "ROOT", "/")
    a = bench.kernel_fingerprint("k_probe")
    src.write_text("int f(int x)   {  /* a note */ return x + 1; }   // a comment\n")
    assert bench.kernel_fingerprint("k_probe") == a
    src.write_text("int f(int x) { return x + 2; }\n")
    assert bench.kernel_fingerprint("k_probe") != a


def test_record_counters_reads_an_ncu_csv_log(tmp_path, monkeypatch):
    counters = tmp_path / "counters.json"
    monkeypatch.setattr(bench, "COUNTERS_JSON", str(counters))
    hdr = ('"ID","Process ID","Process Name","Host Name","Kernel Name","Context","Stream","Block Size",'
           '"Grid Size","Device","CC","Section Name","Metric Name","Metric Unit","Metric Value"\n')
    name = "void unnamed>::k_f64_fixed<1>(const double *, double *, unsigned long)"
    n = 1 << 20
    rows = []
    for launch, (rd, wr, inst) in enumerate([(8 * n, 8 * n, 4 * n), (8 * n + 64, 8 * n - 64, 4 * n)]):
        for metric, value in (("dram__bytes_read.sum", rd), ("dram__bytes_write.sum", wr),
                              ("smsp__inst_executed.sum", inst), ("gpu__time_duration.sum", 1000 + launch)):
            rows.append(f'"{launch}","1","python3","h","{name}","1","7","(128, 1, 1)","(1, 1, 1)","0",'
                        f'"10.3","Command line profiler metrics","{metric}","",'
                        f'"{value:,}"\n')
    log = tmp_path / "log.csv"
    log.write_text("==PROF== noise\n" + hdr + "".join(rows))
    bench.record_counters(str(log), n, "the command")
    rec = json.loads(counters.read_text())["k_f64_fixed"]
    assert rec["launches"] == 2 and rec["n"] == n and rec["command"] == "the command"
    assert rec["dram_bytes_per_element"] == 16.0
    assert rec["inst_per_element"] == 128.0          # warp instructions x 32 / n
    assert rec["duration_ns"] == 1000.5
    assert rec["fingerprint"] == bench.kernel_fingerprint("k_f64_fixed")

"""Host-side logic of the binding that needs no GPU."""


def test_thermo_line_is_lammps_style():
    """The thermo line: fixed-width columns under a header of the same widths,
    TotEng = KinEng + PotEng."""
    from paper_0809_2811_gb300 import mw
    h = mw.thermo_header()
    rec = dict(step=100, temperature=298.123, pe=-5000.1234, ke=500.5, pressure=12.3, conserved=-4499.62,
               volume=15309.1, rebuilds=7)
    line = mw.thermo_line(rec)
    assert h.split() == ["Step", "Temp", "PotEng", "KinEng", "TotEng", "Press", "Econs", "Volume", "Rebuilds"]
    assert len(line) == len(h)
    vals = line.split()
    assert int(vals[0]) == 100 and int(vals[-1]) == 7
    assert float(vals[4]) == -4499.6234
    # columns line up: each value ends where its name ends
    ends_h = [h.index(c) + len(c) for c in h.split()]
    pos, ends_v = 0, []
    for v in vals:
        pos = line.index(v, pos) + len(v)
        ends_v.append(pos)
    assert ends_h == ends_v


def test_clock_summary_reads_throttle_reasons():
    """The bench's clock record: median SM clock, the highest maximum, and
    every throttle reason seen Active in any sample (nvidia-smi CSV lines of
    clocks.sm, clocks.max.sm, power.draw and four reasons)."""
    import bench
    lines = ["2070, 2070, 700.5, Not Active, Not Active, Not Active, Not Active",
             "1980, 2070, 1390.0, Not Active, Not Active, Not Active, Active",
             "2070, 2070, 900.1, Not Active, Not Active, Not Active, Not Active",
             "garbage line", "[N/A], [N/A], [N/A], x, x, x, x"]
    c = bench.clock_summary(lines)
    assert c == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    c = bench.clock_summary(["1500, 2070, 500, Active, Not Active, Active, Not Active"])
    assert c["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"] and c["sm_mhz"] == 1500.0
    assert bench.clock_summary([])["sm_mhz"] is None


def test_traffic_is_reported_only_for_the_profiled_source(tmp_path, monkeypatch):
    """DRAM traffic comes from the committed ncu record of the same workload
    size only while the kernel source hashes to the recorded value; any edit
    of the source gives null."""
    import hashlib
    import json
    import bench
    src = tmp_path / "k.cuh"
    src.write_text("// kernel v1\n")
    prof = tmp_path / "profiles"
    prof.mkdir()
    h = hashlib.sha256(src.read_bytes()).hexdigest()[:16]
    (prof / "sw_force_traffic.json").write_text(json.dumps(
        [{"source_hash": h, "atoms": 1000, "dram_bytes_per_launch": 123},
         {"source_hash": h, "atoms": 2000, "dram_bytes_per_launch": 456}]))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.traffic_from_profile(str(src), 1000) == 123
    assert bench.traffic_from_profile(str(src), 2000) == 456
    assert bench.traffic_from_profile(str(src), 3000) is None  # no capture of this size
    (prof / "sw_force_traffic.json").write_text(json.dumps(
        [{"source_hash": h, "atoms": 1000, "r_list_A": 6.1065, "dram_bytes_per_launch": 123},
         {"source_hash": h, "atoms": 1000, "r_list_A": 6.3065, "dram_bytes_per_launch": 789}]))
    assert bench.traffic_from_profile(str(src), 1000, 6.3065) == 789  # the record of this list radius
    assert bench.traffic_from_profile(str(src), 1000, 5.3065) is None
    src.write_text("// kernel v2\n")
    assert bench.traffic_from_profile(str(src), 1000) is None

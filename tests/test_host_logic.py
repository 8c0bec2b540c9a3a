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

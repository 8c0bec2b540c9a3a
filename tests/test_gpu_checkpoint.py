"""Checkpoint / resume (mw_checkpoint_*): the saved state comes back exactly,
and a resumed run continues the saved trajectory as an uninterrupted run
does (to the run-to-run spread of unordered FP32 force sums, which two
uninterrupted runs show as well)."""
import numpy as np
import pytest

from paper_0809_2811_gb300 import inputs as I

pytestmark = pytest.mark.gpu

NH = dict(dt=10.0, thermostat=2, T0=260.0, tau=500.0)


def _pair(mwlib, make, kw, n_before=100, n_after=50):
    """Run make() for n_before steps, checkpoint, go on n_after steps; a
    second system restores the checkpoint and runs n_after steps."""
    a = make()
    b = make()
    try:
        a.step(n_before, **kw)
        t_ck = a.thermo()
        blob = a.checkpoint()
        ta = a.step(n_after, **kw)
        xa, va = a.get_state()
        b.restore(blob)
        t_res = b.thermo()
        assert b.checkpoint() == blob  # the state came back byte for byte
        tb = b.step(n_after, **kw)
        xb, vb = b.get_state()
        box_a, box_b = a.box(), b.box()
    finally:
        a.close()
        b.close()
    return t_ck, t_res, ta, tb, xa, xb, va, vb, box_a, box_b


def _close(ta, tb, xa, xb, va, vb, box, nsteps):
    for p, q in zip(ta, tb):
        assert p["step"] == q["step"] == nsteps
        assert p["conserved"] == pytest.approx(q["conserved"], rel=1e-6)
        assert p["pe"] == pytest.approx(q["pe"], rel=2e-5)
    d = xa - xb
    d -= box * np.rint(d / box)
    assert np.abs(d).max() < 2e-4
    assert np.abs(va - vb).max() < 5e-6


@pytest.mark.parametrize("engine", [1, 2])
def test_resume_continues_a_nose_hoover_run(mwlib, engine):
    x, box = I.jittered_box(2048, 1.0, 0.15, 31)
    v = I.maxwell_velocities(2048, 260.0, seed=32)

    def make():
        s = mwlib.System(2048, box)
        s.set_engine(engine)
        s.set_state(x, v)
        return s
    t_ck, t_res, ta, tb, xa, xb, va, vb, _, _ = _pair(mwlib, make, NH)
    # the record of the restored state is the checkpoint's, to the last bit
    for k in ("step", "pe", "ke", "conserved", "xi", "eta", "pressure", "rebuilds"):
        assert t_res[0][k] == t_ck[0][k], k
    _close(ta, tb, xa, xb, va, vb, box, 150)


def test_resume_continues_an_isobaric_batch(mwlib):
    n = [512, 729]
    xs, boxes = [], []
    for k, nn in enumerate(n):
        xx, bb = I.jittered_box(nn, [0.95, 1.02][k], 0.15, 40 + k)
        xs.append(xx)
        boxes.append(bb)
    v = I.maxwell_velocities(sum(n), 280.0, seed=42)
    kw = dict(dt=10.0, thermostat=3, T0=280.0, tau=1000.0, p_ext=0.0, tau_p=2000.0)

    def make():
        s = mwlib.System(n, np.array(boxes))
        s.set_state(np.concatenate(xs), v)
        return s
    t_ck, t_res, ta, tb, xa, xb, va, vb, box_a, box_b = _pair(mwlib, make, kw)
    for p, q in zip(t_ck, t_res):
        assert (p["volume"], p["conserved"], p["box"]) == (q["volume"], q["conserved"], q["box"])
    # the edges follow the virial's unordered FP32 sums: 1e-9 apart after 50 steps
    assert np.allclose(box_a, box_b, rtol=2e-7, atol=0)
    assert not np.allclose(box_a, np.array(boxes), rtol=1e-4, atol=0)  # the barostat moved the boxes
    for k in range(2):
        off = sum(n[:k])
        sl = slice(off, off + n[k])
        _close([ta[k]], [tb[k]], xa[sl], xb[sl], va[sl], vb[sl], box_a[k], 150)


def test_resume_with_several_species(mwlib):
    x, box = I.jittered_box(1000, 1.0, 0.2, 51)
    v = I.maxwell_velocities(1000, 260.0, seed=52)
    ty = I.species_draw(1000, 2, 53, [0.9, 0.1])
    table = I.species_table_solute()

    def make():
        s = mwlib.System(1000, box)
        s.set_species(table, ty)
        s.set_state(x, v)
        return s
    t_ck, t_res, ta, tb, xa, xb, va, vb, _, _ = _pair(mwlib, make, NH)
    assert t_res[0]["pe"] == t_ck[0]["pe"]
    _close(ta, tb, xa, xb, va, vb, box, 150)


def test_checkpoint_refuses_another_system(mwlib):
    x, box = I.jittered_box(512, 1.0, 0.15, 61)
    s = mwlib.System(512, box)
    t = mwlib.System(513, box)
    u = mwlib.System(512, box, skin=1.5)
    try:
        s.set_state(x)
        blob = s.checkpoint()
        with pytest.raises(mwlib.MWError):
            t.restore(blob)
        with pytest.raises(mwlib.MWError):
            u.restore(blob)
        with pytest.raises(mwlib.MWError):
            s.restore(blob[: len(blob) // 2])
        with pytest.raises(mwlib.MWError):
            s.restore(b"x" * len(blob))
    finally:
        s.close()
        t.close()
        u.close()

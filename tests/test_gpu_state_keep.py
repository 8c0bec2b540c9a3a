"""mw_set_state on a system whose atom order and neighbour lists are current
keeps them (no re-sort, no list build) while every atom lies within half the
skin of its list position, and rebuilds the boxes where one does not.
Either way the state loaded and the forces computed are the same as on a
fresh system (checked against the FP64 oracle, Sec. II.A)."""
import numpy as np
import pytest

from paper_0809_2811_gb300 import inputs as I
from _parity import compare

pytestmark = pytest.mark.gpu


def test_set_state_keeps_lists_within_half_skin(mwlib, orc):
    x, box = I.jittered_box(3000, 1.0, 0.3, 401)
    x = I.snap_to_grid(x, box)
    v = I.maxwell_velocities(len(x), 300.0, seed=402)
    ref = orc.energy_forces(x, box)
    s = mwlib.System(len(x), box)
    try:
        s.set_state(x, v)
        f, e, w = s.energy_forces()
        assert s.info()["rebuild_steps"] == 1  # a fresh state is sorted and listed once
        compare("keep: first state", f, e[0], w[0], ref)
        # the same positions again: nothing moved, the lists stay
        s.set_state(x, v)
        f, e, w = s.energy_forces()
        assert s.info()["rebuild_steps"] == 0
        compare("keep: same state again", f, e[0], w[0], ref)
        xs, vs = s.get_state()
        assert np.array_equal(xs, x) and np.allclose(vs, v, rtol=2.0 ** -47, atol=0)
        # positions moved by less than half the skin (0.5 A): still no rebuild
        rng = np.random.default_rng(403)
        d = rng.normal(0.0, 1.0, x.shape)
        d *= 0.2 / np.linalg.norm(d, axis=1, keepdims=True)
        x2 = I.snap_to_grid(x + d, box)
        s.set_state(x2, v)
        f, e, w = s.energy_forces()
        assert s.info()["rebuild_steps"] == 0
        compare("keep: moved 0.2 A", f, e[0], w[0], orc.energy_forces(x2, box))
        # one atom moved by more than half the skin: its box is rebuilt
        x3 = x.copy()
        x3[17] += np.array([0.6, 0.0, 0.0])
        x3 = I.snap_to_grid(x3, box)
        s.set_state(x3, v)
        f, e, w = s.energy_forces()
        assert s.info()["rebuild_steps"] == 1
        compare("keep: one atom moved 0.6 A", f, e[0], w[0], orc.energy_forces(x3, box))
    finally:
        s.close()


def test_set_state_after_steps_rebuilds_moved_boxes(mwlib, orc):
    """A batch run far enough for atoms to leave their list positions, then the
    starting state set again: every box is rebuilt and the forces match."""
    n = [512, 729]
    xs, boxes = [], []
    for k, (nn, rho) in enumerate(zip(n, [1.0, 0.95])):
        x, b = I.jittered_box(nn, rho, 0.25, 410 + k)
        xs.append(I.snap_to_grid(x, b))
        boxes.append(b)
    x = np.concatenate(xs)
    v = I.maxwell_velocities(len(x), 350.0, seed=412)
    s = mwlib.System(n, np.array(boxes))
    try:
        s.set_state(x, v)
        s.step(300, dt=10.0, thermostat=mwlib.MW_NOSE_HOOVER, T0=350.0, tau=500.0)
        s.set_state(x, v)
        f, e, w = s.energy_forces()
        off = 0
        for b in range(2):
            compare(f"keep: batch box {b} after 300 steps", f[off:off + n[b]], e[b], w[b],
                    orc.energy_forces(xs[b], boxes[b]))
            off += n[b]
        th = s.step(20, dt=10.0, thermostat=mwlib.MW_NOSE_HOOVER, T0=350.0, tau=500.0)
        assert all(t["step"] == 20 for t in th)
    finally:
        s.close()


def test_set_state_kept_order_refuses_non_finite_velocity(mwlib, orc):
    """In the kept-order path the velocities are loaded after the force call
    at the new positions; a non-finite velocity is still refused by
    mw_set_state itself (MW_EINVAL, no state left), and a valid state set
    afterwards gives the oracle's forces."""
    x, box = I.jittered_box(1000, 1.0, 0.3, 421)
    x = I.snap_to_grid(x, box)
    v = I.maxwell_velocities(len(x), 300.0, seed=422)
    s = mwlib.System(len(x), box)
    try:
        s.set_state(x, v)
        s.energy_forces()  # the order and lists are now current: the next state keeps them
        vb = v.copy()
        vb[123, 1] = np.nan
        with pytest.raises(mwlib.MWError) as ei:
            s.set_state(x, vb)
        assert ei.value.status == mwlib.MW_EINVAL
        with pytest.raises(mwlib.MWError) as ei:
            s.energy_forces()
        assert ei.value.status == mwlib.MW_ESTATE
        s.set_state(x, v)
        f, e, w = s.energy_forces()
        compare("keep: after a refused velocity", f, e[0], w[0], orc.energy_forces(x, box))
        xs, vs = s.get_state()
        assert np.array_equal(xs, x) and np.allclose(vs, v, rtol=2.0 ** -47, atol=0)
    finally:
        s.close()

"""Parity at the benchmarked sizes, through the launch the bench times.

The bench advances its workloads with the persistent engine (one cooperative
launch, the force phase inlined in it) at the skin the autotuner picks.
These tests take the forces, energies and virial of that engine's force phase
element by element against the FP64 oracle (Sec. II.A) on:
  * the two-box workload (32768-atom ice Ih at 0.92 g/cm^3 and a 32768-atom
    liquid-like box at 0.9998: the same lattice with 0.35 A Gaussian jitter)
    at skin 2.6 A (list radius 6.9 A, 88-slot rows);
  * the 2^20-atom ice / liquid slab (Lz = 453 A) with the engine, skin and
    grid the autotuner picks for it, neighbour sets checked on a sample;
  * a thin box 453 A long (18 x 16 A across), where the fixed-point
    coordinates matter most, both on the snapped grid and against the
    unsnapped FP64 positions.
How the engine's own force phase is read: from rest, one NVE step with
dt = 1e-9 fs moves no 64-bit position (the drift rounds to zero), so the
step's force phase evaluates exactly the positions given; the test checks
that the positions on the device grid did not change, then reads the forces
the step left behind.
"""
import numpy as np
import pytest

from paper_0809_2811_gb300 import inputs as I
from _parity import compare, neighbor_mismatch, record

pytestmark = pytest.mark.gpu


def engine_force_phase(mwlib, s, x, boxes):
    """Forces (n,3), energies (nbox,3), virial (nbox,6) of one step of the
    system's engine at the positions x (snapped, box-major)."""
    s.step(1, dt=1e-9, thermostat=mwlib.MW_NVE)
    xs, _ = s.get_state()
    off = 0
    for b, (n, box) in enumerate(boxes):
        assert np.array_equal(I.snap_to_grid(xs[off:off + n], box), x[off:off + n]), "positions moved"
        off += n
    return s.energy_forces()


def check_neighbors_rows(orc, s, x, box, off, n, case, sample=None):
    info = s.info()
    counts, nbr = s.neighbors(width=max(info["max_count"], 1))
    counts, nbr = counts[off:off + n], nbr[off:off + n] - off
    rc, rn, band = orc.neighbors_raw(x, box, info["r_list"], band_rel=1e-5, width=max(info["max_count"], 8) + 8)
    if sample is not None:
        rng = np.random.default_rng(7)
        rows = np.sort(rng.choice(n, size=min(sample, n), replace=False))
        rowset = set(rows.tolist())
        keep = {(i, j) for (i, j) in band if i in rowset}
        # rows renumbered 0..len(rows)-1 for the key arithmetic; partners keep their index
        remap = {int(r): k for k, r in enumerate(rows)}
        mism, nb = neighbor_mismatch_rows(counts[rows], nbr[rows], rc[rows], rn[rows],
                                          {(remap[i], j) for (i, j) in keep}, len(rows), n)
    else:
        mism, nb = neighbor_mismatch(counts, nbr, rc, rn, band, n)
    record(case + " [neighbour sets]", force=0.0, energy=0.0, virial=0.0, strict_force_rel=0.0)
    assert mism == 0, f"{case}: {mism} neighbour entries differ outside the band ({nb} band pairs)"


def neighbor_mismatch_rows(counts, nbr, rc, rn, band, nrows, n):
    """neighbor_mismatch on a subset of rows (rows renumbered, partner indices < n)."""
    counts = np.asarray(counts, np.int64)
    rc = np.asarray(rc, np.int64)
    ig = np.repeat(np.arange(nrows, dtype=np.int64), counts)
    jg = nbr[np.arange(nbr.shape[1])[None, :] < counts[:, None]].astype(np.int64)
    ir = np.repeat(np.arange(nrows, dtype=np.int64), rc)
    jr = rn[np.arange(rn.shape[1])[None, :] < rc[:, None]].astype(np.int64)
    kg, kr = ig * n + jg, ir * n + jr
    assert len(np.unique(kg)) == len(kg), "duplicate neighbour entries"
    diff = np.setxor1d(kg, kr, assume_unique=True)
    if band:
        bk = np.array([a * n + b for a, b in band], np.int64)
        diff = diff[~np.isin(diff, bk)]
    return int(len(diff)), len(band)


def two_box_workload():
    xi, bi = I.ice_ih(16, 16, 16, 0.92)
    xl, bl = I.ice_ih(16, 16, 16, 0.9998)
    xl = xl + np.random.default_rng(3).normal(0.0, 0.35, xl.shape)
    return [(I.snap_to_grid(xi, bi), bi), (I.snap_to_grid(xl, bl), bl)]


def test_two_box_65536_persistent_skin_2p6(mwlib, orc):
    parts = two_box_workload()
    x = np.concatenate([p[0] for p in parts])
    n = [len(p[0]) for p in parts]
    s = mwlib.System(n, np.stack([p[1] for p in parts]), skin=2.6)
    try:
        s.set_engine(mwlib.MW_ENGINE_PERSISTENT)
        s.set_state(x)
        f, e, w = engine_force_phase(mwlib, s, x, [(len(p[0]), p[1]) for p in parts])
        info = s.info()
        assert info["engine"] == mwlib.MW_ENGINE_PERSISTENT
        assert abs(info["r_list"] - 6.9065) < 1e-3 and info["nbr_width"] >= 80
        off = 0
        for b, (xb, box) in enumerate(parts):
            ref = orc.energy_forces(xb, box)
            name = ("ice_32768_0.92" if b == 0 else "liquidlike_32768_0.9998") + " [persistent, skin 2.6]"
            compare(name, f[off:off + len(xb)], e[b], w[b], ref)
            check_neighbors_rows(orc, s, xb, box, off, len(xb), name)
            off += len(xb)
    finally:
        s.close()


def test_slab_2p20_atoms_autotuned_launch(mwlib, orc):
    """The bench's headline workload at full size, in the launch the bench
    times (autotuned engine, skin and grid for NH 250 K at dt = 10 fs)."""
    x, box, _ = I.ice_liquid_slab()
    x = I.snap_to_grid(x, box)
    n = len(x)
    s = mwlib.System(n, box)
    try:
        s.set_state(x)
        integ = mwlib.make_integrator(10.0, mwlib.MW_NOSE_HOOVER, 250.0, 1000.0)
        mwlib.mw_autotune(s.h, integ, 50)
        s.set_state(x)  # from rest again (the autotuner restores the state it was given)
        f, e, w = engine_force_phase(mwlib, s, x, [(n, box)])
        ref = orc.energy_forces(x, box)
        compare(f"ice_liquid_slab_{n} [autotuned launch]", f, e[0], w[0], ref)
        check_neighbors_rows(orc, s, x, box, 0, n, f"ice_liquid_slab_{n} [autotuned launch]", sample=20000)
    finally:
        s.close()


def test_long_thin_box_fixed_point(mwlib, orc):
    """Lz = 453 A: the fixed-point minimum-image differences keep FP32's
    relative precision whatever the box length, so the forces match the
    oracle on the grid positions and on the unsnapped FP64 ones alike."""
    xr, box, _ = I.ice_liquid_slab(4, 2, 32)
    assert box[2] > 440.0
    x = I.snap_to_grid(xr, box)
    ref = orc.energy_forces(x, box)
    for engine, tag in ((mwlib.MW_ENGINE_GRAPH, "k_force"), (mwlib.MW_ENGINE_PERSISTENT, "persistent")):
        s = mwlib.System(len(x), box, skin=2.6)
        try:
            s.set_engine(engine)
            s.set_state(x)
            f, e, w = s.energy_forces()
            compare(f"long_box_{len(x)}_Lz{box[2]:.0f} [{tag} prime]", f, e[0], w[0], ref)
            f, e, w = engine_force_phase(mwlib, s, x, [(len(x), box)])
            compare(f"long_box_{len(x)}_Lz{box[2]:.0f} [{tag} step]", f, e[0], w[0], ref)
            check_neighbors_rows(orc, s, x, box, 0, len(x), f"long_box_{len(x)} [{tag}]")
        finally:
            s.close()
    # unsnapped input: the device rounds it to its grid (<= 5e-8 A here); the
    # force change that causes stays far inside the tolerance
    ref_u = orc.energy_forces(xr, box)
    s = mwlib.System(len(x), box, skin=2.6)
    try:
        s.set_state(xr)
        f, e, w = s.energy_forces()
        compare(f"long_box_{len(x)}_Lz{box[2]:.0f} [unsnapped FP64 input]", f, e[0], w[0], ref_u)
    finally:
        s.close()

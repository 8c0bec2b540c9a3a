"""GPU path vs the FP64 oracle, element by element, through the C ABI.

Tolerances and the margin record are in _parity.py: neighbour sets bit-exact
outside the FP32/FP64 ambiguity band, per-atom forces within 1e-5 (floored
relative), E, E2, E3 within 1e-6 of |E2| + |E3|, the virial within 1e-6 of
the summed magnitude of its diagonal contributions.  The oracle is fed the
same positions the kernels see: inputs are snapped to the 2^-32 box-fraction
grid of the device's fixed-point coordinates.
"""
import numpy as np
import pytest

from paper_0809_2811_gb300 import inputs as I
from _parity import E_TOL, F_TOL, compare, force_err

pytestmark = pytest.mark.gpu


def check_box(mwlib, orc, x, box, v=None, neighbors=True, case="box"):
    x = I.snap_to_grid(np.asarray(x, float), box)
    ref = orc.energy_forces(x, box)
    s = mwlib.System(len(x), box)
    try:
        s.set_state(x, v)
        f, e, w = s.energy_forces()
        compare(case, f, e[0], w[0], ref, w_tol=F_TOL if len(x) <= 3 else E_TOL)
        if neighbors:
            check_neighbors(s, orc, x, box)
        return s, ref, f
    except Exception:
        s.close()
        raise


def check_neighbors(s, orc, x, box):
    info = s.info()
    rl = info["r_list"]
    sets, band = orc.neighbors(x, box, rl, band_rel=1e-5)
    counts, nbr = s.neighbors(width=max(info["max_count"], 1))
    mism = 0
    for i in range(len(x)):
        g = set(nbr[i, :counts[i]].tolist())
        r = set(sets[i].tolist())
        diff = g.symmetric_difference(r)
        diff = {j for j in diff if (i, j) not in band}
        mism += len(diff)
        assert len(g) == counts[i], "duplicate neighbour entries"
    assert mism == 0


CASES = {
    "sc512_nve_start": lambda: I.nve512()[0::2],
    "ice_ih_288": lambda: I.ice_ih(4, 3, 3, 0.92),
    "ice_ic_216": lambda: I.diamond_cubic(3, 0.92),
    "liquidlike_1000": lambda: I.jittered_box(1000, 1.0, 0.3, 101),
    "dense_729_rho1.10": lambda: I.jittered_box(729, 1.10, 0.3, 102),
    "ragged_1237": lambda: I.jittered_box(1237, 0.97, 0.25, 103),
    "slab_2048": lambda: I.ice_liquid_slab(8, 4, 4)[:2],
    "liquid_vapor_slab_1024": lambda: I.liquid_vapor_slab(),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_energy_forces_parity(mwlib, orc, case):
    x, box = CASES[case]()
    s, _, _ = check_box(mwlib, orc, x, box, case=case)
    s.close()


def test_overflow_legs_path(mwlib, orc):
    """Dense box (32 legs per atom on average, up to 36): centres beyond the 24 staged legs
    take the overflow kernel; results must not change."""
    x, box = I.jittered_box(512, 3.5, 0.1, 104)
    s, ref, _ = check_box(mwlib, orc, x, box, case="overflow_legs_512_rho3.5")
    s.close()


def test_dense_cells_many_centres_and_stencil_chunks(mwlib, orc):
    """4096 atoms at 2.6 g/cm^3 with a 3 A skin: 4 cells per edge of ~64
    atoms each, so every cell's warp runs two groups of 32 centres, stages its
    ~1700-candidate stencil in 7 chunks, and every centre has ~26-30 legs (the
    staged-leg limit of 24 sends some to the overflow kernel).  Neighbour sets
    and forces against the oracle as in every other case."""
    x, box = I.jittered_box(4096, 2.6, 0.1, 105)
    x = I.snap_to_grid(np.asarray(x, float), box)
    ref = orc.energy_forces(x, box)
    s = mwlib.System(len(x), box, skin=3.0)
    try:
        s.set_state(x)
        f, e, w = s.energy_forces()
        info = s.info()
        assert info["max_count"] > 32 * 27 // 8  # the rows are long: well past one staging chunk per cell
        compare("dense_cells_4096_rho2.6_skin3", f, e[0], w[0], ref)
        check_neighbors(s, orc, x, box)
    finally:
        s.close()


def test_tiny_systems(mwlib, orc):
    # two atoms inside the cutoff: pair term only
    box = np.array([12.0, 12.0, 12.0])
    s, ref, f = check_box(mwlib, orc, np.array([[1.0, 1.0, 1.0], [3.7, 1.2, 0.9]]), box, case="tiny_pair")
    assert ref["ntriplets"] == 0 and ref["npairs"] == 1
    s.close()
    # three atoms: one triplet per centre that has two legs
    s, ref, f = check_box(mwlib, orc, np.array([[1.0, 1.0, 1.0], [3.7, 1.2, 0.9], [1.5, 3.6, 1.1]]), box,
                          case="tiny_triplet")
    assert ref["ntriplets"] >= 1
    s.close()
    # two atoms far apart: all zero
    s, ref, f = check_box(mwlib, orc, np.array([[1.0, 1.0, 1.0], [7.0, 7.0, 7.0]]), box, case="tiny_apart")
    assert np.abs(f).max() == 0.0
    s.close()
    # across the periodic boundary (minimum image)
    s, ref, f = check_box(mwlib, orc, np.array([[0.2, 11.9, 6.0], [11.5, 0.8, 6.3], [0.5, 1.9, 5.0]]), box,
                          case="tiny_periodic")
    s.close()


def test_box_at_two_list_radii(mwlib, orc):
    """Edge = 2 r_list gives 2 cells per dimension: the stencil must not visit a cell twice."""
    p = orc.default_params()
    rl = p[3] * p[2] + 1.0
    L = 2 * rl + 1e-9
    rng = np.random.default_rng(5)
    x = I.simple_cubic(4, L, 0.0) + rng.normal(0, 0.2, (64, 3))
    s, _, _ = check_box(mwlib, orc, x, np.array([L, L, L]), case="edge_2_rlist_64")
    s.close()


def test_batch_parity(mwlib, orc):
    n = [216, 300, 517, 1000, 250]
    rho = [0.92, 1.0, 1.05, 0.97, 1.10]
    xs, boxes = [], []
    for k, (nn, r) in enumerate(zip(n, rho)):
        x, b = I.jittered_box(nn, r, 0.25, 200 + k)
        xs.append(I.snap_to_grid(x, b))
        boxes.append(b)
    s = mwlib.System(n, np.array(boxes))
    try:
        s.set_state(np.concatenate(xs))
        f, e, w = s.energy_forces()
        off = 0
        for b in range(len(n)):
            ref = orc.energy_forces(xs[b], boxes[b])
            compare(f"batch5_box{b}_n{n[b]}", f[off:off + n[b]], e[b], w[b], ref)
            off += n[b]
    finally:
        s.close()


def test_state_roundtrip_and_wrap(mwlib):
    x, v, box = I.nve512()
    x = x + np.array([25.0, -50.0, 3.0])  # outside the box: wrapped on entry
    s = mwlib.System(512, box)
    try:
        s.set_state(x, v)
        x2, v2 = s.get_state()
        np.testing.assert_allclose(x2, np.mod(x, box), atol=1e-12)
        # velocities are held as hi + lo FP32 pairs: |v - (hi + lo)| <= 2^-48 |v|
        np.testing.assert_allclose(v2, v, rtol=2.0 ** -47, atol=0)
    finally:
        s.close()


def test_count_terms_matches_oracle(mwlib, orc):
    x, box = I.jittered_box(1000, 1.0, 0.3, 101)
    x = I.snap_to_grid(x, box)
    ref = orc.energy_forces(x, box)
    s = mwlib.System(len(x), box)
    try:
        s.set_count_terms(True)
        s.set_state(x)
        s.energy_forces()
        info = s.info()
        assert info["npairs"] == ref["npairs"]
        assert info["ntriplets"] == ref["ntriplets"]
    finally:
        s.close()


def test_neighbor_overflow_recovery(mwlib, orc):
    """A list far too narrow is grown internally and results do not change."""
    x, box = I.jittered_box(729, 1.0, 0.25, 105)
    x = I.snap_to_grid(x, box)
    ref = orc.energy_forces(x, box)
    s = mwlib.System(len(x), box)
    try:
        mwlib.mw_set_nbr_width(s.h, 4)
        s.set_state(x)
        f, e, _ = s.energy_forces()
        assert force_err(f, ref["forces"]) <= F_TOL
        assert s.info()["nbr_width"] > 4
    finally:
        s.close()


def test_rejects_bad_input(mwlib):
    with pytest.raises(mwlib.MWError) as ei:
        mwlib.System(64, [9.0, 9.0, 9.0])  # shorter than 2 r_list
    assert ei.value.status == mwlib.MW_EBOX
    s = mwlib.System(8, [20.0, 20.0, 20.0])
    try:
        x = np.zeros((8, 3))
        x[3, 1] = np.nan
        with pytest.raises(mwlib.MWError) as ei:
            s.set_state(x)
        assert ei.value.status == mwlib.MW_EINVAL
        with pytest.raises(mwlib.MWError) as ei:
            s.energy_forces()
        assert ei.value.status == mwlib.MW_ESTATE
    finally:
        s.close()


def test_pinned_host_state_matches_pageable(mwlib, orc):
    """Page-locked host arrays are read in place by the loading kernel,
    pageable ones through a staging copy: the loaded state is the same to the
    bit, the forces match the oracle, and a non-finite pinned value is refused
    like a pageable one."""
    import torch
    x, v, box = I.nve512()
    x = I.snap_to_grid(x, box)
    xp = torch.from_numpy(np.ascontiguousarray(x)).pin_memory()
    vp = torch.from_numpy(np.ascontiguousarray(v)).pin_memory()
    a = mwlib.System(len(x), box)
    b = mwlib.System(len(x), box)
    try:
        a.set_state(x.copy(), v.copy())
        b.set_state(xp.numpy(), vp.numpy())
        xa, va = a.get_state()
        xb, vb = b.get_state()
        assert np.array_equal(xa, xb) and np.array_equal(va, vb)
        f, e, w = b.energy_forces()
        ref = orc.energy_forces(x, box)
        assert force_err(f, ref["forces"]) <= F_TOL
        assert abs(e[0, 0] - ref["energy"]) <= E_TOL * (abs(ref["e2"]) + abs(ref["e3"]))
        ta = a.step(5, dt=10.0)
        tb = b.step(5, dt=10.0)
        assert ta[0]["step"] == tb[0]["step"] == 5
        xp[7, 2] = float("inf")
        with pytest.raises(mwlib.MWError) as ei:
            b.set_state(xp.numpy(), vp.numpy())
        assert ei.value.status == mwlib.MW_EINVAL
    finally:
        a.close()
        b.close()


@pytest.mark.parametrize("shape", [(4, 8, 0), (2, 8, 0), (8, 8, 0), (4, 7, 0), (4, 8, 1)])
def test_force_kernel_shapes_agree_with_oracle(mwlib, orc, shape):
    """Every launch shape the autotuner may pick (lanes per centre x blocks per
    SM x scatter or owner-computes) computes the same forces, energies and
    virial; the dense box has centres over the staged-leg limit, which the
    owner-computes passes leave to the scatter path."""
    for case, (x, box) in (("liquidlike_1000", I.jittered_box(1000, 1.0, 0.3, 101)),
                           ("ice_ih_288", I.ice_ih(4, 3, 3, 0.92)),
                           ("dense_512_rho3.5", I.jittered_box(512, 3.5, 0.1, 104))):
        x = I.snap_to_grid(x, box)
        ref = orc.energy_forces(x, box)
        s = mwlib.System(len(x), box)
        try:
            mwlib.mw_set_force_shape(s.h, *shape)
            s.set_state(x)
            f, e, w = s.energy_forces()
            info = s.info()
            assert (info["force_lanes"], info["force_blocks_per_sm"], info["force_owner"]) == shape
            compare(f"{case} [force shape {shape[0]}x{shape[1]}{' owner' if shape[2] else ''}]", f, e[0], w[0], ref)
        finally:
            s.close()


def test_autotuner_picks_and_reports_a_force_shape(mwlib):
    x, box = I.jittered_box(4096, 1.0, 0.25, 120)
    s = mwlib.System(len(x), box)
    try:
        s.set_state(x)
        integ = mwlib.make_integrator(10.0, mwlib.MW_NOSE_HOOVER, 300.0, 1000.0)
        mwlib.mw_autotune(s.h, integ, 10)
        info = s.info()
        assert (info["force_lanes"], info["force_blocks_per_sm"], info["force_owner"]) in {
            (4, 8, 0), (2, 8, 0), (8, 8, 0), (4, 7, 0), (4, 8, 1)}
        # rows fitted to the chosen skin, whole 128-byte lines, and the list built in them
        s.energy_forces()
        info = s.info()
        assert info["nbr_width"] % 32 == 0 and info["max_count"] <= info["nbr_width"]
        rl, n_per_a3 = info["r_list"], len(x) / float(np.prod(box))
        assert info["nbr_width"] <= ((int(np.ceil(1.5 * n_per_a3 * 4.18879020478639 * rl ** 3 + 16)) + 31) // 32) * 32
        with pytest.raises(mwlib.MWError):
            mwlib.mw_set_force_shape(s.h, 3, 8)
        with pytest.raises(mwlib.MWError):
            mwlib.mw_set_force_shape(s.h, 2, 8, True)
    finally:
        s.close()

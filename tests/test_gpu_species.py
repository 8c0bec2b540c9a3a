"""Several species (mw_set_species) vs the oracle's energy_forces_species and
md_species, through the C ABI.

Tolerances are those of the one-species parity tests (test_gpu_parity): the
kernel's arithmetic per term is the same FP32 with FP64 sums, only the
parameters now come per pair and per triplet.
"""
import numpy as np
import pytest

from paper_0809_2811_gb300 import inputs as I

from test_gpu_parity import E_TOL, F_TOL, check_neighbors, force_err

pytestmark = pytest.mark.gpu

CASES = {
    "mixed2_1000": lambda: (*I.jittered_box(1000, 1.0, 0.3, 201), I.species_draw(1000, 2, 11),
                            I.species_table_mixed(2, 5)),
    "mixed3_ragged_777": lambda: (*I.jittered_box(777, 0.97, 0.25, 202), I.species_draw(777, 3, 12),
                                  I.species_table_mixed(3, 6)),
    "mw_solute_1200": lambda: (*I.jittered_box(1200, 1.0, 0.25, 203), I.species_draw(1200, 2, 13, [0.9, 0.1]),
                               I.species_table_solute()),
    "sw_family_1331": lambda: (*I.jittered_box(1331, 0.95, 0.25, 204), I.species_draw(1331, 4, 14),
                               I.species_table_sw_family()),
}


def _check(s, orc, x, box, ty, table, ref=None):
    ref = orc.energy_forces_species(x, box, ty, table) if ref is None else ref
    f, e, w = s.energy_forces()
    assert force_err(f, ref["forces"]) <= F_TOL
    escale = abs(ref["e2"]) + abs(ref["e3"])
    for k, name in ((0, "energy"), (1, "e2"), (2, "e3")):
        assert abs(e[0, k] - ref[name]) <= E_TOL * escale, name
    assert np.abs(w[0] - ref["virial"]).max() <= F_TOL * ref["virial_abs"]
    return ref


@pytest.mark.parametrize("case", sorted(CASES))
def test_species_energy_forces_match_oracle(mwlib, orc, case):
    x, box, ty, table = CASES[case]()
    x = I.snap_to_grid(x, box)
    assert orc.species_table_ok(table)
    s = mwlib.System(len(x), box)
    try:
        s.set_species(table, ty)
        s.set_state(x)
        ref = _check(s, orc, x, box, ty, table)
        assert ref["ntriplets"] > 0
        rc = max(table[a, b, b, 3] * table[a, b, b, 2] for a in range(len(table)) for b in range(len(table)))
        info = s.info()
        assert info["r_list"] == pytest.approx(rc + 1.0, rel=1e-12)
        assert info["species"] == len(table)
        # geometric-mean family and the lambda = 0 solute factor into leg weights
        assert info["species_moments"] == (1 if case in ("mw_solute_1200", "sw_family_1331") else 0)
        check_neighbors(s, orc, x, box)
    finally:
        s.close()


@pytest.mark.parametrize("table", ["sw_family", "mixed3"])
def test_species_dense_box_more_legs_than_staged(mwlib, orc, table):
    """Dense boxes: the Fig. 2 family at 4.5 g/cm^3 has 50 legs per centre on
    average (at most 56), so the moment kernel, which stages 48, hands most
    centres to the per-centre walker; the every-entry-different table at 3.5
    has 45 on average and at most 60 (the walker holds 64)."""
    x, box = I.jittered_box(512, 4.5 if table == "sw_family" else 3.5, 0.1, 104)
    x = I.snap_to_grid(x, box)
    t = I.species_table_sw_family() if table == "sw_family" else I.species_table_mixed(3, 17)
    ty = I.species_draw(512, len(t), 18)
    s = mwlib.System(512, box)
    try:
        s.set_species(t, ty)
        s.set_state(x)
        _check(s, orc, x, box, ty, t)
    finally:
        s.close()


def test_species_count_terms_match_oracle(mwlib, orc):
    for t in (I.species_table_solute(), I.species_table_mixed(2, 5)):
        x, box = I.jittered_box(1000, 1.0, 0.3, 205)
        x = I.snap_to_grid(x, box)
        ty = I.species_draw(1000, 2, 19, [0.8, 0.2])
        s = mwlib.System(1000, box)
        try:
            s.set_species(t, ty)
            mwlib.mw_set_count_terms(s.h, True)
            s.set_state(x)
            s.energy_forces()
            info = s.info()
        finally:
            s.close()
        ref = orc.energy_forces_species(x, box, ty, t)
        assert (info["npairs"], info["ntriplets"]) == (ref["npairs"], ref["ntriplets"])


def test_species_set_before_or_after_state_and_back_to_one(mwlib, orc):
    """Species given after the state (atoms already cell-sorted) land on the
    right atoms; mw_set_params returns to the one-species kernel."""
    x, box, ty, table = CASES["mixed2_1000"]()
    x = I.snap_to_grid(x, box)
    s = mwlib.System(len(x), box)
    try:
        s.set_state(x)
        s.energy_forces()  # sorts the atoms
        s.set_species(table, ty)
        _check(s, orc, x, box, ty, table)
        s.set_params(mwlib.mw_params_default())
        _check(s, orc, x, box, np.zeros(len(x), int), orc.species_table(1, lambda a, b, c: orc.default_params()))
    finally:
        s.close()


def test_species_batch_of_uneven_boxes(mwlib, orc):
    n = [300, 451, 200]
    xs, boxes, tys = [], [], []
    for k, nn in enumerate(n):
        x, b = I.jittered_box(nn, [0.95, 1.0, 1.05][k], 0.25, 210 + k)
        xs.append(I.snap_to_grid(x, b))
        boxes.append(b)
        tys.append(I.species_draw(nn, 3, 220 + k))
    table = I.species_table_mixed(3, 9)
    s = mwlib.System(n, np.array(boxes))
    try:
        s.set_species(table, np.concatenate(tys))
        s.set_state(np.concatenate(xs))
        f, e, w = s.energy_forces()
        off = 0
        for k in range(3):
            ref = orc.energy_forces_species(xs[k], boxes[k], tys[k], table)
            assert force_err(f[off:off + n[k]], ref["forces"]) <= F_TOL
            escale = abs(ref["e2"]) + abs(ref["e3"])
            assert abs(e[k, 0] - ref["energy"]) <= E_TOL * escale
            assert np.abs(w[k] - ref["virial"]).max() <= F_TOL * ref["virial_abs"]
            off += n[k]
    finally:
        s.close()


@pytest.mark.parametrize("table_kind", ["mixed", "solute"])
@pytest.mark.parametrize("kind", [0, 2])
def test_species_dynamics_match_oracle(mwlib, orc, kind, table_kind):
    """20 steps of a two-species mixture from the 512-atom start (every set
    different: the leg-pair walker; mW with a solute: the moment kernel):
    same tolerances as the one-species trajectory test."""
    x, v, box = I.nve512()
    x = I.snap_to_grid(x, box)
    ty = I.species_draw(512, 2, 15, None if table_kind == "mixed" else [0.85, 0.15])
    table = I.species_table_mixed(2, 16) if table_kind == "mixed" else I.species_table_solute()
    s = mwlib.System(512, box)
    try:
        s.set_species(table, ty)
        s.set_state(x, v)
        th = s.step(20, dt=10.0, thermostat=kind, T0=250.0, tau=200.0)[0]
        xg, vg = s.get_state()
        assert s.info()["engine"] == mwlib.MW_ENGINE_GRAPH
    finally:
        s.close()
    xo, vo, st, tho = orc.md_species(x, v, box, ty, table, 20, dt=10.0, kind=kind, T0=250.0, tau=200.0)
    d = xg - xo
    d -= box * np.rint(d / box)
    assert np.abs(d).max() < 5e-5
    assert np.abs(vg - vo).max() < 1e-6
    assert th["pe"] == pytest.approx(tho[-1, 0], rel=3e-6)
    assert th["conserved"] == pytest.approx(tho[-1, 5], rel=3e-6)
    if kind == 2:
        assert th["xi"] == pytest.approx(st[0], rel=1e-4, abs=1e-9)


def test_species_table_rules_and_adjoint_are_enforced(mwlib):
    x, box, ty, table = CASES["mixed2_1000"]()
    s = mwlib.System(len(x), box)
    try:
        bad = table.copy()
        bad[0, 1, 1, 1] *= 1.01  # pair (0, 1) differs from (1, 0)
        with pytest.raises(mwlib.MWError):
            s.set_species(bad, ty)
        bad = table.copy()
        bad[1, 0, 1, 7] += 0.1  # cos theta0 of (1; 0, 1) differs from (1; 1, 0)
        with pytest.raises(mwlib.MWError):
            s.set_species(bad, ty)
        with pytest.raises(mwlib.MWError):
            s.set_species(table, np.full(len(x), 2))
        s.set_species(table, ty)
        s.set_state(x)
        import torch
        wd = torch.zeros((len(x), 3), dtype=torch.float32, device="cuda")
        gx = torch.empty_like(wd)
        with pytest.raises(mwlib.MWError):
            mwlib.mw_energy_forces_vjp(s.h, wd, gx, 1)
    finally:
        s.close()

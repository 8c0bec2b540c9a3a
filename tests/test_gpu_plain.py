"""The plain GPU path (MW_ENGINE_PLAIN: one thread per atom, leg pairs looped
per centre, leg forces scattered with red.global, per-phase launches with no
graph) against the FP64 oracle, element by element through the C ABI, with
the tolerances of _parity.py.  It is the baseline the batched, persistent
and adjoint paths are timed against, so it must compute the same thing."""
import numpy as np
import pytest

from paper_0809_2811_gb300 import inputs as I
from _parity import compare

pytestmark = pytest.mark.gpu

CASES = {
    "liquidlike_1000": lambda: I.jittered_box(1000, 1.0, 0.3, 101),
    "ice_ih_288": lambda: I.ice_ih(4, 3, 3, 0.92),
    "dense_729_rho1.10": lambda: I.jittered_box(729, 1.10, 0.3, 102),
    "dense_512_rho3.5": lambda: I.jittered_box(512, 3.5, 0.1, 104),
    "slab_2048": lambda: I.ice_liquid_slab(8, 4, 4)[:2],
    "liquid_vapor_slab_1024": lambda: I.liquid_vapor_slab(),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_plain_force_parity(mwlib, orc, case):
    x, box = CASES[case]()
    x = I.snap_to_grid(x, box)
    ref = orc.energy_forces(x, box)
    s = mwlib.System(len(x), box)
    try:
        s.set_engine(mwlib.MW_ENGINE_PLAIN)
        s.set_state(x)
        f, e, w = s.energy_forces()
        compare(case + " [plain]", f, e[0], w[0], ref)
    finally:
        s.close()


def test_plain_steps_at_32768_atoms(mwlib, orc):
    """The plain engine's own force kernel inside its steps, at the size of one
    box of the two-box workload (forces read after a dt = 1e-9 fs step from
    rest, which moves no position)."""
    xl, bl = I.ice_ih(16, 16, 16, 0.9998)
    xl = I.snap_to_grid(xl + np.random.default_rng(3).normal(0.0, 0.35, xl.shape), bl)
    s = mwlib.System(len(xl), bl)
    try:
        s.set_engine(mwlib.MW_ENGINE_PLAIN)
        s.set_state(xl)
        s.step(1, dt=1e-9, thermostat=mwlib.MW_NVE)
        assert s.info()["engine"] == mwlib.MW_ENGINE_PLAIN
        xs, _ = s.get_state()
        assert np.array_equal(I.snap_to_grid(xs, bl), xl)
        f, e, w = s.energy_forces()
        compare("liquidlike_32768 [plain step]", f, e[0], w[0], orc.energy_forces(xl, bl))
    finally:
        s.close()


def test_plain_counts_terms_like_the_oracle(mwlib, orc):
    x, box = I.jittered_box(1000, 1.0, 0.3, 101)
    x = I.snap_to_grid(x, box)
    ref = orc.energy_forces(x, box)
    s = mwlib.System(len(x), box)
    try:
        s.set_engine(mwlib.MW_ENGINE_PLAIN)
        s.set_count_terms(True)
        s.set_state(x)
        s.energy_forces()
        info = s.info()
        assert info["npairs"] == ref["npairs"] and info["ntriplets"] == ref["ntriplets"]
    finally:
        s.close()


def test_plain_engine_refuses_several_species(mwlib):
    x, box = I.jittered_box(512, 1.0, 0.1, 5)
    ty = I.species_draw(len(x), 2, 5, [0.9, 0.1])
    s = mwlib.System(len(x), box)
    try:
        s.set_engine(mwlib.MW_ENGINE_PLAIN)
        with pytest.raises(mwlib.MWError) as ei:
            s.set_species(I.species_table_solute(), ty)
        assert ei.value.status == mwlib.MW_EINVAL
        s.set_engine(mwlib.MW_ENGINE_GRAPH)
        s.set_species(I.species_table_solute(), ty)
        with pytest.raises(mwlib.MWError) as ei:
            s.set_engine(mwlib.MW_ENGINE_PLAIN)
        assert ei.value.status == mwlib.MW_EINVAL
    finally:
        s.close()

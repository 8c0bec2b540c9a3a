"""The allocation-free entry point against the regular one.

mw_energy_forces_noalloc is for callers that may not allocate device memory
(all its scratch is a static device array).  Through the C ABI it must give
the same forces, energies and virial as mw_energy_forces_dev, within the
tolerances of the parity tests, on two calls in a row (the second call reuses
the array the first one left behind).  This file sorts last so that a
stop-at-first-failure run has already run every other test.
"""
import numpy as np
import pytest

from paper_0809_2811_gb300 import inputs as I
from _parity import E_TOL, F_TOL, W_TOL, force_err as _force_err, record

pytestmark = pytest.mark.gpu


def _regular(mwlib, torch, x, box):
    n = len(x)
    s = mwlib.System(n, box, stream=torch.cuda.current_stream().cuda_stream or None)
    try:
        xd = torch.from_numpy(x).cuda()
        f = torch.empty((n, 3), dtype=torch.float32, device="cuda")
        e = torch.empty(3, dtype=torch.float64, device="cuda")
        w = torch.empty(6, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()  # inputs ready before the library's own stream reads them
        mwlib.mw_energy_forces_dev(s.h, xd, f, e, w)
        torch.cuda.synchronize()
        return f.cpu().numpy(), e.cpu().numpy(), w.cpu().numpy()
    finally:
        s.close()


def _noalloc(mwlib, torch, x, box):
    n = len(x)
    xd = torch.from_numpy(x).cuda()
    f = torch.full((n, 3), float("nan"), dtype=torch.float32, device="cuda")
    e = torch.full((3,), float("nan"), dtype=torch.float64, device="cuda")
    w = torch.full((6,), float("nan"), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    mwlib.mw_energy_forces_noalloc(n, box, xd, f, e, w)
    torch.cuda.synchronize()
    return f.cpu().numpy(), e.cpu().numpy(), w.cpu().numpy()


def test_noalloc_matches_regular_entry_point_twice(mwlib):
    torch = pytest.importorskip("torch")
    cases = [I.jittered_box(4096, 1.0, 0.3, 61), I.ice_ih(8, 5, 5, 0.92)]  # second call: other size and box
    for x, box in cases:
        x = I.snap_to_grid(x, box)
        fr, er, wr = _regular(mwlib, torch, x, box)
        fn, en, wn = _noalloc(mwlib, torch, x, box)
        assert np.isfinite(fn).all() and np.isfinite(en).all() and np.isfinite(wn).all()
        _same_within_tolerance(f"noalloc_vs_regular_n{len(x)}", fn, en, wn, fr, er, wr)


def _same_within_tolerance(case, fn, en, wn, fr, er, wr):
    fe = _force_err(fn, fr)
    escale = abs(er[1]) + abs(er[2])
    ee = np.abs(en - er).max() / escale
    # the regular path's virial stands in for the oracle's diagonal scale
    we = np.abs(wn - wr).max() / max(np.abs(wr[:3]).sum(), 1.0)
    record(case, force=fe / F_TOL, energy=ee / E_TOL, virial=we / W_TOL, strict_force_rel=float("nan"))
    assert fe <= F_TOL and ee <= E_TOL and we <= W_TOL, (fe, ee, we)


def test_noalloc_unsnapped_positions_match_regular(mwlib):
    """Positions off the fixed-point grid are converted exactly as the regular
    path converts them (box fraction, 64-bit fraction, 32-bit rounding), so the
    two entry points agree on unsnapped input too."""
    torch = pytest.importorskip("torch")
    x, box = I.jittered_box(3000, 0.98, 0.3, 63)
    fr, er, wr = _regular(mwlib, torch, x, box)
    fn, en, wn = _noalloc(mwlib, torch, x, box)
    _same_within_tolerance("noalloc_vs_regular_unsnapped_3000", fn, en, wn, fr, er, wr)


def test_noalloc_rejects_non_finite_position(mwlib):
    """A NaN coordinate is refused with MW_EINVAL and the outputs are left as
    they were."""
    torch = pytest.importorskip("torch")
    x, box = I.jittered_box(512, 1.0, 0.1, 64)
    x[17, 2] = np.nan
    xd = torch.from_numpy(x).cuda()
    f = torch.full((512, 3), 7.0, dtype=torch.float32, device="cuda")
    e = torch.full((3,), 7.0, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    with pytest.raises(mwlib.MWError) as ei:
        mwlib.mw_energy_forces_noalloc(512, box, xd, f, e)
    assert ei.value.status == mwlib.MW_EINVAL and "17" in str(ei.value)
    torch.cuda.synchronize()
    assert bool((f == 7.0).all()) and bool((e == 7.0).all())


def test_noalloc_rejects_sizes_beyond_its_limit(mwlib):
    torch = pytest.importorskip("torch")
    n = 16385
    x, box = I.jittered_box(n, 1.0, 0.1, 62)
    xd = torch.from_numpy(x).cuda()
    with pytest.raises(mwlib.MWError) as ei:
        mwlib.mw_energy_forces_noalloc(n, box, xd)
    assert ei.value.status == mwlib.MW_EINVAL and "16384" in str(ei.value)

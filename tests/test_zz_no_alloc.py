"""The allocation-free entry point against the regular one.

mw_energy_forces_noalloc is for callers that may not allocate device memory
(all its scratch is a static device array).  Through the C ABI it must give
the same forces, energies and virial as mw_energy_forces_dev, within the
tolerances of the parity tests, on two calls in a row (the second call reuses
the array the first one left behind).  This file sorts last so that a
stop-at-first-failure run has already run every other test.
"""
import math

import numpy as np
import pytest

from paper_0809_2811_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _force_err(fg, fr):
    mag = np.linalg.norm(fr, axis=1)
    den = np.maximum(np.maximum(mag, math.sqrt(np.mean(mag ** 2))), 6.189 / 2.3925)
    return float((np.linalg.norm(fg - fr, axis=1) / den).max())


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
        assert _force_err(fn, fr) <= 1e-5
        escale = abs(er[1]) + abs(er[2])
        assert np.abs(en - er).max() <= 1e-6 * escale
        assert np.abs(wn - wr).max() <= 1e-5 * max(np.abs(wr[:3]).sum(), 1.0)


def test_noalloc_rejects_sizes_beyond_its_limit(mwlib):
    torch = pytest.importorskip("torch")
    n = 16385
    x, box = I.jittered_box(n, 1.0, 0.1, 62)
    xd = torch.from_numpy(x).cuda()
    with pytest.raises(mwlib.MWError) as ei:
        mwlib.mw_energy_forces_noalloc(n, box, xd)
    assert ei.value.status == mwlib.MW_EINVAL and "16384" in str(ei.value)

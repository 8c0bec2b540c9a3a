"""Tolerances and comparisons shared by the GPU parity tests.

The bar (the method's specification of this engine; Sec. II.A of the paper
defines what is compared):
  * neighbour sets bit-exact, except pairs in the band
    | |d|^2 - r_list^2 | <= 1e-5 r_list^2 (FP32 vs FP64 distance; counted);
  * per-atom forces: max_i |F_gpu,i - F_ref,i| / max(|F_ref,i|, F_rms, eps/sigma)
    <= 1e-5 (eps/sigma = 2.59 kcal/mol/A, the force unit of the reduced form,
    is a floor for lattices whose exact forces and F_rms are zero);
  * energies (E, E2, E3) within 1e-6 of |E2| + |E3| (equal to "relative to E"
    up to a factor < 2 for liquid and ice; on strained inputs E2 and E3
    cancel and |E| alone would demand digits FP32 terms cannot carry);
  * virial within 1e-6 (the energy tolerance) of the summed magnitude of its
    diagonal contributions (the oracle's virial_abs; the trace is a
    cancelling sum like E); systems of two or three atoms at the force
    tolerance (see compare).
Besides the floored force measure, the strict per-atom relative error
|dF_i| / |F_ref,i| over atoms with |F_ref,i| >= eps/sigma is recorded
(reported, not asserted).  Every comparison records its errors as fractions
of the tolerances; conftest prints them in the terminal summary.
"""
from __future__ import annotations

import math

import numpy as np

F_TOL = 1e-5
E_TOL = 1e-6
W_TOL = 1e-6
F_UNIT = 6.189 / 2.3925  # eps / sigma, kcal/mol/A

MARGINS: list = []  # (case, {quantity: error / tolerance, ...})


def force_err(fg, fr):
    """Floored per-atom relative force error (the asserted measure)."""
    fr = np.asarray(fr, np.float64).reshape(-1, 3)
    fg = np.asarray(fg, np.float64).reshape(-1, 3)
    mag = np.linalg.norm(fr, axis=1)
    frms = math.sqrt(np.mean(mag ** 2)) if len(mag) else 1.0
    den = np.maximum(np.maximum(mag, frms), F_UNIT)
    return float((np.linalg.norm(fg - fr, axis=1) / den).max())


def strict_force_err(fg, fr, thresh=F_UNIT):
    """max |dF_i| / |F_ref,i| over atoms with |F_ref,i| >= thresh, and how many
    atoms fell below the threshold."""
    fr = np.asarray(fr, np.float64).reshape(-1, 3)
    fg = np.asarray(fg, np.float64).reshape(-1, 3)
    mag = np.linalg.norm(fr, axis=1)
    sel = mag >= thresh
    if not sel.any():
        return 0.0, int(len(mag))
    return float((np.linalg.norm(fg - fr, axis=1)[sel] / mag[sel]).max()), int((~sel).sum())


def record(case, **fracs):
    MARGINS.append((case, {k: float(v) for k, v in fracs.items()}))


def compare(case, f, e, w, ref, force_only=False, w_tol=W_TOL):
    """Asserts one box's forces (n,3), energies e = (E, E2, E3) and virial w[6]
    against an oracle dict; records the margins.  w_tol: the virial
    tolerance; only systems of two or three atoms take the force tolerance
    there (a lone pair's virial is one leg force times its leg vector, with
    no sum for rounding to average over, and near the phi2 minimum that force
    changes by ~1e2 times the relative FP32 rounding of the displacement)."""
    fe = force_err(f, ref["forces"])
    se, nlow = strict_force_err(f, ref["forces"])
    escale = abs(ref["e2"]) + abs(ref["e3"])
    ee = max(abs(e[0] - ref["energy"]), abs(e[1] - ref["e2"]), abs(e[2] - ref["e3"])) / max(escale, 1e-300)
    we = float(np.abs(np.asarray(w) - ref["virial"]).max()) / max(ref["virial_abs"], 1e-300)
    record(case, force=fe / F_TOL, energy=ee / E_TOL, virial=we / w_tol, strict_force_rel=se,
           atoms_below_force_unit=nlow)
    assert fe <= F_TOL, f"{case}: force error {fe:.3e}"
    if force_only:
        return
    assert ee <= E_TOL, f"{case}: energy error {ee:.3e} of |E2|+|E3|"
    assert we <= w_tol, f"{case}: virial error {we:.3e} of virial_abs"


def neighbor_mismatch(counts, nbr, ref_counts, ref_nbr, band, n):
    """Vectorised set comparison of GPU rows (any order) against the oracle's
    sorted rows; returns (mismatches outside the band, band pairs seen).
    counts/nbr: GPU rows (n, width); ref_*: oracle rows; band: set of (i, j)."""
    counts = np.asarray(counts, np.int64)
    ref_counts = np.asarray(ref_counts, np.int64)
    w = nbr.shape[1]
    wr = ref_nbr.shape[1]
    assert counts.max(initial=0) <= w and ref_counts.max(initial=0) <= wr, "rows truncated"
    ig = np.repeat(np.arange(n, dtype=np.int64), counts)
    jg = nbr[np.arange(w)[None, :] < counts[:, None]].astype(np.int64)
    ir = np.repeat(np.arange(n, dtype=np.int64), ref_counts)
    jr = ref_nbr[np.arange(wr)[None, :] < ref_counts[:, None]].astype(np.int64)
    kg = ig * n + jg
    kr = ir * n + jr
    assert len(np.unique(kg)) == len(kg), "duplicate neighbour entries"
    diff = np.setxor1d(kg, kr, assume_unique=True)
    if len(band):
        bk = np.array([a * n + b for a, b in band], np.int64)
        diff = diff[~np.isin(diff, bk)]
    return int(len(diff)), len(band)

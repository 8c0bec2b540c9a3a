"""FP64 CPU oracle for the mW water model (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library
(``paper_0809_2811_gb300``) neither imports nor links it, and the two share
no code.  The arithmetic lives in ``mw_oracle.c``; this module only builds
and loads that file and marshals numpy arrays.

Function map (section of the paper each follows):
  phi2, dphi2, phi3            Sec. II.A two- and three-body equations
  energy_forces_brute          Sec. II.A total energy, O(N^2)/O(N^3) loops
  energy_forces_cell           same, cell-list owner loop
  energy_forces(method="owner") same sums, owner-computes on several threads
                               (the multi-core CPU baseline)
  neighbors, neighbors_raw      neighbour sets {j : |d_ij| < r_list}
  md                           Sec. II.B velocity-Verlet run (thermostat reading)
  md_npt                       Sec. II.B isobaric-isothermal run (barostat reading)
  energy_forces_species        Sec. II.A equations with a parameter vector per
                               species triple (mW with solutes, Sec. IV)
  md_species                   md with that potential
  force_vjp                    force-matching adjoint (no counterpart in the paper)
  energy_param_grad            dE/d(lambda, epsilon, sigma)
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mw_oracle.c")
_LIB = os.path.join(_HERE, "libmw_oracle.so")

KB = 0.0019872042586408316  # kcal/mol/K
FCONV = 4.184e-4  # (kcal/mol/A)/(g/mol) -> A/fs^2
PARAM_NAMES = ("lambda", "epsilon", "sigma", "a", "gamma", "A", "B", "cos_theta0", "p", "q")


def build(force: bool = False) -> str:
    """Compiles mw_oracle.c into libmw_oracle.so next to it: gcc -O3, with
    OpenMP for the owner-computes routine when the compiler has it (without
    it that routine runs serially).  No -march=native and no FMA contraction
    (-ffp-contract=off), so that the x86 host and the Arm GPU host compute the
    same FP64 results."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        base = ["gcc", "-O3", "-ffp-contract=off", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        try:
            subprocess.check_call(base[:1] + ["-fopenmp"] + base[1:], stderr=subprocess.DEVNULL)
        except subprocess.CalledProcessError:
            subprocess.check_call(base)
        os.replace(tmp, _LIB)
    return _LIB


def openmp_enabled() -> bool:
    """Whether the built oracle has OpenMP (the owner routine then uses threads)."""
    return int(lib().or_openmp_threads()) > 0


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        d = ctypes.POINTER(ctypes.c_double)
        i = ctypes.POINTER(ctypes.c_int)
        _lib.or_params_default.argtypes = [d]
        _lib.or_phi2.argtypes = [d, ctypes.c_double]
        _lib.or_phi2.restype = ctypes.c_double
        _lib.or_dphi2.argtypes = [d, ctypes.c_double]
        _lib.or_dphi2.restype = ctypes.c_double
        _lib.or_phi3.argtypes = [d, ctypes.c_double, ctypes.c_double, ctypes.c_double]
        _lib.or_phi3.restype = ctypes.c_double
        for name in ("or_energy_forces_brute", "or_energy_forces_cell"):
            getattr(_lib, name).argtypes = [d, ctypes.c_int, d, d, d, d]
        _lib.or_energy_forces_owner.argtypes = [d, ctypes.c_int, d, d, d, d, ctypes.c_int]
        _lib.or_md_owner.argtypes = [d, ctypes.c_int, d, d, d, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int, d, d, ctypes.c_int]
        _lib.or_openmp_threads.restype = ctypes.c_int
        _lib.or_neighbors.argtypes = [ctypes.c_int, d, d, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_int, i, i, ctypes.c_int, i, i]
        _lib.or_md.argtypes = [d, ctypes.c_int, d, d, d, ctypes.c_double, ctypes.c_double,
                               ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int, d, d]
        _lib.or_md_npt.argtypes = [d, ctypes.c_int, d, d, d, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                   ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int, d, d]
        _lib.or_force_vjp.argtypes = [d, ctypes.c_int, d, d, d, d, d]
        _lib.or_species_table_check.argtypes = [d, ctypes.c_int]
        _lib.or_energy_forces_species.argtypes = [d, ctypes.c_int, i, ctypes.c_int, d, d, d, d]
        _lib.or_md_npt_species.argtypes = [d, ctypes.c_int, i, ctypes.c_int, d, d, d, ctypes.c_double,
                                           ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                           ctypes.c_double, ctypes.c_int, d, d]
        _lib.or_md_species.argtypes = [d, ctypes.c_int, i, ctypes.c_int, d, d, d, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int, d, d]
        _lib.or_energy_param_grad.argtypes = [d, ctypes.c_int, d, d, d]
        ll = ctypes.POINTER(ctypes.c_longlong)
        _lib.or_pair_histogram.argtypes = [ctypes.c_int, d, d, ctypes.c_double, ctypes.c_int, ctypes.c_double, ll, ll]
        _lib.or_angle_histogram.argtypes = [ctypes.c_int, d, d, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                            ctypes.c_double, ll, ll, ll]
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def default_params() -> np.ndarray:
    p = np.zeros(10)
    lib().or_params_default(_dp(p))
    return p


def params(**kw) -> np.ndarray:
    p = default_params()
    for k, v in kw.items():
        p[PARAM_NAMES.index(k)] = v
    return p


def phi2(r, prm=None):
    prm = default_params() if prm is None else np.ascontiguousarray(prm, np.float64)
    return np.array([lib().or_phi2(_dp(prm), float(x)) for x in np.atleast_1d(r)])


def dphi2(r, prm=None):
    prm = default_params() if prm is None else np.ascontiguousarray(prm, np.float64)
    return np.array([lib().or_dphi2(_dp(prm), float(x)) for x in np.atleast_1d(r)])


def phi3(r, s, cos_t, prm=None):
    prm = default_params() if prm is None else np.ascontiguousarray(prm, np.float64)
    return lib().or_phi3(_dp(prm), float(r), float(s), float(cos_t))


def _check(rc, what):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with code {rc}")


def energy_forces(x, box, prm=None, method="cell", threads=1):
    """Returns dict(e2, e3, energy, forces (n,3), virial[6], npairs, ntriplets,
    virial_abs): virial_abs is the summed magnitude of the diagonal virial
    contributions, the scale against which the (cancelling) trace is judged.
    method: "cell" (cell-list owner loop), "brute" (all pairs / triplets) or
    "owner" (owner-computes on `threads` threads)."""
    prm = default_params() if prm is None else np.ascontiguousarray(prm, np.float64)
    x = np.ascontiguousarray(x, np.float64).reshape(-1, 3)
    box = np.ascontiguousarray(box, np.float64)
    n = x.shape[0]
    f = np.zeros((n, 3))
    out = np.zeros(11)
    if method == "owner":
        rc = lib().or_energy_forces_owner(_dp(prm), n, _dp(x), _dp(box), _dp(f), _dp(out), int(threads))
    else:
        fn = lib().or_energy_forces_cell if method == "cell" else lib().or_energy_forces_brute
        rc = fn(_dp(prm), n, _dp(x), _dp(box), _dp(f), _dp(out))
    _check(rc, "energy_forces")
    return dict(e2=out[0], e3=out[1], energy=out[0] + out[1], forces=f, virial=out[2:8].copy(),
                npairs=int(out[8]), ntriplets=int(out[9]), virial_abs=out[10])


def neighbors(x, box, rlist, band_rel=1e-5, width=256, band_cap=100000):
    """Returns (sets, band) with sets[i] a sorted int array and band a set of (i, j)."""
    x = np.ascontiguousarray(x, np.float64).reshape(-1, 3)
    box = np.ascontiguousarray(box, np.float64)
    n = x.shape[0]
    counts = np.zeros(n, np.int32)
    nbr = np.zeros((n, width), np.int32)
    band = np.zeros((band_cap, 2), np.int32)
    nband = np.zeros(1, np.int32)
    rc = lib().or_neighbors(n, _dp(x), _dp(box), float(rlist), float(band_rel), width, _ip(counts),
                            _ip(nbr), band_cap, _ip(band), _ip(nband))
    _check(rc, "neighbors")
    sets = [nbr[i, :counts[i]].copy() for i in range(n)]
    nb = min(int(nband[0]), band_cap)
    return sets, {(int(a), int(b)) for a, b in band[:nb]}


def neighbors_raw(x, box, rlist, band_rel=1e-5, width=128, band_cap=1000000):
    """neighbors() as padded arrays: (counts[n], nbr[n, width] sorted rows,
    band set of (i, j)); raises if a row is wider than width."""
    x = np.ascontiguousarray(x, np.float64).reshape(-1, 3)
    box = np.ascontiguousarray(box, np.float64)
    n = x.shape[0]
    counts = np.zeros(n, np.int32)
    nbr = np.zeros((n, width), np.int32)
    band = np.zeros((band_cap, 2), np.int32)
    nband = np.zeros(1, np.int32)
    rc = lib().or_neighbors(n, _dp(x), _dp(box), float(rlist), float(band_rel), width, _ip(counts),
                            _ip(nbr), band_cap, _ip(band), _ip(nband))
    _check(rc, "neighbors")
    nb = min(int(nband[0]), band_cap)
    return counts, nbr, {(int(a), int(b)) for a, b in band[:nb]}


def md(x, v, box, nsteps, dt=10.0, kind=0, T0=300.0, tau=1000.0, mass=18.015, prm=None, state=(0.0, 0.0),
       threads=0):
    """Runs the oracle's velocity-Verlet; returns (x, v, state, thermo[nsteps+1, 8]).

    thermo columns: pe, e2, e3, ke, T, conserved, xi, eta.  kind: 0 NVE,
    1 Berendsen, 2 Nose-Hoover.  threads > 0: owner-computes forces and
    threaded loops on that many threads (the multi-core CPU baseline)."""
    prm = default_params() if prm is None else np.ascontiguousarray(prm, np.float64)
    x = np.array(x, np.float64).reshape(-1, 3)
    v = np.array(v, np.float64).reshape(-1, 3)
    box = np.ascontiguousarray(box, np.float64)
    st = np.array(state, np.float64)
    th = np.zeros((nsteps + 1, 8))
    if threads > 0:
        rc = lib().or_md_owner(_dp(prm), x.shape[0], _dp(x), _dp(v), _dp(box), mass, dt, kind, T0, tau, nsteps,
                               _dp(st), _dp(th), int(threads))
    else:
        rc = lib().or_md(_dp(prm), x.shape[0], _dp(x), _dp(v), _dp(box), mass, dt, kind, T0, tau, nsteps,
                         _dp(st), _dp(th))
    _check(rc, "md")
    return x, v, (float(st[0]), float(st[1])), th


# kcal/mol per A^3 in atm (101325 Pa per atm)
KCAL_PER_A3_ATM = 4184.0 / 6.02214076e23 / 1e-30 / 101325.0


def md_npt(x, v, box, nsteps, dt=10.0, T0=298.0, tau=1000.0, p_atm=0.0, tau_p=2500.0, mass=18.015, prm=None,
           state=(0.0, 0.0, 0.0)):
    """Isobaric-isothermal run (Nose-Hoover thermostat and isotropic barostat,
    Martyna-Tobias-Klein split); returns (x, v, box, state, thermo[nsteps+1, 10]).

    thermo columns: pe, e2, e3, ke, T, conserved, xi, eta, V (A^3), P (kcal/mol/A^3)."""
    prm = default_params() if prm is None else np.ascontiguousarray(prm, np.float64)
    x = np.array(x, np.float64).reshape(-1, 3)
    v = np.array(v, np.float64).reshape(-1, 3)
    box = np.array(box, np.float64)
    st = np.array(state, np.float64)
    th = np.zeros((nsteps + 1, 10))
    _check(lib().or_md_npt(_dp(prm), x.shape[0], _dp(x), _dp(v), _dp(box), mass, dt, T0, tau,
                           p_atm / KCAL_PER_A3_ATM, tau_p, nsteps, _dp(st), _dp(th)), "md_npt")
    return x, v, box, (float(st[0]), float(st[1]), float(st[2])), th


def force_vjp(x, box, w, prm=None):
    """Returns (dL/dx (n,3), dL/d(lambda, epsilon, sigma)) for dL/dF = w."""
    prm = default_params() if prm is None else np.ascontiguousarray(prm, np.float64)
    x = np.ascontiguousarray(x, np.float64).reshape(-1, 3)
    w = np.ascontiguousarray(w, np.float64).reshape(-1, 3)
    box = np.ascontiguousarray(box, np.float64)
    gx = np.zeros_like(x)
    gt = np.zeros(3)
    _check(lib().or_force_vjp(_dp(prm), x.shape[0], _dp(x), _dp(box), _dp(w), _dp(gx), _dp(gt)), "force_vjp")
    return gx, gt


def energy_param_grad(x, box, prm=None):
    prm = default_params() if prm is None else np.ascontiguousarray(prm, np.float64)
    x = np.ascontiguousarray(x, np.float64).reshape(-1, 3)
    box = np.ascontiguousarray(box, np.float64)
    g = np.zeros(3)
    _check(lib().or_energy_param_grad(_dp(prm), x.shape[0], _dp(x), _dp(box), _dp(g)), "energy_param_grad")
    return g


def _llp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong))


def pair_histogram(x, box, dr, nbins, rel=1e-5):
    """Sec. II.C: ordered pairs i != j by minimum-image distance bin (the raw
    histogram behind g(r)); also the pairs within rel of a bin edge, per bin."""
    x = np.ascontiguousarray(x, np.float64)
    box = np.ascontiguousarray(box, np.float64)
    h = np.zeros(nbins, np.int64)
    a = np.zeros(nbins, np.int64)
    _check(lib().or_pair_histogram(len(x), _dp(x), _dp(box), float(dr), int(nbins), float(rel), _llp(h), _llp(a)),
           "or_pair_histogram")
    return h, a


def angle_histogram(x, box, nc=8, nbins=180, tol_deg=1e-3, rel=1e-5):
    """Sec. II.C: angles theta_ikj at each atom k over ordered pairs of its nc
    nearest neighbours, binned over [0, 180] degrees; also the angles within
    tol_deg of a bin edge, per bin, and the number of atoms whose nc-th
    neighbour is within rel of the next (an ambiguous selection)."""
    x = np.ascontiguousarray(x, np.float64)
    box = np.ascontiguousarray(box, np.float64)
    h = np.zeros(nbins, np.int64)
    a = np.zeros(nbins, np.int64)
    t = np.zeros(1, np.int64)
    _check(lib().or_angle_histogram(len(x), _dp(x), _dp(box), int(nc), int(nbins), float(tol_deg), float(rel),
                                    _llp(h), _llp(a), _llp(t)), "or_angle_histogram")
    return h, a, int(t[0])


def species_table(nt, entry):
    """nt^3 parameter vectors from entry(a, b, c) -> parameter vector (or dict of overrides)."""
    t = np.zeros((nt, nt, nt, 10))
    for a in range(nt):
        for b in range(nt):
            for c in range(nt):
                e = entry(a, b, c)
                t[a, b, c] = params(**e) if isinstance(e, dict) else np.asarray(e, np.float64)
    return t


def species_table_ok(table) -> bool:
    t = np.ascontiguousarray(table, np.float64)
    return lib().or_species_table_check(_dp(t), t.shape[0]) == 0


def energy_forces_species(x, box, types, table):
    """Several species (brute force): same dict as energy_forces."""
    t = np.ascontiguousarray(table, np.float64)
    x = np.ascontiguousarray(x, np.float64).reshape(-1, 3)
    box = np.ascontiguousarray(box, np.float64)
    ty = np.ascontiguousarray(types, np.int32)
    n = x.shape[0]
    f = np.zeros((n, 3))
    out = np.zeros(11)
    _check(lib().or_energy_forces_species(_dp(t), t.shape[0], _ip(ty), n, _dp(x), _dp(box), _dp(f), _dp(out)),
           "energy_forces_species")
    return {"e2": out[0], "e3": out[1], "energy": out[0] + out[1], "forces": f, "virial": out[2:8].copy(),
            "npairs": int(out[8]), "ntriplets": int(out[9]), "virial_abs": out[10]}


def md_species(x, v, box, types, table, nsteps, dt=10.0, kind=0, T0=300.0, tau=1000.0, mass=18.015,
               state=(0.0, 0.0)):
    """md() with the several-species potential; returns (x, v, state, thermo[nsteps+1, 8])."""
    t = np.ascontiguousarray(table, np.float64)
    ty = np.ascontiguousarray(types, np.int32)
    x = np.array(x, np.float64).reshape(-1, 3)
    v = np.array(v, np.float64).reshape(-1, 3)
    box = np.ascontiguousarray(box, np.float64)
    st = np.array(state, np.float64)
    th = np.zeros((nsteps + 1, 8))
    _check(lib().or_md_species(_dp(t), t.shape[0], _ip(ty), x.shape[0], _dp(x), _dp(v), _dp(box), mass, dt, kind,
                               T0, tau, nsteps, _dp(st), _dp(th)), "md_species")
    return x, v, (float(st[0]), float(st[1])), th


def md_npt_species(x, v, box, types, table, nsteps, dt=10.0, T0=298.0, tau=1000.0, p_atm=0.0, tau_p=2500.0,
                   mass=18.015, state=(0.0, 0.0, 0.0)):
    """md_npt() with the several-species potential; same returns."""
    t = np.ascontiguousarray(table, np.float64)
    ty = np.ascontiguousarray(types, np.int32)
    x = np.array(x, np.float64).reshape(-1, 3)
    v = np.array(v, np.float64).reshape(-1, 3)
    box = np.array(box, np.float64)
    st = np.array(state, np.float64)
    th = np.zeros((nsteps + 1, 10))
    _check(lib().or_md_npt_species(_dp(t), t.shape[0], _ip(ty), x.shape[0], _dp(x), _dp(v), _dp(box), mass, dt,
                                   T0, tau, p_atm / KCAL_PER_A3_ATM, tau_p, nsteps, _dp(st), _dp(th)),
           "md_npt_species")
    return x, v, box, (float(st[0]), float(st[1]), float(st[2])), th

"""Thin Python binding of libmw (include/mw.h): same names, argument marshalling only.

Every computation runs in the CUDA library; this module converts numpy arrays
or torch tensors to pointers and raises MWError on a non-zero mw_status.
There is no CPU fallback: if libmw.so is missing or cannot reach a GPU the
calls raise.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmw.so")

(MW_OK, MW_EINVAL, MW_EBOX, MW_ENLIST_OVERFLOW, MW_ENAN, MW_ELOST, MW_ETIMEOUT, MW_ECUDA, MW_ENOMEM, MW_ESTATE,
 MW_EGRID) = range(11)
STATUS_NAMES = {0: "MW_OK", 1: "MW_EINVAL", 2: "MW_EBOX", 3: "MW_ENLIST_OVERFLOW", 4: "MW_ENAN", 5: "MW_ELOST",
                6: "MW_ETIMEOUT", 7: "MW_ECUDA", 8: "MW_ENOMEM", 9: "MW_ESTATE", 10: "MW_EGRID"}
MW_NVE, MW_BERENDSEN, MW_NOSE_HOOVER, MW_NPT = 0, 1, 2, 3
MW_ENGINE_AUTO, MW_ENGINE_GRAPH, MW_ENGINE_PERSISTENT, MW_ENGINE_PLAIN = 0, 1, 2, 3

# every symbol include/mw.h declares
EXPORTS = (
    "mw_params_default", "mw_system_create", "mw_batch_create", "mw_system_destroy", "mw_set_state",
    "mw_set_state_dev", "mw_get_state", "mw_get_state_dev", "mw_set_params", "mw_build_neighbors",
    "mw_get_neighbors", "mw_energy_forces", "mw_energy_forces_dev", "mw_step", "mw_get_thermo",
    "mw_energy_forces_vjp", "mw_set_engine", "mw_set_nbr_width", "mw_autotune", "mw_get_info",
    "mw_set_count_terms", "mw_forces_async", "mw_step_async", "mw_sync", "mw_energy_forces_noalloc", "mw_set_skin", "mw_set_force_shape", "mw_phase_times",
    "mw_pair_histogram", "mw_angle_histogram", "mw_get_unwrapped", "mw_get_box", "mw_set_species",
    "mw_checkpoint_size", "mw_checkpoint_save", "mw_checkpoint_load", "mw_set_wait_limit",
    "mw_set_phase_marks", "mw_get_phase_marks", "mw_last_error",
)


class mw_params(ctypes.Structure):
    _fields_ = [("lambda_", ctypes.c_double), ("epsilon", ctypes.c_double), ("sigma", ctypes.c_double),
                ("a", ctypes.c_double), ("gamma", ctypes.c_double), ("A", ctypes.c_double),
                ("B", ctypes.c_double), ("cos_theta0", ctypes.c_double), ("p", ctypes.c_int),
                ("q", ctypes.c_int)]


class mw_integrator(ctypes.Structure):
    _fields_ = [("dt", ctypes.c_double), ("thermostat", ctypes.c_int), ("T0", ctypes.c_double),
                ("T0_per_box", ctypes.POINTER(ctypes.c_double)), ("tau", ctypes.c_double),
                ("p_ext", ctypes.c_double), ("tau_p", ctypes.c_double)]


class mw_thermo(ctypes.Structure):
    _fields_ = [("step", ctypes.c_int64), ("pe", ctypes.c_double), ("e2", ctypes.c_double),
                ("e3", ctypes.c_double), ("ke", ctypes.c_double), ("temperature", ctypes.c_double),
                ("conserved", ctypes.c_double), ("pressure", ctypes.c_double),
                ("virial", ctypes.c_double * 6), ("xi", ctypes.c_double), ("eta", ctypes.c_double),
                ("rebuilds", ctypes.c_int64), ("volume", ctypes.c_double), ("box", ctypes.c_double * 3)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_ if k not in ("virial", "box")}
        d["virial"] = list(self.virial)
        d["box"] = list(self.box)
        return d


class mw_info(ctypes.Structure):
    _fields_ = [("nbox", ctypes.c_int), ("n_total", ctypes.c_int), ("nbr_width", ctypes.c_int),
                ("max_count", ctypes.c_int), ("ncell_total", ctypes.c_int), ("engine", ctypes.c_int),
                ("persistent_blocks", ctypes.c_int), ("persistent_threads", ctypes.c_int),
                ("r_list", ctypes.c_double), ("npairs", ctypes.c_int64), ("ntriplets", ctypes.c_int64),
                ("rebuild_steps", ctypes.c_int64), ("regrids", ctypes.c_int64), ("species", ctypes.c_int),
                ("species_moments", ctypes.c_int), ("force_lanes", ctypes.c_int), ("force_blocks_per_sm", ctypes.c_int),
                ("force_owner", ctypes.c_int), ("pad_", ctypes.c_int)]


class MWError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None


def lib():
    """Loads libmw.so (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libmw.so not built ({LIB_PATH}); run paper_0809_2811_gb300/build.py")
        L = ctypes.CDLL(LIB_PATH)
        P = ctypes.c_void_p
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        sig = {
            "mw_params_default": [ctypes.POINTER(mw_params)],
            "mw_system_create": [ctypes.POINTER(P), ctypes.c_int, dp, ctypes.POINTER(mw_params), ctypes.c_double,
                                 ctypes.c_double, P],
            "mw_batch_create": [ctypes.POINTER(P), ctypes.c_int, ip, dp, ctypes.POINTER(mw_params), ctypes.c_double,
                                ctypes.c_double, P],
            "mw_system_destroy": [P],
            "mw_set_state": [P, dp, dp],
            "mw_set_state_dev": [P, P, P],
            "mw_get_state": [P, dp, dp],
            "mw_get_state_dev": [P, P, P],
            "mw_set_params": [P, ctypes.POINTER(mw_params)],
            "mw_build_neighbors": [P, ip],
            "mw_get_neighbors": [P, ip, ip, ctypes.c_int],
            "mw_energy_forces": [P, dp, dp, dp],
            "mw_energy_forces_dev": [P, P, P, P, P],
            "mw_step": [P, ctypes.POINTER(mw_integrator), ctypes.c_int, ctypes.POINTER(mw_thermo)],
            "mw_get_thermo": [P, ctypes.POINTER(mw_thermo)],
            "mw_energy_forces_vjp": [P, P, P, dp],
            "mw_set_engine": [P, ctypes.c_int],
            "mw_set_nbr_width": [P, ctypes.c_int],
            "mw_autotune": [P, ctypes.POINTER(mw_integrator), ctypes.c_int, ip],
            "mw_get_info": [P, ctypes.POINTER(mw_info)],
            "mw_set_count_terms": [P, ctypes.c_int],
            "mw_forces_async": [P],
            "mw_step_async": [P, ctypes.POINTER(mw_integrator), ctypes.c_int],
            "mw_sync": [P],
            "mw_set_skin": [P, ctypes.c_double],
            "mw_set_force_shape": [P, ctypes.c_int, ctypes.c_int, ctypes.c_int],
            "mw_phase_times": [P, ctypes.POINTER(mw_integrator), ctypes.c_int, dp],
            "mw_pair_histogram": [P, ctypes.c_double, ctypes.c_int, ctypes.POINTER(ctypes.c_ulonglong)],
            "mw_get_unwrapped": [P, dp],
            "mw_get_box": [P, dp],
            "mw_checkpoint_size": [P, ctypes.POINTER(ctypes.c_size_t)],
            "mw_set_wait_limit": [P, ctypes.c_double],
            "mw_set_phase_marks": [P, ctypes.c_int],
            "mw_get_phase_marks": [P, ctypes.POINTER(ctypes.c_ulonglong), ctypes.c_int],
            "mw_checkpoint_save": [P, P, ctypes.c_size_t],
            "mw_checkpoint_load": [P, P, ctypes.c_size_t],
            "mw_set_species": [P, ctypes.c_int, ctypes.POINTER(mw_params), ip],
            "mw_angle_histogram": [P, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_ulonglong)],
            "mw_energy_forces_noalloc": [ctypes.c_int, dp, ctypes.POINTER(mw_params), ctypes.c_double, P, P, P, P,
                                         P],
        }
        for name, args in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = ctypes.c_int
        L.mw_last_error.argtypes = []
        L.mw_last_error.restype = ctypes.c_char_p
        _lib = L
    return _lib


def _check(st: int):
    if st != MW_OK:
        raise MWError(st, lib().mw_last_error().decode())


def _dp(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def _ptr(t) -> Optional[int]:
    """Device pointer of a torch tensor (or an int), None for None."""
    if t is None:
        return None
    if isinstance(t, int):
        return t
    return t.data_ptr()


# ----------------------------------------------------------------- C names

def mw_params_default() -> mw_params:
    p = mw_params()
    _check(lib().mw_params_default(ctypes.byref(p)))
    return p


def mw_system_create(n: int, box, prm: Optional[mw_params] = None, mass: float = 18.015, skin: float = 1.0,
                     stream: Optional[int] = None) -> int:
    prm = prm or mw_params_default()
    b = np.ascontiguousarray(box, np.float64)
    h = ctypes.c_void_p()
    _check(lib().mw_system_create(ctypes.byref(h), int(n), _dp(b), ctypes.byref(prm), mass, skin, stream))
    return h.value


def mw_batch_create(n: Sequence[int], box, prm: Optional[mw_params] = None, mass: float = 18.015,
                    skin: float = 1.0, stream: Optional[int] = None) -> int:
    prm = prm or mw_params_default()
    nn = np.ascontiguousarray(n, np.int32)
    b = np.ascontiguousarray(box, np.float64).reshape(-1, 3)
    h = ctypes.c_void_p()
    _check(lib().mw_batch_create(ctypes.byref(h), len(nn), _ip(nn), _dp(b), ctypes.byref(prm), mass, skin, stream))
    return h.value


def mw_system_destroy(h: int):
    _check(lib().mw_system_destroy(h))


def mw_set_state(h: int, x, v=None):
    x = np.ascontiguousarray(x, np.float64)
    v = None if v is None else np.ascontiguousarray(v, np.float64)
    _check(lib().mw_set_state(h, _dp(x), _dp(v)))


def mw_set_state_dev(h: int, x_dev, v_dev=None):
    _check(lib().mw_set_state_dev(h, _ptr(x_dev), _ptr(v_dev)))


def mw_get_state(h: int, n_total: int, x_out: Optional[np.ndarray] = None, v_out: Optional[np.ndarray] = None):
    """Positions and velocities (n_total, 3) into new arrays, or into the given
    C-contiguous float64 arrays (e.g. page-locked ones)."""
    x = np.empty((n_total, 3)) if x_out is None else x_out
    v = np.empty((n_total, 3)) if v_out is None else v_out
    for a in (x, v):
        if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"] or a.size != 3 * n_total:
            raise ValueError("state outputs must be C-contiguous float64 arrays of n_total x 3")
    _check(lib().mw_get_state(h, _dp(x), _dp(v)))
    return x, v


def mw_get_state_dev(h: int, x_dev=None, v_dev=None):
    _check(lib().mw_get_state_dev(h, _ptr(x_dev), _ptr(v_dev)))


def mw_set_params(h: int, prm: mw_params):
    _check(lib().mw_set_params(h, ctypes.byref(prm)))


def mw_build_neighbors(h: int) -> int:
    m = ctypes.c_int()
    _check(lib().mw_build_neighbors(h, ctypes.byref(m)))
    return m.value


def mw_get_neighbors(h: int, n_total: int, width: int):
    counts = np.zeros(n_total, np.int32)
    nbr = np.full((n_total, width), -1, np.int32)
    _check(lib().mw_get_neighbors(h, _ip(counts), _ip(nbr), width))
    return counts, nbr


def mw_energy_forces(h: int, n_total: int, nbox: int):
    f = np.empty((n_total, 3))
    e = np.empty((nbox, 3))
    w = np.empty((nbox, 6))
    _check(lib().mw_energy_forces(h, _dp(f), _dp(e), _dp(w)))
    return f, e, w


def mw_energy_forces_dev(h: int, x_dev=None, f_dev=None, energy_dev=None, virial_dev=None):
    _check(lib().mw_energy_forces_dev(h, _ptr(x_dev), _ptr(f_dev), _ptr(energy_dev), _ptr(virial_dev)))


MW_MAX_SPECIES = 8
PARAM_FIELDS = ("lambda_", "epsilon", "sigma", "a", "gamma", "A", "B", "cos_theta0", "p", "q")


def species_params(table) -> "ctypes.Array":
    """nt^3 mw_params from an (nt, nt, nt, 10) array whose last axis is
    (lambda, epsilon, sigma, a, gamma, A, B, cos_theta0, p, q), or from a
    flat sequence of mw_params in (a nt + b) nt + c order."""
    if isinstance(table, np.ndarray):
        t = np.asarray(table, np.float64)
        nt = t.shape[0]
        assert t.shape == (nt, nt, nt, 10), t.shape
        arr = (mw_params * (nt ** 3))()
        for k, row in enumerate(t.reshape(-1, 10)):
            for f, v in zip(PARAM_FIELDS, row):
                setattr(arr[k], f, int(v) if f in ("p", "q") else float(v))
        return arr
    arr = (mw_params * len(table))()
    for k, e in enumerate(table):
        arr[k] = e
    return arr


def mw_set_species(h: int, table, types):
    arr = species_params(table)
    nt = int(round(len(arr) ** (1.0 / 3.0)))
    ty = np.ascontiguousarray(types, np.int32) if types is not None else None
    _check(lib().mw_set_species(h, nt, arr, ty.ctypes.data_as(ctypes.POINTER(ctypes.c_int)) if ty is not None
                                else None))


THERMO_COLUMNS = (("Step", "step", "{:>10d}"), ("Temp", "temperature", "{:>10.3f}"), ("PotEng", "pe", "{:>14.4f}"),
                  ("KinEng", "ke", "{:>12.4f}"), ("TotEng", None, "{:>14.4f}"), ("Press", "pressure", "{:>11.2f}"),
                  ("Econs", "conserved", "{:>14.4f}"), ("Volume", "volume", "{:>12.2f}"),
                  ("Rebuilds", "rebuilds", "{:>9d}"))


def thermo_header() -> str:
    """Column names of thermo_line (LAMMPS-style)."""
    return " ".join("{:>%d}" % len(f.format(0 if "d" in f else 0.0)) for _, _, f in THERMO_COLUMNS).format(
        *[c for c, _, _ in THERMO_COLUMNS])


def thermo_line(rec: dict) -> str:
    """One LAMMPS-style thermo line of a record (mw_thermo as a dict); TotEng = KinEng + PotEng."""
    vals = []
    for _, key, f in THERMO_COLUMNS:
        v = rec["ke"] + rec["pe"] if key is None else rec[key]
        vals.append(f.format(int(v) if "d" in f else float(v)))
    return " ".join(vals)


def make_integrator(dt=10.0, thermostat=MW_NVE, T0=300.0, tau=1000.0, T0_per_box=None, p_ext=1.0,
                    tau_p=5000.0):
    """tau, tau_p in fs; p_ext in atm (MW_NPT only)."""
    it = mw_integrator()
    it.dt = dt
    it.thermostat = thermostat
    it.T0 = T0
    it.tau = tau
    it.p_ext = p_ext
    it.tau_p = tau_p
    if T0_per_box is not None:
        arr = np.ascontiguousarray(T0_per_box, np.float64)
        it._keep = arr
        it.T0_per_box = _dp(arr)
    return it


def mw_step(h: int, integ: mw_integrator, nsteps: int, nbox: int = 1):
    th = (mw_thermo * nbox)()
    _check(lib().mw_step(h, ctypes.byref(integ), int(nsteps), th))
    return [t.as_dict() for t in th]


def mw_get_thermo(h: int, nbox: int = 1):
    th = (mw_thermo * nbox)()
    _check(lib().mw_get_thermo(h, th))
    return [t.as_dict() for t in th]


def mw_energy_forces_vjp(h: int, dL_dF_dev, dL_dx_dev, nbox: int = 1):
    g = np.zeros((nbox, 3))
    _check(lib().mw_energy_forces_vjp(h, _ptr(dL_dF_dev), _ptr(dL_dx_dev), _dp(g)))
    return g


def mw_set_engine(h: int, engine: int):
    _check(lib().mw_set_engine(h, engine))


def mw_set_nbr_width(h: int, width: int):
    _check(lib().mw_set_nbr_width(h, width))


def mw_autotune(h: int, integ: mw_integrator, steps: int = 50) -> int:
    e = ctypes.c_int()
    _check(lib().mw_autotune(h, ctypes.byref(integ), steps, ctypes.byref(e)))
    return e.value


def mw_get_info(h: int) -> dict:
    i = mw_info()
    _check(lib().mw_get_info(h, ctypes.byref(i)))
    return {k: getattr(i, k) for k, _ in i._fields_}


def mw_set_count_terms(h: int, on: bool):
    _check(lib().mw_set_count_terms(h, 1 if on else 0))


def mw_forces_async(h: int):
    _check(lib().mw_forces_async(h))


def mw_step_async(h: int, integ: mw_integrator, nsteps: int):
    _check(lib().mw_step_async(h, ctypes.byref(integ), int(nsteps)))


def mw_sync(h: int):
    _check(lib().mw_sync(h))


def mw_energy_forces_noalloc(n: int, box, x_dev, f_dev=None, energy_dev=None, virial_dev=None,
                             prm: Optional[mw_params] = None, skin: float = 1.0, stream: Optional[int] = None):
    """Energy/forces of one box without any device allocation (see mw.h)."""
    prm = prm or mw_params_default()
    b = np.ascontiguousarray(box, np.float64)
    _check(lib().mw_energy_forces_noalloc(int(n), _dp(b), ctypes.byref(prm), skin, _ptr(x_dev), _ptr(f_dev),
                                          _ptr(energy_dev), _ptr(virial_dev), stream))


def mw_set_skin(h: int, skin: float):
    _check(lib().mw_set_skin(h, float(skin)))


def mw_set_force_shape(h: int, lanes_per_centre: int, blocks_per_sm: int, owner_computes: bool = False):
    """Launch shape of the per-phase force kernel: scatter 4/8, 2/8, 8/8, 4/7 or
    owner-computes 4/8."""
    _check(lib().mw_set_force_shape(h, int(lanes_per_centre), int(blocks_per_sm), int(bool(owner_computes))))


PHASES = ("kick1", "bin", "scan", "scatter", "copyback", "neigh", "force", "kick2")


def mw_phase_times(h: int, integ: mw_integrator, nsteps: int) -> dict:
    out = np.zeros(8)
    _check(lib().mw_phase_times(h, ctypes.byref(integ), int(nsteps), _dp(out)))
    return dict(zip(PHASES, out.tolist()))


def mw_pair_histogram(h: int, nbox: int, dr: float, nbins: int) -> np.ndarray:
    """Per box, ordered pairs by distance bin (the raw count behind g(r)); uint64 [nbox, nbins]."""
    out = np.zeros((nbox, nbins), np.uint64)
    _check(lib().mw_pair_histogram(h, float(dr), int(nbins), out.ctypes.data_as(ctypes.POINTER(ctypes.c_ulonglong))))
    return out


def mw_angle_histogram(h: int, nbox: int, nc: int, nbins: int) -> np.ndarray:
    """Per box, angles at each atom between ordered pairs of its nc nearest
    neighbours, over [0, 180] degrees; uint64 [nbox, nbins]."""
    out = np.zeros((nbox, nbins), np.uint64)
    _check(lib().mw_angle_histogram(h, int(nc), int(nbins), out.ctypes.data_as(ctypes.POINTER(ctypes.c_ulonglong))))
    return out


def mw_last_error() -> str:
    return lib().mw_last_error().decode()


# ----------------------------------------------------------------- convenience

class System:
    """One box (n atoms, box[3]) or a batch (n = list, box = [nbox, 3]) on the GPU."""

    def __init__(self, n, box, prm: Optional[mw_params] = None, mass: float = 18.015, skin: float = 1.0,
                 stream: Optional[int] = None):
        if np.ndim(n) == 0:
            self.nbox = 1
            self.n = [int(n)]
            self.h = mw_system_create(int(n), box, prm, mass, skin, stream)
        else:
            self.nbox = len(n)
            self.n = [int(k) for k in n]
            self.h = mw_batch_create(n, box, prm, mass, skin, stream)
        self.n_total = int(sum(self.n))

    def close(self):
        if self.h:
            mw_system_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_state(self, x, v=None):
        mw_set_state(self.h, x, v)

    def get_state(self, x_out=None, v_out=None):
        return mw_get_state(self.h, self.n_total, x_out, v_out)

    def energy_forces(self):
        return mw_energy_forces(self.h, self.n_total, self.nbox)

    def build_neighbors(self):
        return mw_build_neighbors(self.h)

    def neighbors(self, width: int = 128):
        return mw_get_neighbors(self.h, self.n_total, width)

    def step(self, nsteps: int, dt=10.0, thermostat=MW_NVE, T0=300.0, tau=1000.0, T0_per_box=None, p_ext=1.0,
             tau_p=5000.0):
        it = make_integrator(dt, thermostat, T0, tau, T0_per_box, p_ext, tau_p)
        return mw_step(self.h, it, nsteps, self.nbox)

    def set_species(self, table, types):
        """Several species: table (nt, nt, nt, 10) or nt^3 mw_params, types per atom (caller's order)."""
        mw_set_species(self.h, table, types)

    def set_phase_marks(self, cap: int):
        """Record the persistent engine's phase marks for the first cap steps of each launch (0: off)."""
        _check(lib().mw_set_phase_marks(self.h, int(cap)))

    def phase_marks(self, cap: int) -> np.ndarray:
        """SM-clock marks (cycles) of the last persistent launch: [cap, 16] (see mw_set_phase_marks)."""
        out = np.zeros((cap, 16), np.uint64)
        _check(lib().mw_get_phase_marks(self.h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_ulonglong)), int(cap)))
        return out

    def set_wait_limit(self, seconds: float):
        """Limit of each device-side wait of the persistent engine (MW_ETIMEOUT past it)."""
        _check(lib().mw_set_wait_limit(self.h, float(seconds)))

    def checkpoint(self) -> bytes:
        """The exact engine state as bytes (mw_checkpoint_save)."""
        n = ctypes.c_size_t()
        _check(lib().mw_checkpoint_size(self.h, ctypes.byref(n)))
        buf = ctypes.create_string_buffer(n.value)
        _check(lib().mw_checkpoint_save(self.h, buf, n.value))
        return buf.raw

    def restore(self, blob: bytes):
        """Continues from a checkpoint taken on a system of the same make (mw_checkpoint_load)."""
        buf = ctypes.create_string_buffer(blob, len(blob))
        _check(lib().mw_checkpoint_load(self.h, buf, len(blob)))

    def run(self, nsteps: int, every: int = 100, log=print, **integ):
        """nsteps steps with a thermo line per box every `every` steps (and the
        header first); returns the last records."""
        log(thermo_header())
        th = self.thermo()
        for t in th:
            log(thermo_line(t))
        done = 0
        while done < nsteps:
            k = min(every, nsteps - done)
            th = self.step(k, **integ)
            done += k
            for t in th:
                log(thermo_line(t))
        return th

    def box(self) -> np.ndarray:
        """Current edges of every box (nbox x 3, A); they change under MW_NPT."""
        b = np.empty((self.nbox, 3))
        _check(lib().mw_get_box(self.h, _dp(b)))
        return b

    def thermo(self):
        return mw_get_thermo(self.h, self.nbox)

    def get_unwrapped(self) -> np.ndarray:
        """Positions plus the periodic images crossed since set_state (n_total x 3, A)."""
        x = np.empty((self.n_total, 3))
        _check(lib().mw_get_unwrapped(self.h, _dp(x)))
        return x

    def pair_histogram(self, dr: float, nbins: int) -> np.ndarray:
        return mw_pair_histogram(self.h, self.nbox, dr, nbins)

    def angle_histogram(self, nc: int = 8, nbins: int = 180) -> np.ndarray:
        return mw_angle_histogram(self.h, self.nbox, nc, nbins)

    def info(self):
        return mw_get_info(self.h)

    def set_engine(self, engine: int):
        mw_set_engine(self.h, engine)

    def set_params(self, prm: mw_params):
        mw_set_params(self.h, prm)

    def set_count_terms(self, on: bool):
        mw_set_count_terms(self.h, on)

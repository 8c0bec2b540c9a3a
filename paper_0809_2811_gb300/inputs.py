"""Seeded synthetic inputs for the mW engine and its oracle.

This module holds geometry and random numbers only, none of the model's
arithmetic; the oracle and the CUDA path both read its arrays.  It imports
numpy alone.

Recipes (workloads of the paper's kind; there is no dataset to stand in for):
  * density -> volume per molecule: v = M / (N_A rho), M = 18.015 g/mol
    (Sec. II.C of the paper), so v = 29.9146 A^3 at 1 g/cm^3.
  * simple-cubic lattice with Gaussian jitter (the 512-atom NVE check:
    8^3 sites, L = 24.834 A at 1.000 g/cm^3, jitter 0.1 A).
  * ice Ih oxygen lattice = hexagonal diamond (Sec. II.C: ice without
    hydrogens is hexagonal / cubic diamond), orthorhombic 8-atom cell
    a x sqrt(3) a x sqrt(8/3) a; cubic diamond for ice Ic.
  * Maxwell velocities: Gaussian per component with variance kB T / m, centre
    of mass removed, rescaled to exactly T with Ndf = 3N - 3.
  * batches: N uniform in [216, 8000], density uniform in [0.92, 1.10] g/cm^3,
    T uniform in [200, 320] K, jittered simple-cubic start of
    n = ceil(N^(1/3)) sites per edge with N sites picked by a seeded
    permutation.
  * several species: parameter tables (nt, nt, nt, 10), entry (a, b, c) the
    set of centre a with legs to b and c, last axis (lambda, epsilon, sigma,
    a, gamma, A, B, cos theta0, p, q).  Three recipes: every pair and triplet
    different (seeded factors around the paper's mW values, the pair set
    shared by (a, b, b) and (b, a, a), the triplet set by (a, b, c) and
    (a, c, b)); mW with a solute that has two-body terms only; the SW family
    of Fig. 2 (lambda 20, 21, 23.15, 26.2) mixed by geometric means.
    Species are assigned to atoms by a seeded draw.
"""
from __future__ import annotations

import math

import numpy as np

M_WATER = 18.015  # g/mol, Sec. II.C
N_A = 6.02214076e23
KB = 0.0019872042586408316  # kcal/mol/K (exact SI R / 4184)
FCONV = 4.184e-4  # (kcal/mol/A)/(g/mol) -> A/fs^2
BASE_SEED = 20260101


def volume_per_molecule(rho: float) -> float:
    """A^3 per molecule at density rho (g/cm^3)."""
    return M_WATER / (N_A * rho) * 1e24


def cubic_box_edge(n: int, rho: float) -> float:
    return (n * volume_per_molecule(rho)) ** (1.0 / 3.0)


def simple_cubic(nside: int, L: float, jitter: float = 0.0, seed: int = 0) -> np.ndarray:
    s = L / nside
    g = np.arange(nside) * s
    x = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    if jitter > 0:
        x = x + np.random.default_rng(seed).normal(0.0, jitter, x.shape)
    return x


def diamond_cubic(ncell: int, rho: float):
    """Cubic diamond (ice Ic oxygens): 8 atoms per cube; returns (x, box)."""
    ac = (8 * volume_per_molecule(rho)) ** (1.0 / 3.0)
    basis = np.array([[0, 0, 0], [0, .5, .5], [.5, 0, .5], [.5, .5, 0]], float)
    basis = np.concatenate([basis, basis + 0.25])
    cells = np.stack(np.meshgrid(*[np.arange(ncell)] * 3, indexing="ij"), -1).reshape(-1, 1, 3)
    x = ((cells + basis[None]) * ac).reshape(-1, 3)
    return x, np.array([ncell * ac] * 3)


def ice_ih(nx: int, ny: int, nz: int, rho: float):
    """Hexagonal diamond (ice Ih oxygens), ideal c/a; returns (x, box).

    Orthorhombic cell a x sqrt(3) a x sqrt(8/3) a holding 8 atoms at the
    fractional positions below; nearest-neighbour spacing sqrt(3/8) a."""
    v = volume_per_molecule(rho)
    a = (2.0 * math.sqrt(2.0) * v) ** (1.0 / 3.0)  # 8 v = sqrt(3) a * a * sqrt(8/3) a
    cell = np.array([a, math.sqrt(3.0) * a, math.sqrt(8.0 / 3.0) * a])
    frac = np.array([
        [0.0, 1 / 3, 0.0], [0.5, 5 / 6, 0.0],
        [0.5, 1 / 6, 0.5], [0.0, 2 / 3, 0.5],
        [0.0, 1 / 3, 3 / 8], [0.5, 5 / 6, 3 / 8],
        [0.5, 1 / 6, 7 / 8], [0.0, 2 / 3, 7 / 8],
    ])
    idx = np.stack(np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij"), -1).reshape(-1, 1, 3)
    x = ((idx + frac[None]) * cell).reshape(-1, 3)
    return x, cell * np.array([nx, ny, nz])


def maxwell_velocities(n: int, T: float, mass: float = M_WATER, seed: int = 0) -> np.ndarray:
    """A/fs; exactly temperature T with 3N - 3 degrees of freedom."""
    rng = np.random.default_rng(seed)
    sd = math.sqrt(KB * T / mass * FCONV)
    v = rng.normal(0.0, sd, (n, 3))
    v -= v.mean(0)
    if T <= 0 or n < 2:
        return np.zeros((n, 3))
    ke = 0.5 * mass * (v * v).sum() / FCONV
    t_now = 2 * ke / ((3 * n - 3) * KB)
    return v * math.sqrt(T / t_now)


def snap_to_grid(x: np.ndarray, box) -> np.ndarray:
    """Rounds positions to the 2^-32 box-fraction grid (wrapped into [0, L))."""
    box = np.asarray(box, np.float64)
    xw = np.mod(x, box)
    q = np.rint(xw / box * 2.0 ** 32)
    q = np.mod(q, 2.0 ** 32)
    return q * (box / 2.0 ** 32)


# ---------------------------------------------------------------- workloads

def nve512(seed: int = BASE_SEED + 1):
    """512 atoms, SC 8^3 at 1.000 g/cm^3 with 0.1 A jitter, 298 K Maxwell."""
    L = cubic_box_edge(512, 1.000)
    x = simple_cubic(8, L, 0.1, seed)
    v = maxwell_velocities(512, 298.0, seed=seed + 1000)
    return x, v, np.array([L, L, L])


def ice_box(nx=16, ny=16, nz=16, rho=0.92):
    return ice_ih(nx, ny, nz, rho)


def jittered_box(n: int, rho: float, jitter: float = 0.1, seed: int = 0):
    """n atoms on a jittered SC lattice of ceil(n^(1/3)) sites per edge, n of the
    sites picked by a seeded permutation; cubic box at density rho."""
    rng = np.random.default_rng(seed)
    L = cubic_box_edge(n, rho)
    m = int(math.ceil(round(n ** (1.0 / 3.0), 9)))
    sites = simple_cubic(m, L)
    pick = np.sort(rng.permutation(m ** 3)[:n])
    x = sites[pick] + rng.normal(0.0, jitter, (n, 3))
    return x, np.array([L, L, L])


def batch_spec(nbox: int = 256, seed: int = BASE_SEED + 3, nmin: int = 216, nmax: int = 8000,
               rho_range=(0.92, 1.10), t_range=(200.0, 320.0)):
    rng = np.random.default_rng(seed)
    n = rng.integers(nmin, nmax + 1, nbox)
    rho = rng.uniform(*rho_range, nbox)
    T = rng.uniform(*t_range, nbox)
    return n.astype(np.int32), rho, T


def batch_boxes(nbox: int = 256, seed: int = BASE_SEED + 3, **kw):
    """Returns (n[nbox], box[nbox,3], x[sum n,3], v[sum n,3], T[nbox])."""
    n, rho, T = batch_spec(nbox, seed, **kw)
    xs, vs, boxes = [], [], []
    for b in range(nbox):
        x, box = jittered_box(int(n[b]), float(rho[b]), 0.1, seed * 1000 + b)
        xs.append(x)
        boxes.append(box)
        vs.append(maxwell_velocities(int(n[b]), float(T[b]), seed=seed * 1000 + 500000 + b))
    return n, np.array(boxes), np.concatenate(xs), np.concatenate(vs), T


def lattice_fill(n: int, lo, hi, rho_hint: float, jitter: float = 0.1, seed: int = 0) -> np.ndarray:
    """n atoms on a jittered orthorhombic grid filling the region [lo, hi)
    (n of the grid sites picked by a seeded permutation)."""
    rng = np.random.default_rng(seed)
    lo = np.asarray(lo, float)
    ext = np.asarray(hi, float) - lo
    s0 = volume_per_molecule(rho_hint) ** (1.0 / 3.0)
    mx = max(1, int(round(ext[0] / s0)))
    my = max(1, int(round(ext[1] / s0)))
    mz = max(1, int(math.ceil(n / (mx * my))))
    gx = (np.arange(mx) + 0.5) * ext[0] / mx
    gy = (np.arange(my) + 0.5) * ext[1] / my
    gz = (np.arange(mz) + 0.5) * ext[2] / mz
    sites = np.stack(np.meshgrid(gx, gy, gz, indexing="ij"), -1).reshape(-1, 3)
    pick = np.sort(rng.permutation(len(sites))[:n])
    return lo + sites[pick] + rng.normal(0.0, jitter, (n, 3))


def ice_liquid_slab(nx: int = 64, ny: int = 32, nz: int = 32, rho_ice: float = 0.92, rho_liq: float = 0.9998,
                    seed: int = BASE_SEED + 5):
    """Ice Ih slab (nx*ny*nz orthorhombic cells, 8 atoms each) with an equal
    number of liquid-start atoms stacked above it along z at rho_liq (jittered
    grid start; the liquid forms once dynamics run).  Returns (x, box, is_ice)."""
    xi, bi = ice_ih(nx, ny, nz, rho_ice)
    xi = xi + np.array([0.0, 0.0, bi[2] / nz / 16.0])  # centre the ice layers in [0, Lz_ice)
    n_liq = len(xi)
    lz = n_liq * volume_per_molecule(rho_liq) / (bi[0] * bi[1])
    xl = lattice_fill(n_liq, [0.0, 0.0, bi[2]], [bi[0], bi[1], bi[2] + lz], rho_liq, 0.1, seed)
    box = np.array([bi[0], bi[1], bi[2] + lz])
    x = np.concatenate([xi, xl])
    is_ice = np.concatenate([np.ones(len(xi), bool), np.zeros(n_liq, bool)])
    return x, box, is_ice


def liquid_vapor_slab(n: int = 1024, lxy: float = 30.0, lz: float = 100.0, rho: float = 0.997,
                      jitter: float = 0.2, seed: int = BASE_SEED + 6):
    """The liquid-vapour slab of Sec. II.C: n molecules filling a slab of
    density rho centred along z in an lxy x lxy x lz periodic cell, the rest
    of z empty (two interfaces perpendicular to z).  Jittered-grid start; the
    liquid forms once dynamics run.  Returns (x, box)."""
    t = n * volume_per_molecule(rho) / (lxy * lxy)
    z0 = 0.5 * (lz - t)
    x = lattice_fill(n, [0.0, 0.0, z0], [lxy, lxy, z0 + t], rho, jitter, seed)
    return x, np.array([lxy, lxy, lz])


# ---------------------------------------------------------------------------
# Several species.

# The paper's mW set (Sec. II.A and II.D) in table layout: lambda, epsilon,
# sigma, a, gamma, A, B, cos theta0, p, q.
MW_SET = np.array([23.15, 6.189, 2.3925, 1.8, 1.2, 7.049556277, 0.6022245584, -1.0 / 3.0, 4.0, 0.0])


def species_table_mixed(nt: int, seed: int = 0) -> np.ndarray:
    """Every pair and triplet set different: seeded factors on epsilon, sigma,
    a, gamma, A, B of each unordered pair and on lambda, epsilon, cos theta0
    of each centre and unordered leg pair."""
    rng = np.random.default_rng(seed)
    pair = {}
    for a in range(nt):
        for b in range(a, nt):
            q = MW_SET.copy()
            q[1] *= rng.uniform(0.7, 1.3)
            q[2] *= rng.uniform(0.9, 1.1)
            q[3] *= rng.uniform(0.95, 1.05)
            q[4] *= rng.uniform(0.8, 1.2)
            q[5] *= rng.uniform(0.9, 1.1)
            q[6] *= rng.uniform(0.9, 1.1)
            pair[(a, b)] = pair[(b, a)] = q
    t = np.zeros((nt, nt, nt, 10))
    for a in range(nt):
        for b in range(nt):
            for c in range(b, nt):
                lam = MW_SET[0] * rng.uniform(0.6, 1.3)
                c0 = rng.uniform(-0.5, -0.2)
                eps = pair[(a, b)][1] if b == c else MW_SET[1] * rng.uniform(0.7, 1.3)
                for bb, cc in ((b, c), (c, b)):
                    e = pair[(a, bb)].copy()
                    e[0], e[1], e[7] = lam, eps, c0
                    t[a, bb, cc] = e
    return t


def species_table_solute(eps_ss: float = 0.34, sig_ss: float = 3.4, eps_ws: float = 0.25,
                         sig_ws: float = 2.9) -> np.ndarray:
    """Species 0 = mW, species 1 = a solute with two-body terms only (lambda
    = 0 in every triplet that holds it): a hydrophobic particle of the kind
    Sec. IV discusses.  Sizes in A, energies in kcal/mol."""
    t = np.zeros((2, 2, 2, 10))
    for a in range(2):
        for b in range(2):
            for c in range(2):
                e = MW_SET.copy()
                if (a, b) == (1, 1):
                    e[1], e[2] = eps_ss, sig_ss
                elif a != b:
                    e[1], e[2] = eps_ws, sig_ws
                if a == 1 or b == 1 or c == 1:
                    e[0] = 0.0
                    if b != c:
                        e[1] = MW_SET[1]
                t[a, b, c] = e
    # the (a, b, b) sets carry the pair's epsilon, sigma; mixed triplets use
    # lambda = 0, so their epsilon is immaterial but kept symmetric
    return t


def species_table_sw_family() -> np.ndarray:
    """Fig. 2's tetrahedral family as four species: lambda = 20 (Ge), 21 (Si),
    23.15 (water), 26.2 (C), all in the mW energy and length scales; a pair
    or triplet takes the geometric mean of the lambdas involved."""
    lams = [20.0, 21.0, 23.15, 26.2]
    nt = len(lams)
    t = np.zeros((nt, nt, nt, 10))
    for a in range(nt):
        for b in range(nt):
            for c in range(nt):
                e = MW_SET.copy()
                e[0] = (lams[a] * lams[min(b, c)] * lams[max(b, c)]) ** (1.0 / 3.0)  # same for (a, c, b)
                t[a, b, c] = e
    return t


def species_draw(n: int, nt: int, seed: int = 0, weights=None) -> np.ndarray:
    """Seeded species of n atoms (int32), drawn with the given weights."""
    rng = np.random.default_rng(seed)
    return rng.choice(nt, size=n, p=weights).astype(np.int32)

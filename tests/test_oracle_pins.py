"""Pins of the FP64 oracle against facts that do not come from the oracle.

Each test targets a mistake the oracle could plausibly contain: a wrong SW
constant or exponent (phi2 minimum), a dropped / miscounted three-body term
(simple-cubic closed form with its 1/9 and 4/9 angle factors, brute force vs
cell list), a wrong force sign or factor (finite differences), a wrong virial
(strain finite differences, closed form on diamond / ice Ih), a wrong
adjoint (finite differences and the reduced-form identities of Sec. II.A),
and a wrong integrator (energy conservation, time reversibility, free
flight).
"""
import json
import math
import os

import numpy as np
import pytest

from paper_0809_2811_gb300 import inputs as I

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def test_default_params_are_the_papers(orc):
    p = orc.default_params()
    for name, key in [("lambda", "lambda"), ("epsilon", "epsilon_kcal_mol"), ("sigma", "sigma_A"),
                      ("a", "a"), ("gamma", "gamma"), ("A", "A"), ("B", "B"), ("p", "p"), ("q", "q")]:
        assert p[orc.PARAM_NAMES.index(name)] == GOLD[key]["value"], name
    # cos(theta0): tetrahedral reading of 109.47 deg; the printed angle agrees to 2e-5
    assert p[7] == -1.0 / 3.0
    assert abs(math.cos(math.radians(GOLD["theta0_deg"]["value"])) - p[7]) < 3e-5
    # the cutoff a*sigma lies below the paper's "forces zero beyond 4.32 A"
    assert p[3] * p[2] <= GOLD["cutoff_upper_bound_A"]["value"]


def test_phi2_minimum_is_minus_epsilon(orc):
    """A and B of the SW form put the pair minimum at 2^(1/6) sigma with depth
    epsilon (Sec. II.A calls epsilon the depth of the two-body potential)."""
    p = orc.default_params()
    r0 = 2 ** (1 / 6) * p[2]
    assert orc.phi2(r0)[0] == pytest.approx(-p[1], rel=1e-9)
    assert abs(orc.dphi2(r0)[0]) < 1e-7
    rs = np.linspace(2.2, 4.3, 2000)
    assert orc.phi2(rs).min() >= -p[1] * (1 + 1e-9)
    # scaling: epsilon scales phi2 linearly, sigma moves the minimum
    p2 = orc.params(epsilon=2.0, sigma=3.0)
    assert orc.phi2(2 ** (1 / 6) * 3.0, p2)[0] == pytest.approx(-2.0, rel=1e-9)


def test_terms_vanish_smoothly_at_cutoff(orc):
    p = orc.default_params()
    rc = p[3] * p[2]
    assert orc.phi2(rc)[0] == 0.0 and orc.phi2(rc + 0.1)[0] == 0.0
    assert abs(orc.phi2(rc - 1e-3)[0]) < 1e-100
    assert abs(orc.dphi2(rc - 1e-3)[0]) < 1e-100
    assert orc.phi3(rc - 1e-3, 2.7, 0.5) < 1e-100
    assert orc.phi3(rc, 2.7, 0.5) == 0.0
    # three-body term is zero at the tetrahedral angle, positive elsewhere
    assert orc.phi3(2.7, 2.8, -1.0 / 3.0) == 0.0
    assert orc.phi3(2.7, 2.8, 0.0) > 0


def _rand_box(rng, n, L, dmin=1.8, periodic=True):
    """Random points with a minimum separation (rejection) in a cube of edge L;
    periodic distances unless periodic is False (a cluster)."""
    x = []
    tries = 0
    while len(x) < n:
        tries += 1
        assert tries < 200000, "rejection sampler stuck"
        c = rng.uniform(0, L, 3)
        ok = True
        for y in x:
            d = c - y
            if periodic:
                d -= L * np.rint(d / L)
            if d @ d < dmin * dmin:
                ok = False
                break
        if ok:
            x.append(c)
    return np.array(x)


@pytest.mark.parametrize("seed,n,L", [(1, 8, 8.7), (2, 24, 9.5), (3, 40, 10.8), (4, 64, 12.4), (5, 64, 11.0)])
def test_brute_force_equals_cell_list(orc, seed, n, L):
    rng = np.random.default_rng(seed)
    x = _rand_box(rng, n, L)
    box = np.array([L, L, L])
    a = orc.energy_forces(x, box, method="cell")
    b = orc.energy_forces(x, box, method="brute")
    assert a["ntriplets"] == b["ntriplets"] > 0 and a["npairs"] == b["npairs"]
    for k in ("e2", "e3"):
        assert a[k] == pytest.approx(b[k], rel=1e-12, abs=1e-12)
    np.testing.assert_allclose(a["forces"], b["forces"], rtol=1e-11, atol=1e-11)
    np.testing.assert_allclose(a["virial"], b["virial"], rtol=1e-11, atol=1e-10)


def test_dense_cluster_brute_force(orc):
    """A tight cluster (most atoms legs of most others) in a padded box."""
    rng = np.random.default_rng(7)
    x = _rand_box(rng, 10, 5.0, dmin=2.2, periodic=False) + 4.0
    box = np.array([14.0, 14.0, 14.0])
    a = orc.energy_forces(x, box, method="cell")
    b = orc.energy_forces(x, box, method="brute")
    assert a["energy"] == pytest.approx(b["energy"], rel=1e-12)
    np.testing.assert_allclose(a["forces"], b["forces"], rtol=1e-11, atol=1e-11)


@pytest.mark.parametrize("rho", [0.92, 0.978, 0.9998])
def test_ice_ih_and_diamond_closed_form(orc, rho):
    """Perfect tetrahedral lattice with spacing d in (a sig / sqrt(8/3), a sig):
    four legs per atom at the tetrahedral angle, so E3 = 0, E/N = 2 phi2(d),
    F = 0, and the virial is isotropic with trace -2 N d phi2'(d)."""
    p = orc.default_params()
    for x, box in (I.ice_ih(4, 3, 3, rho), I.diamond_cubic(3, rho)):
        n = len(x)
        d = (3 * math.sqrt(3) / 8 * I.volume_per_molecule(rho)) ** (1 / 3)
        assert p[3] * p[2] / math.sqrt(8 / 3) < d < p[3] * p[2]
        r = orc.energy_forces(x, box)
        assert r["npairs"] == 2 * n
        assert r["ntriplets"] == 6 * n
        assert abs(r["e3"]) < 1e-20 * n
        assert r["energy"] / n == pytest.approx(2 * orc.phi2(d)[0], rel=1e-12)
        assert np.abs(r["forces"]).max() < 1e-10
        w = r["virial"]
        tr = -2 * n * d * orc.dphi2(d)[0]
        assert w[:3].sum() == pytest.approx(tr, rel=1e-10)
        np.testing.assert_allclose(w[:3], tr / 3, rtol=1e-9)
        # only pair terms, all of one sign on the diagonal: the scale equals |trace|
        assert r["virial_abs"] == pytest.approx(abs(tr), rel=1e-10)
        assert np.abs(w[3:]).max() < 1e-9 * abs(tr)


def test_ice_worked_values(orc):
    """Geometry and energy per molecule of the ice Ih lattice at 0.92 and
    0.978 g/cm^3 (0.978 is the mW ice density at T_m, Table 1)."""
    for rho, d_exp, e_exp in [(0.92, 2.764156, -12.245839), (0.978, 2.708396, -12.366348)]:
        x, box = I.ice_ih(4, 3, 3, rho)
        d = (3 * math.sqrt(3) / 8 * I.volume_per_molecule(rho)) ** (1 / 3)
        assert d == pytest.approx(d_exp, abs=2e-6)
        assert orc.energy_forces(x, box)["energy"] / len(x) == pytest.approx(e_exp, abs=2e-6)


def test_simple_cubic_closed_form(orc):
    """SC lattice, spacing s in (a sig/sqrt2, a sig): six legs per atom, 12 leg
    pairs at 90 deg ((0 + 1/3)^2 = 1/9) and 3 at 180 deg ((-1 + 1/3)^2 = 4/9):
    E3/N = (12/9 + 12/9) lam eps exp(2 gam sig / (s - a sig)), E2/N = 3 phi2(s)."""
    p = orc.default_params()
    lam, eps, sig, a, gam = p[:5]
    L = I.cubic_box_edge(512, 1.0)
    s = L / 8
    x = I.simple_cubic(8, L)
    r = orc.energy_forces(x, np.array([L] * 3))
    e3 = (8.0 / 3.0) * lam * eps * math.exp(2 * gam * sig / (s - a * sig))
    assert r["e3"] / 512 == pytest.approx(e3, rel=1e-12)
    assert r["e2"] / 512 == pytest.approx(3 * orc.phi2(s)[0], rel=1e-12)
    assert np.abs(r["forces"]).max() < 1e-10
    # worked numbers for s = L/8 at 1.000 g/cm^3
    assert r["e2"] / 512 == pytest.approx(-14.089228, abs=2e-6)
    assert r["e3"] / 512 == pytest.approx(3.220146, abs=2e-6)
    assert r["ntriplets"] == 15 * 512 and r["npairs"] == 3 * 512


def _jittered(seed=11, n=216, rho=1.0, jitter=0.25):
    return I.jittered_box(n, rho, jitter, seed)


def test_forces_are_minus_gradient(orc):
    x, box = _jittered()
    r = orc.energy_forces(x, box)
    h = 1e-5
    rng = np.random.default_rng(0)
    for i in rng.choice(len(x), 12, replace=False):
        for k in range(3):
            xp = x.copy()
            xp[i, k] += h
            xm = x.copy()
            xm[i, k] -= h
            fd = -(orc.energy_forces(xp, box)["energy"] - orc.energy_forces(xm, box)["energy"]) / (2 * h)
            assert r["forces"][i, k] == pytest.approx(fd, rel=1e-6, abs=1e-6)


def test_virial_is_strain_derivative(orc):
    """Diagonal: W_aa = -dE/d eps_aa under x_a -> (1+eps) x_a, L_a -> (1+eps) L_a."""
    x, box = _jittered(seed=12)
    r = orc.energy_forces(x, box)
    h = 1e-6
    for a in range(3):
        s = np.ones(3)
        s[a] = 1 + h
        ep = orc.energy_forces(x * s, box * s)["energy"]
        s[a] = 1 - h
        em = orc.energy_forces(x * s, box * s)["energy"]
        assert r["virial"][a] == pytest.approx(-(ep - em) / (2 * h), rel=1e-6)


def test_virial_off_diagonal_by_shear_of_isolated_cluster(orc):
    rng = np.random.default_rng(5)
    x = _rand_box(rng, 20, 6.5, dmin=2.3, periodic=False) + 6.0
    box = np.array([20.0, 20.0, 20.0])
    r = orc.energy_forces(x, box)
    c = x.mean(0)
    h = 1e-6
    for comp, (a, b) in zip(range(3, 6), [(0, 1), (0, 2), (1, 2)]):
        def E(e):
            y = x - c
            y2 = y.copy()
            y2[:, a] += e * y[:, b]
            return orc.energy_forces(y2 + c, box)["energy"]
        assert r["virial"][comp] == pytest.approx(-(E(h) - E(-h)) / (2 * h), rel=1e-5, abs=1e-7)


def test_invariants(orc):
    x, box = _jittered(seed=13)
    r = orc.energy_forces(x, box)
    F = r["forces"]
    assert np.abs(F.sum(0)).max() < 1e-9 * np.abs(F).max()
    # translation with wrapping
    t = orc.energy_forces(np.mod(x + np.array([3.3, -7.1, 11.9]), box), box)
    assert t["energy"] == pytest.approx(r["energy"], rel=1e-12)
    np.testing.assert_allclose(t["forces"], F, atol=1e-9)
    # axis permutation and reflection of the cubic box
    perm = [2, 0, 1]
    p = orc.energy_forces(x[:, perm], box)
    assert p["energy"] == pytest.approx(r["energy"], rel=1e-12)
    np.testing.assert_allclose(p["forces"], F[:, perm], atol=1e-9)
    m = orc.energy_forces(np.mod(-x, box), box)
    assert m["energy"] == pytest.approx(r["energy"], rel=1e-12)
    np.testing.assert_allclose(m["forces"], -F, atol=1e-9)


def test_rotation_of_isolated_cluster(orc):
    rng = np.random.default_rng(9)
    x = _rand_box(rng, 24, 7.0, dmin=2.3, periodic=False)
    x -= x.mean(0)
    box = np.array([30.0, 30.0, 30.0])
    q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    if np.linalg.det(q) < 0:
        q[:, 0] *= -1
    a = orc.energy_forces(x + 15, box)
    b = orc.energy_forces(x @ q.T + 15, box)
    assert a["energy"] == pytest.approx(b["energy"], rel=1e-12)
    np.testing.assert_allclose(a["forces"] @ q.T, b["forces"], atol=1e-9)


def test_neighbor_sets_match_direct_enumeration(orc):
    x, box = _jittered(seed=14, n=343, rho=1.05)
    rl = 5.3065
    sets, band = orc.neighbors(x, box, rl)
    d = x[None, :, :] - x[:, None, :]
    d -= box * np.rint(d / box)
    r2 = (d * d).sum(-1)
    np.fill_diagonal(r2, np.inf)
    for i in range(len(x)):
        assert np.array_equal(sets[i], np.nonzero(r2[i] < rl * rl)[0])
    nb = {(i, j) for i, j in zip(*np.nonzero(np.abs(r2 - rl * rl) <= 1e-5 * rl * rl))}
    assert band == nb


def test_parameter_gradient_identities(orc):
    """Reduced form (Sec. II.A): E = eps * E~(x / sig), E3 linear in lambda, so
    dE/deps = E/eps, dE/dlam = E3/lam, dE/dsig = tr(W)/sig."""
    x, box = _jittered(seed=15)
    p = orc.default_params()
    r = orc.energy_forces(x, box)
    g = orc.energy_param_grad(x, box)
    assert g[0] == pytest.approx(r["e3"] / p[0], rel=1e-10)
    assert g[1] == pytest.approx(r["energy"] / p[1], rel=1e-10)
    assert g[2] == pytest.approx(r["virial"][:3].sum() / p[2], rel=1e-9)
    # and against plain central differences
    for t in range(3):
        h = 1e-6 * p[t]
        pp = p.copy()
        pp[t] += h
        pm = p.copy()
        pm[t] -= h
        fd = (orc.energy_forces(x, box, pp)["energy"] - orc.energy_forces(x, box, pm)["energy"]) / (2 * h)
        assert g[t] == pytest.approx(fd, rel=1e-6)


def test_force_vjp_against_finite_differences(orc):
    """dL/dx and dL/dtheta of L = sum_i w_i . F_i against central differences
    (h = 1e-4 A in x, 1e-4 relative in theta) and the reduced-form identities
    dL/deps = L/eps, dL/dlam = (w . F3)/lam."""
    x, box = _jittered(seed=16, n=125, rho=1.0)
    rng = np.random.default_rng(3)
    w = rng.normal(size=x.shape)
    p = orc.default_params()
    gx, gt = orc.force_vjp(x, box, w)

    def L(xx, pp=p):
        return float((w * orc.energy_forces(xx, box, pp)["forces"]).sum())

    for i in rng.choice(len(x), 6, replace=False):
        for k in range(3):
            h = 1e-4
            xp = x.copy()
            xp[i, k] += h
            xm = x.copy()
            xm[i, k] -= h
            fd = (L(xp) - L(xm)) / (2 * h)
            assert gx[i, k] == pytest.approx(fd, rel=2e-5, abs=1e-4)
    for t in range(3):
        h = 1e-4 * p[t]
        pp = p.copy()
        pp[t] += h
        pm = p.copy()
        pm[t] -= h
        fd = (L(x, pp) - L(x, pm)) / (2 * h)
        assert gt[t] == pytest.approx(fd, rel=1e-6)
    assert gt[1] == pytest.approx(L(x) / p[1], rel=1e-10)
    p0 = p.copy()
    p0[0] = 0.0
    f2 = orc.energy_forces(x, box, p0)["forces"]
    f3 = orc.energy_forces(x, box)["forces"] - f2
    assert gt[0] == pytest.approx(float((w * f3).sum()) / p[0], rel=1e-10)
    # the x-gradient of a one-atom probe equals minus a Hessian column
    w1 = np.zeros_like(x)
    w1[0, 0] = 1.0
    g1, _ = orc.force_vjp(x, box, w1)
    h = 1e-5
    xp = x.copy()
    xp[0, 0] += h
    xm = x.copy()
    xm[0, 0] -= h
    col = (orc.energy_forces(xp, box)["forces"] - orc.energy_forces(xm, box)["forces"]) / (2 * h)
    np.testing.assert_allclose(g1, col, rtol=1e-5, atol=1e-5)


def test_units_reduced_time(orc):
    """10 fs is 0.05 reduced time units (Sec. II.B), tau = sigma sqrt(m/eps)."""
    p = orc.default_params()
    tau = p[2] / math.sqrt(p[1] / I.M_WATER * orc.FCONV)
    assert tau == pytest.approx(199.56, abs=0.01)
    assert GOLD["dt_fs"]["value"] / tau == pytest.approx(GOLD["dt_reduced"]["value"], abs=0.0015)


def test_free_flight_is_exact(orc):
    """Atoms farther apart than a sigma feel nothing: x(t) = x0 + v t."""
    x = np.array([[1.0, 1.0, 1.0], [11.0, 11.0, 11.0]])
    v = np.array([[0.01, -0.02, 0.003], [-0.005, 0.0, 0.01]])
    box = np.array([20.0, 20.0, 20.0])
    x1, v1, _, th = orc.md(x, v, box, 50, dt=10.0)
    np.testing.assert_allclose(x1, np.mod(x + 500 * v, box), atol=1e-12)
    np.testing.assert_allclose(v1, v, atol=1e-15)


def test_nve_conservation_and_reversibility(orc):
    x, v, box = I.nve512()
    x1, v1, _, th = orc.md(x, v, box, 200, dt=10.0)
    e = th[:, 5]
    assert abs(e[-1] - e[0]) / abs(e[0]) < GOLD["nve_relative_drift_bound"]["value"]
    assert np.std(e) / abs(e.mean()) < 1e-4
    # velocity Verlet is time reversible: run back with -v
    x2, v2, _, _ = orc.md(x1, -v1, box, 200, dt=10.0)
    d = x2 - np.mod(x, box)
    d -= box * np.rint(d / box)
    assert np.abs(d).max() < 1e-6
    np.testing.assert_allclose(-v2, v, atol=1e-8)


def test_nose_hoover_conserved_and_thermalises(orc):
    x, v, box = I.nve512()
    v = v * math.sqrt(400.0 / 298.0)
    x1, v1, st, th = orc.md(x, v, box, 400, dt=5.0, kind=2, T0=298.0, tau=200.0)
    c = th[:, 5]
    assert abs(c[-1] - c[0]) / abs(c[0]) < 2e-4
    assert abs(th[-200:, 4].mean() - 298.0) < 60.0
    # a huge relaxation time makes it NVE
    _, _, _, th2 = orc.md(x, v, box, 20, dt=5.0, kind=2, T0=298.0, tau=1e9)
    _, _, _, th3 = orc.md(x, v, box, 20, dt=5.0, kind=0)
    np.testing.assert_allclose(th2[:, 0], th3[:, 0], rtol=1e-9)


def test_berendsen_relaxes_temperature(orc):
    x, v, box = I.nve512()
    x1, v1, _, th = orc.md(x, v * math.sqrt(2.0), box, 300, dt=10.0, kind=1, T0=298.0, tau=100.0)
    assert abs(th[-50:, 4].mean() - 298.0) < 25.0


# --------------------------------------------------------------------------
# Sec. II.C structure: the pair histogram behind g(r) and the adf.

def test_pair_histogram_diamond_shells(orc):
    """Cubic diamond with cube edge a0: coordination shells at r^2 = (3/16) a0^2
    x (1, 8/3, 11/3) hold 4, 12 and 12 atoms; the histogram counts ordered pairs."""
    x, box = I.diamond_cubic(3, 0.92)
    n = len(x)
    a0 = box[0] / 3
    d = math.sqrt(3.0) / 4.0 * a0
    dr = 0.01
    h, amb = orc.pair_histogram(x, box, dr, 600)
    assert amb.sum() == 0
    for f, c in ((1.0, 4), (8.0 / 3.0, 12), (11.0 / 3.0, 12)):
        k = int(math.floor(d * math.sqrt(f) / dr))
        assert h[k] == c * n
    k3 = int(math.floor(d * math.sqrt(11.0 / 3.0) / dr))
    assert h[: k3 + 1].sum() == (4 + 12 + 12) * n  # nothing in between


def test_pair_histogram_simple_cubic_shells_and_total(orc):
    """Simple cubic (spacing s): 6, 12, 8 neighbours at s, sqrt2 s, sqrt3 s;
    with the range past the largest minimum-image distance every ordered pair
    is counted once: N (N - 1) in all."""
    L = 8 * 3.104282
    x = I.simple_cubic(8, L)
    n = len(x)
    s = L / 8
    h, amb = orc.pair_histogram(x, np.array([L, L, L]), 0.01, 3000)
    assert amb.sum() == 0
    for f, c in ((1.0, 6), (2.0, 12), (3.0, 8)):
        assert h[int(math.floor(s * math.sqrt(f) / 0.01))] == c * n
    assert h.sum() == n * (n - 1)


def test_angle_histogram_tetrahedral_and_cubic(orc):
    """adf with n_c = 4 in diamond: every angle is the tetrahedral one
    (acos(-1/3) = 109.47 deg), 4 x 3 ordered pairs per atom; with n_c = 6 in
    simple cubic: 24 right angles and 6 straight ones per atom."""
    x, box = I.diamond_cubic(2, 0.92)
    n = len(x)
    h, amb, ties = orc.angle_histogram(x, box, nc=4, nbins=7)
    w = 180.0 / 7
    assert amb.sum() == 0 and ties == 0
    assert h[int(math.degrees(math.acos(-1.0 / 3.0)) // w)] == 12 * n
    assert h.sum() == 12 * n
    L = 6 * 3.104282
    xs = I.simple_cubic(6, L)
    hs, amb, ties = orc.angle_histogram(xs, np.array([L, L, L]), nc=6, nbins=7)
    m = len(xs)
    assert ties == 0
    assert hs[int(90.0 // w)] == 24 * m
    assert hs[6] == 6 * m
    assert hs.sum() == 30 * m


# --------------------------------------------------------------------------
# Sec. II.B isobaric dynamics (Nose-Hoover barostat, read as the isotropic
# Martyna-Tobias-Klein split).

def test_npt_reduces_to_nose_hoover_without_barostat_coupling(orc):
    """With an infinitely heavy barostat (tau_p -> inf) the box stays fixed and
    the NPT split is the Nose-Hoover one, step for step."""
    x, v, box = I.nve512()
    xa, va, ba, _, _ = orc.md_npt(x, v, box, 40, dt=10.0, T0=298.0, tau=1000.0, p_atm=0.0, tau_p=1e12)
    xb, vb, _, _ = orc.md(x, v, box, 40, dt=10.0, kind=2, T0=298.0, tau=1000.0)
    assert np.array_equal(ba, box)
    assert np.abs(xa - xb).max() < 1e-9 and np.abs(va - vb).max() < 1e-12


def test_npt_conserved_quantity_is_second_order(orc):
    """H' = KE + PE + P V + pe^2/2W + Q xi^2/2 + Ndf kB T0 eta: its excursion
    over a fixed 1 ps, from a start far from equilibrium (box under tension),
    falls as dt^2 (a dropped or mis-signed term in the barostat force would
    leave a dt-independent drift), and stays below 5e-4 |H'| at 10 fs."""
    x, v, box = I.nve512()
    dev = []
    for dt in (10.0, 5.0):
        _, _, _, _, th = orc.md_npt(x, v, box, int(1000 / dt), dt=dt, T0=298.0, tau=1000.0, p_atm=0.0,
                                    tau_p=2500.0)
        c = th[:, 5]
        dev.append((c.max() - c.min()) / abs(c[0]))
        assert th[-1, 8] != th[0, 8]  # the box did move
    assert dev[0] < 5e-4
    assert 3.0 < dev[0] / dev[1] < 5.0


# ---------------------------------------------------------------------------
# Several species (Sec. IV's mW with solutes of other lambda, epsilon, sigma,
# and the SW family of Fig. 2): a parameter vector per species triple.  Pinned
# by reduction to the one-species oracle, by the entries a few isolated atoms
# select, and by derivatives.

def _mixed_table(orc, seed=0, nt=2):
    """A table with every species pair and triplet different, symmetric in
    the pair and in the two legs (the table rule the oracle checks)."""
    rng = np.random.default_rng(seed)
    p0 = orc.default_params()
    pair = {}
    for a in range(nt):
        for b in range(a, nt):
            q = p0.copy()
            q[1] *= rng.uniform(0.7, 1.3)   # epsilon
            q[2] *= rng.uniform(0.9, 1.1)   # sigma
            q[3] *= rng.uniform(0.95, 1.05)  # a
            q[4] *= rng.uniform(0.8, 1.2)   # gamma
            q[5] *= rng.uniform(0.9, 1.1)   # A
            q[6] *= rng.uniform(0.9, 1.1)   # B
            pair[(a, b)] = pair[(b, a)] = q
    tri = {}
    for a in range(nt):
        for b in range(nt):
            for c in range(b, nt):
                tri[(a, b, c)] = tri[(a, c, b)] = (rng.uniform(10, 30), rng.uniform(4, 8), rng.uniform(-0.5, -0.2))

    def entry(a, b, c):
        e = pair[(a, b)].copy() if b == c else p0.copy()
        if b != c:  # (gamma, sigma, a) of a mixed entry are never read; lambda, epsilon, cos theta0 are
            e[1:7] = pair[(a, b)][1:7]
        if b == c:
            e[0] = tri[(a, b, c)][0]
            # the pair term reads epsilon from (a, b, b): the triplet (a, b, b) shares it
            e[7] = tri[(a, b, c)][2]
        else:
            e[0], e[1], e[7] = tri[(a, b, c)]
        return e
    return orc.species_table(nt, entry)


def test_species_one_type_is_the_one_species_oracle(orc):
    x, box = _jittered(seed=31, n=300)
    p = orc.default_params()
    r1 = orc.energy_forces_species(x, box, np.zeros(len(x), int), orc.species_table(1, lambda a, b, c: p))
    r0 = orc.energy_forces(x, box)
    assert r1["e2"] == pytest.approx(r0["e2"], rel=1e-13)
    assert r1["e3"] == pytest.approx(r0["e3"], rel=1e-13)
    assert np.abs(r1["forces"] - r0["forces"]).max() < 1e-11
    assert np.allclose(r1["virial"], r0["virial"], rtol=1e-12, atol=1e-9)
    assert (r1["npairs"], r1["ntriplets"]) == (r0["npairs"], r0["ntriplets"])


def test_species_labels_of_identical_species_do_not_matter(orc):
    x, box = _jittered(seed=32, n=250)
    p = orc.default_params()
    ty = np.random.default_rng(3).integers(0, 3, len(x))
    r3 = orc.energy_forces_species(x, box, ty, orc.species_table(3, lambda a, b, c: p))
    r0 = orc.energy_forces(x, box)
    assert r3["energy"] == pytest.approx(r0["energy"], rel=1e-13)
    assert np.abs(r3["forces"] - r0["forces"]).max() < 1e-11


def test_species_pair_term_takes_the_pair_entry(orc):
    """Two atoms of species 0 and 1: the energy is phi2 of entry (0, 1, 1)
    (= entry (1, 0, 0)), the one-species oracle's pair term with those
    parameters, and the force is its derivative."""
    t = _mixed_table(orc, seed=4)
    box = np.array([30.0, 30.0, 30.0])
    for r in (2.6, 3.1, 3.9):
        x = np.array([[5.0, 5.0, 5.0], [5.0 + r * 0.6, 5.0 + r * 0.8, 5.0]])
        res = orc.energy_forces_species(x, box, [0, 1], t)
        pe = t[0, 1, 1]
        assert res["e3"] == 0.0
        assert res["e2"] == pytest.approx(orc.phi2(r, pe)[0], rel=1e-14)
        assert res["forces"][1] == pytest.approx(-orc.dphi2(r, pe)[0] * np.array([0.6, 0.8, 0.0]), rel=1e-12)
        assert orc.energy_forces_species(x, box, [1, 0], t)["e2"] == pytest.approx(res["e2"], rel=1e-14)


def test_species_triplet_takes_the_centre_legs_entry(orc):
    """Centre of species 0 with legs to species 1 and 2 that are out of each
    other's range: the only triplet is (0; 1, 2), and with all leg parameters
    equal its energy is the one-species oracle's with lambda, epsilon and
    cos theta0 of entry (0, 1, 2)."""
    p0 = orc.default_params()
    lam = {(0, 1, 2): 17.0, (0, 2, 1): 17.0}
    eps3 = {(0, 1, 2): 5.5, (0, 2, 1): 5.5}
    c0 = {(0, 1, 2): -0.25, (0, 2, 1): -0.25}

    def entry(a, b, c):
        e = p0.copy()
        if (a, b, c) in lam:
            e[0], e[1], e[7] = lam[(a, b, c)], eps3[(a, b, c)], c0[(a, b, c)]
        return e
    t = orc.species_table(3, entry)
    box = np.array([30.0, 30.0, 30.0])
    ang = math.radians(150.0)
    r1, r2 = 3.0, 3.6
    x = np.array([[10.0, 10.0, 10.0], [10.0 + r1, 10.0, 10.0],
                  [10.0 + r2 * math.cos(ang), 10.0 + r2 * math.sin(ang), 10.0]])
    res = orc.energy_forces_species(x, box, [0, 1, 2], t)
    assert res["ntriplets"] == 1
    pt = p0.copy()
    pt[0], pt[1], pt[7] = 17.0, 5.5, -0.25
    assert res["e3"] == pytest.approx(orc.phi3(r1, r2, math.cos(ang), pt), rel=1e-13)
    assert res["e3"] != pytest.approx(orc.phi3(r1, r2, math.cos(ang), p0), rel=1e-3)
    # the same atoms with the centre of another species take that centre's entries
    res2 = orc.energy_forces_species(x, box, [1, 0, 2], t)
    assert res2["e3"] == pytest.approx(orc.phi3(r1, r2, math.cos(ang), p0), rel=1e-13)


def test_species_forces_and_virial_are_derivatives(orc):
    """A two-species mixture with every pair and triplet entry different:
    F = -grad E (central differences) and tr W = -dE/d(ln s) under a uniform
    scaling of positions and box."""
    t = _mixed_table(orc, seed=7)
    x, box = _jittered(seed=33, n=160)
    ty = np.random.default_rng(8).integers(0, 2, len(x))
    r = orc.energy_forces_species(x, box, ty, t)
    assert r["e3"] > 0 and r["ntriplets"] > 0
    h = 1e-5
    rng = np.random.default_rng(9)
    for i in rng.choice(len(x), 8, replace=False):
        for k in range(3):
            xp = x.copy()
            xp[i, k] += h
            xm = x.copy()
            xm[i, k] -= h
            fd = -(orc.energy_forces_species(xp, box, ty, t)["energy"]
                   - orc.energy_forces_species(xm, box, ty, t)["energy"]) / (2 * h)
            assert r["forces"][i, k] == pytest.approx(fd, rel=1e-6, abs=1e-6)
    hs = 1e-6
    ep = orc.energy_forces_species(x * (1 + hs), box * (1 + hs), ty, t)["energy"]
    em = orc.energy_forces_species(x * (1 - hs), box * (1 - hs), ty, t)["energy"]
    assert sum(r["virial"][:3]) == pytest.approx(-(ep - em) / (2 * hs), rel=1e-6)


def test_species_table_rule_is_checked(orc):
    t = _mixed_table(orc, seed=10)
    assert orc.species_table_ok(t)
    bad = t.copy()
    bad[0, 1, 1, 1] *= 1.01  # pair (0, 1) no longer equals pair (1, 0)
    assert not orc.species_table_ok(bad)
    bad = t.copy()
    bad[1, 0, 1, 0] += 1.0  # lambda of (1; 0, 1) differs from (1; 1, 0)
    assert not orc.species_table_ok(bad)
    with pytest.raises(RuntimeError):
        orc.energy_forces_species(*_jittered(seed=34, n=50), np.zeros(50, int), bad)


def test_species_dynamics_with_one_type_is_the_one_species_run(orc):
    x, v, box = I.nve512()
    p = orc.default_params()
    t = orc.species_table(2, lambda a, b, c: p)
    ty = np.arange(512) % 2
    xa, va, sa, tha = orc.md_species(x, v, box, ty, t, 20, dt=10.0, kind=2, T0=298.0, tau=1000.0)
    xb, vb, sb, thb = orc.md(x, v, box, 20, dt=10.0, kind=2, T0=298.0, tau=1000.0)
    assert np.abs(xa - xb).max() < 1e-9 and np.abs(va - vb).max() < 1e-12
    assert tha[-1, 5] == pytest.approx(thb[-1, 5], rel=1e-12)


def test_species_npt_with_one_type_is_the_one_species_run(orc):
    x, v, box = I.nve512()
    p = orc.default_params()
    t = orc.species_table(2, lambda a, b, c: p)
    ty = np.arange(512) % 2
    xa, va, ba, sa, tha = orc.md_npt_species(x, v, box, ty, t, 20, dt=10.0, T0=298.0, tau=1000.0, tau_p=2000.0)
    xb, vb, bb, sb, thb = orc.md_npt(x, v, box, 20, dt=10.0, T0=298.0, tau=1000.0, tau_p=2000.0)
    assert np.abs(xa - xb).max() < 1e-9 and np.abs(va - vb).max() < 1e-12
    assert np.abs(ba - bb).max() < 1e-12 and ba[0] != box[0]
    assert tha[-1, 5] == pytest.approx(thb[-1, 5], rel=1e-12)


# ---- owner-computes routine (the multi-core CPU baseline) -----------------

@pytest.mark.parametrize("threads", [1, 4])
@pytest.mark.parametrize("case", ["liquidlike", "ice", "dense_overflow", "small_box", "cluster"])
def test_owner_computes_equals_cell_list(orc, case, threads):
    """The owner-computes grouping (pair halves, terms centred on the atom, the
    atom as a leg of its neighbours' terms) is the same sum as the cell-list
    loop; the brute-force pin above ties that loop to the definition.  A
    dropped two-hop term, a wrong sign of a reaction or a double-counted pair
    half shows up here as an O(1) difference."""
    if case == "liquidlike":
        x, box = I.jittered_box(1000, 1.0, 0.3, 301)
    elif case == "ice":
        x, box = I.ice_ih(4, 3, 3, 0.92)
    elif case == "dense_overflow":
        x, box = I.jittered_box(512, 3.5, 0.1, 302)
    elif case == "small_box":
        rng = np.random.default_rng(303)
        L = 9.5
        x, box = _rand_box(rng, 24, L), np.array([L, L, L])
    else:
        rng = np.random.default_rng(304)
        x = _rand_box(rng, 10, 5.0, dmin=2.2, periodic=False) + 4.0
        box = np.array([14.0, 14.0, 14.0])
    a = orc.energy_forces(x, box, method="cell")
    b = orc.energy_forces(x, box, method="owner", threads=threads)
    assert a["npairs"] == b["npairs"] and a["ntriplets"] == b["ntriplets"]
    for k in ("e2", "e3"):
        assert b[k] == pytest.approx(a[k], rel=1e-12, abs=1e-9)
    scale = max(np.abs(a["forces"]).max(), 1.0)
    np.testing.assert_allclose(b["forces"], a["forces"], rtol=0, atol=1e-11 * scale)
    np.testing.assert_allclose(b["virial"], a["virial"], rtol=0, atol=1e-12 * a["virial_abs"] + 1e-12)
    assert b["virial_abs"] == pytest.approx(a["virial_abs"], rel=1e-12)


def test_owner_computes_dynamics_follow_the_serial_run(orc):
    """Nose-Hoover steps with the threaded owner forces stay on the serial
    run's trajectory (rounding-order differences only)."""
    x, v, box = I.nve512()
    xa, va, sa, tha = orc.md(x, v, box, 20, dt=10.0, kind=2, T0=298.0, tau=1000.0)
    xb, vb, sb, thb = orc.md(x, v, box, 20, dt=10.0, kind=2, T0=298.0, tau=1000.0, threads=4)
    d = np.mod(xa - xb + box / 2, box) - box / 2
    assert np.abs(d).max() < 1e-9
    np.testing.assert_allclose(thb[:, 5], tha[:, 5], rtol=1e-10)

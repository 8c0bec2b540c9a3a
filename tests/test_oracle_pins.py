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

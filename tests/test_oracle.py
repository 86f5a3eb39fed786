"""Pins for the FP64 CPU oracle (CPU only).

Each test ties the oracle to something other than itself: closed forms of
Eq. (1), textbook limits, invariances of a pair potential, an independent
image-enumeration brute force, finite differences of the energy, the
order of the velocity-Verlet error, time reversibility, the published
SplitMix64 test vector, the configuration's density endpoints for Eq. (3),
and hand-built cluster geometries plus an independent BFS for Sec. II.C.
"""
import json
import math
from pathlib import Path

import numpy as np
import pytest

import oracle
import inputs

GOLD = Path(__file__).resolve().parent / "golden"
T1 = json.loads((GOLD / "table1_params.json").read_text())


def P(r_C=20.0, **kw):
    return oracle.params(r_C, **kw)


# ---------------------------------------------------------------- Eq. (1)

def test_default_params_match_table_I():
    p = P()
    assert (p.a, p.b, p.c, p.Lambda) == (T1["a_MeV"], T1["b_MeV"], T1["c_MeV"], T1["Lambda_fm2"])
    assert p.lambda_s == T1["lambda_fm"] and p.M == T1["M_MeV"] and p.r_nuc == T1["r_nuc_fm"]
    # alpha*hbar*c from CODATA: 1.4399645 MeV fm
    assert abs(p.alpha - 1.4399645) < 1e-6


@pytest.mark.parametrize("ti,tj,s", [(1, 0, T1["b_MeV"] - T1["c_MeV"]),
                                     (0, 1, T1["b_MeV"] - T1["c_MeV"]),
                                     (0, 0, T1["b_MeV"] + T1["c_MeV"]),
                                     (1, 1, T1["b_MeV"] + T1["c_MeV"])])
def test_nuclear_minimum_closed_form(ti, tj, s):
    """V = a g^2 + s g with g = exp(-r^2/2Lambda) is minimal at g* = -s/2a:
    V_min = -s^2/(4a) at r*^2 = 2 Lambda ln(2a/|s|) and the force vanishes."""
    a, Lam = T1["a_MeV"], T1["Lambda_fm2"]
    p = P(coulomb=False)
    r2 = 2.0 * Lam * math.log(2.0 * a / abs(s))
    vn, vc, g = oracle.pair(ti, tj, r2, p)
    assert vc == 0.0
    assert abs(vn - (-s * s / (4.0 * a))) < 1e-13
    assert abs(g) < 1e-12
    # and it is a minimum: larger on both sides
    for d in (-0.05, 0.05):
        rr = (math.sqrt(r2) + d) ** 2
        assert oracle.pair(ti, tj, rr, p)[0] > vn


def test_np_minimum_values():
    """Numbers derivable from Table I: V_np,min = -5.681818 MeV at 1.92458 fm;
    V_nn,min = -0.00909091 MeV at 3.42800 fm."""
    p = P(coulomb=False)
    r_np = math.sqrt(2 * 1.25 * math.log(220 / 50))
    r_nn = math.sqrt(2 * 1.25 * math.log(220 / 2))
    assert abs(r_np - 1.92458) < 1e-5 and abs(r_nn - 3.42800) < 1e-5
    assert abs(oracle.pair(1, 0, r_np ** 2, p)[0] + 5.681818) < 1e-6
    assert abs(oracle.pair(0, 0, r_nn ** 2, p)[0] + 0.00909091) < 1e-8


def test_coulomb_limits():
    """Screened Coulomb of V_pp: V r e^{r/lambda} = alpha for any r, and with
    lambda -> infinity the textbook alpha/r, |F| = alpha/r^2."""
    p = P(r_C=30.0)
    pn = P(r_C=30.0, coulomb=False)
    for r in (0.7, 2.0, 5.5, 12.0, 29.0):
        vn, vc, g = oracle.pair(1, 1, r * r, p)
        vn0, _, g0 = oracle.pair(1, 1, r * r, pn)
        assert vn == vn0
        assert abs(vc * r * math.exp(r / 10.0) - p.alpha) < 1e-12 * p.alpha
        # Coulomb part of the force, from the derivative of alpha e^{-r/l}/r
        fc = (g - g0) * r
        expect = p.alpha * math.exp(-r / 10.0) * (1 / r ** 2 + 1 / (10.0 * r))
        assert abs(fc - expect) < 1e-12 * expect
    pinf = P(r_C=30.0, lambda_s=1e300)
    for r in (0.5, 3.0, 17.0):
        vn, vc, g = oracle.pair(1, 1, r * r, pinf)
        vn0, _, g0 = oracle.pair(1, 1, r * r, pn)
        assert abs(vc * r - p.alpha) < 1e-13
        assert abs((g - g0) * r ** 3 - p.alpha) < 1e-12
    # no Coulomb between unlike or neutral pairs
    assert oracle.pair(1, 0, 4.0, p)[1] == 0.0 and oracle.pair(0, 0, 4.0, p)[1] == 0.0


def test_cutoffs_strict():
    p = P(r_C=15.0)
    eps = 1e-9
    assert oracle.pair(0, 0, (11.5 - eps) ** 2, p)[0] != 0.0
    assert oracle.pair(0, 0, (11.5 + eps) ** 2, p)[0] == 0.0
    assert oracle.pair(0, 0, 11.5 ** 2, p)[0] == 0.0
    assert oracle.pair(1, 1, (15.0 - eps) ** 2, p)[1] != 0.0
    assert oracle.pair(1, 1, (15.0 + eps) ** 2, p)[1] == 0.0
    # nuclear tail at the cutoff is below 1e-20 MeV
    assert abs(oracle.pair(1, 0, (11.5 - eps) ** 2, p)[0]) < 1e-20


def test_spot_values_two_body():
    """Spot values of Eq. (1) at r = 1 fm."""
    p = P(r_C=20.0)
    vn, vc, g = oracle.pair(1, 0, 1.0, p)
    assert abs(vn - 15.910184) < 1e-6 and abs(g - 52.269096) < 1e-6
    vn, vc, g = oracle.pair(0, 0, 1.0, p)
    assert abs(vn - 48.085546) < 1e-6
    vn, vc, g = oracle.pair(1, 1, 1.0, p)
    assert abs(vn + vc - 49.388480) < 1e-6 and abs(g - 79.442613) < 1e-6


# -------------------------------------------------------- sums over pairs

def _images_bruteforce(x, t, L, p):
    """Independent O(27 N^2) sum: enumerate all 27 images of each source and
    keep those inside the cutoffs (valid because r_cut <= L/2)."""
    N = len(x)
    F = np.zeros((N, 3))
    E = np.zeros(2)
    shifts = np.array([(i, j, k) for i in (-1, 0, 1) for j in (-1, 0, 1) for k in (-1, 0, 1)], float) * L
    for i in range(N):
        for j in range(N):
            if i == j:
                continue
            for s in shifts:
                d = x[i] - (x[j] + s)
                r2 = float(d @ d)
                vn, vc, g = oracle.pair(int(t[i]), int(t[j]), r2, p)
                F[i] += g * d
                E += 0.5 * np.array([vn, vc])
    return F, E


def test_forces_match_image_enumeration():
    L = 24.0
    x, t = inputs.uniform(40, 0.4, L, seed=11, min_sep=0.8)
    p = P(r_C=L / 2)
    F, (en, ec, w) = oracle.forces(x, t, L, p)
    Fb, Eb = _images_bruteforce(x, t, L, p)
    assert np.allclose(F, Fb, rtol=1e-11, atol=1e-11)
    assert abs(en - Eb[0]) < 1e-10 * (abs(Eb[0]) + 1)
    assert abs(ec - Eb[1]) < 1e-10 * (abs(Eb[1]) + 1)


def test_newton_third_law_and_invariances():
    L = 30.0
    x, t = inputs.uniform(120, 0.3, L, seed=5, min_sep=0.9)
    p = P(r_C=L / 2)
    F, E = oracle.forces(x, t, L, p)
    scale = np.abs(F).sum()
    assert np.abs(F.sum(0)).max() <= 1e-12 * scale
    # translation invariance (shift mod L)
    rng = np.random.default_rng(3)
    xs = np.mod(x + rng.random(3) * L, L)
    F2, E2 = oracle.forces(xs, t, L, p)
    assert np.allclose(F2, F, rtol=1e-9, atol=1e-10 * scale / len(x))
    assert all(abs(a - b) <= 1e-10 * (abs(a) + 1) for a, b in zip(E, E2))
    # permutation invariance
    perm = rng.permutation(len(x))
    F3, E3 = oracle.forces(x[perm], t[perm], L, p)
    assert np.allclose(F3, F[perm], rtol=1e-11, atol=1e-12)
    assert all(abs(a - b) <= 1e-11 * (abs(a) + 1) for a, b in zip(E, E3))


def test_force_is_minus_energy_gradient():
    """Central finite differences of the total potential energy (drop that
    straddles the periodic corner, all pairs inside both cutoffs)."""
    L = 60.0
    x, t = inputs.drop(9, 11, L, center=(0.3, 59.8, 0.1), seed=2, spacing=1.7)
    p = P(r_C=25.0)
    F, _ = oracle.forces(x, t, L, p)

    def pe(xx):
        _, e = oracle.forces(xx, t, L, p)
        return e[0] + e[1]

    h = 1e-4
    for i in (0, 3, 9, 15, 19):
        for a in range(3):
            xp = x.copy(); xp[i, a] += h
            xm = x.copy(); xm[i, a] -= h
            fd = -(pe(xp) - pe(xm)) / (2 * h)
            assert abs(fd - F[i, a]) <= 1e-6 * (abs(F[i, a]) + 1e-3)


def test_target_range_and_virial():
    L = 26.0
    x, t = inputs.uniform(60, 0.5, L, seed=8, min_sep=0.8)
    p = P(r_C=L / 2)
    F, (en, ec, w) = oracle.forces(x, t, L, p)
    Fa, ea = oracle.forces(x, t, L, p, 0, 25)
    Fb, eb = oracle.forces(x, t, L, p, 25, 60)
    assert np.array_equal(Fa[:25], F[:25]) and np.array_equal(Fb[25:], F[25:])
    assert abs(ea[0] + eb[0] - en) < 1e-11 * abs(en)
    # virial W = sum_{i<j} r_ij . F_ij equals 1/2 sum_i x_i^(unwrapped pair) ...
    # check against an explicit pair loop
    wsum = 0.0
    for i in range(60):
        for j in range(i + 1, 60):
            d = x[i] - x[j]
            d -= L * np.round(d / L)
            g = oracle.pair(int(t[i]), int(t[j]), float(d @ d), p)[2]
            wsum += g * float(d @ d)
    assert abs(wsum - w) < 1e-10 * (abs(w) + 1)


# ------------------------------------------------------------ integrator

def _energy(x, v, t, L, p):
    _, e = oracle.forces(x, t, L, p)
    return oracle.kinetic(v) + e[0] + e[1]


def test_verlet_energy_error_second_order():
    L = 90.0
    x, t = inputs.drop(6, 8, L, center=(45, 45, 45), seed=4, spacing=1.9)
    v = inputs.maxwell(len(x), 0.5, seed=9)
    p = P(r_C=40.0)
    E0 = _energy(x, v, t, L, p)
    errs = []
    dts = [2.0, 1.0, 0.5, 0.25]
    for dt in dts:
        n = int(round(60.0 / dt))
        xx, vv = x.copy(), v.copy()
        F = None
        dev = 0.0
        tt, st = 0.0, 0
        for _ in range(4):
            r = oracle.run(xx, vv, t, L, p, n // 4, dt=dt, F=F, t=tt, step=st)
            xx, vv, F, tt, st = r["x"], r["v"], r["F"], r["t"], r["step"]
            dev = max(dev, abs(_energy(xx, vv, t, L, p) - E0))
        errs.append(dev)
    slope = np.polyfit(np.log(dts), np.log(errs), 1)[0]
    assert 1.8 <= slope <= 2.2, (errs, slope)


def test_verlet_time_reversible():
    L = 40.0
    x, t = inputs.drop(5, 7, L, center=(20, 20, 20), seed=6)
    v = inputs.maxwell(len(x), 1.0, seed=1)
    p = P(r_C=20.0)
    r = oracle.run(x, v, t, L, p, 50)
    back = oracle.run(r["x"], -r["v"], t, L, p, 50, F=r["F"])
    d = back["x"] - x
    d -= L * np.round(d / L)
    assert np.abs(d).max() < 1e-9
    assert np.abs(-back["v"] - v).max() < 1e-11


def test_two_body_head_on_conserves_momentum_and_energy():
    L = 50.0
    x = np.array([[20.0, 25.0, 25.0], [30.0, 25.0, 25.0]])
    t = np.array([0, 0], dtype=np.int8)
    v = np.array([[0.08, 0.0, 0.0], [-0.08, 0.0, 0.0]])
    p = P(r_C=20.0)
    E0 = _energy(x, v, t, L, p)
    r = oracle.run(x, v, t, L, p, 200, dt=0.5)
    assert np.abs(r["v"].sum(0)).max() < 1e-15
    assert abs(_energy(r["x"], r["v"], t, L, p) - E0) < 1e-4 * abs(E0)
    # they bounced: relative velocity reversed
    assert r["v"][0, 0] < 0 < r["v"][1, 0]


def test_expansion_law_and_no_position_rescaling():
    """Eq. (3): L(t) = L(0)(1 + xi t).  The configuration's 20,000 steps of
    dt = 2 fm/c at xi = 3/40000 c/fm take the side from L0 to 4 L0
    (density 0.080 -> 0.00125).  Positions are not rescaled (Sec. II.A): two
    non-interacting neutrons move ballistically whatever the rate."""
    g = json.loads((GOLD / "expansion_endpoints.json").read_text())
    for N, L0, Le in zip(g["N"], g["L0_fm"], g["L_end_fm"]):
        assert abs(inputs.box_side(N, g["rho_start"]) - L0) < 1e-3
        assert abs(inputs.box_side(N, g["rho_end"]) - Le) < 1e-2
    x = np.array([[35.0, 40.0, 45.0], [60.0, 62.0, 66.0]])
    t = np.array([0, 0], dtype=np.int8)
    v = np.array([[0.015, -0.012, 0.01], [0.0, 0.013, -0.014]])
    p = P(r_C=10.0)
    L0 = 100.0
    xi = 3.0 / 40000.0
    r = oracle.run(x, v, t, L0, p, 1000, xi_dot=xi)
    assert r["L"] == L0 * (1.0 + xi * r["t"])
    assert abs(r["L"] / L0 - (1 + xi * 2000.0)) < 1e-15
    assert np.array_equal(r["v"], v)
    # the chosen velocities keep both particles inside [0, L0) for 2000 fm/c
    assert np.abs(r["x"] - (x + v * 2000.0)).max() < 1e-9
    r0 = oracle.run(x, v, t, L0, p, 1000, xi_dot=0.0)
    assert r0["L"] == L0 and np.allclose(r0["x"], r["x"], atol=1e-9)
    # full-run endpoint: side grows by exactly the golden ratio 4
    assert abs((1.0 + xi * 20000 * 2.0) - g["side_ratio"]) < 1e-15


def test_wrap_into_box():
    L = 7.3
    for x in (-1e-18, -0.5, 0.0, 3.1, 7.3, 7.3 + 1e-12, 14.0):
        w = oracle.wrap(x, L)
        assert 0.0 <= w < L
        k = round((x - w) / L)
        assert abs(x - w - k * L) < 1e-12


def test_thermostat_rescales_to_three_halves_T():
    L = 30.0
    x, t = inputs.lattice_liquid(216, 0.3, L, seed=1)
    v = inputs.maxwell(216, 2.0, seed=2)
    p = P(r_C=15.0)
    r = oracle.run(x, v, t, L, p, 100, T=1.0, thermostat_every=100)
    ke = oracle.kinetic(r["v"])
    assert abs(ke - 1.5 * 216 * 1.0) < 1e-12 * ke
    r = oracle.run(x, v, t, L, p, 99, T=1.0, thermostat_every=100)
    assert abs(oracle.kinetic(r["v"]) - 1.5 * 216) > 1e-3


# ----------------------------------------------------------- initial state

def test_splitmix64_reference_vector():
    g = json.loads((GOLD / "splitmix64_vectors.json").read_text())
    out = [oracle.splitmix64(g["seed"], k) for k in range(5)]
    assert out == [int(s) for s in g["outputs"]]


def test_init_state_properties():
    N, Yp, rho, T = 20000, 0.3, 0.08, 1.0
    x, v, t, L = oracle.init(N, Yp, rho, T, 7, P())
    assert abs(L - (N / rho) ** (1 / 3)) < 1e-12
    assert int(t.sum()) == 6000 and t[:6000].all() and not t[6000:].any()
    assert x.min() >= 0 and x.max() < L
    # positions are U(k) * L with U from the stream
    u0 = (oracle.splitmix64(7, 0) >> 11) * 2.0 ** -53
    assert x[0, 0] == u0 * L
    assert np.abs(x.mean(0) / L - 0.5).max() < 0.01
    assert np.abs(v.sum(0)).max() < 1e-12
    assert abs(oracle.kinetic(v) - 1.5 * N * T) < 1e-10 * 1.5 * N * T
    # Gaussian shape: excess kurtosis ~ 0 (uniform would give -1.2)
    z = v.ravel() / v.std()
    assert abs((z ** 4).mean() - 3.0) < 0.1
    x0, v0, _, _ = oracle.init(N, Yp, rho, 0.0, 7, P())
    assert np.array_equal(x0, x) and not v0.any()


def test_relax_lowers_energy():
    N = 300
    x, v, t, L = oracle.init(N, 0.3, 0.08, 1.0, 3, P())
    p = P(r_C=L / 2)
    e0 = sum(oracle.forces(x, t, L, p)[1][:2])
    x1 = oracle.relax(x, t, L, p, 30)
    e1 = sum(oracle.forces(x1, t, L, p)[1][:2])
    assert e1 < e0
    d = x1 - x
    d -= L * np.round(d / L)
    assert np.sqrt((d * d).sum(1)).max() <= 30 * 0.1 + 1e-12
    assert x1.min() >= 0 and x1.max() < L


@pytest.mark.parametrize("r,clamped", [(1.6, False), (1.3, True)])
def test_relax_one_iteration_by_hand(r, clamped):
    """One steepest-descent iteration on two neutrons, written out from Table I.

    Two neutrons (nn: s = b + c) at separation r along the diagonal (1, 1, 0)/sqrt(2).
    The force on neutron 0 is F = r_vec ((2a/Lambda) g^2 + (s/Lambda) g),
    g = exp(-r^2 / 2 Lambda) (Eq. 1), so each moves by gamma |F| along the
    separation, outward, unless gamma |F| > dmax, when the displacement VECTOR is
    scaled to length dmax.  At r = 1.6 fm gamma |F| = 0.0708 fm (no clamp); at
    r = 1.3 fm gamma |F| = 0.1163 fm > 0.1 while each component is 0.0822 < 0.1,
    so a per-component clamp would leave it unchanged and fails here, as would a
    wrong gamma, a wrong sign or a dropped Gaussian."""
    a, b, c, Lam = T1["a_MeV"], T1["b_MeV"], T1["c_MeV"], T1["Lambda_fm2"]
    gamma, dmax = 0.002, 0.1
    s = b + c
    g = math.exp(-r * r / (2.0 * Lam))
    fmag = r * ((2.0 * a / Lam) * g * g + (s / Lam) * g)        # |F|, repulsive here
    step = gamma * fmag
    assert (step > dmax) == clamped
    if clamped:
        assert step / math.sqrt(2.0) < dmax                     # components below the clamp
        step = dmax
    u = np.array([1.0, 1.0, 0.0]) / math.sqrt(2.0)
    L = 100.0
    c0 = np.array([40.0, 40.0, 40.0])
    x = np.array([c0, c0 + r * u])
    t = np.zeros(2, dtype=np.int8)                               # two neutrons
    p = P(r_C=20.0)
    x1 = oracle.relax(x, t, L, p, 1, gamma=gamma, dmax=dmax)
    expect = np.array([c0 - step * u, c0 + (r + step) * u])
    assert np.abs(x1 - expect).max() < 1e-12


# ---------------------------------------------------------------- clusters

def test_cluster_chain_threshold():
    L = 200.0
    for sp, expect in ((4.49, 1), (4.51, 10)):
        x = np.array([[10 + k * sp, 50.0, 50.0] for k in range(10)])
        t = np.ones(10, dtype=np.int8)
        lab, hA, hZ, st = oracle.clusters(x, t, L)
        assert st[0] == expect
        if expect == 1:
            assert (lab == 0).all() and hA[10] == 1 and hZ[10] == 1
        else:
            assert (lab == np.arange(10)).all() and hA[1] == 10


def test_cluster_neutron_radius_periodic_and_ties():
    L = 40.0
    x = np.array([[0.5, 20.0, 20.0],      # p0
                  [39.0, 20.0, 20.0],     # p1, 1.5 fm from p0 through the face
                  [20.0, 20.0, 20.0],     # p2 alone
                  [10.0, 10.0, 10.0],     # p3
                  [15.0, 10.0, 10.0],     # p4, 5 fm from p3: separate cluster
                  [20.0, 22.99, 20.0],    # n: 2.99 from p2 -> bound
                  [20.0, 16.99, 20.0],    # n: 3.01 from p2 -> free
                  [12.5, 10.0, 10.0],     # n: 2.5 from p3 and p4 -> tie -> p3
                  [37.5, 20.0, 20.0]])    # n: 1.5 from p1, 3 from p0(through face)
    t = np.array([1, 1, 1, 1, 1, 0, 0, 0, 0], dtype=np.int8)
    lab, hA, hZ, st = oracle.clusters(x, t, L)
    assert list(lab) == [0, 0, 2, 3, 4, 2, -1, 3, 0]
    assert st[0] == 4 and st[1] == 1 / 9
    assert hA[3] == 1 and hA[2] == 2 and hA[1] == 1
    assert hZ[2] == 1 and hZ[1] == 3


def _bfs_clusters(x, t, L, rpp=4.5, rnp=3.0):
    N = len(x)
    pi = np.flatnonzero(t == 1)
    d = x[:, None, :] - x[None, :, :]
    d -= L * np.round(d / L)
    D2 = (d * d).sum(-1)
    lab = -np.ones(N, dtype=np.int64)
    seen = set()
    for a in pi:
        if a in seen:
            continue
        comp, stack = [a], [a]
        seen.add(a)
        while stack:
            u = stack.pop()
            for b in pi:
                if b not in seen and D2[u, b] < rpp * rpp:
                    seen.add(b); comp.append(b); stack.append(b)
        m = min(comp)
        for c in comp:
            lab[c] = m
    for n in np.flatnonzero(t == 0):
        best = None
        for b in pi:
            if D2[n, b] < rnp * rnp and (best is None or D2[n, b] < D2[n, best]):
                best = b
        if best is not None:
            lab[n] = lab[best]
    return lab


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_clusters_match_bfs(seed):
    L = 22.0
    x, t = inputs.uniform(150, 0.35, L, seed=seed)
    lab, hA, hZ, st = oracle.clusters(x, t, L)
    assert np.array_equal(lab, _bfs_clusters(x, t, L))
    assert hA.sum() == st[0] and (np.arange(len(hA)) * hA).sum() == (lab >= 0).sum()
    assert (np.arange(len(hZ)) * hZ).sum() == (t == 1).sum()


def test_expansion_rebase_keeps_L_continuous():
    """Changing the rate mid-run re-bases Eq. (3) at the current time: the
    side is continuous and then grows linearly from its current value."""
    x = np.array([[35.0, 40.0, 45.0], [60.0, 62.0, 66.0]])
    t = np.array([0, 0], dtype=np.int8)
    v = np.zeros((2, 3))
    p = P(r_C=10.0)
    L0 = 100.0
    r1 = oracle.run(x, v, t, L0, p, 100, xi_dot=1e-4)
    L1, t1 = r1["L"], r1["t"]
    assert abs(L1 - L0 * (1 + 1e-4 * 200.0)) < 1e-12
    r2 = oracle.run(r1["x"], r1["v"], t, L1, p, 1, xi_dot=3e-4, t=t1, step=r1["step"],
                    L_base=L1, t_base=t1, F=r1["F"])
    assert abs(r2["L"] - L1 * (1 + 3e-4 * 2.0)) < 1e-12
    r3 = oracle.run(r1["x"], r1["v"], t, L1, p, 50, xi_dot=3e-4, t=t1, step=r1["step"],
                    L_base=L1, t_base=t1, F=r1["F"])
    assert abs(r3["L"] - L1 * (1 + 3e-4 * 100.0)) < 1e-12


def test_thomas_fermi_lambda_eq2_limits():
    """Eq. (2): for k_F >> m_e, lambda -> sqrt(pi)/(2 sqrt(alpha) k_F); for
    k_F << m_e, lambda -> sqrt(pi)/(2 sqrt(alpha)) (k_F m_e)^(-1/2).  At
    the Y_p = 0.4 proton density 0.032 fm^-3 it is slightly above the 10 fm
    the paper fixes (Sec. II.A)."""
    alpha = 1 / 137.035999084
    me = 0.51099895 / 197.3269804
    pre = math.sqrt(math.pi) / (2 * math.sqrt(alpha))
    ne = 10.0
    kF = (3 * math.pi ** 2 * ne) ** (1 / 3)
    assert abs(oracle.lambda_tf(ne) / (pre / kF) - 1) < 1e-5
    ne = 1e-14
    kF = (3 * math.pi ** 2 * ne) ** (1 / 3)
    assert abs(oracle.lambda_tf(ne) / (pre / math.sqrt(kF * me)) - 1) < 1e-3
    lam = oracle.lambda_tf(0.4 * 0.08)
    assert 10.0 < lam < 11.0
    assert oracle.lambda_tf(0.05 * 0.08) > lam     # decreasing in density


def test_affine_option_scales_positions_with_the_box():
    x = np.array([[35.0, 40.0, 45.0], [60.0, 62.0, 66.0]])
    t = np.array([0, 0], dtype=np.int8)
    v = np.zeros((2, 3))
    p = P(r_C=10.0)
    r = oracle.run(x, v, t, 100.0, p, 10, xi_dot=1e-3, affine=True)
    assert np.allclose(r["x"] / x, r["L"] / 100.0, rtol=1e-13)
    r0 = oracle.run(x, v, t, 100.0, p, 10, xi_dot=1e-3)
    assert np.array_equal(r0["x"], x)


# ------------------------------------------------------------------ MSTE
# Energy-criterion clusters (reading of Sec. II.C: the paper names MSTE
# without defining it): i, j bound when V_ij + (M/4)|v_i - v_j|^2 < 0.

def _pair_min_r(s, a=110.0, Lam=1.25):
    """Eq. (1) nuclear term a g^2 + s g, g = exp(-r^2/(2 Lambda)): minimum
    -s^2/(4a) at g = -s/(2a)."""
    r2 = 2.0 * Lam * math.log(2.0 * a / abs(s))
    return math.sqrt(r2), -s * s / (4.0 * a)


def _mste2(t0, t1, r, dv=0.0, L=60.0, coulomb=True):
    x = np.array([[20.0, 20.0, 20.0], [20.0 + r, 20.0, 20.0]])
    v = np.zeros((2, 3))
    v[1, 1] = dv
    t = np.array([t0, t1], dtype=np.int8)
    return oracle.mste(x, v, t, L, P(r_C=20.0, coulomb=coulomb))


def test_mste_np_pair_binding_threshold():
    r, vmin = _pair_min_r(-26.0 - 24.0)                 # unlike species: s = b - c
    lab, hA, hZ, st = _mste2(1, 0, r)
    assert list(lab) == [0, 0] and hA[2] == 1 and hZ[1] == 1 and st[0] == 1 and st[1] == 0
    M = 939.0
    for f, bound in ((1.0 - 1e-9, True), (1.0 + 1e-9, False)):
        dv = math.sqrt(4.0 * (-vmin) * f / M)          # (M/4) dv^2 = f |V_min|
        lab, hA, hZ, st = _mste2(1, 0, r, dv)
        if bound:
            assert list(lab) == [0, 0]
        else:                                            # lone proton is a cluster, neutron free
            assert list(lab) == [0, -1] and hA[1] == 1 and st[1] == 0.5


def test_mste_like_pairs_and_coulomb():
    r, vmin = _pair_min_r(-26.0 + 24.0)                 # like species: s = b + c
    lab, hA, hZ, st = _mste2(0, 0, r)                    # nn at rest: bound, no proton
    assert list(lab) == [0, 0] and hZ[0] == 1 and st[0] == 1
    lab, _, _, st = _mste2(1, 1, r)                       # pp: Coulomb (~0.3 MeV) unbinds
    assert list(lab) == [0, 1] and st[0] == 2
    lab, _, _, _ = _mste2(1, 1, r, coulomb=False)        # without it the pp pair binds
    assert list(lab) == [0, 0]


def test_mste_strict_nuclear_range_and_periodic_image():
    # at rest any r < r_nuc binds an np pair (V < 0, however small); r_nuc is strict
    assert list(_mste2(1, 0, 11.4)[0]) == [0, 0]
    assert list(_mste2(1, 0, 11.6)[0]) == [0, -1]
    assert list(_mste2(1, 0, 11.5)[0]) == [0, -1]        # r^2 = 132.25 exactly, not < r_nuc^2
    # the same pair across the periodic face
    r, _ = _pair_min_r(-50.0)
    x = np.array([[0.2, 5.0, 5.0], [0.2 - r + 30.0, 5.0, 5.0]])
    lab, _, _, _ = oracle.mste(x, np.zeros((2, 3)), np.array([0, 1], dtype=np.int8), 30.0, P(r_C=10.0))
    assert list(lab) == [0, 0]


def test_mste_chain_connectivity():
    """n - p - n, each neutron at the np minimum distance from the proton:
    connected through the proton, one cluster A = 3, Z = 1."""
    r, _ = _pair_min_r(-50.0)
    x = np.array([[20.0 - r, 20.0, 20.0], [20.0, 20.0, 20.0], [20.0 + r, 20.0, 20.0]])
    v = np.zeros((3, 3))
    v[0, 2], v[2, 2] = 0.01, -0.01
    t = np.array([0, 1, 0], dtype=np.int8)
    lab, hA, hZ, st = oracle.mste(x, v, t, 60.0, P(r_C=20.0))
    assert list(lab) == [0, 0, 0] and hA[3] == 1 and hZ[1] == 1


def test_mste_bfs_on_random_inputs():
    """Independent brute force: the bound-pair matrix from numpy and a BFS."""
    rng = np.random.default_rng(5)
    for trial in range(4):
        N, L = 60, 14.0
        x = rng.uniform(0, L, (N, 3))
        v = rng.normal(0, 0.02, (N, 3))
        t = (rng.uniform(size=N) < 0.4).astype(np.int8)
        p = P(r_C=7.0)
        lab, hA, hZ, st = oracle.mste(x, v, t, L, p)
        d = x[:, None, :] - x[None, :, :]
        d -= L * np.round(d / L)
        r2 = (d ** 2).sum(-1)
        g = np.exp(-r2 / 2.5)
        s = np.where(t[:, None] == t[None, :], -2.0, -50.0)
        V = 110.0 * g * g + s * g
        pp = (t[:, None] == 1) & (t[None, :] == 1) & (r2 < 49.0)
        with np.errstate(divide="ignore", invalid="ignore"):
            r = np.sqrt(r2)
            V = V + np.where(pp, 1.4399645 * np.exp(-r / 10.0) / np.where(r > 0, r, 1.0), 0.0)
        e = V + 0.25 * 939.0 * ((v[:, None, :] - v[None, :, :]) ** 2).sum(-1)
        B = (e < 0.0) & (r2 < 11.5 ** 2)
        np.fill_diagonal(B, False)
        ref = np.full(N, -1)
        for i in range(N):
            if ref[i] >= 0 or (t[i] == 0 and not B[i].any()):
                continue
            comp, stack = {i}, [i]
            while stack:
                k = stack.pop()
                for j in np.nonzero(B[k])[0]:
                    if j not in comp:
                        comp.add(j)
                        stack.append(j)
            for j in comp:
                ref[j] = min(comp)
        assert np.array_equal(lab, ref), trial
        assert B.sum() > 0

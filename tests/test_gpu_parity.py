"""GPU path vs the FP64 oracle, element by element, through the C ABI.

Tolerances (the path's stated targets):
  forces, split precision   relative L2 <= 1e-5 per evaluation
  forces, FP64 mode         relative L2 <= 1e-11
  energies                  |dE| <= 1e-6 (|KE| + |PE_nuc| + |PE_coul|)
  FP64 trajectory, 50 steps positions within 1e-6 fm, velocities rel L2 1e-6
  clusters                  bit-exact labels, histograms and statistics
"""
import numpy as np
import pytest

import inputs
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def md():
    from paper_1412_8502_b300 import md as m
    return m


def make(md, N, Yp, rho, T=1.0, seed=1, precision=0, relax=0, **kw):
    p = md.md_params_default()
    p.precision = precision
    p.relax_iters = relax
    for k, v in kw.items():
        setattr(p, k, v)
    return md.System(N, Yp, rho, T, seed, p)


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def oparams(sys):
    p = sys.params
    return oracle.params(p.r_C, coulomb=bool(p.coulomb), r_nuc=p.r_nuc, lambda_s=p.lambda_s)


def min_img(d, L):
    return d - L * np.round(d / L)


# --------------------------------------------------------------- configurations
def cfg_liquid(N, Yp, rho, seed):
    L = inputs.box_side(N, rho)
    x, t = inputs.lattice_liquid(N, Yp, L, seed)
    return x, t, L


def cfg_drops(N, Yp, rho, seed):
    """Nucleus-like drops (Z ~ 20-45, A ~ 50-110) on a jittered coarse grid of
    centres (no overlaps) plus a free-neutron gas at least 1 fm from all
    other particles; low mean density."""
    L = inputs.box_side(N, rho)
    rng = np.random.default_rng(seed)
    Np = int(np.floor(Yp * N + 0.5))
    ng = max(1, int(L // 16.0))
    cells = rng.permutation(ng ** 3)
    xs_p, xs_n = [], []
    left_p, left_n = Np, N - Np
    k = 0
    while left_p > 0:
        c = cells[k % len(cells)]
        centre = (np.array([c // (ng * ng), (c // ng) % ng, c % ng]) + 0.5 + 0.2 * (rng.random(3) - 0.5)) * (L / ng)
        zp = min(left_p, int(rng.integers(20, 45)))
        zn = min(left_n, int(zp * 1.4))
        x, t = inputs.drop(zp, zn, L, centre, seed + 17 * k, spacing=1.85)
        xs_p.append(x[t == 1]); xs_n.append(x[t == 0])
        left_p -= zp; left_n -= zn; k += 1
    taken = np.concatenate(xs_p + xs_n)
    gas = []
    while len(gas) < left_n:
        q = rng.random(3) * L
        d = taken - q
        d -= L * np.round(d / L)
        if (d * d).sum(1).min() > 1.0:
            gas.append(q)
            taken = np.vstack([taken, q])
    if gas:
        xs_n.append(np.array(gas))
    x = np.concatenate(xs_p + xs_n)
    return x, inputs.species(N, Yp), L


def cfg_relaxed(N, Yp, rho, seed, iters=40):
    x, v, t, L = oracle.init(N, Yp, rho, 1.0, seed, oracle.params(min(40.0, 0.5 * inputs.box_side(N, rho))))
    x = oracle.relax(x, t, L, oracle.params(min(40.0, L / 2)), iters)
    return x, t, L


PARITY_CASES = {
    "liquid_2000": lambda: cfg_liquid(2000, 0.30, 0.080, 3),
    "liquid_8000_yp04": lambda: cfg_liquid(8000, 0.40, 0.080, 4),
    "drops_3000_dilute": lambda: cfg_drops(3000, 0.30, 0.005, 5),
    "relaxed_1500": lambda: cfg_relaxed(1500, 0.30, 0.080, 6),
    "liquid_4096_yp005": lambda: cfg_liquid(4096, 0.05, 0.030, 7),
    # the late expansion: drops in a 464 fm box (coordinates as large as at
    # the end of the 409,600 run's schedule, where the FP32 screens and the
    # hi + lo separations work on the largest magnitudes)
    "drops_20000_L464": lambda: cfg_drops(20000, 0.40, 0.0002, 8),
}


def load(md, x, t, L, precision, T=1.0, seed=11, **kw):
    N = len(x)
    Yp = float(t.sum()) / N
    rho = N / L ** 3
    s = make(md, N, Yp, rho, precision=precision, **kw)
    assert s.Np == int(t.sum())
    v = inputs.maxwell(N, T, seed)
    s.set_state(x, v, L)
    return s, v


# --------------------------------------------------------------- generator
@pytest.mark.parametrize("args", [(2000, 0.30, 0.080, 1.0, 1), (777, 0.05, 0.010, 0.5, 9), (64, 1.0, 0.05, 0.0, 3)])
def test_create_generator_matches_oracle(md, args):
    N, Yp, rho, T, seed = args
    s = make(md, N, Yp, rho, T=T, seed=seed, relax=0)
    st = s.state()
    x, v, t, L = oracle.init(N, Yp, rho, T, seed, oracle.params(1.0))
    assert st["L"] == L
    assert np.array_equal(st["x"], x)
    assert np.array_equal(st["type"], t)
    scale = max(np.abs(v).max(), 1e-300)
    assert np.abs(st["v"] - v).max() <= 1e-13 * scale


def test_relax_fp64_matches_oracle(md):
    N, Yp, rho = 400, 0.3, 0.08
    s = make(md, N, Yp, rho, relax=6, precision=1)
    x, v, t, L = oracle.init(N, Yp, rho, 1.0, 1, oracle.params(1.0))
    xr = oracle.relax(x, t, L, oparams(s), 6)
    d = min_img(s.state()["x"] - xr, L)
    assert np.abs(d).max() < 1e-9


# --------------------------------------------------------------- forces
@pytest.mark.parametrize("name", list(PARITY_CASES))
@pytest.mark.parametrize("precision", [0, 1])
def test_forces_and_energy_vs_oracle(md, name, precision):
    x, t, L = PARITY_CASES[name]()
    s, v = load(md, x, t, L, precision)
    F = s.forces()
    Fo, (en, ec, w) = oracle.forces(x, t, L, oparams(s))
    tol = 1e-5 if precision == 0 else 1e-11
    assert rel_l2(F, Fo) <= tol, rel_l2(F, Fo)
    e = s.energy()
    ke = oracle.kinetic(v)
    scale = abs(ke) + abs(en) + abs(ec)
    etol = 1e-6 if precision == 0 else 1e-12
    assert abs(e["KE"] - ke) <= 1e-12 * ke
    assert abs(e["PE_nuc"] - en) <= etol * scale, (e["PE_nuc"], en)
    assert abs(e["PE_coul"] - ec) <= etol * scale, (e["PE_coul"], ec)
    assert abs(e["virial"] - w) <= etol * (abs(w) + scale)
    # md_energy must leave the cached forces alone
    assert np.array_equal(s.forces(), F)


@pytest.mark.parametrize("precision", [0, 1])
def test_edge_cases(md, precision):
    L = 30.0
    cases = [
        (np.array([[10.0, 10.0, 10.0], [11.5, 10.0, 10.0]]), np.array([1, 0], np.int8)),         # N = 2
        (np.array([[0.0, 0.0, 0.0], [29.9, 29.5, 0.4], [15.0, 0.0, 29.999999]]),
         np.array([1, 1, 0], np.int8)),                                                          # faces
    ]
    rng = np.random.default_rng(0)
    x, _ = inputs.uniform(200, 0.0, L, seed=1, min_sep=0.9)
    cases.append((x, np.zeros(200, np.int8)))                                                     # all neutrons
    x, _ = inputs.uniform(150, 1.0, L, seed=2, min_sep=0.9)
    cases.append((x, np.ones(150, np.int8)))                                                      # all protons
    for x, t in cases:
        s, v = load(md, x, t, L, precision)
        F = s.forces()
        Fo, _ = oracle.forces(x, t, L, oparams(s))
        tol = 1e-5 if precision == 0 else 1e-11
        assert rel_l2(F, Fo) <= tol, (len(x), rel_l2(F, Fo))


def test_ragged_tiles_and_many_sizes(md):
    """Sizes that leave partial 32-particle tiles in both species."""
    for N, Yp in ((33, 0.5), (65, 0.3), (97, 0.71), (1000, 0.013), (1025, 0.5)):
        x, t, L = cfg_liquid(N, Yp, 0.08 if N > 500 else 0.02, N)
        s, _ = load(md, x, t, L, 0)
        F = s.forces()
        Fo, _ = oracle.forces(x, t, L, oparams(s))
        assert rel_l2(F, Fo) <= 1e-5, (N, Yp, rel_l2(F, Fo))


# --------------------------------------------------------------- dynamics
def test_trajectory_fp64_50_steps(md):
    x, t, L = cfg_liquid(2000, 0.30, 0.080, 21)
    s, v = load(md, x, t, L, 1, T=1.0, thermostat_every=0)
    s.step(50, 0.0)
    g = s.state()
    r = oracle.run(x, v, t, L, oparams(s), 50)
    assert g["t"] == r["t"] and g["step"] == 50
    assert np.abs(min_img(g["x"] - r["x"], L)).max() < 1e-6
    assert rel_l2(g["v"], r["v"]) < 1e-6
    e = s.energy()
    _, (en, ec, _) = oracle.forces(r["x"], t, L, oparams(s))
    ke = oracle.kinetic(r["v"])
    assert abs(e["KE"] + e["PE_nuc"] + e["PE_coul"] - (ke + en + ec)) < 1e-6 * (ke + abs(en) + abs(ec))


def test_trajectory_fp64_expansion_and_thermostat(md):
    x, t, L = cfg_liquid(1200, 0.40, 0.080, 22)
    s, v = load(md, x, t, L, 1, T=1.0, thermostat_every=20)
    p = s.params
    p.T = 1.0
    s.params = p
    xi = 7.5e-5
    s.step(50, xi)
    g = s.state()
    r = oracle.run(x, v, t, L, oparams(s), 50, xi_dot=xi, T=1.0, thermostat_every=20)
    assert g["L"] == r["L"] and g["t"] == r["t"]
    assert np.abs(min_img(g["x"] - r["x"], r["L"])).max() < 1e-6
    assert rel_l2(g["v"], r["v"]) < 1e-6
    Fo = r["F"]
    assert rel_l2(s.forces(), Fo) < 1e-9


def test_split_single_step_from_oracle_state(md):
    x, t, L = cfg_relaxed(2000, 0.30, 0.080, 23)
    s, v = load(md, x, t, L, 0, T=1.0, thermostat_every=0)
    s.step(1, 0.0)
    g = s.state()
    r = oracle.run(x, v, t, L, oparams(s), 1)
    assert np.abs(min_img(g["x"] - r["x"], L)).max() < 1e-6
    assert rel_l2(g["v"], r["v"]) < 1e-5
    assert rel_l2(s.forces(), r["F"]) < 1e-5


def test_split_trajectory_50_steps_vs_oracle(md):
    """Split precision (FP32 pair arithmetic) over 50 steps from an oracle
    state, 2,000-nucleon liquid, NVE, against the FP64 oracle (Sec. II.A).
    While the trajectories are close (through step 5) positions agree within
    1e-6 fm and velocities within 1e-6 relative; the total energy of the two
    trajectories agrees within 1e-6 relative through step 20.  The positions
    then separate exponentially (measured: 1.3e-7 fm after 1 step, 1.5e-6
    after 10, 1e-5 after 20, 2.7e-3 after 50): the dynamics amplify
    differences at the FP32 rounding level.  The oracle shows the same:
    started from positions moved by 1e-7 fm (random signs), it separates from
    its own unperturbed run by the same order after 50 steps.  At step 50 the
    two runs are therefore different states, whose total energies differ by
    the integrator's own fluctuation (the oracle's total energy moves by
    1e-3 relative between steps 20 and 50 of this start); there the energies
    the GPU records are compared with the oracle's on the GPU's own state,
    and the separation with the oracle's own amplification.  Beyond the
    first steps the split mode is compared statistically
    (test_gpu_statistics)."""
    x, t, L = cfg_liquid(2000, 0.30, 0.080, 21)
    s, v = load(md, x, t, L, 0, T=1.0, thermostat_every=0)
    op = oparams(s)

    def e_oracle(xx, vv):
        _, (en, ec, _) = oracle.forces(xx, t, L, op)
        ke = oracle.kinetic(vv)
        return ke + en + ec, ke + abs(en) + abs(ec)

    s.step(5, 0.0)
    g = s.state()
    r5 = oracle.run(x, v, t, L, op, 5)
    assert np.abs(min_img(g["x"] - r5["x"], L)).max() < 1e-6
    assert rel_l2(g["v"], r5["v"]) < 1e-6
    s.step(15, 0.0)
    e = s.energy()
    r20 = oracle.run(r5["x"], r5["v"], t, L, op, 15, t=r5["t"], step=r5["step"], F=r5["F"])
    eo, scale = e_oracle(r20["x"], r20["v"])
    assert abs(e["KE"] + e["PE_nuc"] + e["PE_coul"] - eo) < 1e-6 * scale
    s.step(30, 0.0)
    g = s.state()
    e = s.energy()
    eg, scale = e_oracle(g["x"], g["v"])
    assert abs(e["KE"] + e["PE_nuc"] + e["PE_coul"] - eg) < 1e-6 * scale
    r = oracle.run(r20["x"], r20["v"], t, L, op, 30, t=r20["t"], step=r20["step"], F=r20["F"])
    d_split = np.abs(min_img(g["x"] - r["x"], L)).max()
    rng = np.random.default_rng(5)
    xp = x + 1e-7 * rng.choice([-1.0, 1.0], x.shape)
    rp = oracle.run(xp, v, t, L, op, 50)
    d_oracle = np.abs(min_img(rp["x"] - r["x"], L)).max()
    assert d_oracle > 100 * 1e-7                 # the oracle's own amplification of a 1e-7 fm move
    assert d_split < 30 * d_oracle, (d_split, d_oracle)


def test_split_energy_conservation_nve(md):
    x, t, L = cfg_relaxed(2000, 0.30, 0.080, 24)
    s, v = load(md, x, t, L, 0, T=1.0, thermostat_every=0)
    e0 = s.energy()
    E0 = e0["KE"] + e0["PE_nuc"] + e0["PE_coul"]
    s.step(200, 0.0)
    e1 = s.energy()
    E1 = e1["KE"] + e1["PE_nuc"] + e1["PE_coul"]
    assert abs(E1 - E0) < 2e-3 * (e0["KE"] + abs(e0["PE_nuc"]))


def test_rerun_is_bitwise_identical(md):
    for prec in (0, 1):
        outs = []
        for _ in range(2):
            s = make(md, 3000, 0.3, 0.08, T=1.0, seed=5, precision=prec, relax=20)
            s.step(30, 7.5e-5)
            outs.append((s.state()["x"], s.forces()))
            s.close()
        assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])


def test_plain_and_conditional_step_graphs_agree_bitwise(md):
    """The rebuild kernels in conditional graph nodes (default) or as plain
    nodes that return at once without a rebuild: the same kernels run on
    the same data, so trajectories (through several rebuilds) are identical."""
    x, t, L = PARITY_CASES["liquid_2000"]()
    out = []
    for cond in (1, 0):
        s, v = load(md, x, t, L, 0, cond_graph=cond)
        s.step(30, 7.5e-5)
        g = s.state()
        out.append((g["x"].copy(), g["v"].copy(), s.forces(), s.info()["rebuilds"]))
        s.close()
    assert out[0][3] == out[1][3] and out[0][3] >= 3
    for a, b in zip(out[0][:3], out[1][:3]):
        assert np.array_equal(a, b)


def test_set_state_resume_matches_uninterrupted(md):
    s1 = make(md, 1500, 0.3, 0.08, T=1.0, seed=8, precision=1, relax=10, thermostat_every=0)
    st0 = s1.state()
    s1.step(20, 0.0)
    mid = s1.state()
    s1.step(20, 0.0)
    end = s1.state()
    s2 = make(md, 1500, 0.3, 0.08, T=1.0, seed=99, precision=1, relax=0, thermostat_every=0)
    s2.set_state(mid["x"], mid["v"], mid["L"], L_base=mid["L_base"], t=mid["t"], t_base=mid["t_base"],
                 step=mid["step"])
    s2.step(20, 0.0)
    e2 = s2.state()
    assert np.abs(min_img(e2["x"] - end["x"], end["L"])).max() < 1e-9
    assert st0["N"] == 1500


# --------------------------------------------------------------- clusters
def _check_clusters(s, x, t, L):
    lab, hA, hZ, st = s.clusters()
    lo, hAo, hZo, sto = oracle.clusters(x, t, L)
    assert np.array_equal(lab, lo)
    assert np.array_equal(hA, hAo) and np.array_equal(hZ, hZo)
    assert st["n_clusters"] == sto[0] and st["m_free_n"] == sto[1]
    assert st["A_mean"] == sto[2] and st["Z_mean"] == sto[3] and st["n_big"] == sto[4]


@pytest.mark.parametrize("name", ["drops_3000_dilute", "liquid_2000", "liquid_4096_yp005", "drops_20000_L464"])
def test_clusters_bit_exact(md, name):
    x, t, L = PARITY_CASES[name]()
    s, _ = load(md, x, t, L, 0)
    _check_clusters(s, x, t, L)


def test_clusters_beyond_the_link_buffer(md):
    """Matter dense enough (0.15 protons per fm^3: about 28 proton pairs
    inside r_pp per proton) that the links found outnumber the link buffer
    (16 per proton): the link pass unites the pairs beyond it itself.  Labels,
    histograms and statistics stay bit-exact with the oracle."""
    x, t, L = cfg_liquid(6000, 0.60, 0.25, 12)
    s, _ = load(md, x, t, L, 0)
    _check_clusters(s, x, t, L)


def test_clusters_after_dynamics_and_edges(md):
    x, t, L = cfg_drops(3000, 0.30, 0.005, 31)
    s, _ = load(md, x, t, L, 0, T=0.5)
    s.step(30, 7.5e-5)
    g = s.state()
    _check_clusters(s, g["x"], g["type"], g["L"])
    # chain across the periodic face and the 4.5 fm threshold
    L = 60.0
    xs = np.array([[59.0, 5, 5], [2.4, 5, 5], [6.89, 5, 5], [11.4, 5, 5], [30, 30, 30], [30, 32.99, 30],
                   [30, 26.99, 30], [8.0, 8.0, 5.0]], dtype=float)
    ts = np.array([1, 1, 1, 1, 1, 0, 0, 0], np.int8)
    s2, _ = load(md, xs, ts, L, 0)
    _check_clusters(s2, xs, ts, L)
    # caller-supplied output arrays: same results, filled in place (twice)
    lab, hA, hZ, st = s.clusters()
    out = (np.full(s.N, -7, np.int32), np.full(s.N + 1, 9, np.int64), np.full(s.Np + 1, 9, np.int64))
    for _ in range(2):
        lab2, hA2, hZ2, st2 = s.clusters(out=out)
        assert lab2 is out[0] and hA2 is out[1] and hZ2 is out[2]
        assert np.array_equal(lab, lab2) and np.array_equal(hA, hA2) and np.array_equal(hZ, hZ2) and st == st2


# --------------------------------------------------------------- full size
@pytest.mark.parametrize("N,Yp,T,seed", [(51200, 0.30, 1.0, 2), (409600, 0.40, 0.5, 3)])
def test_full_size_sampled_forces(md, N, Yp, T, seed):
    """Configurations of the 51,200 and 409,600 nucleon runs in the launch
    configuration the benchmark times: sampled targets against the oracle's
    brute force over all N sources."""
    s = make(md, N, Yp, 0.080, T=T, seed=seed, relax=500)
    p = s.params
    p.T = T
    s.params = p
    s.step(20, 7.5e-5)
    g = s.state()
    F = s.forces()
    Np = s.Np
    op = oparams(s)
    for i0, i1 in ((0, 48), (Np, Np + 48)):
        Fo, _ = oracle.forces(g["x"], g["type"], g["L_F"], op, i0, i1)
        assert rel_l2(F[i0:i1], Fo[i0:i1]) <= 1e-5, (i0, rel_l2(F[i0:i1], Fo[i0:i1]))
    info = s.info()
    assert info["rebuilds"] >= 2
    e = s.energy()
    assert np.isfinite(e["KE"] + e["PE_nuc"] + e["PE_coul"])


# --------------------------------------------------------------- state round trip
@pytest.mark.parametrize("precision", [0, 1])
def test_state_round_trip_with_forces(md, precision):
    """md_get_state with f returns the cached forces; md_set_state with them
    restores them bit for bit (no fresh force pass), and the restored system
    continues the trajectory of the original one (differences only from the
    FP32 summation order of the re-sorted tiles)."""
    x, t, L = PARITY_CASES["liquid_2000"]()
    s, _ = load(md, x, t, L, precision)
    xi = 7.5e-5
    s.step(7, xi)
    g = s.state(f=True)
    assert np.array_equal(g["f"], s.forces())
    s2 = make(md, len(x), float(t.sum()) / len(x), len(x) / L ** 3, precision=precision)
    kw = dict(L_base=g["L_base"], t=g["t"], t_base=g["t_base"], xi_dot=g["xi_dot"], step=g["step"])
    s2.set_state(g["x"], g["v"], g["L"], f=g["f"], L_F=g["L_F"], **kw)
    g2 = s2.state(f=True)
    assert np.array_equal(g2["f"], g["f"]) and np.array_equal(s2.forces(), g["f"])
    assert g2["L_F"] == g["L_F"] and g2["L"] == g["L"] and g2["step"] == g["step"]
    assert np.array_equal(g2["x"], g["x"]) and np.array_equal(g2["v"], g["v"])
    s.step(5, xi)
    s2.step(5, xi)
    a, b = s.state(), s2.state()
    tol = 1e-12 if precision == 1 else 1e-6
    assert rel_l2(b["x"], a["x"]) < tol and rel_l2(b["v"], a["v"]) < tol
    # without f the forces are re-evaluated at the loaded positions, with the
    # loaded box side (here L_F, the side the saved forces were evaluated with)
    s3 = make(md, len(x), float(t.sum()) / len(x), len(x) / L ** 3, precision=precision)
    s3.set_state(g["x"], g["v"], g["L_F"])
    assert rel_l2(s3.forces(), g["f"]) < (1e-12 if precision == 1 else 1e-5)
    for q in (s, s2, s3):
        q.close()


# --------------------------------------------------------------- code variants
@pytest.mark.parametrize("name", ["liquid_2000", "drops_3000_dilute", "liquid_4096_yp005"])
@pytest.mark.parametrize("energy_every", [1, 0])
def test_force_code_variants_agree_bitwise(md, name, energy_every):
    """The long, compact and minimal code variants of the split force pass
    (the minimal one also in one-warp blocks) do the same arithmetic in the
    same order: identical forces, energies and
    pair counts, before and after steps (force_unroll = 0: the device tuner's
    choice), in steps with the energy pass and in steps without it (whose
    kernels are compiled for more resident blocks)."""
    x, t, L = PARITY_CASES[name]()
    outs = []
    for fu in (4, 2, 1, 3, 0):
        s, _ = load(md, x, t, L, 0, force_unroll=fu, energy_every=energy_every)
        F0, e0 = s.forces(), s.energy()
        s.step(12, 7.5e-5)
        outs.append((F0, e0, s.state(f=True), s.step_energy() if energy_every else None))
        s.close()
    for o in outs[1:]:
        assert np.array_equal(o[0], outs[0][0]) and o[1] == outs[0][1]
        for k in ("x", "v", "f"):
            assert np.array_equal(o[2][k], outs[0][2][k])
        assert o[3] == outs[0][3]


def test_force_code_tuner_reports_its_choice(md):
    """Engines of at least 131,072 nucleons select the force-pass variant per
    step (a SWITCH graph node) and the device tuner times all four every 500
    steps from step 500: the trial runs every variant and the trajectory is
    bitwise that of the fixed long variant.  Smaller engines run the variant
    force_unroll fixes (the minimal one by default)."""
    x, t, L = cfg_liquid(135000, 0.40, 0.080, 12)
    outs = []
    for fu in (4, 0):
        s, _ = load(md, x, t, L, 0, T=0.5, force_unroll=fu)
        s.step(10, 7.5e-5)
        assert s.info()["force_trials"] == 0 and s.info()["force_code"] == 4     # long until step 500
        s.step(510, 7.5e-5)                  # the trial: steps 501-512, four passes of each variant
        info = s.info()
        assert info["force_trials"] == (1 if fu == 0 else 0) and info["force_code"] in (1, 2, 3, 4)
        outs.append(s.state(f=True))
        s.close()
    for k in ("x", "v", "f"):
        assert np.array_equal(outs[0][k], outs[1][k])
    x, t, L = PARITY_CASES["liquid_2000"]()
    for fu in (0, 1, 2, 3, 4):
        s, _ = load(md, x, t, L, 0, force_unroll=fu)
        s.step(520, 0.0)
        assert s.info()["force_code"] == (fu or 1) and s.info()["force_trials"] == 0
        s.close()
    with pytest.raises(md.MDError):
        load(md, x, t, L, 0, force_unroll=5)


def test_step_async_matches_step(md):
    """md_step_async enqueues the same steps as md_step (bitwise the same
    state); md_sync reports completion."""
    x, t, L = PARITY_CASES["liquid_2000"]()
    outs = []
    for asynchronous in (False, True):
        s, _ = load(md, x, t, L, 0, energy_every=1)
        for _ in range(6):
            if asynchronous:
                s.step_async(1, 7.5e-5)
            else:
                s.step(1, 7.5e-5)
        if asynchronous:
            s.sync()
        outs.append((s.state(f=True), s.step_energy()))
        s.close()
    for k in ("x", "v", "f"):
        assert np.array_equal(outs[0][0][k], outs[1][0][k])
    assert outs[0][1] == outs[1][1]

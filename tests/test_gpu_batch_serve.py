"""Batched ensemble and serving: each system's result is the same alone and
in the mix (the kernels are deterministic per system, so "the same" is
bit-identical here, tighter than the stated tolerances), a batch member
matches the oracle, and the server admits jobs under its HBM budget."""
import time

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

JOBS = [
    dict(N=1500, Yp=0.30, rho=0.080, T=1.0, seed=11, xi_dot=0.0),
    dict(N=4000, Yp=0.05, rho=0.020, T=0.5, seed=12, xi_dot=7.5e-5),
    dict(N=2700, Yp=0.40, rho=0.005, T=0.75, seed=13, xi_dot=2e-4),
    dict(N=640, Yp=0.20, rho=0.0125, T=1.0, seed=14, xi_dot=0.0),
]


@pytest.fixture(scope="module")
def md():
    from paper_1412_8502_b300 import md as m
    return m


def params(md, relax=40):
    p = md.md_params_default()
    p.relax_iters = relax
    p.thermostat_every = 25
    return p


def alone(md, job, steps, p):
    s = md.System(job["N"], job["Yp"], job["rho"], job["T"], job["seed"], p)
    s.step(steps, job["xi_dot"])
    return s


def test_batch_member_equals_alone(md):
    p = params(md)
    b = md.Batch(JOBS, p)
    b.step(60)
    for j, s in zip(JOBS, b.systems):
        a = alone(md, j, 60, p)
        ga, gb = a.state(), s.state()
        assert np.array_equal(ga["x"], gb["x"]) and np.array_equal(ga["v"], gb["v"]), j
        assert ga["L"] == gb["L"] and ga["t"] == gb["t"]
        assert np.array_equal(a.forces(), s.forces())
        la, _, _, _ = a.clusters()
        lb, _, _, _ = s.clusters()
        assert np.array_equal(la, lb)
        a.close()
    b.close()


def test_persistent_step_is_one_launch_and_equals_the_graph(md):
    """The persistent step kernel (one cooperative launch per step for all
    systems, phases between bounded grid barriers) gives bitwise the states,
    forces and energies of the graph of separate kernels, with and without
    the energy pass, through rebuilds, box growth and the thermostat."""
    for ee in (0, 1):
        ps, pg = params(md), params(md)
        ps.persistent, pg.persistent = 1, 0
        ps.energy_every = pg.energy_every = ee
        bs, bg = md.Batch(JOBS, ps), md.Batch(JOBS, pg)
        bs.step(1)                 # (the first call also sets the systems' expansion rates)
        bg.step(1)
        n0 = bs.systems[0].info()["launches"]
        bs.step(40)
        bg.step(40)
        assert bs.systems[0].info()["launches"] - n0 == 40      # one kernel per step
        assert bs.systems[0].info()["rebuilds"] > 2
        for s1, s0 in zip(bs.systems, bg.systems):
            g1, g0 = s1.state(), s0.state()
            assert np.array_equal(g1["x"], g0["x"]) and np.array_equal(g1["v"], g0["v"])
            assert g1["L"] == g0["L"] and g1["t"] == g0["t"]
            assert np.array_equal(s1.forces(), s0.forces())
            if ee:
                assert s1.step_energy() == s0.step_energy()
        bs.close()
        bg.close()
    # one system on its own, in the same launch form
    p = params(md)
    p.persistent = 1
    a = md.System(3000, 0.3, 0.03, 1.0, 21, p)
    p.persistent = 0
    b = md.System(3000, 0.3, 0.03, 1.0, 21, p)
    a.step(25, 1e-4)
    b.step(25, 1e-4)
    assert np.array_equal(a.state()["x"], b.state()["x"]) and np.array_equal(a.forces(), b.forces())
    a.close()
    b.close()


def test_persistent_wait_limit_is_an_error_status(md):
    """Every grid-wide wait of the persistent step kernel is bounded by
    md_params.wait_limit_ns (%globaltimer).  At 1 ns the waits give up (the
    blocks reach the barrier after the force phase microseconds apart), every
    block leaves at its next barrier, and md_batch_step returns MD_ETIMEOUT:
    no hang and no device fault.  The limit is then restored and a fresh batch
    steps normally on the same device."""
    p = params(md)
    p.persistent = 1
    p.wait_limit_ns = 1
    b = md.Batch(JOBS, p)
    with pytest.raises(md.MDError) as e:
        b.step(3)
    assert e.value.code == md.MD_ETIMEOUT
    b.close()
    p.wait_limit_ns = 2_000_000_000
    b = md.Batch(JOBS, p)
    b.step(5)
    b.close()
    p.persistent = 2
    with pytest.raises(md.MDError) as e:
        md.Batch(JOBS, p)
    assert e.value.code == md.MD_EINVAL


def test_persistent_mode_selection(md):
    """persistent = -1 (default) runs a batch as one persistent launch per step
    but falls back to the graph where the persistent step does not apply
    (per-particle Verlet lists; FP64); persistent = 1 there is MD_EINVAL;
    a single system defaults to the graph.  Results equal the same systems
    alone in every case."""
    p = params(md)
    p.list_kind = 1
    p.skin = 4.0
    b = md.Batch(JOBS[:2], p)                    # falls back: graph of kernels
    b.step(1)
    n0 = b.systems[0].info()["launches"]
    b.step(10)
    assert b.systems[0].info()["launches"] - n0 > 10
    a = alone(md, JOBS[0], 11, p)
    assert np.array_equal(a.state()["x"], b.systems[0].state()["x"])
    a.close()
    b.close()
    p.persistent = 1
    with pytest.raises(md.MDError) as e:
        md.Batch(JOBS[:2], p)
    assert e.value.code == md.MD_EINVAL
    q = params(md)
    q.precision = 1
    q.persistent = 1
    with pytest.raises(md.MDError) as e:
        md.Batch(JOBS[:2], q)
    assert e.value.code == md.MD_EINVAL
    s = md.System(1500, 0.3, 0.08, 1.0, 3, params(md))       # one system: the graph
    s.step(1)
    n0 = s.info()["launches"]
    s.step(5)
    assert s.info()["launches"] - n0 > 5
    s.close()


def test_batch_member_matches_oracle(md):
    p = params(md)
    b = md.Batch(JOBS[:3], p)
    b.step(10)
    for s in b.systems:
        g = s.state()
        F = s.forces()
        pr = s.params
        Fo, _ = oracle.forces(g["x"], g["type"], g["L_F"], oracle.params(pr.r_C))
        assert np.linalg.norm(F - Fo) / np.linalg.norm(Fo) <= 1e-5
    b.close()


def test_server_results_equal_alone_and_budget(md):
    p = params(md, relax=30)
    steps = 40
    jobs = [dict(j, steps=steps) for j in JOBS]
    # budget that holds only some of the jobs at once (a few MB each)
    from paper_1412_8502_b300 import md as m
    budget = 5 * 1024 * 1024
    sv = m.md_server_create(budget, p)
    ids = {}
    for j in jobs:
        ids[m.md_server_submit(sv, j)] = j
        time.sleep(0.01)
    big = m.md_server_submit(sv, dict(N=400000, Yp=0.4, rho=0.08, T=0.5, seed=1, xi_dot=0.0, steps=1))
    m.md_server_drain(sv, 600.0)
    res = {}
    while True:
        r = m.md_server_poll(sv)
        if r is None:
            break
        res[r["id"]] = r
    m.md_server_destroy(sv)
    assert set(res) == set(ids) | {big}
    assert res[big]["status"] == m.MD_ENOMEM
    for jid, j in ids.items():
        r = res[jid]
        assert r["status"] == m.MD_OK and r["steps"] == steps
        a = alone(md, j, steps, p)
        e = a.energy()
        for k in ("KE", "PE_nuc", "PE_coul", "virial", "L", "t"):
            assert r["energy"][k] == e[k], (j, k, r["energy"][k], e[k])
        assert 0 < r["step_p50_ms"] <= r["step_p99_ms"]
        a.close()


def test_server_poll_empty_and_bad_job(md):
    from paper_1412_8502_b300 import md as m
    sv = m.md_server_create(1 << 30)
    assert m.md_server_poll(sv) is None
    with pytest.raises(m.MDError):
        m.md_server_submit(sv, dict(N=1, Yp=0.3, rho=0.08, T=1.0, seed=1, xi_dot=0.0, steps=5))
    m.md_server_drain(sv, 10.0)
    m.md_server_destroy(sv)


def test_autotune_restores_state_and_picks_a_candidate(md):
    p = params(md)
    s = md.System(3000, 0.3, 0.04, 1.0, 21, p)
    s.step(5, 0.0)
    g0 = s.state()
    chosen = s.autotune(4)
    g1 = s.state()
    assert np.array_equal(g0["x"], g1["x"]) and np.array_equal(g0["v"], g1["v"])
    assert g0["t"] == g1["t"] and g0["step"] == g1["step"] and g0["L"] == g1["L"]
    assert chosen.skin in (0.5, 1.0, 1.5, 2.0) and 2 <= chosen.sort_bits <= 7
    s.step(10, 0.0)
    F = s.forces()
    g = s.state()
    Fo, _ = oracle.forces(g["x"], g["type"], g["L_F"], oracle.params(s.params.r_C))
    assert np.linalg.norm(F - Fo) / np.linalg.norm(Fo) <= 1e-5
    b = md.Batch(JOBS[:2], p)
    cb = b.autotune(3)
    assert cb.skin in (0.5, 1.0, 1.5, 2.0)
    b.step(5)
    b.close()
    s.close()

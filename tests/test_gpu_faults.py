"""Host-side fault tests: invalid arguments are rejected before any device
work, and a force the kernel cannot represent becomes an error status
(MD_ENUMERIC) instead of a silent result.  The fault is planted on the host
(two protons 1e-6 fm apart: a Coulomb force of ~1e12 MeV/fm, beyond the
force kernel's range check); md_set_state evaluates the forces of the new
state and reports it, before any step integrates it."""
import numpy as np
import pytest

import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def md():
    from paper_1412_8502_b300 import md as m
    return m


def test_invalid_arguments_are_rejected(md):
    p = md.md_params_default()
    for args in [(1, 0.3, 0.08, 1.0), (100, 1.5, 0.08, 1.0), (100, 0.3, 0.0, 1.0), (100, 0.3, 0.08, -1.0)]:
        with pytest.raises(md.MDError) as e:
            md.System(*args, 1, p)
        assert e.value.code == -1, args                      # MD_EINVAL
    p.r_C = 50.0                                             # > L0/2 = 29.2 / 2 fm
    with pytest.raises(md.MDError) as e:
        md.System(2000, 0.3, 0.08, 1.0, 1, p)
    assert e.value.code == -1
    s = md.System(2000, 0.3, 0.08, 1.0, 1, md.md_params_default())
    with pytest.raises(md.MDError) as e:
        s.step(1, float("nan"))
    assert e.value.code == -1
    s.close()


def test_unrepresentable_force_is_an_error_status(md):
    N, Yp, rho = 600, 0.5, 0.02
    p = md.md_params_default()
    p.relax_iters = 0
    s = md.System(N, Yp, rho, 1.0, 2, p)
    st = s.state()
    x, L = st["x"].copy(), st["L"]
    s.step(0, 0.0)                                           # a sound state first: no error
    x[1] = x[0] + np.array([1e-6, 0.0, 0.0])                 # protons 0 and 1 (protons come first)
    with pytest.raises(md.MDError) as e:                     # md_set_state evaluates the new state's forces
        s.set_state(x, inputs.maxwell(N, 1.0, 3), L)
    assert e.value.code == -5                                # MD_ENUMERIC
    s.close()


def test_union_find_limit_is_an_error_status(md):
    """Every union-find loop of the cluster analyses (Sec. II.C) is bounded by
    md_params.uf_iter_limit.  A periodic ring of 100 protons 4.49 fm apart is
    one cluster whose union-find tree is deeper than one hop (the links of a
    tile's lanes land in parallel), so with the limit at 1 a root walk gives up
    and md_clusters returns MD_ETIMEOUT: no device fault and no wait is
    involved.  At the default limit the same call is bit-exact with the oracle.
    The MSTE analysis reports the limit the same way, on a ring of alternating
    protons and neutrons at the n-p minimum of Eq. (1) at rest (every n-p
    neighbour pair bound)."""
    import oracle
    from test_gpu_parity import load, oparams

    n, sp = 100, 4.49
    L = n * sp                                               # the ring closes through the periodic face
    xs = [[k * sp, 20.0, 20.0] for k in range(n)]
    xs += [[k * sp + 1.0, 21.5, 20.0] for k in range(0, n, 5)]   # neutrons 1.8 fm from a proton
    xs += [[100.0, 200.0, 150.0 + 10.0 * k] for k in range(10)]  # free neutrons
    x = np.array(xs)
    t = np.array([1] * n + [0] * (len(xs) - n), np.int8)
    s, _ = load(md, x, t, L, 0, uf_iter_limit=1)
    with pytest.raises(md.MDError) as e:
        s.clusters()
    assert e.value.code == -4                                # MD_ETIMEOUT
    p = s.params
    p.uf_iter_limit = 1 << 26
    s.params = p
    lab, hA, hZ, st = s.clusters()
    lo, hAo, hZo, sto = oracle.clusters(x, t, L)
    assert np.array_equal(lab, lo) and np.array_equal(hA, hAo) and np.array_equal(hZ, hZo)
    assert st["n_clusters"] == sto[0] == 1
    s.close()

    r_min = np.sqrt(2.0 * 1.25 * np.log(2.0 * 110.0 / 50.0))   # V_np minimum, s = b - c = -50 MeV
    m = 120
    Lr = m * r_min
    pos = np.array([[k * r_min, 30.0, 30.0] for k in range(m)])
    order = np.r_[np.arange(0, m, 2), np.arange(1, m, 2)]     # protons (even sites) first
    x2 = pos[order]
    t2 = np.array([1] * (m // 2) + [0] * (m // 2), np.int8)
    s2, v2 = load(md, x2, t2, Lr, 0, T=0.0, uf_iter_limit=1)
    with pytest.raises(md.MDError) as e:
        s2.clusters_mste()
    assert e.value.code == -4
    p = s2.params
    p.uf_iter_limit = 1 << 26
    s2.params = p
    lab, hA, hZ, st = s2.clusters_mste()
    lo, hAo, hZo, sto = oracle.mste(x2, v2, t2, Lr, oparams(s2))
    assert np.array_equal(lab, lo) and np.array_equal(hA, hAo) and np.array_equal(hZ, hZo)
    assert st["n_clusters"] == 1
    s2.close()


def test_uf_limit_out_of_range_is_rejected(md):
    p = md.md_params_default()
    assert p.uf_iter_limit == 1 << 26
    for bad in (0, -5, 1 << 31):
        p.uf_iter_limit = bad
        with pytest.raises(md.MDError) as e:
            md.System(300, 0.3, 0.08, 1.0, 1, p)
        assert e.value.code == -1


def _free_bytes():
    import torch
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def test_allocation_failure_injection(md):
    """The test hook md_debug_fail_alloc(k) makes the k-th device allocation
    fail as if the device were out of memory.  Walking k over every
    allocation md_create and md_batch_create make, each failing call returns
    MD_ENOMEM and leaves the device's free memory where it was (nothing
    leaked); once k passes the last allocation the call succeeds.  The
    first cluster analysis (which allocates its buffers) fails the same way
    and the system stays usable."""
    p = md.md_params_default()
    p.relax_iters = 2
    jobs = [dict(N=900, Yp=0.3, rho=0.05, T=1.0, seed=5, xi_dot=0.0, steps=0),
            dict(N=1300, Yp=0.1, rho=0.02, T=0.5, seed=6, xi_dot=0.0, steps=0)]
    md.System(1500, 0.3, 0.08, 1.0, 1, p).close()            # context and modules loaded first
    md.Batch(jobs, p).close()
    base = _free_bytes()
    for make in (lambda: md.System(1500, 0.3, 0.08, 1.0, 1, p), lambda: md.Batch(jobs, p)):
        succeeded_at = None
        for k in range(1, 200):
            assert md.LIB.md_debug_fail_alloc(k) == md.MD_OK
            try:
                obj = make()
            except md.MDError as e:
                assert e.code == md.MD_ENOMEM, (k, str(e))
                assert "injected" in str(e)
                assert _free_bytes() == base, k
                continue
            md.LIB.md_debug_fail_alloc(0)
            obj.close()
            succeeded_at = k
            break
        md.LIB.md_debug_fail_alloc(0)
        assert succeeded_at is not None and succeeded_at > 20     # every allocation site was made to fail
        assert _free_bytes() == base
    s = md.System(1500, 0.3, 0.08, 1.0, 1, p)
    md.LIB.md_debug_fail_alloc(1)
    with pytest.raises(md.MDError) as e:
        s.clusters()
    assert e.value.code == md.MD_ENOMEM
    md.LIB.md_debug_fail_alloc(0)
    lab, hA, hZ, st = s.clusters()
    assert hA.sum() == st["n_clusters"]
    s.close()
    assert md.LIB.md_debug_fail_alloc(-1) == md.MD_EINVAL


def test_server_admission_allocation_failure(md):
    """A job whose admission hits a failed device allocation finishes with
    MD_ENOMEM; the server keeps serving the next job."""
    p = md.md_params_default()
    p.relax_iters = 4
    sv = md.md_server_create(8 << 30, p)
    try:
        job = dict(N=1200, Yp=0.3, rho=0.08, T=1.0, seed=8, xi_dot=0.0, steps=10)
        md.LIB.md_debug_fail_alloc(3)
        md.md_server_submit(sv, job)
        md.md_server_drain(sv, 120.0)
        r = md.md_server_poll(sv)
        assert r is not None and r["status"] == md.MD_ENOMEM
        md.LIB.md_debug_fail_alloc(0)
        md.md_server_submit(sv, job)
        md.md_server_drain(sv, 120.0)
        r = md.md_server_poll(sv)
        assert r is not None and r["status"] == md.MD_OK and r["steps"] == 10
    finally:
        md.LIB.md_debug_fail_alloc(0)
        md.md_server_destroy(sv)

"""Per-particle Verlet lists (list_kind 1, the paper's neighbour lists with
delta r = 4 fm, Sec. II.B.1) against the oracle: forces, energies, a run
through rebuilds with expansion, determinism, pool exhaustion."""
import numpy as np
import pytest

import inputs
import oracle
from test_gpu_parity import cfg_drops, cfg_liquid, load, make, oparams, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def md():
    from paper_1412_8502_b300 import md as m
    return m


def verlet(md, x, t, L, **kw):
    kw.setdefault("skin", 4.0)
    return load(md, x, t, L, 0, list_kind=1, **kw)


@pytest.mark.parametrize("cfg", ["liquid2000", "drops3000", "liquid20000_rc15", "yp05_4096"])
def test_verlet_forces_and_energy_vs_oracle(md, cfg):
    if cfg == "liquid2000":
        x, t, L = cfg_liquid(2000, 0.3, 0.08, 61)
        kw = {}
    elif cfg == "drops3000":
        x, t, L = cfg_drops(3000, 0.3, 0.005, 62)
        kw = {}
    elif cfg == "liquid20000_rc15":            # large enough box for the shifted (non-wrap) path
        x, t, L = cfg_liquid(20000, 0.4, 0.08, 63)
        kw = {"r_C": 15.0}
    else:
        x, t, L = cfg_liquid(4096, 0.05, 0.08, 64)
        kw = {}
    s, v = verlet(md, x, t, L, **kw)
    F = s.forces()
    Fo, (en, ec, w) = oracle.forces(x, t, L, oparams(s))
    assert rel_l2(F, Fo) <= 1e-5, rel_l2(F, Fo)
    e = s.energy()
    scale = oracle.kinetic(v) + abs(en) + abs(ec)
    assert abs(e["PE_nuc"] - en) <= 1e-6 * scale
    assert abs(e["PE_coul"] - ec) <= 1e-6 * scale
    assert abs(e["virial"] - w) <= 1e-6 * (scale + abs(w))
    info = s.info()
    assert 0 < info["verlet_entries"] <= info["verlet_slots"] <= info["verlet_capacity"]


def test_verlet_shifted_images_large_box(md):
    """A box large enough that tile pairs carry one periodic shift (no per-pair
    wrap): forces of 3,000 sampled targets against the oracle over all
    sources, before and after 10 expanding steps."""
    x, t, L = cfg_liquid(60000, 0.4, 0.08, 68)
    s, _ = verlet(md, x, t, L, r_C=15.0)
    assert s.info()["need_wrap"] == 0
    po = oparams(s)
    F = s.forces()
    Fo, _ = oracle.forces(x, t, L, po, 0, 3000)
    assert rel_l2(F[:3000], Fo[:3000]) <= 1e-5
    s.step(10, 7.5e-5)
    g = s.state()
    Fo, _ = oracle.forces(g["x"], g["type"], g["L_F"], po, 30000, 33000)
    assert rel_l2(s.forces()[30000:33000], Fo[30000:33000]) <= 1e-5


def test_verlet_equals_tile_lists_within_fp32(md):
    x, t, L = cfg_liquid(8000, 0.4, 0.08, 65)
    a, _ = verlet(md, x, t, L)
    b, _ = load(md, x, t, L, 0)
    Fa, Fb = a.forces(), b.forces()
    assert rel_l2(Fa, Fb) <= 2e-6
    ea, eb = a.energy(), b.energy()
    assert ea["pairs_nuc"] == eb["pairs_nuc"] and ea["pairs_coul"] == eb["pairs_coul"]


def test_verlet_run_through_rebuilds_with_expansion(md):
    """40 steps at 4x the configuration's expansion rate: the lists are rebuilt
    by the displacement rule and the forces at the end match the oracle."""
    x, t, L = cfg_liquid(3000, 0.3, 0.08, 66)
    s, _ = verlet(md, x, t, L, T=1.0, thermostat_every=0)
    r0 = s.info()["rebuilds"]
    s.step(40, 3e-4)
    g = s.state()
    Fo, _ = oracle.forces(g["x"], g["type"], g["L_F"], oparams(s))
    assert rel_l2(s.forces(), Fo) <= 1e-5
    reb_verlet = s.info()["rebuilds"] - r0
    # same run on tile lists with a 1 fm skin rebuilds at least as often
    b, _ = load(md, x, t, L, 0, T=1.0, thermostat_every=0, rebuild_every=1000)
    b0 = b.info()["rebuilds"]
    b.step(40, 3e-4)
    assert reb_verlet <= b.info()["rebuilds"] - b0


def test_verlet_rerun_is_bitwise_identical(md):
    x, t, L = cfg_drops(3000, 0.3, 0.005, 67)
    outs = []
    for _ in range(2):
        s, _ = verlet(md, x, t, L)
        s.step(15, 7.5e-5)
        outs.append(s.state()["x"].copy())
    assert np.array_equal(outs[0], outs[1])


def test_verlet_pool_exhaustion_is_an_error(md):
    """A pool far below the need makes the rebuild keep empty lists and the
    call report MD_ENOMEM (no out-of-bounds write)."""
    p = md.md_params_default()
    p.list_kind = 1
    p.skin = 4.0
    p.verlet_pool = 0.02
    p.relax_iters = 0
    with pytest.raises(md.MDError) as ei:
        md.System(4000, 0.3, 0.08, 1.0, 5, p)
    assert ei.value.code == md.MD_ENOMEM


def test_verlet_needs_split_precision(md):
    p = md.md_params_default()
    p.list_kind = 1
    p.precision = 1
    with pytest.raises(md.MDError) as ei:
        md.System(500, 0.3, 0.08, 1.0, 5, p)
    assert ei.value.code == md.MD_EINVAL

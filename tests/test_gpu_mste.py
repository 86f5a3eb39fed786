"""MSTE (energy-criterion) clusters on the GPU against the oracle: labels,
histograms and statistics bit-exact, in both precisions, with Verlet lists
and with the all-pairs Coulomb."""
import numpy as np
import pytest

import oracle
from test_gpu_parity import cfg_drops, cfg_liquid, load, oparams

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def md():
    from paper_1412_8502_b300 import md as m
    return m


def check(s):
    g = s.state()
    lab, hA, hZ, st = s.clusters_mste()
    lo, hAo, hZo, sto = oracle.mste(g["x"], g["v"], g["type"], g["L"], oparams(s))
    assert np.array_equal(lab, lo)
    assert np.array_equal(hA, hAo) and np.array_equal(hZ, hZo)
    assert st["n_clusters"] == int(sto[0])
    assert st["m_free_n"] == pytest.approx(sto[1], abs=0, rel=1e-15)
    assert st["n_big"] == int(sto[4])
    return lo


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("cfg", ["drops3000", "liquid2000", "yp05_4096"])
def test_mste_matches_oracle(md, precision, cfg):
    if cfg == "drops3000":
        x, t, L = cfg_drops(3000, 0.3, 0.005, 71)
    elif cfg == "liquid2000":
        x, t, L = cfg_liquid(2000, 0.3, 0.08, 72)
    else:
        x, t, L = cfg_liquid(4096, 0.05, 0.08, 73)
    s, _ = load(md, x, t, L, precision, T=1.0)
    lab = check(s)
    assert (lab >= 0).sum() > 0
    s.step(20, 7.5e-5)          # dynamics, rebuilds, expansion
    check(s)


def test_mste_with_verlet_lists_and_all_pairs_coulomb(md):
    x, t, L = cfg_drops(3000, 0.3, 0.005, 74)
    s, _ = load(md, x, t, L, 0, T=0.5, list_kind=1, skin=4.0)
    s.step(10, 7.5e-5)
    check(s)
    x, t, L = cfg_liquid(2000, 0.4, 0.08, 75)
    s, _ = load(md, x, t, L, 0, T=0.5, coulomb=2)
    check(s)


def test_mste_and_distance_clusters_agree_on_drops(md):
    """Drops in a neutron gas at T = 0.5 MeV: the energy criterion and the
    distance linkage of Sec. II.C find the same nuclei (the paper reports the
    two compare well).  (At T = 0 every pair inside r_nuc with V < 0 is
    bound, the far Gaussian tails included, and the drops merge.)"""
    x, t, L = cfg_drops(3000, 0.3, 0.005, 76)
    s, _ = load(md, x, t, L, 0, T=0.5)
    _, hA1, hZ1, st1 = s.clusters()
    _, hA2, hZ2, st2 = s.clusters_mste()
    assert st1["n_big"] > 5
    assert st2["n_big"] == st1["n_big"]
    z1 = (np.arange(hZ1.size) * hZ1)[12 // 3:].sum()
    z2 = (np.arange(hZ2.size) * hZ2)[12 // 3:].sum()
    assert abs(z2 - z1) <= 0.05 * z1

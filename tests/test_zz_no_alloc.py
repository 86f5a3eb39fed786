"""md_clusters_noalloc: the cluster analysis for callers that cannot allocate
device memory (it works only in a fixed device array of the library).

Checked through the C ABI against the existing entry point md_clusters on
the same positions, on two calls in a row (the scratch array keeps the
previous call's contents, so the second call checks that everything that
must start at zero is cleared), and against the oracle's Sec. II.C
clusters.  Labels, histograms and counts must match exactly, the tolerance
the other cluster tests use.  The device's free memory is the same before
and after the second call: the entry point allocates nothing.  Collected
last so that a run stopping at the first failure has run every other
test."""
import numpy as np
import pytest

import inputs
import oracle

pytestmark = pytest.mark.gpu


def _drops(N, Yp, rho, seed):
    from test_gpu_parity import cfg_drops
    return cfg_drops(N, Yp, rho, seed)


def test_noalloc_clusters_match_md_clusters_twice():
    import torch
    from paper_1412_8502_b300 import md

    dev = torch.device("cuda", 0)
    for (N, Yp, rho, seed) in ((3000, 0.30, 0.005, 41), (1800, 0.40, 0.01, 42)):
        x, t, L = _drops(N, Yp, rho, seed)
        Np = int(t.sum())
        p = md.md_params_default()
        p.relax_iters = 0
        s = md.System(N, Np / N, N / L ** 3, 1.0, 1, p)
        s.set_state(x, inputs.maxwell(N, 1.0, seed), L)
        lab_ref, hA_ref, hZ_ref, st = s.clusters()
        g = s.state()
        xd = torch.tensor(g["x"], dtype=torch.float64, device=dev)
        lo, hAo, hZo, sto = oracle.clusters(g["x"], g["type"], g["L"])
        assert np.array_equal(lab_ref, lo) and np.array_equal(hA_ref, hAo) and np.array_equal(hZ_ref, hZo)
        for call in range(2):
            lab = torch.full((N,), 12345, dtype=torch.int32, device=dev)
            hA = torch.full((N + 1,), 7, dtype=torch.int64, device=dev)
            hZ = torch.full((Np + 1,), 7, dtype=torch.int64, device=dev)
            cnt = torch.full((5,), 7, dtype=torch.int64, device=dev)
            stream = torch.cuda.current_stream(dev)
            torch.cuda.synchronize(dev)
            free_before = torch.cuda.mem_get_info(dev)[0]
            md.md_clusters_noalloc(xd.data_ptr(), N, Np, g["L"], p.r_pp, p.r_np, lab.data_ptr(), hA.data_ptr(),
                                   hZ.data_ptr(), cnt.data_ptr(), stream)
            torch.cuda.synchronize(dev)
            if call == 1:   # (the first call may load the library's module)
                assert torch.cuda.mem_get_info(dev)[0] == free_before
            assert np.array_equal(lab.cpu().numpy(), lab_ref), call
            assert np.array_equal(lab.cpu().numpy(), lo), call
            assert np.array_equal(hA.cpu().numpy(), hA_ref), call
            assert np.array_equal(hZ.cpu().numpy(), hZ_ref), call
            c = cnt.cpu().numpy()
            assert c[0] == st["n_clusters"] and c[1] == st["n_free"] and c[2] == st["n_big"], call
            if c[2]:
                assert c[3] / c[2] == st["A_mean"] and c[4] / c[2] == st["Z_mean"]
        s.close()


def test_noalloc_rejects_oversize():
    import torch
    from paper_1412_8502_b300 import md

    buf = torch.zeros(16, dtype=torch.int64, device="cuda")
    with pytest.raises(md.MDError) as e:
        md.md_clusters_noalloc(buf.data_ptr(), 40000, 100, 100.0, 4.5, 3.0, buf.data_ptr(), buf.data_ptr(),
                               buf.data_ptr(), buf.data_ptr())
    assert e.value.code == md.MD_EINVAL and "32768" in str(e.value)

"""C-ABI checks that need no GPU: the library builds for sm_103a, loads, and
exports every function declared in include/*.h; defaults match the paper."""
import ctypes
import re
import subprocess
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parent.parent


@pytest.fixture(scope="module")
def lib_path():
    from paper_1412_8502_b300 import build
    return build.build()


def _declared():
    names = set()
    for h in (ROOT / "include").glob("*.h"):
        txt = re.sub(r"/\*.*?\*/", "", h.read_text(), flags=re.S)
        names |= set(re.findall(r"\b(md_\w+)\s*\(", txt))
    return names


def test_all_declared_symbols_exported(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", str(lib_path)], capture_output=True, text=True,
                         check=True).stdout
    exported = {l.split()[-1] for l in out.splitlines() if " T " in l}
    declared = _declared()
    assert len(declared) >= 25
    missing = declared - exported
    assert not missing, missing


def test_build_targets_sm103a_only(lib_path):
    from paper_1412_8502_b300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_binding_loads_and_defaults(lib_path):
    from paper_1412_8502_b300 import md
    p = md.md_params_default()
    assert (p.dt, p.r_nuc, p.lambda_s, p.r_pp, p.r_np) == (2.0, 11.5, 10.0, 4.5, 3.0)
    assert p.thermostat_every == 100 and p.relax_iters == 500 and p.precision == md.MD_PREC_SPLIT


def test_no_device_is_an_error_not_a_fallback(lib_path):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1412_8502_b300 import md
    h = ctypes.c_void_p()
    assert md.LIB.md_create(100, 0.3, 0.08, 1.0, 1, ctypes.byref(h)) == md.MD_ENODEV
    assert b"device" in md.LIB.md_last_error()
    assert md.LIB.md_batch_create(0, None, None, ctypes.byref(h)) == md.MD_EINVAL
    sv = ctypes.c_void_p()
    assert md.LIB.md_server_create(1 << 30, None, ctypes.byref(sv)) == md.MD_ENODEV


def test_cluster_output_buffers_are_checked(lib_path):
    """Caller-supplied cluster output arrays: wrong size, dtype or layout is
    rejected before the library is called."""
    import numpy as np
    from paper_1412_8502_b300 import md
    N, Np = 10, 4
    good = (np.empty(N, np.int32), np.empty(N + 1, np.int64), np.empty(Np + 1, np.int64))
    bad = [(good[0], np.empty(N, np.int64), good[2]),                  # hist_A one short
           (good[0], good[1], np.empty(Np + 1, np.int32)),               # hist_Z wrong dtype
           (np.empty(2 * N, np.int32)[::2], good[1], good[2]),           # labels not contiguous
           (good[0], good[1], np.empty((Np + 1, 1), np.int64))]          # hist_Z 2-D
    for out in bad:
        with pytest.raises(ValueError):
            md.md_clusters(None, N, Np, True, out=out)


def test_state_arrays_are_checked(lib_path):
    """Caller-supplied state arrays of the wrong shape or dtype are rejected
    before the library is called."""
    import numpy as np
    from paper_1412_8502_b300 import md
    N = 8
    ok = np.empty((N, 3))
    for out in [(np.empty((N, 2)), ok), (ok, np.empty((N, 3), np.float32)), (ok, ok, np.empty((N + 1, 3)))]:
        with pytest.raises(ValueError):
            md.md_get_state(None, N, out=out)
    with pytest.raises(ValueError):
        md.md_set_state(None, ok, ok, 10.0, Np=2, f=np.empty((N, 2)))

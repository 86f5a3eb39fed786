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

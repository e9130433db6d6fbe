"""Failure detection on the GPU without a GPU fault: a device wait that cannot end gives
up after its limit and the context stays usable; non-finite data and an unconverged
solve come back as status codes."""
import numpy as np
import pytest

from paper_2304_08159_gb300 import wl
from paper_2304_08159_gb300.wl import Sim

pytestmark = pytest.mark.gpu


def test_wait_probe_gives_up_and_context_survives():
    limit = 0.05
    rc, ms = wl.wl_wait_probe(limit)
    assert rc == wl.WL_ETIMEOUT
    assert 0.9 * limit * 1e3 <= ms <= limit * 1e3 + 500.0, ms
    # the context is still usable: a small simulation steps normally afterwards
    s = Sim((32, 16), 0.05, (1.0, 0.0), body={"kind": wl.WL_BODY_SPHERE, "center": (8, 8), "radius": 3})
    s.step(2)
    assert s.status()[0] == 0
    assert np.isfinite(s.get(wl.WL_FIELD_U)).all()
    s.close()


def test_nonfinite_velocity_poisons_the_sim():
    s = Sim((32, 16), 0.05, (1.0, 0.0), use_graph=False)
    u = s.get(wl.WL_FIELD_U)
    u.reshape(-1)[100] = np.nan
    s.set(wl.WL_FIELD_U, u)
    s.step(1)
    with pytest.raises(wl.WLError) as e:
        s.status()
    assert e.value.rc == wl.WL_ENONFINITE
    with pytest.raises(wl.WLError) as e:  # poisoned: later calls refuse
        s.step(1)
    assert e.value.rc == wl.WL_ENONFINITE
    s.close()


def test_unconverged_solve_is_a_warning_with_a_valid_state():
    s = Sim((32, 16), 0.05, (1.0, 0.0), body={"kind": wl.WL_BODY_SPHERE, "center": (8, 8), "radius": 3},
            tol=1e-14, max_vcycles=1)
    s.step(2)
    rc, last, total, worst = s.status()
    assert rc == wl.WL_WNOTCONV
    assert worst > 1e-14
    assert np.isfinite(s.get(wl.WL_FIELD_U)).all() and np.isfinite(s.get(wl.WL_FIELD_P)).all()
    s.close()

"""Checkpoint / resume (wl_save, wl_load): a run split into two halves, the second
resumed from the saved state in a freshly created sim, gives the same bits as the run
done in one go (velocity, pressure, dt, time and step count), with the state held in host
memory or on the device; states of another setup are refused."""
import numpy as np
import pytest

from tests.gpu_cases import make_pair

pytestmark = pytest.mark.gpu

CASES = [
    dict(id="sphere64x32x32", dims=(64, 32, 32), nu=0.02, U=(1.0, 0.0, 0.0), periodic=0,
         body=dict(kind=1, center=(20.0, 16.2, 15.7), radius=5.0), kw={}),
    dict(id="cyl96x48_exit", dims=(96, 48), nu=0.05, U=(1.0, 0.0), periodic=0,
         body=dict(kind=1, center=(30.0, 24.3), radius=6.0), kw=dict(exit_bc=True)),
    dict(id="zper48x32x32_fp32", dims=(48, 32, 32), nu=0.02, U=(1.0, 0.0, 0.0), periodic=4,
         body=dict(kind=2, center=(16.0, 16.0, 16.0), radius=7.0, radius2=2.5), kw=dict(precision=0)),
]


@pytest.mark.parametrize("device", [False, True], ids=["host", "device"])
@pytest.mark.parametrize("case", CASES, ids=lambda c: c["id"])
def test_split_run_resumes_bitwise(case, device):
    whole, _ = make_pair(case, oracle=False, **case["kw"])
    whole.step(10)
    first, _ = make_pair(case, oracle=False, **case["kw"])
    first.step(5)
    state = first.save(device=device)
    first.close()
    second, _ = make_pair(case, oracle=False, **case["kw"])
    second.load(state)
    second.step(5)
    for f in (0, 1):
        assert np.array_equal(whole.get(f), second.get(f)), f
    assert whole.dt == second.dt
    assert whole.time() == second.time()
    if case["kw"].get("exit_bc"):
        assert np.array_equal(whole.get(7), second.get(7))
    whole.close()
    second.close()


def test_load_refuses_other_setup():
    from paper_2304_08159_gb300 import wl

    case = CASES[0]
    a, _ = make_pair(case, oracle=False)
    a.step(1)
    state = a.save()
    other = dict(case, dims=(64, 32, 16))
    b, _ = make_pair(other, oracle=False)
    assert wl.wl_load(b.h, state.ctypes.data, state.nbytes, 0) == wl.WL_EINVAL
    bad = state.copy()
    bad[0] ^= 0xFF  # not a saved state
    assert wl.wl_load(a.h, bad.ctypes.data, bad.nbytes, 0) == wl.WL_EINVAL
    assert wl.wl_load(a.h, state.ctypes.data, state.nbytes - 4, 0) == wl.WL_EINVAL
    assert wl.wl_load(a.h, state.ctypes.data, state.nbytes, 0) == wl.WL_OK
    a.close()
    b.close()

"""GPU parity of the convective exit (wl_opts.exit_bc) against the FP64 oracle, whose
exit is pinned in tests/test_oracle_exit.py, and bitwise agreement of its code paths.
Bars as the other whole-step parity tests: velocity (and the exit plane) relative L2
<= 1e-5, pressure (mean over active cells removed) <= 1e-5 at Poisson tol 1e-8, drag
relative <= 1e-4; the exit plane's mean equals U_x to FP32 rounding."""
import numpy as np
import pytest

import oracle as O
from tests.gpu_cases import rel_l2, active_mask

pytestmark = pytest.mark.gpu


def _pair(case, tol=1e-8, oracle=True, **kw):
    from paper_2304_08159_gb300 import Sim

    sim = Sim(case["dims"], case["nu"], case["U"], body=case["body"], periodic=case["periodic"], tol=tol,
              exit_bc=True, **kw)
    ref = None
    if oracle:
        ref = O.Oracle(case["dims"], case["nu"], U=case["U"], periodic=case["periodic"], body=case["body"])
        ref.set_exit(True)
        ref.set_ic(0)
    return sim, ref


CYL = dict(id="cyl", dims=(128, 64), nu=0.064, U=(1.0, 0.0), periodic=0,
           body=dict(kind=1, center=(32.0, 32.0), radius=8.0))
SPH = dict(id="sph", dims=(64, 32, 32), nu=0.02, U=(1.0, 0.0, 0.0), periodic=0,
           body=dict(kind=1, center=(16.3, 15.8, 16.2), radius=5.0))
ZPER = dict(id="zper", dims=(64, 32, 32), nu=0.02, U=(1.0, 0.0, 0.0), periodic=4,
            body=dict(kind=1, center=(20.0, 16.0, 16.0), radius=5.0))


@pytest.mark.parametrize("case,steps", [(CYL, 10), (SPH, 6), (ZPER, 6)], ids=["cyl", "sph", "zper"])
def test_exit_steps_parity(case, steps):
    from paper_2304_08159_gb300 import wl

    sim, ref = _pair(case)
    sim.step(steps)
    ref.step(steps, tol=1e-12)
    rc, last, tot, worst = sim.status()
    assert rc == 0, (rc, last, tot, worst)
    eu = rel_l2(sim.get(0).astype(np.float64), ref.get_u())
    act = active_mask(ref)
    pg, po = sim.get(1).astype(np.float64), ref.get_p()
    pg = (pg - pg[act].mean()) * act
    po = (po - po[act].mean()) * act
    ep = rel_l2(pg, po)
    eg = sim.get(wl.WL_FIELD_EXIT).astype(np.float64)
    eo = ref.get_exit()
    ee = rel_l2(eg.reshape(-1), eo.reshape(-1))
    Fg, Fo = sim.forces(), ref.forces()
    ef = abs(Fg[0] - Fo[0]) / abs(Fo[0])
    print(f"{case['id']}: u {eu:.2e} p {ep:.2e} exit {ee:.2e} drag {ef:.2e}")
    assert eu <= 1e-5 and ep <= 1e-5 and ee <= 1e-5 and ef <= 1e-4, (eu, ep, ee, ef)
    assert abs(eg.mean() - case["U"][0]) <= 1e-6
    assert np.abs(eg - case["U"][0]).max() > 1e-5  # the wake reached the exit


def test_exit_free_stream_exact():
    from paper_2304_08159_gb300 import wl

    case = dict(id="fs", dims=(96, 48, 40), nu=0.01, U=(0.7, 0.0, 0.0), periodic=0, body=None)
    sim, _ = _pair(case, oracle=False)
    sim.step(3)
    u = sim.get(0)
    assert np.all(u[0] == np.float32(0.7)) and np.all(u[1:] == 0.0)
    assert np.all(sim.get(wl.WL_FIELD_EXIT) == np.float32(0.7))


@pytest.mark.parametrize("env", ["WL_NO_TMA", "WL_NO_UNIFORM", "WL_NO_TAIL"])
def test_exit_code_paths_agree(env, monkeypatch):
    """With the exit, the staged and table kernels, the uniform split and the small-level
    tail give the same bits as their alternatives (three steps)."""
    from paper_2304_08159_gb300 import wl

    case = dict(SPH, dims=(128, 64, 64), body=dict(kind=1, center=(40.3, 31.8, 32.2), radius=6.0))
    monkeypatch.setenv("WL_UNIFORM_ALL", "1")
    a, _ = _pair(case, oracle=False, tol=1e-6)
    monkeypatch.delenv("WL_UNIFORM_ALL")
    monkeypatch.setenv(env, "1")
    b, _ = _pair(case, oracle=False, tol=1e-6)
    monkeypatch.delenv(env)
    a.step(3)
    b.step(3)
    assert np.array_equal(a.get(0), b.get(0))
    assert np.array_equal(a.get(1), b.get(1))
    assert np.array_equal(a.get(wl.WL_FIELD_EXIT), b.get(wl.WL_FIELD_EXIT))


def test_exit_graph_and_host_loop_agree():
    case = dict(CYL, dims=(96, 48), body=dict(kind=1, center=(24.0, 24.0), radius=6.0))
    a, _ = _pair(case, oracle=False, use_graph=True)
    b, _ = _pair(case, oracle=False, use_graph=False)
    a.step(4)
    b.step(4)
    assert np.array_equal(a.get(0), b.get(0))
    assert np.array_equal(a.get(1), b.get(1))


def test_exit_argument_checks():
    from paper_2304_08159_gb300 import Sim, wl

    with pytest.raises(wl.WLError):  # x periodic
        Sim((32, 16), 0.05, (1.0, 0.0), periodic=1, exit_bc=True)
    with pytest.raises(wl.WLError):  # no outflow through the upper x face
        Sim((32, 16), 0.05, (-1.0, 0.0), exit_bc=True)
    sim = Sim((32, 16), 0.05, (1.0, 0.0), body=dict(kind=1, center=(8.0, 8.0), radius=3.0), exit_bc=True,
              dt_fixed=0.2)
    with pytest.raises(wl.WLError):  # not differentiated
        sim.grad_forward(2, 1)
    sim.close()

"""Per-step metric ring (wl_get_metrics): each step's record matches what the sim reports
through its other entry points (clock, dt, V-cycles, status) and, with wl_opts.metrics,
the kinetic energy, max |div u| and pressure force of its end state computed here from
the fields; the ring keeps the last WL_METRIC_RING steps in order."""
import numpy as np
import pytest

from tests.gpu_cases import make_pair

pytestmark = pytest.mark.gpu


def _ke_maxdiv(sim, case):
    """Kinetic energy and max |div u| of the sim's velocity, from the definitions: the
    divergence sums u_c[I+e_c] - u_c[I], the upper face of a non-periodic side carrying U_c."""
    u = sim.get(0).astype(np.float64)
    D = sim.D
    ke = 0.5 * (u ** 2).sum() / sim.ncell
    div = np.zeros(sim.shape)
    for c in range(D):
        ax = D - 1 - c
        up = np.roll(u[c], -1, axis=ax)
        if not (case["periodic"] >> c) & 1:
            idx = [slice(None)] * D
            idx[ax] = -1
            up[tuple(idx)] = case["U"][c]
        div += up - u[c]
    return ke, np.abs(div).max()


@pytest.mark.parametrize("case", [
    dict(id="sphere48x32x32", dims=(48, 32, 32), nu=0.02, U=(1.0, 0.0, 0.0), periodic=0,
         body=dict(kind=1, center=(16.0, 16.2, 15.7), radius=5.0)),
    dict(id="cyl64x32", dims=(64, 32), nu=0.064, U=(1.0, 0.0), periodic=0,
         body=dict(kind=1, center=(16.0, 16.0), radius=5.0)),
    dict(id="tgv32", dims=(32, 32, 32), nu=0.01, U=(0.0, 0.0, 0.0), periodic=7, body=None),
], ids=lambda c: c["id"])
def test_metric_records_match_the_state(case):
    sim, _ = make_pair(case, oracle=False, metrics=True)
    if case["body"] is None:
        sim.set_ic(1, 1.0)
    t_prev, n = 0.0, 6
    for s in range(n):
        dt = sim.dt
        sim.step(1)
        m = sim.metrics(1)
        t, steps = sim.time()
        rc, last, tot, worst = sim.status()
        assert m["step"][0] == steps == s + 1
        assert m["time"][0] == t and m["dt"][0] == dt
        assert abs(t - t_prev - dt) <= 1e-12 * t
        t_prev = t
        assert (m["vcycles1"][0], m["vcycles2"][0]) == tuple(last)
        assert max(m["resid1"][0], m["resid2"][0]) <= 1e-6
        ke, md = _ke_maxdiv(sim, case)
        assert abs(m["ke"][0] - ke) <= 1e-12 * ke
        assert abs(m["maxdiv"][0] - md) <= 1e-6 * max(md, 1.0)
        # dt of the next step follows from the recorded CFL maximum
        assert abs(sim.dt - min(10.0, 1.0 / (m["cfl"][0] + 2 * sim.D * case["nu"]))) <= 1e-12 * sim.dt
        if case["body"] is not None:
            F = sim.forces()
            assert np.allclose([m["F0"][0], m["F1"][0], m["F2"][0]][: sim.D], F, rtol=0, atol=1e-12 * np.abs(F).max())
    allm = sim.metrics()
    assert list(allm["step"]) == list(range(1, n + 1))
    sim.close()


def test_ring_keeps_the_last_steps_in_order():
    from paper_2304_08159_gb300 import wl

    case = dict(id="c16", dims=(16, 16), nu=0.05, U=(1.0, 0.0), periodic=0, body=None)
    sim, _ = make_pair(case, oracle=False)
    n = wl.METRIC_RING + 37
    sim.step(n)
    m = sim.metrics()
    assert len(m["step"]) == wl.METRIC_RING
    assert list(m["step"]) == list(range(n - wl.METRIC_RING + 1, n + 1))
    assert np.all(np.diff(m["time"]) > 0)
    assert np.all(np.isnan(m["ke"])) and np.all(np.isnan(m["F0"]))  # metrics off: not measured
    last5 = sim.metrics(5)
    assert list(last5["step"]) == list(range(n - 4, n + 1))
    sim.close()

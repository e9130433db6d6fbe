"""Serving on the GPU: every request's result is the same alone and in the mix."""
import numpy as np
import pytest

from paper_2304_08159_gb300 import serve, wl

pytestmark = pytest.mark.gpu


def small_requests():
    reqs = []
    for i, (dims, R, steps) in enumerate([((64, 64), 5.0, 12), ((32, 32, 32), 4.0, 7), ((96, 96), 8.0, 9),
                                          ((48, 48, 48), 6.0, 5), ((64, 64), 6.5, 10), ((32, 32, 32), 4.5, 8)]):
        c = tuple([dims[0] / 4] + [d / 2 for d in dims[1:]])
        reqs.append(serve.Request(i, 0.5 * i, dims, 2.0 * R / 250.0, dict(kind=wl.WL_BODY_SPHERE, center=c, radius=R),
                                  steps))
    return reqs


def test_results_same_alone_and_in_the_mix():
    import torch

    reqs = small_requests()
    alone = {}
    for r in reqs:
        s = wl.Sim(r.dims, r.nu, (1.0,) + (0.0,) * (len(r.dims) - 1), body=r.body)
        s.step(r.steps)
        alone[r.rid] = (s.get(wl.WL_FIELD_U), s.get(wl.WL_FIELD_P), s.dt)
        s.close()
    mixed = {}

    def on_finish(req, sim):
        mixed[req.rid] = (sim.get(wl.WL_FIELD_U), sim.get(wl.WL_FIELD_P), sim.dt)

    # a budget of three of the larger workspaces: requests queue, overlap and replace one another
    budget = 3 * max(serve.workspace_bytes(r) for r in reqs)
    stats, lat = serve.serve_gpu(reqs, budget_bytes=budget, on_finish=on_finish)
    assert sorted(mixed) == [r.rid for r in reqs] and not stats["rejected"]
    assert max(n for n, _, _ in stats["rounds"]) > 1
    for rid, (u, p, dt) in alone.items():
        um, pm, dtm = mixed[rid]
        assert np.array_equal(u, um) and np.array_equal(p, pm) and dt == dtm, rid
    assert len(lat) == len(stats["rounds"]) and min(lat) > 0


def test_mix_requests_match_oracle():
    """Requests served in the mix against the FP64 oracle stepping the same flow alone
    (projections to 1e-10): a 2-D one (64 x 64 cylinder, 12 steps) and a 3-D one (32^3
    sphere, 7 steps).  Velocity within the stated 1e-5 relative L2, dt and time within
    1e-5, drag coefficient within 1e-4; the pressure (mean over active cells removed)
    within the tolerance gap of the mix's Poisson tol 1e-6 (1e-3)."""
    import oracle as O
    from tests.gpu_cases import rel_l2

    reqs = small_requests()
    mixed = {}

    def on_finish(req, sim):
        mixed[req.rid] = (sim.get(wl.WL_FIELD_U), sim.get(wl.WL_FIELD_P), sim.dt, sim.time(), sim.forces())

    budget = 3 * max(serve.workspace_bytes(r) for r in reqs)
    serve.serve_gpu(reqs, budget_bytes=budget, on_finish=on_finish)
    for r in (reqs[0], reqs[1]):
        U = (1.0,) + (0.0,) * (len(r.dims) - 1)
        ref = O.Oracle(r.dims, r.nu, U=U, body=r.body)
        ref.set_ic(0)
        ref.step(r.steps, tol=1e-10, maxit=200, solver=1)
        u, p, dt, (t, n), F = mixed[r.rid]
        uo = ref.get_u()
        act = ref.poisson_diag() > 0
        po = ref.get_p()
        pg = p.astype(np.float64)
        pg = (pg - pg[act].mean()) * act
        po = (po - po[act].mean()) * act
        print(f"request {r.rid} {r.dims}: u {rel_l2(u.astype(np.float64), uo):.2e}, p {rel_l2(pg, po):.2e}")
        assert n == r.steps
        assert rel_l2(u.astype(np.float64), uo) <= 1e-5
        assert rel_l2(pg, po) <= 1e-3
        assert abs(dt - ref.dt) <= 1e-5 * ref.dt and abs(t - ref.time) <= 1e-5 * ref.time
        Fo = ref.forces()
        assert abs(F[0] - Fo[0]) <= 1e-4 * abs(Fo[0])

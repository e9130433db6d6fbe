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

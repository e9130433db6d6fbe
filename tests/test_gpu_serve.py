"""Serving on the GPU: every request's result is the same alone and in the mix, stepped
with its own graph or in a batched graph, and matches the oracle."""
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


@pytest.mark.parametrize("batch_cells", [0, 10000, 1 << 18], ids=["graphs", "batch2d", "batchall"])
def test_results_same_alone_and_in_the_mix(batch_cells):
    """batch_cells 0: every resident steps with its own graph; 10000: the 2-D grids step in
    one batched graph, the 3-D ones with their own; 2^18: all of them batched."""
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
    stats, lat = serve.serve_gpu(reqs, budget_bytes=budget, on_finish=on_finish, batch_cells=batch_cells)
    assert sorted(mixed) == [r.rid for r in reqs] and not stats["rejected"]
    assert max(n for n, _, _ in stats["rounds"]) > 1
    for rid, (u, p, dt) in alone.items():
        um, pm, dtm = mixed[rid]
        assert np.array_equal(u, um) and np.array_equal(p, pm) and dt == dtm, rid
    assert len(lat) == len(stats["rounds"]) and min(lat) > 0
    if batch_cells:
        small, large = serve.class_latencies_ms(stats)
        ns = sum(r.steps for r in reqs if r.cells <= batch_cells)
        assert len(small) == ns and len(large) == sum(r.steps for r in reqs) - ns
        assert min(small) > 0


def test_batch_steps_through_the_c_abi():
    """wl_batch_step directly: three small sims (2-D and 3-D, with and without a body)
    advanced five rounds in one batch, and a large one beside them, give the bits each
    gets from wl_step alone; the small-done event is recorded."""
    import torch

    cases = [((64, 32), dict(kind=wl.WL_BODY_SPHERE, center=(16.0, 16.0), radius=5.0)),
             ((48, 48), None),
             ((32, 16, 16), dict(kind=wl.WL_BODY_SPHERE, center=(10.0, 8.0, 8.0), radius=3.0)),
             ((64, 32, 32), dict(kind=wl.WL_BODY_SPHERE, center=(20.0, 16.0, 16.0), radius=5.0))]

    def make(dims, body):
        stream = torch.cuda.Stream()
        with torch.cuda.stream(stream):
            sim = wl.Sim(dims, 0.02, (1.0,) + (0.0,) * (len(dims) - 1), body=body)
        return sim, stream

    ref = []
    for dims, body in cases:
        sim, _ = make(dims, body)
        sim.step(5)
        ref.append((sim.get(0), sim.get(1), sim.dt))
        sim.close()
    sims = [make(d, b) for d, b in cases]
    batch = wl.Batch(20000)  # the 64 x 32 x 32 sim steps with its own graph
    stream = torch.cuda.Stream()
    for _ in range(5):
        done = torch.cuda.Event(enable_timing=True)
        done.record(stream)  # creates the event (wl_batch_step records it again)
        assert batch.step([s.h for s, _ in sims], stream.cuda_stream, done.cuda_event) == wl.WL_OK
    torch.cuda.synchronize()
    for (sim, _), (u, p, dt) in zip(sims, ref):
        assert np.array_equal(sim.get(0), u) and np.array_equal(sim.get(1), p) and sim.dt == dt
        assert sim.time()[1] == 5
    batch.close()
    for sim, _ in sims:
        sim.close()


def test_mix_requests_match_oracle():
    """Requests served in the mix (batched steps) against the FP64 oracle stepping the same flow alone
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
    serve.serve_gpu(reqs, budget_bytes=budget, on_finish=on_finish, batch_cells=1 << 18)
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

"""Host logic of the serving loop (no GPU): the seeded request stream and the
admission / stepping / retirement schedule, with stand-in simulations."""
import numpy as np

from paper_2304_08159_gb300 import serve


def test_request_stream_is_seeded_and_in_range():
    a = serve.request_stream(200)
    b = serve.request_stream(200)
    assert [(r.dims, r.nu, r.steps, r.arrival) for r in a] == [(r.dims, r.nu, r.steps, r.arrival) for r in b]
    arr = [r.arrival for r in a]
    assert all(x < y for x, y in zip(arr, arr[1:]))
    n2 = n3 = 0
    for r in a:
        N = r.dims[0]
        assert all(d == N for d in r.dims) and N % 16 == 0
        R = r.body["radius"]
        Re = 2.0 * R / r.nu
        assert 4.0 <= R <= 24.0 and 100.0 <= Re <= 1000.0 + 1e-9 and 20 <= r.steps <= 200
        c = r.body["center"]
        assert all(R < c[d] < N - R for d in range(len(r.dims)))
        if len(r.dims) == 2:
            assert 64 <= N <= 512
            n2 += 1
        else:
            assert 32 <= N <= 192
            n3 += 1
    assert n2 > 60 and n3 > 60


class FakeSim:
    live = set()

    def __init__(self, req):
        self.req = req
        self.steps = 0
        FakeSim.live.add(req.rid)

    def close(self):
        FakeSim.live.discard(self.req.rid)


def run_fake(requests, budget, max_slots=256):
    log = []
    sizes = {r.rid: serve.workspace_bytes(r) for r in requests}

    def make_sim(req):
        return FakeSim(req), None

    def step_batch(residents):
        used = sum(sizes[r.req.rid] for r in residents)
        assert used <= budget and len(residents) <= max_slots
        for r in residents:
            r.sim.steps += 1
        log.append([r.req.rid for r in residents])
        return None

    done = {}

    def on_finish(req, sim):
        done[req.rid] = sim.steps

    srv = serve.Server(budget, max_slots=max_slots, on_finish=on_finish, make_sim=make_sim, step_batch=step_batch)
    stats = srv.run(requests)
    return stats, log, done, sizes


def test_schedule_respects_budget_and_finishes_everything():
    reqs = serve.request_stream(40, rate=3.0)
    sizes = [serve.workspace_bytes(r) for r in reqs]
    budget = 3 * max(sizes)
    stats, log, done, _ = run_fake(reqs, budget)
    assert not stats["rejected"] and not FakeSim.live
    assert done == {r.rid: r.steps for r in reqs}  # every request got exactly its steps
    assert stats["peak_bytes"] <= budget
    assert max(len(x) for x in log) > 1  # work overlapped
    # admission is first come, first served
    order = [rid for rid, _ in stats["admitted"]]
    assert order == [r.rid for r in sorted(reqs, key=lambda r: (r.arrival, r.rid))]
    # nothing is admitted before it arrives
    arrival = {r.rid: r.arrival for r in reqs}
    assert all(rnd >= arrival[rid] for rid, rnd in stats["admitted"])


def test_slots_limit_and_oversized_requests():
    reqs = serve.request_stream(30, rate=5.0)
    stats, log, done, sizes = run_fake(reqs, budget=1 << 50, max_slots=4)
    assert max(len(x) for x in log) <= 4 and len(done) == 30
    big = max(reqs, key=lambda r: sizes[r.rid])
    stats, log, done, _ = run_fake(reqs, budget=sizes[big.rid] - 1)
    assert big.rid in stats["rejected"] and big.rid not in done
    assert len(done) + len(stats["rejected"]) == 30

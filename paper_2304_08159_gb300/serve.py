"""Serving: many simulations of different sizes resident on one GPU.

Requests (a grid, a body, a viscosity and a number of steps) arrive over time and
wait in a FIFO queue; a request is admitted as soon as its workspace fits the memory
budget and a slot is free, and leaves when its last step is done, which frees its
memory for the next one (continuous batching).  Every round advances all resident
simulations by one time step together: `wl_step_batch` launches each simulation's
step graph (its whole time step, V-cycle loops included, captured once) on its own
stream, forked from and joined back to the server's stream, so the steps of all
resident simulations overlap on the device and the host issues one call per round.
The device time of a round is the step latency every resident request sees.

Each simulation keeps its own workspace and stream and shares nothing with the
others, so its result is the same alone and in any mix (bit for bit).
"""
from __future__ import annotations

import collections
import dataclasses
import math
import time

import numpy as np

from . import wl


@dataclasses.dataclass
class Request:
    rid: int
    arrival: float  # in rounds of the server's clock
    dims: tuple
    nu: float
    body: dict
    steps: int

    @property
    def cells(self) -> int:
        return int(np.prod(self.dims))


def request_stream(n, seed=20230417, rate=2.0):
    """n requests of the serving mix: Poisson arrivals (`rate` per round); half are 2-D
    flows past a circle on N x N cells (N from 64 to 512), half 3-D flows past a sphere
    on N^3 cells (N from 32 to 192), N a multiple of 16 drawn log-uniformly; radius 4 to
    24 cells within the box, a quarter of the way down it; inflow U = 1 along x;
    Re uniform in [100, 1000] on the diameter; 20 to 200 steps."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(n):
        t += rng.exponential(1.0 / rate)
        if rng.random() < 0.5:
            N = 16 * int(round(2 ** rng.uniform(6.0, 9.0) / 16))
            R = float(rng.uniform(4.0, min(24.0, N / 8)))
            dims, center = (N, N), (N / 4, N / 2)
        else:
            N = 16 * int(round(2 ** rng.uniform(5.0, math.log2(192.0)) / 16))
            R = float(rng.uniform(4.0, min(24.0, N / 6)))
            dims, center = (N, N, N), (N / 4, N / 2, N / 2)
        Re = float(rng.uniform(100.0, 1000.0))
        steps = int(rng.integers(20, 201))
        out.append(Request(i, t, dims, 2.0 * R / Re, dict(kind=wl.WL_BODY_SPHERE, center=center, radius=R), steps))
    return out


def workspace_bytes(req, tol=1e-6):
    o = wl.wl_default_opts()
    o.tol = tol
    return int(wl.wl_workspace_bytes(req.dims, o))


class _Resident:
    __slots__ = ("req", "sim", "stream", "left", "nbytes", "admitted")

    def __init__(self, req, sim, stream, nbytes, admitted):
        self.req, self.sim, self.stream, self.nbytes, self.admitted = req, sim, stream, nbytes, admitted
        self.left = req.steps


class Server:
    """Continuous batching of simulations on one GPU (see the module docstring).

    budget_bytes: device memory the resident workspaces may take together;
    max_slots: most simulations resident at once; on_finish(req, sim): called when a
    request's last step is done, before its simulation is closed (read results there).
    `make_sim` and `step_batch` are the GPU hooks (defaults: wl.Sim on its own stream
    and wl_step_batch); the scheduling itself is plain host logic.
    """

    def __init__(self, budget_bytes, max_slots=256, tol=1e-6, on_finish=None, make_sim=None, step_batch=None,
                 timer=None, batch_cells=0):
        self.budget = int(budget_bytes)
        self.max_slots = int(max_slots)
        self.tol = tol
        self.on_finish = on_finish
        self._make_sim = make_sim or self._gpu_sim
        self._step_batch = step_batch or self._gpu_step_batch
        self._timer = timer
        self.stream = None
        # batch_cells > 0: simulations of at most that many cells step together in one
        # batched graph per dimension (wl_batch_step), the others with their own graphs
        self.batch_cells = int(batch_cells)
        self.batch = None

    # ---- GPU hooks
    def _gpu_sim(self, req):
        import torch

        stream = torch.cuda.Stream()
        with torch.cuda.stream(stream):
            sim = wl.Sim(req.dims, req.nu, (1.0,) + (0.0,) * (len(req.dims) - 1), body=req.body, tol=self.tol)
        return sim, stream

    def _gpu_step_batch(self, residents):
        import torch

        if self.stream is None:
            # with a batch, the server's stream (which runs the batched graphs) takes the
            # higher priority, so the small simulations' blocks are scheduled ahead of the
            # large ones' and their step latency stays short
            self.stream = torch.cuda.Stream(priority=-1 if self.batch_cells > 0 else 0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(self.stream)
        if self.batch_cells > 0:
            if self.batch is None:
                self.batch = wl.Batch(self.batch_cells)
            es = torch.cuda.Event(enable_timing=True)
            es.record(self.stream)  # creates the event; wl_batch_step records it again where the batch ends
            self.batch.step([r.sim.h for r in residents], self.stream.cuda_stream, es.cuda_event)
            e1.record(self.stream)
            small = sum(1 for r in residents if r.req.cells <= self.batch_cells)
            return (e0, e1, es, small, len(residents) - small)
        rc = wl.wl_step_batch([r.sim.h for r in residents], 1, self.stream.cuda_stream)
        e1.record(self.stream)
        if rc < 0:
            raise wl.WLError(rc, "wl_step_batch")
        return (e0, e1)

    # ---- the request loop
    def run(self, requests):
        """Serve `requests` to completion.  Returns a dict of statistics: rounds,
        wall time, cells*steps, per-round (occupancy, timing token), admissions."""
        pending = collections.deque(sorted(requests, key=lambda r: (r.arrival, r.rid)))
        queue = collections.deque()
        active = []
        used = 0
        rnd = 0
        rounds = []
        admitted = []
        rejected = []
        finished = []
        peak_used = 0
        t0 = time.perf_counter()
        while pending or queue or active:
            while pending and pending[0].arrival <= rnd:
                queue.append(pending.popleft())
            if not active and not queue:
                rnd = max(rnd + 1, int(math.ceil(pending[0].arrival)))
                continue
            # admission: FIFO while the head fits the memory budget and a slot is free
            while queue and len(active) < self.max_slots:
                req = queue[0]
                nb = workspace_bytes(req, self.tol)
                if nb > self.budget:
                    rejected.append(queue.popleft().rid)
                    continue
                if used + nb > self.budget:
                    break
                queue.popleft()
                sim, stream = self._make_sim(req)
                active.append(_Resident(req, sim, stream, nb, rnd))
                used += nb
                peak_used = max(peak_used, used)
                admitted.append((req.rid, rnd))
            if not active:
                rnd += 1
                continue
            token = self._step_batch(active)
            rounds.append((len(active), sum(r.req.cells for r in active), token))
            keep = []
            for r in active:
                r.left -= 1
                if r.left == 0:
                    if self.on_finish:
                        self.on_finish(r.req, r.sim)
                    r.sim.close()
                    used -= r.nbytes
                    finished.append((r.req.rid, r.admitted, rnd))
                else:
                    keep.append(r)
            active = keep
            rnd += 1
        if self._timer:
            self._timer()
        wall = time.perf_counter() - t0
        done = {rid for rid, _, _ in finished}
        cs = sum(q.cells * q.steps for q in requests if q.rid in done)
        return dict(rounds=rounds, wall_s=wall, cells_steps=cs, admitted=admitted, finished=finished,
                    rejected=rejected, peak_bytes=peak_used)


def round_latencies_ms(stats):
    """Device time of each round (ms) from the timing events of a GPU run."""
    import torch

    torch.cuda.synchronize()
    return [tok[0].elapsed_time(tok[1]) for _, _, tok in stats["rounds"]]


def class_latencies_ms(stats):
    """Step latencies (ms) seen by the small (batched) and the large simulations of a run
    with a batch: every resident request's step of a round counts once, a small one at the
    batch's completion, a large one at the round's end.  Returns (small, large) lists."""
    import torch

    torch.cuda.synchronize()
    small, large = [], []
    for _, _, tok in stats["rounds"]:
        if len(tok) < 5:
            continue
        e0, e1, es, ns, nl = tok
        # es was recorded by the library (wl_batch_step), so its time comes through it
        small += [wl.wl_event_elapsed(e0.cuda_event, es.cuda_event)] * ns
        large += [e0.elapsed_time(e1)] * nl
    return small, large


def serve_gpu(requests, budget_bytes=None, max_slots=256, tol=1e-6, on_finish=None, batch_cells=0):
    """Batched run on the current GPU; returns (stats, per-round latencies in ms).
    batch_cells > 0: the simulations of at most that many cells step in batched graphs."""
    import torch

    if budget_bytes is None:
        free, _ = torch.cuda.mem_get_info()
        budget_bytes = int(0.5 * free)
    srv = Server(budget_bytes, max_slots=max_slots, tol=tol, on_finish=on_finish, timer=torch.cuda.synchronize,
                 batch_cells=batch_cells)
    stats = srv.run(requests)
    lat = round_latencies_ms(stats)
    if srv.batch is not None:
        srv.batch.close()
    return stats, lat


def sequential_gpu(requests, tol=1e-6, on_finish=None):
    """The same requests one at a time (each alone on the device, graph-launched steps).
    Returns (wall seconds, cells*steps, per-step latencies in ms: one per request)."""
    import torch

    stream = torch.cuda.Stream()
    t0 = time.perf_counter()
    lat = []
    cs = 0
    with torch.cuda.stream(stream):
        for req in sorted(requests, key=lambda r: (r.arrival, r.rid)):
            sim = wl.Sim(req.dims, req.nu, (1.0,) + (0.0,) * (len(req.dims) - 1), body=req.body, tol=tol)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sim.step(req.steps)
            e1.record(stream)
            if on_finish:
                on_finish(req, sim)
            e1.synchronize()
            lat.append(e0.elapsed_time(e1) / req.steps)
            sim.close()
            cs += req.cells * req.steps
    torch.cuda.synchronize()
    return time.perf_counter() - t0, cs, lat

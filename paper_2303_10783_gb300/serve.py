"""Continuous-batching simulation server.

Requests (a case dictionary and an arrival time) are admitted in arrival
order as soon as they have arrived and their device workspace fits the HBM
budget; admitted requests keep their fields on the device. Each request
advances on its own CUDA stream in chunks of a few graph-replayed steps, with
up to `depth` chunks in flight; the host polls each request's CUDA events and
never waits for a round: a request whose last chunk has completed is retired
at once (its fields read back if asked, its workspace freed), and the
requests waiting for memory are admitted in the same pass. Requests of
different sizes therefore overlap on the GPU and a small late request can
finish before a large early one. Latency is measured per request from
admission to completion and reported per 100 steps (p50/p99), beside queue
waits and the aggregate cell-steps/s. A request's result does not depend on
what runs beside it: the kernels' reductions are deterministic and cases
share no data.
"""
import collections
import time

from . import cases as cases_mod
from . import solid


class Request:
    def __init__(self, rid, arrival, case):
        self.rid = rid
        self.arrival = arrival
        self.case = case
        self.steps = int(case["steps"])
        self.cells = case["nx"] * case["ny"] * (case["nz"] if case["dim"] == 3 else 1)
        self.done_steps = 0
        self.admitted = None
        self.finished = None
        self.sim = None
        self.stream = None
        self.bytes = 0
        self.result = None
        self.inflight = []      # CUDA events of the chunks enqueued and not yet seen complete


class Server:
    """``budget_bytes``: HBM the active requests' workspaces may hold.
    ``chunk``: steps per enqueued chunk; ``depth``: chunks a request keeps in
    flight. ``keep_results``: copy each finished request's fields to the host
    (for checks). ``block_cap``: blocks per cooperative solver launch of each
    request (0: no cap; -1: in proportion to the request's size); requests
    that share the GPU run more of their solves at once with a cap.
    ``precond``: pressure solver for every request ("dct", "mg", "jacobi";
    None keeps each request's own). ``slots``: requests on the GPU at once at
    most (0: only the memory budget limits them); fewer slots give each
    admitted request a larger share of the GPU, so it finishes sooner, while
    later arrivals wait longer in the queue."""

    def __init__(self, budget_bytes, precision=solid.SS_MIXED, chunk=10, keep_results=False, block_cap=0, depth=2,
                 precond=None, slots=0):
        self.budget = int(budget_bytes)
        self.slots = int(slots)
        self.depth = max(1, int(depth))
        self.precond = precond
        self.block_cap = int(block_cap)
        self.precision = precision
        self.chunk = int(chunk)
        self.keep = keep_results
        self.used = 0
        self.max_active = 0
        self.max_used = 0

    @staticmethod
    def _cap_for(r):
        """Blocks per solver launch in proportion to the request's size: one
        per 8192 cells, at least 16; no cap once that reaches 152 (one block
        per SM of a GB300)."""
        cap = max(16, r.cells // 8192)
        return 0 if cap >= 152 else cap

    def _admit(self, r, now):
        import torch
        r.stream = torch.cuda.Stream()
        with torch.cuda.stream(r.stream):
            r.sim = solid.Case(r.case, precision=self.precision, stream=r.stream)
            cap = self._cap_for(r) if self.block_cap < 0 else self.block_cap
            if cap:
                r.sim.set_block_cap(cap)
            f = cases_mod.initial_fields(r.case)
            r.sim.initialize(f["T"], f["C"])
        r.admitted = now
        self.used += r.bytes

    def _retire(self, r, now):
        r.sim.sync()
        if self.keep:
            r.result = r.sim.get_fields()
        r.sim.close()
        r.sim = None
        r.finished = now
        self.used -= r.bytes

    def _pump(self, r, now):
        """Advance request r without waiting: drop its completed chunks,
        retire it when everything it needs has run, else keep up to `depth`
        chunks in flight. Returns (progressed, cell-steps enqueued, retired)."""
        import torch
        progressed = False
        while r.inflight and r.inflight[0].query():
            r.inflight.pop(0)
            progressed = True
        if r.done_steps >= r.steps and not r.inflight:
            self._retire(r, now)
            return True, 0, True
        enq = 0
        while len(r.inflight) < self.depth and r.done_steps < r.steps:
            k = min(self.chunk, r.steps - r.done_steps)
            r.sim.step_graph(k)
            r.done_steps += k
            enq += k * r.cells
            ev = torch.cuda.Event()
            ev.record(r.stream)
            r.inflight.append(ev)
            progressed = True
        return progressed, enq, False

    def run(self, requests, time_scale=1.0):
        """Serve ``requests`` (list of (arrival_s, case)); arrivals are replayed
        in real time scaled by ``time_scale``. Returns a report dict."""
        reqs = []
        for q, (t, c) in enumerate(requests):
            if self.precond:
                c = dict(c, precond_p=self.precond)
            reqs.append(Request(q, t * time_scale, c))
        for r in reqs:
            r.bytes = solid.workspace_bytes(r.case, self.precision)
            if r.bytes > self.budget:
                raise ValueError("request %d needs %d bytes, more than the whole budget" % (r.rid, r.bytes))
        pending = collections.deque(sorted(reqs, key=lambda r: r.arrival))
        active = []
        t0 = time.perf_counter()
        cell_steps = 0
        while pending or active:
            now = time.perf_counter() - t0
            # admission: every arrived request, in arrival order, while its workspace fits
            while (pending and pending[0].arrival <= now and self.used + pending[0].bytes <= self.budget
                   and (self.slots <= 0 or len(active) < self.slots)):
                r = pending.popleft()
                self._admit(r, now)
                active.append(r)
            self.max_active = max(self.max_active, len(active))
            self.max_used = max(self.max_used, self.used)
            progressed = False
            still = []
            for r in active:
                moved, enq, retired = self._pump(r, time.perf_counter() - t0)
                progressed = progressed or moved
                cell_steps += enq
                if not retired:
                    still.append(r)
            active = still
            if not progressed:
                # every active request has its chunks in flight (or none is admitted yet)
                wait = 2e-4
                if not active and pending:
                    wait = max(0.0, min(pending[0].arrival - (time.perf_counter() - t0), 0.01))
                time.sleep(wait)
        wall = time.perf_counter() - t0
        lat = sorted((r.finished - r.admitted) / (r.steps / 100.0) for r in reqs)
        tot = sorted((r.finished - r.arrival) / (r.steps / 100.0) for r in reqs)
        wait = sorted(r.admitted - r.arrival for r in reqs)

        def pct(v, p):
            return v[min(len(v) - 1, int(round(p / 100.0 * (len(v) - 1))))]

        per = [dict(rid=r.rid, arrival=r.arrival, admitted=r.admitted, finished=r.finished, steps=r.steps,
                    cells=r.cells) for r in reqs]
        return dict(requests=len(reqs), wall_s=wall, cell_steps=cell_steps, cell_steps_per_s=cell_steps / wall,
                    p50_ms_per_100_steps=1e3 * pct(lat, 50), p99_ms_per_100_steps=1e3 * pct(lat, 99),
                    p50_total_ms_per_100_steps=1e3 * pct(tot, 50), p99_total_ms_per_100_steps=1e3 * pct(tot, 99),
                    p50_queue_s=pct(wait, 50), p99_queue_s=pct(wait, 99), max_active=self.max_active,
                    max_used_bytes=self.max_used, budget_bytes=self.budget, per_request=per,
                    results={r.rid: r.result for r in reqs} if self.keep else None)

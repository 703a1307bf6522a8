"""Continuous-batching simulation server.

Requests (a case dictionary and an arrival time) are admitted in arrival
order while the sum of their device workspaces fits an HBM budget; admitted
requests keep their fields on the device and are stepped together, each on
its own CUDA stream with graph-replayed steps, in rounds of a few steps. A
request that finishes frees its workspace at once, so waiting requests join
the running ones at the next round (no batch barrier: the set of active
requests changes every round). Latency is measured per request from
admission to completion and reported per 100 steps (p50/p99), beside the
aggregate cell-steps/s. A request's result does not depend on what runs
beside it: the kernels' reductions are deterministic and cases share no data.
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


class Server:
    """``budget_bytes``: HBM the active requests' workspaces may hold.
    ``chunk``: steps per request per round. ``keep_results``: copy each
    finished request's fields to the host (for checks). ``block_cap``: blocks
    per cooperative solver launch of each request (0: no cap; -1: in
    proportion to the request's size); requests that share the GPU run more
    of their solves at once with a cap."""

    def __init__(self, budget_bytes, precision=solid.SS_MIXED, chunk=10, keep_results=False, block_cap=0):
        self.budget = int(budget_bytes)
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

    def run(self, requests, time_scale=1.0):
        """Serve ``requests`` (list of (arrival_s, case)); arrivals are replayed
        in real time scaled by ``time_scale``. Returns a report dict."""
        import torch
        reqs = [Request(q, t * time_scale, c) for q, (t, c) in enumerate(requests)]
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
            while pending and pending[0].arrival <= now and self.used + pending[0].bytes <= self.budget:
                r = pending.popleft()
                self._admit(r, now)
                active.append(r)
            self.max_active = max(self.max_active, len(active))
            self.max_used = max(self.max_used, self.used)
            if not active:
                if pending:
                    time.sleep(max(0.0, min(pending[0].arrival - now, 0.01)))
                continue
            # one round: every active request advances up to `chunk` steps on its stream
            for r in active:
                k = min(self.chunk, r.steps - r.done_steps)
                r.sim.step_graph(k)
                r.done_steps += k
                cell_steps += k * r.cells
            for r in active:
                r.stream.synchronize()
            now = time.perf_counter() - t0
            still = []
            for r in active:
                if r.done_steps >= r.steps:
                    self._retire(r, now)
                else:
                    still.append(r)
            active = still
        wall = time.perf_counter() - t0
        lat = sorted((r.finished - r.admitted) / (r.steps / 100.0) for r in reqs)
        wait = sorted(r.admitted - r.arrival for r in reqs)

        def pct(v, p):
            return v[min(len(v) - 1, int(round(p / 100.0 * (len(v) - 1))))]

        return dict(requests=len(reqs), wall_s=wall, cell_steps=cell_steps, cell_steps_per_s=cell_steps / wall,
                    p50_ms_per_100_steps=1e3 * pct(lat, 50), p99_ms_per_100_steps=1e3 * pct(lat, 99),
                    p50_queue_s=pct(wait, 50), p99_queue_s=pct(wait, 99), max_active=self.max_active,
                    max_used_bytes=self.max_used, budget_bytes=self.budget,
                    results={r.rid: r.result for r in reqs} if self.keep else None)

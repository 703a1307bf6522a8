"""Many independent cases stepped side by side on one GPU.

Each case owns a CUDA stream and a device workspace; one time step of a case
is a captured CUDA graph (``ss_step_graph``) replayed on its stream, so the
host issues one launch per case per step and the small cases' cooperative
solver grids (a few blocks each) run concurrently on the GPU. Every case is
independent: a case gives bit-identical fields alone or in a batch (the
kernels' reductions are deterministic and no data crosses cases).
"""
import time

from . import cases as cases_mod
from . import solid


class Batch:
    """A set of cases stepped together. ``case_dicts`` come from
    :mod:`paper_2303_10783_gb300.cases`; initial fields are the seeded ones."""

    def __init__(self, case_dicts, precision=solid.SS_MIXED, graphs=True):
        import torch
        self.graphs = graphs
        self.members = []
        for cd in case_dicts:
            stream = torch.cuda.Stream()
            with torch.cuda.stream(stream):
                c = solid.Case(cd, precision=precision, stream=stream)
                f = cases_mod.initial_fields(cd)
                c.initialize(f["T"], f["C"])
            self.members.append((cd, c, stream))

    @property
    def cells(self):
        return sum(cd["nx"] * cd["ny"] * (cd["nz"] if cd["dim"] == 3 else 1) for cd, _, _ in self.members)

    def step(self, n=1):
        """Enqueue n steps of every case (each on its own stream) and return."""
        for _ in range(n):
            for _, c, _ in self.members:
                if self.graphs:
                    c.step_graph(1)
                else:
                    c.step(1)

    def sync(self, allow=()):
        """Wait for every case; returns the worst sticky solver status."""
        worst = solid.SS_OK
        for _, c, _ in self.members:
            st = c.sync(allow=allow)
            worst = max(worst, st)
        return worst

    def run(self, steps, warmup=0):
        """Step every case `warmup` then `steps` steps; returns (seconds of the
        timed part, aggregate cell-steps/s)."""
        import torch
        if warmup:
            self.step(warmup)
            self.sync()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        self.step(steps)
        self.sync()
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        return dt, self.cells * steps / dt

    def set_block_cap(self, max_blocks):
        for _, c, _ in self.members:
            c.set_block_cap(max_blocks)

    def autotune(self, caps=(0, 64, 32, 16, 8), steps=2):
        """Choose the solver block cap (``ss_set_block_cap``) that steps this
        batch fastest. A cooperative solve of a small case is bound by its
        synchronisations, not by its SMs; fewer blocks per case let more
        cases' solves run at once, but too few starve the larger cases.
        Each candidate steps the batch ``steps`` times from the same state;
        the state (every field and the case time) is saved before and
        restored after each trial, so tuning leaves the cases where they
        were. Returns (best cap, {cap: seconds per step})."""
        import torch
        saved = []
        for _, c, _ in self.members:
            f = c.get_fields(device=True)
            saved.append((f, c.get_time()))

        def restore():
            for (f, t), (_, c, _) in zip(saved, self.members):
                c.set_fields(f)
                c.set_time(t)
            for _, c, _ in self.members:
                c.sync()

        timing = {}
        for cap in caps:
            self.set_block_cap(cap)
            self.step(1)                 # captures each case's graph with this launch shape
            self.sync()
            restore()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            self.step(steps)
            self.sync()
            torch.cuda.synchronize()
            timing[cap] = (time.perf_counter() - t0) / steps
            restore()
        best = min(timing, key=timing.get)
        self.set_block_cap(best)
        return best, timing

    def fields(self, q):
        return self.members[q][1].get_fields()

    def close(self):
        for _, c, _ in self.members:
            c.close()
        self.members = []

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

    def fields(self, q):
        return self.members[q][1].get_fields()

    def close(self):
        for _, c, _ in self.members:
            c.close()
        self.members = []

"""Many independent cases stepped side by side on one GPU.

Two ways:
- streams (default): each case owns a CUDA stream and a device workspace;
  one time step of a case is a captured CUDA graph (``ss_step_graph``)
  replayed on its stream, so the host issues one launch per case per step and
  the small cases' cooperative solver grids run concurrently. A case gives
  bit-identical fields alone or in such a batch.
- packed (``packed=True``, ``ss_batch_*``): one launch per stage of the step
  for all cases at once (packed row tiles for assembly and pointwise stages,
  one team of blocks per case in each cooperative solve), captured once into
  a graph. Its schedule (team sizes ~ cells^gamma, rows per tile) is chosen by
  ``autotune``. Members agree with the same case stepped alone to rounding.
"""
import time

from . import cases as cases_mod
from . import solid


class Batch:
    """A set of cases stepped together. ``case_dicts`` come from
    :mod:`paper_2303_10783_gb300.cases`; initial fields are the seeded ones."""

    def __init__(self, case_dicts, precision=solid.SS_MIXED, graphs=True, packed=False):
        import torch
        self.graphs = graphs
        self.members = []
        self.packed = None
        self.launches = 0
        for cd in case_dicts:
            stream = torch.cuda.Stream()
            with torch.cuda.stream(stream):
                c = solid.Case(cd, precision=precision, stream=stream)
                f = cases_mod.initial_fields(cd)
                c.initialize(f["T"], f["C"])
            self.members.append((cd, c, stream))
        if packed:
            self.packed = solid.PackedBatch([c for _, c, _ in self.members])

    @property
    def cells(self):
        return sum(cd["nx"] * cd["ny"] * (cd["nz"] if cd["dim"] == 3 else 1) for cd, _, _ in self.members)

    def step(self, n=1):
        """Enqueue n steps of every case and return."""
        if self.packed is not None:
            self.packed.step(n)
            return
        for _ in range(n):
            for _, c, _ in self.members:
                if self.graphs:
                    c.step_graph(1)
                else:
                    c.step(1)

    def sync(self, allow=()):
        """Wait for every case; returns the worst sticky solver status."""
        if self.packed is not None:
            st, self.launches = self.packed.sync(allow)
            return st
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

    def kernels(self):
        """Library kernels launched so far (packed) or since the members' last profile read (streams)."""
        if self.packed is not None:
            self.sync()
            return self.launches
        return sum(c.get_profile()["kernels"] for _, c, _ in self.members)

    def set_block_cap(self, max_blocks):
        for _, c, _ in self.members:
            c.set_block_cap(max_blocks)

    def _timed_trials(self, settings, apply, steps):
        """Time `steps` batch steps under each setting from the same saved
        state (every field and the case time), restoring it after each trial;
        returns (best setting, {setting: seconds per step})."""
        import torch
        self.sync()
        saved = []
        for _, c, _ in self.members:
            f = c.get_fields(device=True)
            saved.append((f, c.get_time()))

        def restore():
            self.sync()
            for (f, t), (_, c, _) in zip(saved, self.members):
                c.set_fields(f)
                c.set_time(t)
            for _, c, _ in self.members:
                c.sync()

        timing = {}
        for setting in settings:
            apply(setting)
            self.step(1)                 # captures the step graph with this setting
            self.sync()
            restore()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            self.step(steps)
            self.sync()
            torch.cuda.synchronize()
            timing[setting] = (time.perf_counter() - t0) / steps
            restore()
        best = min(timing, key=timing.get)
        apply(best)
        return best, timing

    def autotune(self, caps=(0, 64, 32, 16, 8), steps=2, gammas=(0.5, 0.75, 1.0), tiles=(1024, 4096, 16384)):
        """Choose the launch schedule that steps this batch fastest, from
        timed trials that leave the cases where they were. Streams: the solver
        block cap (``ss_set_block_cap``): a cooperative solve of a small case
        is bound by its synchronisations, not by its SMs, so fewer blocks per
        case let more cases' solves run at once, but too few starve the larger
        cases. Packed: the team sizes (blocks ~ cells^gamma) and the rows per
        tile of the packed stages. Returns (best setting, {setting: seconds
        per step})."""
        if self.packed is not None:
            settings = [(g, t) for g in gammas for t in tiles]
            return self._timed_trials(settings, lambda gt: self.packed.set_schedule(*gt), steps)
        return self._timed_trials(caps, self.set_block_cap, steps)

    def fields(self, q):
        if self.packed is not None:
            self.sync()
        return self.members[q][1].get_fields()

    def close(self):
        if self.packed is not None:
            self.packed.close()
            self.packed = None
        for _, c, _ in self.members:
            c.close()
        self.members = []

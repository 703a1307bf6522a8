"""Graph-replayed steps, batches of independent cases, and the
continuous-batching server: each must give the same fields as the plain
single-case path (bit for bit: the kernels are deterministic and cases
share no data), and the server must respect its HBM budget."""
import numpy as np
import pytest

from paper_2303_10783_gb300 import cases, solid
from paper_2303_10783_gb300.batch import Batch
from paper_2303_10783_gb300.serve import Server

pytestmark = pytest.mark.gpu


def _alone(case, nsteps, precision=solid.SS_MIXED, graph=False):
    import torch
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        c = solid.Case(case, precision=precision, stream=stream)
        f = cases.initial_fields(case)
        c.initialize(f["T"], f["C"])
        for _ in range(nsteps):
            if graph:
                c.step_graph(1)
            else:
                c.step(1)
        c.sync()
        out = c.get_fields()
        c.close()
    return out


def _same(a, b):
    return all(np.array_equal(a[k], b[k]) for k in a)


@pytest.mark.parametrize("prec", [solid.SS_FP64, solid.SS_MIXED], ids=["fp64", "mixed"])
def test_graph_step_equals_plain_step(lib, prec):
    case = cases.box_3d(24, 16, 12)
    assert _same(_alone(case, 6, prec, graph=True), _alone(case, 6, prec, graph=False))


def test_batch_member_equals_alone(lib):
    cs = [cases.cavity_2d(64, 40), cases.box_3d(32, 24, 16), cases.cavity_2d(48, 32, seed=5),
          cases.box_3d(16, 16, 16, seed=7)]
    b = Batch(cs, precision=solid.SS_MIXED)
    b.step(8)
    assert b.sync() == solid.SS_OK
    for q, cd in enumerate(cs):
        assert _same(b.fields(q), _alone(cd, 8)), q
    b.close()


def _tight_mixed(case):
    # T* to 1e-14: the transform pre-solve stops just below its tolerance (a
    # sweep gains ~3 digits), and these cavities' buoyancy-driven velocity
    # (|v| ~ 3e-4) reflects a 1e-13 T* residual at ~1e-9 of its size
    return dict(case, tol_p=1e-13, tol_t=1e-14, max_it_p=50000, max_it_t=5000, precond_p="dct")


PACKED_CASES = [_tight_mixed(cases.cavity_2d(40, 24, T0=498.2)), _tight_mixed(cases.box_3d(19, 13, 11, T0=498.2)),
                _tight_mixed(cases.box_3d(16, 12, 8, seed=3, T0=498.2)), _tight_mixed(cases.cavity_2d(50, 30, T0=498.2))]


def _packed_run(cs, nsteps, schedule=None):
    b = Batch(cs, precision=solid.SS_MIXED, packed=True)
    if schedule:
        b.packed.set_schedule(*schedule)
    b.step(nsteps)
    assert b.sync() == solid.SS_OK
    out = [b.fields(q) for q in range(len(cs))]
    teams = b.packed.teams()
    launches = b.kernels()
    b.close()
    return out, teams, launches


def test_packed_batch_matches_oracle(lib):
    """Uneven 2D and 3D cases stepped by the packed batch (one launch per stage
    for all of them, each solve by a team of blocks per case) match the oracle
    after 20 steps at the parity tolerances, starting inside the mushy range."""
    import oracle
    out, teams, launches = _packed_run(PACKED_CASES, 20)
    assert len(teams) == len(PACKED_CASES) and min(teams) >= 1
    assert launches == 20 * 10        # ten launches per batch step
    for q, case in enumerate(PACKED_CASES):
        f = cases.initial_fields(case)
        g = oracle.Grid(case)
        st = oracle.initial_state(case, f["T"], f["C"])
        for _ in range(20):
            st = oracle.step(g, st, case)
        gpu = out[q]
        for k in ("p", "T", "C", "gl", "Cl", "Cs"):
            ref = getattr(st, k)
            assert np.abs(gpu[k] - ref).max() <= 1e-9 * np.abs(ref).max(), (q, k)
        vmax = max(np.abs(x).max() for x in st.vel)
        for a, k in enumerate("uvw"[: case["dim"]]):
            assert np.abs(gpu[k] - st.vel[a]).max() <= 1e-9 * vmax, (q, k)
        assert st.gl.min() < 1.0


def test_packed_batch_is_deterministic_and_agrees_with_alone(lib):
    """Two packed runs with the same schedule agree bit for bit; another
    schedule (other team sizes and tiles) and the case stepped alone agree to
    rounding."""
    cs = [dict(c, precond_p="dct") for c in (cases.cavity_2d(64, 40), cases.box_3d(32, 24, 16),
                                              cases.box_3d(16, 16, 16, seed=7))]
    a, ta, _ = _packed_run(cs, 6)
    b, tb, _ = _packed_run(cs, 6)
    assert ta == tb
    for x, y in zip(a, b):
        assert _same(x, y)
    c2, tc, _ = _packed_run(cs, 6, schedule=(0.5, 1024))
    for q, cd in enumerate(cs):
        alone = _alone(cd, 6)
        for other in (alone, c2[q]):
            for k in ("T", "C", "gl", "p"):
                assert np.abs(a[q][k] - other[k]).max() <= 1e-9 * np.abs(other[k]).max(), (q, k)


def test_packed_autotune_restores_state_and_rejects_bad_cases(lib):
    import ctypes
    cs = [dict(cases.box_3d(20, 12, 10, seed=4), precond_p="dct"), dict(cases.cavity_2d(48, 32), precond_p="dct")]
    bt = Batch(cs, precision=solid.SS_MIXED, packed=True)
    bt.step(2)
    bt.sync()
    before = [bt.fields(q) for q in range(len(cs))]
    best, timing = bt.autotune(steps=1, gammas=(0.5, 1.0), tiles=(1024, 4096))
    assert best in timing and len(timing) == 4
    after = [bt.fields(q) for q in range(len(cs))]
    for x, y in zip(before, after):
        assert _same(x, y)
    assert lib.ss_batch_set_schedule(bt.packed.h, -1.0, 4096) == solid.SS_EINVAL
    assert lib.ss_batch_set_schedule(bt.packed.h, 1.0, 16) == solid.SS_EINVAL
    bt.close()
    # FP64 cases, multigrid pressure solves and repeated cases are refused
    for cd, prec in ((dict(cs[1], precond_p="dct"), solid.SS_FP64), (dict(cs[1], precond_p="mg"), solid.SS_MIXED)):
        c = solid.Case(cd, precision=prec)
        arr = (ctypes.c_void_p * 1)(c.h.value)
        nb = ctypes.c_size_t(0)
        assert lib.ss_batch_workspace_bytes(arr, 1, ctypes.byref(nb)) == solid.SS_EINVAL
        c.close()
    c = solid.Case(dict(cs[1], precond_p="dct"), precision=solid.SS_MIXED)
    arr = (ctypes.c_void_p * 2)(c.h.value, c.h.value)
    nb = ctypes.c_size_t(0)
    assert lib.ss_batch_workspace_bytes(arr, 2, ctypes.byref(nb)) == solid.SS_EINVAL
    c.close()


def test_batched_workload_cases_are_valid():
    cs = cases.batch_cases(64)
    assert len(cs) == 64 and {c["dim"] for c in cs} == {2, 3}
    for c in cs:
        assert 0.5 <= c["lx"] / c["ly"] <= 2.5 and 2.0 <= c["alloy"]["C0"] <= 15.0


def test_server_budget_and_isolation(lib):
    reqs = cases.serving_requests(n=6, rate=1000.0, seed=9, steps=20, grids=((16, 16, 16), (24, 16, 16)))
    one = solid.workspace_bytes(reqs[0][1], solid.SS_MIXED)
    big = max(solid.workspace_bytes(c, solid.SS_MIXED) for _, c in reqs)
    srv = Server(budget_bytes=int(2.5 * big), chunk=5, keep_results=True)
    rep = srv.run(reqs)
    # the budget binds (not all six run at once) and is never exceeded
    assert rep["requests"] == 6 and rep["max_active"] < 6 and rep["max_used_bytes"] <= rep["budget_bytes"]
    assert rep["max_active"] <= rep["budget_bytes"] // min(solid.workspace_bytes(c, solid.SS_MIXED) for _, c in reqs)
    assert rep["p50_ms_per_100_steps"] > 0 and rep["p99_ms_per_100_steps"] >= rep["p50_ms_per_100_steps"]
    # results are the same alone and in the mix
    for q in (0, 3):
        assert _same(rep["results"][q], _alone(reqs[q][1], 20)), q
    assert one > 0


def test_server_admits_and_retires_continuously(lib):
    """Continuous batching: a small request that arrives while a large one is
    running is admitted at once and finishes first; a second large request
    that does not fit the budget beside the first waits and is admitted as
    soon as memory frees; every result equals the request run alone."""
    big = dict(cases.box_3d(64, 48, 48, seed=11), steps=80)
    small = dict(cases.box_3d(16, 16, 16, seed=13), steps=10)
    big2 = dict(cases.box_3d(64, 48, 48, seed=12), steps=10)
    reqs = [(0.0, big), (0.002, small), (0.004, big2)]
    wb = solid.workspace_bytes(big, solid.SS_MIXED)
    ws = solid.workspace_bytes(small, solid.SS_MIXED)
    srv = Server(budget_bytes=wb + ws + ws // 2, chunk=5, keep_results=True)
    rep = srv.run(reqs)
    per = {p["rid"]: p for p in rep["per_request"]}
    assert per[1]["arrival"] > per[0]["arrival"] and per[1]["finished"] < per[0]["finished"]
    assert per[1]["admitted"] < per[0]["finished"]                 # admitted while the large one ran
    assert per[2]["admitted"] >= per[0]["finished"]                # waited for the large one's memory
    assert rep["max_used_bytes"] <= rep["budget_bytes"] and rep["max_active"] == 2
    for q, (_, cd) in enumerate(reqs):
        assert _same(rep["results"][q], _alone(cd, cd["steps"])), q


@pytest.mark.parametrize("prec", [solid.SS_FP64, solid.SS_MIXED], ids=["fp64", "mixed"])
@pytest.mark.parametrize("dims", [(24, 16, 12), (64, 48, 48)])
def test_steps_are_bit_reproducible(lib, prec, dims):
    """Deterministic reductions and race-free phases: two runs agree bit for bit."""
    case = cases.box_3d(*dims)
    assert _same(_alone(case, 4, prec), _alone(case, 4, prec))


def test_mixed_pressure_refinement_does_not_stall(lib):
    """Once the mixed pressure solve's FP64 residual is at rounding level, its
    mean (the Neumann null-space part, which no correction can remove) must
    not reach the FP32 inner solve: on this 96x128 batch case it once made the
    inner CG run to the iteration cap at steps 6 and 7. Every step must stay
    at a few V-cycle iterations and meet the tolerance."""
    case = dict(cases.batch_cases(n=64)[48], precond_p="mg")
    assert (case["dim"], case["nx"], case["ny"]) == (2, 96, 128)
    c = solid.Case(case, precision=solid.SS_MIXED)
    f = cases.initial_fields(case)
    c.initialize(f["T"], f["C"])
    for _ in range(8):
        c.step(1)
        assert c.sync() == solid.SS_OK
        s = c.stats()
        assert s["iters"]["p"] <= 40, s["iters"]
        assert s["relres"]["p"] <= case["tol_p"]
    c.close()


def test_block_cap_is_deterministic_and_batch_equals_alone(lib):
    """With a solver block cap the fields are again bit-reproducible, and a
    capped case gives the same fields alone and in a capped batch; the cap only
    reorders reductions, so capped and uncapped runs agree to rounding."""
    import ctypes
    case = cases.box_3d(24, 16, 12)
    def run(cap, graph):
        import torch
        stream = torch.cuda.Stream()
        with torch.cuda.stream(stream):
            c = solid.Case(case, precision=solid.SS_MIXED, stream=stream)
            c.set_block_cap(cap)
            f = cases.initial_fields(case)
            c.initialize(f["T"], f["C"])
            for _ in range(5):
                c.step_graph(1) if graph else c.step(1)
            c.sync()
            out = c.get_fields()
            c.close()
        return out
    a, b = run(4, False), run(4, True)
    assert _same(a, b)
    full = run(0, False)
    for k in ("T", "C", "gl", "p"):
        assert np.abs(a[k] - full[k]).max() <= 1e-9 * np.abs(full[k]).max(), k
    others = [cases.box_3d(16, 12, 8, seed=3), cases.cavity_2d(40, 24)]
    bt = Batch([case] + others, precision=solid.SS_MIXED)
    bt.set_block_cap(4)
    bt.step(5)
    bt.sync()
    assert _same(bt.fields(0), a)
    bt.close()
    c = solid.Case(case)
    assert lib.ss_set_block_cap(c.h, -1) == solid.SS_EINVAL
    c.close()


def test_batch_autotune_restores_state(lib):
    """The batch autotuner times each candidate cap from a saved state and
    restores it: the cases' fields after tuning equal those before."""
    cs = [cases.box_3d(20, 12, 10, seed=4), cases.cavity_2d(48, 32)]
    bt = Batch(cs, precision=solid.SS_MIXED)
    bt.step(2)
    bt.sync()
    before = [bt.fields(q) for q in range(len(cs))]
    best, timing = bt.autotune(caps=(0, 8, 2), steps=1)
    assert best in (0, 8, 2) and set(timing) == {0, 8, 2}
    after = [bt.fields(q) for q in range(len(cs))]
    for x, y in zip(before, after):
        assert _same(x, y)
    bt.close()


def test_restart_from_state_equals_new_case(lib):
    """Each mixed-precision step starts its pressure correction from the
    previous step's; ss_set_fields clears that warm start, so a case restarted
    from a saved state gives the same fields, bit for bit, as a new case set to
    that state, whatever the restarted case ran in between."""
    import torch
    case = cases.box_3d(24, 16, 12)
    f = cases.initial_fields(case)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        a = solid.Case(case, precision=solid.SS_MIXED, stream=stream)
        a.initialize(f["T"], f["C"])
        a.step(3)
        a.sync()
        state, t = a.get_fields(), a.get_time()
        a.step(2)                      # history beyond the saved state
        a.sync()
        a.set_fields(state)
        a.set_time(t)
        a.step(2)
        a.sync()
        ra = a.get_fields()
        a.close()
        b = solid.Case(case, precision=solid.SS_MIXED, stream=stream)
        b.initialize(f["T"], f["C"])
        b.set_fields(state)
        b.set_time(t)
        b.step(2)
        b.sync()
        rb = b.get_fields()
        b.close()
    assert _same(ra, rb)

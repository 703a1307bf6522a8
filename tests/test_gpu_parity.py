"""Parity of the CUDA path (through the C-ABI) with the FP64 CPU oracle.

Stage by stage (assembly planes, lever update, each solve, projection) on
seeded random states, then whole steps: 100 steps on the 2D cavity and on a
ragged 3D box must match the oracle to a relative L-infinity error of 1e-9
on every field. At the full 128x96x96 size the oracle checks what it can
afford: assembly and lever rule on every row, residuals of the GPU solves,
divergence, solute conservation and phase bounds."""
import numpy as np
import pytest

import oracle
from oracle.scheme import State
from paper_2303_10783_gb300 import cases, solid

pytestmark = pytest.mark.gpu

STEP_TOL = 1e-9          # relative L-inf bound on every field after 100 steps (FP64 path)
PLANE_TOL = 1e-12        # assembly planes, relative to the row scale


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _oracle_state(f):
    return State([f["u"], f["v"], f["w"]], f["p"], f["T"], f["C"], f["gl"], f["Cl"], f.get("Cs", 0.1 * f["Cl"]))


def _tight(case):
    case["tol_p"] = 1e-14
    case["tol_t"] = 1e-14
    case["max_it_p"] = 50000
    case["max_it_t"] = 5000
    if case.get("precond_p") == "dct":
        # the transform solver tests the true FP64 residual of its refinement,
        # whose rounding floor can sit above 1e-14 (a CG tests its recursive one)
        case["tol_p"] = 1e-13
    return case


CASES_2D = [cases.cavity_2d(61, 37, robin={"x-": (400.0, 298.0), "y+": (60.0, 300.0)})]
CASES_3D = [cases.box_3d(27, 19, 13, robin={"x-": (400.0, 298.0), "z+": (60.0, 300.0)})]
SMALL = CASES_2D + CASES_3D
# sizes whose multigrid hierarchy has several levels (the ragged ones above have one)
MULTILEVEL = [cases.cavity_2d(64, 40, robin={"x-": (400.0, 298.0), "y+": (60.0, 300.0)}),
              cases.box_3d(32, 24, 16, robin={"x-": (400.0, 298.0), "z+": (60.0, 300.0)})]
SOLVE_CASES = [(c, prec, pre) for c in SMALL + MULTILEVEL for prec in ("fp64", "mixed") for pre in ("mg", "jacobi", "dct")]
SOLVE_IDS = ["%s-%dx%dx%d-%s-%s" % ("2d" if c["dim"] == 2 else "3d", c["nx"], c["ny"], c["nz"], prec, pre)
             for c, prec, pre in SOLVE_CASES]
PREC = {"fp64": solid.SS_FP64, "mixed": solid.SS_MIXED}


def _random_case(case, seed, precision=solid.SS_FP64):
    c = solid.Case(case, precision=precision)
    f = cases.random_state(case, seed)
    c.set_fields(f)
    return c, f


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("case", SMALL, ids=["2d", "3d"])
def test_assembly_planes_match_oracle(lib, case, prec):
    """Every plane and right-hand side of every system against the oracle's
    assembly: FP64 arithmetic on the FP64 path, double-float arithmetic for the
    planes on the mixed path."""
    c, f = _random_case(case, 11, PREC[prec])
    g = oracle.Grid(case)
    st = _oracle_state(f)
    for a, name in enumerate("uvw"[: case["dim"]]):
        c.assemble(name)
        gpu = c.get_system(name)
        ref = oracle.assemble_momentum(g, st, case, a)
        scale = np.abs(ref["P"]).max()
        for k in oracle.PLANES + ("b",):
            s = scale if k != "b" else np.abs(ref["b"]).max()
            assert np.abs(gpu[k] - ref[k]).max() <= PLANE_TOL * s, (name, k)
        assert np.array_equal(gpu["x"], f[name])    # u* starts from u^n
    # pressure right-hand side from u* = u^n
    c.assemble("p")
    gp = c.get_system("p")["b"]
    ref = oracle.poisson_rhs(g, st.vel, case)
    assert _rel(gp - gp.mean(), ref) < 1e-12
    for name, ref in (("C", oracle.assemble_solute(g, st.vel, st.gl, st.C, case)),
                      ("T", oracle.assemble_temperature(g, st.vel, st.T, case))):
        c.assemble(name)
        gpu = c.get_system(name)
        scale = np.abs(ref["P"]).max()
        for k in oracle.PLANES:
            assert np.abs(gpu[k] - ref[k]).max() <= PLANE_TOL * scale, (name, k)
        assert _rel(gpu["b"], ref["b"]) < 1e-14
    c.close()


@pytest.mark.parametrize("with_eutectic", [True, False])
def test_lever_kernel_matches_oracle(lib, with_eutectic):
    case = cases.box_3d(33, 17, 9)
    if not with_eutectic:
        case["alloy"]["Ce"] = None
    al = case["alloy"]
    rng = np.random.default_rng(7)
    shape = cases.cell_shape(case)
    C = al["C0"] * rng.uniform(0.2, 8.0, shape)
    Tl = al["Tm"] + al["m"] * C
    Ts = Tl + rng.uniform(-60.0, 5.0, shape)
    gn = rng.uniform(0.0, 1.0, shape)
    gn[rng.uniform(size=shape) < 0.2] = 1.0
    gn[rng.uniform(size=shape) < 0.1] = 0.0
    c = solid.Case(case)
    c.set_fields({"T": Ts, "gl": gn, "C": C})
    c.lever()
    gpu = c.get_fields(("T", "gl", "Cl", "Cs", "C"))
    T, g, Cl, Cs = oracle.lever_update(Ts, gn, C, al)
    assert np.abs(gpu["gl"] - g).max() < 1e-12
    assert _rel(gpu["T"], T) < 1e-14
    assert _rel(gpu["Cl"], Cl) < 1e-12
    assert _rel(gpu["Cs"], Cs) < 1e-12
    assert np.array_equal(gpu["C"], C)
    c.close()


@pytest.mark.parametrize("case,prec,precond", SOLVE_CASES, ids=SOLVE_IDS)
def test_solves_match_oracle(lib, case, prec, precond):
    case = _tight(dict(case, precond_p=precond))
    c, f = _random_case(case, 12, PREC[prec])
    g = oracle.Grid(case)
    st = _oracle_state(f)
    # predictor components
    ustar = []
    for a, name in enumerate("uvw"[: case["dim"]]):
        c.assemble(name)
        c.solve(name)
        x = c.get_system(name)["x"]
        ref = oracle.solve_system(oracle.assemble_momentum(g, st, case, a))
        assert _rel(x, ref) < 1e-11, name
        ustar.append(ref)
    if case["dim"] == 2:
        ustar.append(np.zeros(g.faces(2)))
    # pressure correction and projection
    c.assemble("p")
    c.solve("p")
    pc = c.get_system("p")["x"]
    pref = oracle.solve_poisson(g, oracle.poisson_rhs(g, ustar, case))
    assert _rel(pc, pref) < 1e-10
    assert abs(pc.mean()) < 1e-12 * np.abs(pref).max()
    c.project()
    out = c.get_fields(("u", "v", "w", "p"))
    vel = oracle.project(g, ustar, pref, case)
    for a, name in enumerate("uvw"[: case["dim"]]):
        assert _rel(out[name], vel[a]) < 1e-10, name
    assert np.abs(oracle.divergence(g, [out["u"], out["v"], out["w"]])).max() < 1e-10
    # solute and temperature with the projected velocity
    st2 = _oracle_state(dict(f, u=vel[0], v=vel[1], w=vel[2]))
    c.assemble("C")
    c.solve("C")
    Cref = oracle.solve_system(oracle.assemble_solute(g, st2.vel, st2.gl, st2.C, case))
    assert _rel(c.get_fields(("C",))["C"], Cref) < 1e-12
    c.assemble("T")
    c.solve("T")
    Tref = oracle.solve_system(oracle.assemble_temperature(g, st2.vel, st2.T, case))
    assert _rel(c.get_fields(("T",))["T"], Tref) < 1e-12
    c.close()


def _run_pair(case, nsteps, T0shift=-0.8, precision=solid.SS_FP64):
    f = cases.initial_fields(case)
    T0 = f["T"] + T0shift
    c = solid.Case(case, precision=precision)
    c.initialize(T0, f["C"])
    g = oracle.Grid(case)
    st = oracle.initial_state(case, T0, f["C"])
    init = c.get_fields()
    for k in ("T", "C", "gl", "Cl", "Cs"):
        assert _rel(init[k], getattr(st, k)) < 1e-15, k
    c.step(nsteps)
    c.sync()
    stats = c.stats()
    gpu = c.get_fields()
    for _ in range(nsteps):
        st = oracle.step(g, st, case)
    c.close()
    return gpu, st, stats


STEP_CASES = [(cases.cavity_2d(), "fp64", "mg"), (cases.box_3d(19, 13, 11), "fp64", "mg"),
              (cases.box_3d(24, 16, 12), "fp64", "mg"), (cases.cavity_2d(), "mixed", "mg"),
              (cases.box_3d(24, 16, 12), "mixed", "mg"),
              (cases.cavity_2d(), "fp64", "dct"), (cases.box_3d(19, 13, 11), "fp64", "dct"),
              (cases.cavity_2d(), "mixed", "dct"), (cases.box_3d(24, 16, 12), "mixed", "dct"),
              (cases.box_3d(19, 13, 11), "mixed", "dct")]


@pytest.mark.parametrize("case,prec,precond", STEP_CASES,
                         ids=["%s-%dx%dx%d-%s-%s" % ("2d" if c["dim"] == 2 else "3d", c["nx"], c["ny"], c["nz"], p, q)
                              for c, p, q in STEP_CASES])
def test_step_parity_100_steps(lib, case, prec, precond):
    """The GPU step matches the oracle to 1e-9 relative L-inf on every field after 100 steps
    (the mixed path reaches the same bound: its outer iterations and residuals are FP64),
    with the multigrid and with the cosine-transform pressure solver."""
    case = _tight(dict(case, precond_p=precond))
    if prec == "mixed":
        # the mixed path stops on the true FP64 residual, which rounding keeps
        # above 1e-14 on some systems (the FP64 path tests its recursive one)
        case.update(tol_p=1e-13, tol_t=1e-13)
    gpu, st, stats = _run_pair(case, 100, precision=PREC[prec])
    assert stats["status"] == solid.SS_OK
    for k in ("p", "T", "C", "gl", "Cl", "Cs"):
        assert _rel(gpu[k], getattr(st, k)) < STEP_TOL, (k, _rel(gpu[k], getattr(st, k)))
    # the velocity is one vector field (Eq. 2.1): its relative error is taken
    # against the largest velocity component, so a small transverse component
    # is not judged against its own, much smaller, scale
    vmax = max(np.abs(x).max() for x in st.vel)
    for a, k in enumerate("uvw"[: case["dim"]]):
        err = np.abs(gpu[k] - st.vel[a]).max() / vmax
        assert err < STEP_TOL, (k, err)
    assert st.gl.min() < 1.0   # the mush formed: the lever rule and Darcy terms were exercised


TC_CASES = [cases.cavity_2d(40, 24), cases.box_3d(19, 13, 11), cases.box_3d(32, 24, 16, seed=3)]


@pytest.mark.parametrize("mode", ["on", "off"])
@pytest.mark.parametrize("case", TC_CASES, ids=["%s-%dx%dx%d" % ("2d" if c["dim"] == 2 else "3d", c["nx"], c["ny"],
                                                                   c["nz"]) for c in TC_CASES])
def test_transform_products_on_and_off_the_tensor_cores_match_oracle(lib, case, mode):
    """Mixed steps with the cosine transforms' products on the tensor cores
    wherever they can run (passes A, C and, in 3D, B: "on") or on the FP32
    pipes ("off") match the oracle after 20 steps at the step-parity bound,
    the pressure solve and the T* pre-solve included."""
    case = _tight(dict(case, precond_p="dct"))
    # T* to 1e-14: the transform pre-solve stops just below its tolerance (a
    # sweep gains ~3 digits), and the 2D cavity's buoyancy-driven velocity
    # reflects a 1e-13 T* residual at ~1e-9 of its size
    case.update(tol_p=1e-13, tol_t=1e-14)
    f = cases.initial_fields(case)
    T0 = f["T"] - 0.8
    c = solid.Case(case, precision=solid.SS_MIXED)
    c.set_tensor_cores(mode)
    c.initialize(T0, f["C"])
    c.get_profile()
    c.step(20)
    assert c.sync() == solid.SS_OK
    prof = c.get_profile()
    gpu = c.get_fields()
    assert lib.ss_set_tensor_cores(c.h, 3) == solid.SS_EINVAL
    c.close()
    g = oracle.Grid(case)
    st = oracle.initial_state(case, T0, f["C"])
    for _ in range(20):
        st = oracle.step(g, st, case)
    for k in ("p", "T", "C", "gl", "Cl", "Cs"):
        assert _rel(gpu[k], getattr(st, k)) < STEP_TOL, (k, _rel(gpu[k], getattr(st, k)))
    vmax = max(np.abs(x).max() for x in st.vel)
    for a, k in enumerate("uvw"[: case["dim"]]):
        assert np.abs(gpu[k] - st.vel[a]).max() / vmax < STEP_TOL, k
    assert prof["iters"]["p"] > 0          # transform sweeps of the pressure solve
    print("tensor cores %s, %s: T* pre-solve sweeps %d" % (mode, case["dim"], prof["presolve_sweeps"]))


def _example2(dim, slip):
    """Example 2's walls (Sec. 5): bottom wall temperature falling linearly in
    time, free-slip or no-slip sides, perturbed centre line; the rate is raised
    so that 100 steps cool the wall by 5 K."""
    if dim == 2:
        case = cases.freckle_2d(20, 60, slip=slip)
        case["dirichlet"] = {"y-": (case["T0"], -50.0)}
    else:
        case = cases.box_3d(19, 13, 11, robin={"x-": (400.0, 298.0)}, dirichlet={"z-": (490.0, -50.0)},
                            slip=("x-", "x+", "y-", "y+") if slip else (), perturb=1.0001)
    return case


EX2_CASES = [(_example2(2, True), "fp64"), (_example2(2, False), "mixed"), (_example2(3, True), "fp64"),
             (_example2(3, True), "mixed")]


@pytest.mark.parametrize("case,prec", EX2_CASES,
                         ids=["2d-20x60-slip-fp64", "2d-20x60-noslip-mixed", "3d-19x13x11-slip-fp64",
                              "3d-19x13x11-slip-mixed"])
def test_example2_walls_step_parity(lib, case, prec):
    """Time-dependent Dirichlet cooling and free-slip walls: 100 GPU steps
    against the oracle; the case time advances by exactly the oracle's sums
    of dt. Scalars are held to 1e-9 relative. In the first second of this
    flow the velocity (~1e-6 m/s) is the small remainder of a hydrostatic
    balance, so a solve at the stated residual tolerance fixes it only to
    ~1e-7 relative: the oracle's own direct and iterative solves differ by
    that much. The velocity bound is therefore the larger of 1e-9 relative
    and four times that spread."""
    case = _tight(dict(case))
    if prec == "mixed":
        case.update(tol_p=1e-13, tol_t=1e-13)
    f = cases.initial_fields(case)
    c = solid.Case(case, precision=PREC[prec])
    c.initialize(f["T"] - 0.8, f["C"])
    c.step(100)
    c.sync()
    gpu = c.get_fields()
    t_gpu = c.get_time()
    c.close()
    g = oracle.Grid(case)
    st = oracle.initial_state(case, f["T"] - 0.8, f["C"])
    alt = st
    for _ in range(100):
        st = oracle.step(g, st, case)
        alt = oracle.step(g, alt, case, method="iterative")
    assert t_gpu == st.t
    for k in ("p", "T", "C", "gl", "Cl", "Cs"):
        assert _rel(gpu[k], getattr(st, k)) < STEP_TOL, (k, _rel(gpu[k], getattr(st, k)))
    vmax = max(np.abs(x).max() for x in st.vel)
    for a, k in enumerate("uvw"[: case["dim"]]):
        spread = np.abs(st.vel[a] - alt.vel[a]).max()
        err = np.abs(gpu[k] - st.vel[a]).max()
        assert err <= max(STEP_TOL * vmax, 4.0 * spread), (k, err, spread, vmax)
    assert st.gl.min() < 1.0


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_minimal_model_step_parity(lib, prec):
    """The minimal model (D_l = 0, Sec. 2): 100 steps of the cavity against the oracle."""
    case = cases.cavity_2d()
    case["alloy"] = dict(case["alloy"], Dl=0.0)
    case = _tight(case)
    if prec == "mixed":
        case.update(tol_p=1e-13, tol_t=1e-13)
    gpu, st, stats = _run_pair(case, 100, precision=PREC[prec])
    assert stats["status"] == solid.SS_OK
    for k in ("p", "T", "C", "gl", "Cl", "Cs"):
        assert _rel(gpu[k], getattr(st, k)) < STEP_TOL, (k, _rel(gpu[k], getattr(st, k)))
    vmax = max(np.abs(x).max() for x in st.vel)
    for a, k in enumerate("uv"):
        assert np.abs(gpu[k] - st.vel[a]).max() / vmax < STEP_TOL, k


def test_temperature_assembly_at_a_given_time(lib):
    """ss_assemble(T) takes the wall temperature at the case's time + dt."""
    case = _example2(3, True)
    c, f = _random_case(case, 12)
    c.set_time(3.7)
    assert c.get_time() == 3.7
    c.assemble("T")
    gpu = c.get_system("T")
    ref = oracle.assemble_temperature(oracle.Grid(case), [f["u"], f["v"], f["w"]], f["T"], case, t=3.7 + case["dt"])
    scale = np.abs(ref["P"]).max()
    for k in oracle.PLANES:
        assert np.abs(gpu[k] - ref[k]).max() <= PLANE_TOL * scale, k
    assert _rel(gpu["b"], ref["b"]) < 1e-14
    c.close()


@pytest.mark.parametrize("dims", [(1, 1, 1), (2, 1, 1), (3, 2, 2), (1, 5, 3)])
def test_degenerate_grids(lib, dims):
    """Single-cell and one-cell-thick grids step without error and keep the invariants."""
    nx, ny, nz = dims
    case = _tight(cases.box_3d(nx, ny, nz))
    gpu, st, stats = _run_pair(case, 5)
    assert stats["status"] == solid.SS_OK
    for k in ("T", "C", "gl", "u", "v", "w"):
        assert np.abs(gpu[k] - getattr(st, k)).max() <= 1e-9 * max(np.abs(getattr(st, k)).max(), 1e-12), k


def test_fully_solid_and_fully_liquid(lib):
    case = _tight(cases.cavity_2d(20, 12))
    for shift in (+5.0, -60.0):
        gpu, st, stats = _run_pair(case, 10, T0shift=shift)
        assert stats["status"] == solid.SS_OK
        for k in ("T", "gl", "C", "u", "v"):
            assert np.abs(gpu[k] - getattr(st, k)).max() <= 1e-9 * max(np.abs(getattr(st, k)).max(), 1e-12), (shift, k)


@pytest.mark.parametrize("precond,tol", [("mg", 1e-14), ("dct", 1e-30)])
def test_iteration_cap_is_reported(lib, precond, tol):
    """A solve that hits its cap records SS_ENOTCONV (sticky) and keeps its iterate; nothing traps."""
    case = cases.cavity_2d(30, 20, tol_p=tol, max_it_p=2, precond_p=precond)
    f = cases.initial_fields(case)
    c = solid.Case(case)
    c.initialize(f["T"] - 0.8, f["C"])
    c.step(2)
    assert c.sync(allow=(solid.SS_ENOTCONV,)) == solid.SS_ENOTCONV
    s = c.stats()
    assert s["iters"]["p"] == 2 if precond == "mg" else 1 <= s["iters"]["p"] <= 2
    assert c.sync() == solid.SS_OK       # cleared by the read
    assert np.all(np.isfinite(c.get_fields(("u", "T"))["u"]))
    c.close()


def test_device_wait_runs_out_and_the_case_recovers(lib):
    """A device-side wait that nothing completes gives up after the case's
    poll limit: the kernel returns, the next sync reports SS_ETIMEOUT (once),
    and the case then steps normally and matches the oracle."""
    case = _tight(cases.cavity_2d(20, 12))
    f = cases.initial_fields(case)
    c = solid.Case(case)
    c.initialize(f["T"] - 0.8, f["C"])
    c.set_wait_limit(4096)
    c.wait_selftest()
    assert c.sync(allow=(solid.SS_ETIMEOUT,)) == solid.SS_ETIMEOUT
    assert b"timed out" in lib.ss_last_error()
    assert c.sync() == solid.SS_OK              # the sticky error was cleared by the read
    assert lib.ss_set_wait_limit(c.h, -1) == solid.SS_EINVAL
    assert lib.ss_set_wait_limit(c.h, 1 << 30) == solid.SS_EINVAL
    c.set_wait_limit(0)
    c.step(3)
    assert c.sync() == solid.SS_OK
    gpu = c.get_fields(("T", "gl"))
    c.close()
    g = oracle.Grid(case)
    st = oracle.initial_state(case, f["T"] - 0.8, f["C"])
    for _ in range(3):
        st = oracle.step(g, st, case)
    assert _rel(gpu["T"], st.T) < STEP_TOL and np.abs(gpu["gl"] - st.gl).max() < STEP_TOL


def test_bad_arguments(lib):
    import ctypes
    case = cases.cavity_2d(10, 8)
    c = solid.Case(case)
    assert lib.ss_step(c.h, -1) == solid.SS_EINVAL
    assert lib.ss_assemble(c.h, 2) == solid.SS_EINVAL    # no w system in 2D
    assert lib.ss_set_boundary(c.h, 7, ctypes.byref(solid.BC(1, 10.0, 300.0))) == solid.SS_EINVAL
    assert lib.ss_set_boundary(c.h, 0, ctypes.byref(solid.BC(3, 10.0, 300.0))) == solid.SS_EINVAL
    assert lib.ss_set_boundary(c.h, 0, ctypes.byref(solid.BC(1, 0.0, 300.0))) == solid.SS_EINVAL
    assert lib.ss_set_boundary(c.h, 0, ctypes.byref(solid.BC(0, 0.0, 0.0, 0.0, 2))) == solid.SS_EINVAL
    assert lib.ss_set_boundary(c.h, 0, ctypes.byref(solid.BC(2, 0.0, 300.0, float("nan")))) == solid.SS_EINVAL
    assert lib.ss_set_time(c.h, float("inf")) == solid.SS_EINVAL
    c.step(1)
    c.sync()
    al = solid.alloy_struct(case)
    assert lib.ss_set_alloy(c.h, ctypes.byref(al)) == solid.SS_ESTATE
    g = solid.grid_struct(case)
    h = ctypes.c_void_p()
    assert lib.ss_create_case(ctypes.byref(g), ctypes.c_void_p(c.workspace.data_ptr()), 1024, None,
                              ctypes.byref(h)) == solid.SS_ENOMEM
    c.close()


# ------------------------------------------------------------------ full size (the benchmark workload)

@pytest.fixture(scope="module")
def full():
    case = cases.box_3d()
    return case


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_full_size_assembly_and_lever(lib, full, prec):
    """128x96x96: every assembled row and every lever-rule cell equals the oracle's."""
    case = full
    c, f = _random_case(case, 21, PREC[prec])
    g = oracle.Grid(case)
    st = _oracle_state(f)
    for a, name in enumerate("uvw"):
        c.assemble(name)
        gpu = c.get_system(name)
        ref = oracle.assemble_momentum(g, st, case, a)
        scale = np.abs(ref["P"]).max()
        for k in oracle.PLANES:
            assert np.abs(gpu[k] - ref[k]).max() <= PLANE_TOL * scale, (name, k)
    c.assemble("T")
    gpu = c.get_system("T")
    ref = oracle.assemble_temperature(g, st.vel, st.T, case)
    assert np.abs(gpu["P"] - ref["P"]).max() <= PLANE_TOL * np.abs(ref["P"]).max()
    c.lever()
    out = c.get_fields(("T", "gl"))
    T, gl, _, _ = oracle.lever_update(f["T"], f["gl"], f["C"], case["alloy"])
    assert np.abs(out["gl"] - gl).max() < 1e-12
    assert _rel(out["T"], T) < 1e-14
    c.close()


def test_full_size_steps_keep_invariants(lib, full):
    """Three benchmark steps at 128x96x96 (bench tolerances): every solve
    converges, the true residual of the last T* solve meets its tolerance,
    the projected velocity is divergence-free, solute mass is conserved and
    0 <= g_l <= 1."""
    case = dict(full)
    f = cases.initial_fields(case)
    c = solid.Case(case)
    c.initialize(f["T"] - 0.8, f["C"])
    C0 = c.get_fields(("C",))["C"].sum()
    c.step(3)
    s = c.stats()
    assert s["status"] == solid.SS_OK, s
    out = c.get_fields()
    g = oracle.Grid(case)
    assert np.abs(oracle.divergence(g, [out["u"], out["v"], out["w"]])).max() < 1e-9
    assert abs(out["C"].sum() - C0) <= 1e-11 * C0
    assert out["gl"].min() >= 0.0 and out["gl"].max() <= 1.0 and out["gl"].min() < 1.0
    for k in ("u", "v", "w", "p", "T", "C"):
        assert np.all(np.isfinite(out[k]))
    # re-solve one T* system and check its true residual with the oracle's sparse view
    c.assemble("T")
    c.solve("T")
    sysT = c.get_system("T")
    A = oracle.sparse_from_planes(sysT)
    r = sysT["b"].ravel() - A @ sysT["x"].ravel()
    assert np.linalg.norm(r) <= 10 * case["tol_t"] * np.linalg.norm(sysT["b"])
    c.close()


FULL_STEPS = 3
FULL_BOUND = 1e-6     # relative L-inf bound on T, C and g_l of the mixed path (and checked on p and u here)


@pytest.fixture(scope="module")
def full_oracle(full):
    """FULL_STEPS oracle steps of the 128x96x96 benchmark workload, started
    inside the mushy range so that the lever rule and the Darcy terms act,
    with the oracle's iterative solves at their 1e-13 floor."""
    case = dict(full)
    f = cases.initial_fields(case)
    T0 = f["T"] - 0.8
    g = oracle.Grid(case)
    st = oracle.initial_state(case, T0, f["C"])
    for _ in range(FULL_STEPS):
        st = oracle.step(g, st, case, method="iterative")
    return case, T0, f["C"], st


@pytest.mark.parametrize("prec,precond", [("mixed", "mg"), ("fp64", "mg"), ("mixed", "dct"), ("fp64", "dct")])
def test_full_size_steps_match_oracle(lib, full_oracle, prec, precond):
    """The benchmarked path at the benchmark size and tolerances (128x96x96,
    pressure tol 1e-10, transport tol 1e-12), element by element against the
    oracle after FULL_STEPS steps. The mixed case takes the one-after-another
    momentum solves and the full pressure hierarchy that the benchmark runs;
    the FP64 case the joint momentum launch. T, C and g_l must be within the
    1e-6 bound of the mixed path; so must p and the velocity (one vector
    field, judged against its largest component)."""
    case, T0, C0, ref = full_oracle
    c = solid.Case(dict(case, precond_p=precond), precision=PREC[prec])
    c.initialize(T0, C0)
    c.step(FULL_STEPS)
    s = c.stats()
    assert s["status"] == solid.SS_OK, s
    gpu = c.get_fields()
    c.close()
    assert s["iters"]["p"] > 0
    errs = {k: _rel(gpu[k], getattr(ref, k)) for k in ("p", "T", "C", "gl", "Cl", "Cs")}
    vmax = max(np.abs(x).max() for x in ref.vel)
    errs["velocity"] = max(np.abs(gpu[k] - ref.vel[a]).max() for a, k in enumerate("uvw")) / vmax
    print("full-size %s %s vs oracle after %d steps: %s" % (prec, precond, FULL_STEPS,
                                                          ", ".join("%s %.2e" % kv for kv in errs.items())))
    for k, e in errs.items():
        assert e < FULL_BOUND, (k, e)
    assert ref.gl.min() < 1.0


@pytest.mark.parametrize("prec,precond", [("fp64", "mg"), ("mixed", "mg"), ("fp64", "dct"), ("mixed", "dct")])
def test_tiny_right_hand_side(lib, prec, precond):
    """A nearly solenoidal u* gives a pressure right-hand side near the
    rounding level; the solves must neither underflow (the mixed path scales
    its FP32 inner problem) nor lose accuracy."""
    case = _tight(dict(cases.box_3d(32, 24, 16), precond_p=precond))
    c = solid.Case(case, precision=PREC[prec])
    f = cases.random_state(case, 31, vel_scale=1e-22)
    c.set_fields(f)
    g = oracle.Grid(case)
    for name in "uvw":
        c.assemble(name)
    c.assemble("p")
    c.solve("p")
    pc = c.get_system("p")["x"]
    assert np.all(np.isfinite(pc))
    pref = oracle.solve_poisson(g, oracle.poisson_rhs(g, [f["u"], f["v"], f["w"]], case))
    assert _rel(pc, pref) < 1e-10
    c.close()


def test_fp32_planes_are_the_rounded_fp64_planes(lib):
    """The inner solves of the mixed path use the FP64 planes rounded to
    nearest (ties to even) and the FP32 reciprocal of the rounded diagonal."""
    case = cases.box_3d(27, 19, 13, robin={"x-": (400.0, 298.0), "z+": (60.0, 300.0)})
    c = solid.Case(case, precision=solid.SS_MIXED)
    c.set_fields(cases.random_state(case, 21))
    for name in ("u", "v", "w", "C", "T"):
        c.assemble(name)
        a64 = c.get_system(name)
        a32 = c.get_system_f32(name)
        for k in oracle.PLANES:
            assert np.array_equal(a32[k].view(np.uint32), a64[k].astype(np.float32).view(np.uint32)), (name, k)
        expect = (np.float32(1.0) / a32["P"]).astype(np.float32)
        assert np.array_equal(a32["idiag"].view(np.uint32), expect.view(np.uint32)), name
    c.close()


def test_fp64_to_fp32_rounding_matches_ieee(lib):
    """The integer-pipe FP64 -> FP32 rounding of the plane copies equals IEEE
    round-to-nearest-even on random values of every magnitude, on exact ties
    (both parities), at the normal/subnormal and overflow edges, and on zeros,
    infinities and NaN."""
    import torch
    rng = np.random.default_rng(5)
    vals = [rng.standard_normal(20000) * np.exp2(rng.integers(-160, 160, 20000).astype(np.float64))]
    f = rng.standard_normal(5000).astype(np.float32)
    ulp = np.spacing(np.abs(f)).astype(np.float64)
    vals += [f.astype(np.float64) + 0.5 * ulp * s for s in (1.0, -1.0)]            # exact ties
    vals += [f.astype(np.float64) + 0.5 * ulp * (1.0 + 2.0 ** -20)]               # just above a tie
    fmax = float(np.finfo(np.float32).max)
    tiny = float(np.finfo(np.float32).tiny)
    edges = [0.0, -0.0, np.inf, -np.inf, fmax, -fmax, fmax * (1 + 2.0 ** -25), fmax * (1 + 2.0 ** -23),
             tiny, -tiny, tiny * (1 - 2.0 ** -30), tiny * 0.75, 2.0 ** -149, 2.0 ** -150, 2.0 ** -151, 1e-300,
             1e300, 1.0, 1.0 + 2.0 ** -24, 1.0 + 3 * 2.0 ** -24, 3.4e38, np.nan]
    vals.append(np.array(edges))
    x = np.concatenate(vals)
    got = solid.convert_f64_to_f32(torch.from_numpy(x).cuda()).cpu().numpy()
    with np.errstate(over="ignore"):
        ref = x.astype(np.float32)
    nan = np.isnan(ref)
    assert np.array_equal(np.isnan(got), nan)
    assert np.array_equal(got[~nan].view(np.uint32), ref[~nan].view(np.uint32))


FORWARD_CASES = [
    cases.box_3d(27, 19, 13, robin={"x-": (400.0, 298.0)}, dirichlet={"z-": (490.0, -50.0)},
                 slip=("y-", "y+")),
    cases.cavity_2d(61, 37, robin={"x-": (400.0, 298.0), "y+": (60.0, 300.0)}),
    cases.box_3d(),
]


@pytest.mark.parametrize("case", FORWARD_CASES[:2], ids=["3d-27x19x13-walls", "2d-61x37"])
def test_forward_assembly_matches_oracle_forward(lib, case):
    """The GPU forward assembly (Sec. 4, Eq. 4.5-4.7) against the oracle's own
    forward assembly, written separately from the paper: every plane and
    right-hand side of every system, with no-slip, free-slip, Robin and
    time-linear Dirichlet walls."""
    from oracle import forward as oforward
    c, f = _random_case(case, 31)
    c.set_time(1.25)
    g = oracle.Grid(case)
    st = _oracle_state(f)
    refs = {name: oforward.forward_momentum(g, st, case, a) for a, name in enumerate("uvw"[: case["dim"]])}
    refs["C"] = oforward.forward_solute(g, st.vel, st.gl, st.C, case)
    refs["T"] = oforward.forward_temperature(g, st.vel, st.T, case, t=1.25 + case["dt"])
    for name, ref in refs.items():
        c.assemble_forward(name)
        fw = c.get_system(name)
        scale = np.abs(ref["P"]).max()
        for k in oracle.PLANES:
            assert np.abs(fw[k] - ref[k]).max() <= PLANE_TOL * scale, (name, k)
        bs = max(np.abs(ref["b"]).max(), 1e-300)
        assert np.abs(fw["b"] - ref["b"]).max() <= PLANE_TOL * bs, (name, "b")
    c.close()


@pytest.mark.parametrize("case", FORWARD_CASES, ids=["3d-27x19x13-walls", "2d-61x37", "3d-128x96x96"])
def test_forward_assembly_matches_termwise(lib, case):
    """Sec. 4 states that the forward (equation-based) assembly yields the
    vectorised matrix up to rounding. On the GPU, the residual-probing
    assembly and the term-wise kernels agree on every plane and right-hand
    side, including at the full 128x96x96 workload (beyond the oracle's
    reach), with no-slip, free-slip, Robin and time-linear Dirichlet walls."""
    c, f = _random_case(case, 31)
    c.set_time(1.25)
    names = ("u", "v", "w", "C", "T") if case["dim"] == 3 else ("u", "v", "C", "T")
    for name in names:
        c.assemble(name)
        tw = c.get_system(name)
        c.assemble_forward(name)
        fw = c.get_system(name)
        scale = np.abs(tw["P"]).max()
        for k in oracle.PLANES:
            assert np.abs(fw[k] - tw[k]).max() <= PLANE_TOL * scale, (name, k)
        bs = max(np.abs(tw["b"]).max(), 1e-300)
        assert np.abs(fw["b"] - tw["b"]).max() <= PLANE_TOL * bs, (name, "b")
    c.close()

"""Pins of the FP64 CPU oracle against things other than itself: the paper's
Table 1, closed-form solutions, conservation laws, the forward assembly of
Sec. 4 and brute-force dense solves. CPU only."""
import os

import numpy as np
import pytest

import oracle
from oracle import forward as fw
from oracle.scheme import State
from paper_2303_10783_gb300 import cases

import _closed_forms as cf

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _state_from_random(case, seed):
    rs = cases.random_state(case, seed)
    return State([rs["u"], rs["v"], rs["w"]], rs["p"], rs["T"], rs["C"], rs["gl"], rs["Cl"], 0.1 * rs["Cl"])


def _small(dim, **kw):
    kw.setdefault("robin", {"x-": (400.0, 298.0), "y+": (60.0, 300.0)})
    return cases.make_case(dim, 7, 5, 4, 0.010, 0.008, 0.006, 0.01, **kw)


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


# ---------------------------------------------------------------- Table 1 (Sec. 5)

def _table1():
    cols = {}
    with open(os.path.join(GOLDEN, "table1_alloys.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            k, a, b = line.split()
            cols.setdefault("PbSn", {})[k] = float(a)
            cols.setdefault("SnPb", {})[k] = float(b)
    return cols


@pytest.mark.parametrize("alloy", ["PbSn", "SnPb"])
def test_table1_initial_temperature_is_liquidus(alloy):
    """Table 1 prints T0 = T_l(C0); the oracle's liquidus (Eq. 2.20) must give it."""
    t = _table1()[alloy]
    al = dict(Tm=t["Tm_C"], m=t["m"], kp=t["kp"])
    assert abs(oracle.liquidus(t["C0"], al) - t["T0_C"]) < 0.05
    # the melt just above its liquidus is fully liquid in equilibrium (Eq. 3.15), just below it is not
    Tl = oracle.liquidus(t["C0"], al)
    assert oracle.equilibrium_fraction(np.array(Tl + 1e-6), np.array(t["C0"]), al) == 1.0
    assert oracle.equilibrium_fraction(np.array(Tl - 1e-3), np.array(t["C0"]), al) < 1.0


# ---------------------------------------------------------------- lever rule (Eq. 3.13-3.19)

def _lever_samples(al, n, seed):
    rng = np.random.default_rng(seed)
    C = al["C0"] * rng.uniform(0.5, 2.0, n)
    Tl = oracle.liquidus(C, al)
    Tstar = Tl + rng.uniform(-30.0, 3.0, n)
    gl = rng.uniform(0.0, 1.0, n)
    gl[: n // 8] = 1.0
    gl[n // 8: n // 4] = 0.0
    return Tstar, gl, C


def test_lever_root_solves_the_coupled_relations():
    """Brute force: for each cell solve Eq. 3.13 + Eq. 3.15 by bracketing the
    scalar equation in g; the quadratic root (Eq. 3.16-3.17) must agree. A
    wrong coefficient in Eq. 3.17 fails this."""
    from scipy.optimize import brentq
    al = cases.sn_pb_alloy()
    al["Ce"] = None
    Tstar, gl, C = _lever_samples(al, 400, 1)
    T, g, Cl, Cs = oracle.lever_update(Tstar, gl, C, al)
    A = al["L"] / al["cp"]
    kp, Tm = al["kp"], al["Tm"]
    checked = 0
    for i in range(len(g)):
        Tl = oracle.liquidus(C[i], al)
        T_of = lambda x: Tstar[i] - A * (x - gl[i])          # energy split step, Eq. 3.13
        lever = lambda x: 1.0 - (T_of(x) - Tl) / ((1.0 - kp) * (T_of(x) - Tm))   # Eq. 3.15
        if 0.0 < g[i] < 1.0:
            # on [x_lo, 1] the temperature stays at or below the liquidus (no pole at T_m)
            x_lo = max(0.0, gl[i] + (Tstar[i] - Tl) / A)
            ref = brentq(lambda x: x - lever(x), x_lo, 1.0, xtol=1e-15)
            assert abs(g[i] - ref) < 1e-10
            checked += 1
        elif g[i] == 1.0:
            assert T_of(1.0) >= Tl - 1e-9          # still above the liquidus: fully liquid
        else:
            assert T_of(0.0) <= Tl and lever(0.0) <= 1e-12   # lever fraction <= 0: fully solid
    assert checked > 100


def test_lever_energy_and_equilibrium_relations():
    """T + (L/c_p) g is conserved by the latent-heat step (Eq. 3.13); inside
    the mush, T is the liquidus of C_l (Eq. 2.20) and C = (g + k(1-g)) C_l
    (Eq. 2.19); C_s = k_p C_l (Eq. 3.19)."""
    al = cases.sn_pb_alloy()
    al["Ce"] = None
    Tstar, gl, C = _lever_samples(al, 2000, 2)
    T, g, Cl, Cs = oracle.lever_update(Tstar, gl, C, al)
    A = al["L"] / al["cp"]
    assert np.all((g >= 0.0) & (g <= 1.0))
    np.testing.assert_allclose(T + A * g, Tstar + A * gl, rtol=0, atol=1e-9)
    mush = (g > 1e-9) & (g < 1 - 1e-9)
    np.testing.assert_allclose(T[mush], al["Tm"] + al["m"] * Cl[mush], rtol=1e-12)
    np.testing.assert_allclose(C, (g + al["kp"] * (1 - g)) * Cl, rtol=1e-13)
    np.testing.assert_allclose(Cs, al["kp"] * Cl, rtol=1e-15)


def test_lever_special_cases():
    al = cases.sn_pb_alloy()
    C = np.full(4, al["C0"])
    Tl = oracle.liquidus(C, al)
    # superheated liquid stays liquid at T*
    T, g, _, _ = oracle.lever_update(Tl + np.array([0.1, 1.0, 5.0, 50.0]), np.ones(4), C, al)
    np.testing.assert_array_equal(g, 1.0)
    np.testing.assert_allclose(T, Tl + np.array([0.1, 1.0, 5.0, 50.0]), rtol=1e-15)
    # a fully solid cell below the eutectic temperature stays solid and cools freely
    Ts = np.array([455.0, 440.0, 400.0, 300.0])
    T, g, _, _ = oracle.lever_update(Ts, np.zeros(4), C, al)
    np.testing.assert_array_equal(g, 0.0)
    np.testing.assert_allclose(T, Ts, rtol=1e-15)
    # without a eutectic, below the lever-rule solidus T_m + m C / k_p
    al["Ce"] = None
    Tsol = al["Tm"] + al["m"] * al["C0"] / al["kp"]
    Ts = Tsol - np.array([0.5, 10.0, 50.0, 100.0])
    T, g, _, _ = oracle.lever_update(Ts, np.zeros(4), C, al)
    np.testing.assert_array_equal(g, 0.0)
    np.testing.assert_allclose(T, Ts, rtol=1e-15)
    # ... and above it a solid cell remelts partially (equilibrium lever rule)
    T, g, _, _ = oracle.lever_update(np.full(4, Tsol + 5.0), np.zeros(4), C, al)
    assert np.all(g > 0.0)


def test_eutectic_plateau_is_isothermal():
    """Below T_e = T_m + m C_e, liquid solidifies at T_e (Sec. 3 after Eq. 3.17)."""
    al = cases.sn_pb_alloy()
    Te = oracle.liquidus(al["Ce"], al)
    A = al["L"] / al["cp"]
    C = np.full(3, al["Ce"])
    gn = np.array([0.5, 0.5, 0.01])
    Tstar = np.array([Te - 1.0, Te - 10.0, Te - 10.0])
    T, g, Cl, _ = oracle.lever_update(Tstar, gn, C, al)
    np.testing.assert_allclose(T[:2], Te, rtol=1e-14)
    np.testing.assert_allclose(g[:2], gn[:2] - (Te - Tstar[:2]) / A, rtol=1e-12)
    # not enough liquid left to absorb the cooling: solid, below T_e
    assert g[2] == 0.0 and abs(T[2] - (Tstar[2] + A * gn[2])) < 1e-12 and T[2] < Te
    assert np.all(Cl <= al["Ce"])


# ---------------------------------------------------------------- assembly (Sec. 4)

@pytest.mark.parametrize("dim", [2, 3])
def test_vectorised_equals_forward_assembly(dim):
    """Sec. 4: the forward (residual-probing) assembly gives the vectorised
    matrix up to rounding. Checked for u, v, (w), C, T and the Poisson operator."""
    case = _small(dim)
    g = oracle.Grid(case)
    st = _state_from_random(case, 3)
    pairs = [(oracle.assemble_momentum(g, st, case, a), fw.forward_momentum(g, st, case, a)) for a in range(dim)]
    pairs.append((oracle.assemble_solute(g, st.vel, st.gl, st.C, case), fw.forward_solute(g, st.vel, st.gl, st.C, case)))
    pairs.append((oracle.assemble_temperature(g, st.vel, st.T, case), fw.forward_temperature(g, st.vel, st.T, case)))
    pairs.append((oracle.poisson_matrix(g), fw.forward_poisson(g)))
    for vec, fwd in pairs:
        for k in vec:
            scale = max(np.abs(vec[k]).max(), np.abs(vec["P"]).max())
            assert np.abs(vec[k] - fwd[k]).max() <= 1e-11 * scale, k


@pytest.mark.parametrize("dim", [2, 3])
def test_forward_equals_vectorised_with_slip_and_dirichlet_walls(dim):
    """The same Sec. 4 cross-check with Example 2's walls: free-slip sides and a
    bottom wall held at a time-dependent temperature."""
    vert = "y-" if dim == 2 else "z-"
    case = _small(dim, robin={"x-": (400.0, 298.0)}, dirichlet={vert: (480.0, -0.05)},
                  slip=("x-", "x+", "y+") if dim == 3 else ("x-", "x+"))
    g = oracle.Grid(case)
    st = _state_from_random(case, 6)
    pairs = [(oracle.assemble_momentum(g, st, case, a), fw.forward_momentum(g, st, case, a)) for a in range(dim)]
    pairs.append((oracle.assemble_temperature(g, st.vel, st.T, case, t=2.5),
                  fw.forward_temperature(g, st.vel, st.T, case, t=2.5)))
    for vec, fwd in pairs:
        for k in vec:
            scale = max(np.abs(vec[k]).max(), np.abs(vec["P"]).max())
            assert np.abs(vec[k] - fwd[k]).max() <= 1e-11 * scale, k


@pytest.mark.parametrize("dim", [2, 3])
def test_dia_pattern(dim):
    """Every system has only the 5 (2D) / 7 (3D) diagonals of Eq. 4.1 and no coupling wraps a row."""
    case = _small(dim)
    g = oracle.Grid(case)
    st = _state_from_random(case, 4)
    systems = [oracle.assemble_momentum(g, st, case, a) for a in range(dim)]
    systems += [oracle.assemble_solute(g, st.vel, st.gl, st.C, case), oracle.assemble_temperature(g, st.vel, st.T, case)]
    for s in systems:
        oracle.sparse_from_planes(s)   # raises on wrap-around couplings
        if dim == 2:
            assert not s["B"].any() and not s["T"].any()


def test_stencil_exactness():
    """Central diffusion is exact on quadratics and upwind convection on linear
    fields in the interior (Eq. 3.27-3.29)."""
    case = cases.make_case(2, 9, 7, 1, 0.009, 0.007, 1.0, 1.0)
    g = oracle.Grid(case)
    yc, xc = np.meshgrid((np.arange(7) + 0.5) * g.h[1], (np.arange(9) + 0.5) * g.h[0], indexing="ij")
    phi = (3.0 * xc ** 2 - 2.0 * yc ** 2 + xc * yc)[None]
    zero = [np.zeros(g.faces(a)) for a in range(3)]
    D = [np.where((oracle.scheme._index(g.faces(a), a) >= 1) & (oracle.scheme._index(g.faces(a), a) <= g.n[a] - 1), 1.0, 0.0) for a in range(2)]
    P, nb = oracle.assemble_scalar(g, zero, D)
    A = dict(nb, P=P)
    Aphi = (oracle.sparse_from_planes(A) @ phi.ravel()).reshape(phi.shape)
    lap = 6.0 - 4.0   # analytic Laplacian of phi
    np.testing.assert_allclose(-Aphi[0, 1:-1, 1:-1], lap, rtol=1e-9)
    # constant velocity field (ux, vy) on every face; walls 0
    ux, vy = 0.3, -0.2
    vel = [np.full(g.faces(0), ux), np.full(g.faces(1), vy), np.zeros(g.faces(2))]
    vel[0][:, :, 0] = vel[0][:, :, -1] = 0.0
    vel[1][:, 0, :] = vel[1][:, -1, :] = 0.0
    lin = (2.0 * xc - 5.0 * yc)[None]
    zeroD = [np.zeros(g.faces(a)) for a in range(2)]
    P, nb = oracle.assemble_scalar(g, vel, zeroD)
    Alin = (oracle.sparse_from_planes(dict(nb, P=P)) @ lin.ravel()).reshape(lin.shape)
    np.testing.assert_allclose(Alin[0, 1:-1, 1:-1], ux * 2.0 + vy * (-5.0), rtol=1e-9)


# ---------------------------------------------------------------- linear solves

def _dense(eq, shape):
    n = int(np.prod(shape))
    base = eq(np.zeros(shape)).ravel()
    A = np.empty((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        A[:, j] = eq(e.reshape(shape)).ravel() - base
    return A, -base


@pytest.mark.parametrize("dim", [2, 3])
def test_step_matches_brute_force_dense_solves(dim):
    """Build each system of a step densely by applying the forward equation
    to unit vectors, solve it with dense LU and compare with the oracle step."""
    case = cases.make_case(dim, 5, 4, 3, 0.005, 0.004, 0.003, 0.01, robin={"x-": (400.0, 298.0)})
    g = oracle.Grid(case)
    st = _state_from_random(case, 5)
    info = {}
    new = oracle.step(g, st, case, info=info)
    for a in range(dim):
        A, b = _dense(lambda phi: fw.momentum_eq(g, st, case, a, phi), g.faces(a))
        assert _rel(np.linalg.solve(A, b).reshape(g.faces(a)), info["ustar"][a]) < 1e-12
    A, _ = _dense(lambda p: fw.poisson_eq(g, p), g.cells)
    bp = oracle.poisson_rhs(g, info["ustar"], case).ravel()
    sol = np.linalg.lstsq(A, bp, rcond=None)[0]
    assert _rel(sol - sol.mean(), info["pc"].ravel()) < 1e-10
    A, b = _dense(lambda c: fw.solute_eq(g, new.vel, st.gl, st.C, case, c), g.cells)
    assert _rel(np.linalg.solve(A, b).reshape(g.cells), new.C) < 1e-12
    A, b = _dense(lambda t: fw.temperature_eq(g, new.vel, st.T, case, t), g.cells)
    assert _rel(np.linalg.solve(A, b).reshape(g.cells), info["Tstar"]) < 1e-12


def test_iterative_path_agrees_with_direct():
    case = cases.make_case(3, 9, 7, 6, 0.009, 0.007, 0.006, 0.01)
    f = cases.initial_fields(case)
    g = oracle.Grid(case)
    st0 = oracle.initial_state(case, f["T"] - 1.0, f["C"])
    a = st0
    b = st0
    for _ in range(3):
        a = oracle.step(g, a, case, method="direct")
        b = oracle.step(g, b, case, method="iterative")
    for k in ("u", "v", "w", "T", "C", "gl"):
        assert _rel(getattr(b, k), getattr(a, k)) < 1e-9, k


# ---------------------------------------------------------------- invariants of the step

def _cavity(nx=20, ny=12, **kw):
    return cases.cavity_2d(nx, ny, **kw)


@pytest.fixture(scope="module")
def cavity_run():
    case = _cavity(T0=499.0)
    f = cases.initial_fields(case)
    g = oracle.Grid(case)
    st = oracle.initial_state(case, f["T"] - 0.8, f["C"])   # start slightly inside the mush
    hist = [st]
    infos = []
    for _ in range(30):
        info = {}
        st = oracle.step(g, st, case, info=info)
        hist.append(st)
        infos.append(info)
    return case, g, hist, infos


def test_solute_mass_conserved(cavity_run):
    """Zero-flux walls and the conservative column-scaled operator (Eq. 3.10):
    sum C is constant to round-off (row scaling would break this)."""
    case, g, hist, _ = cavity_run
    s0 = hist[0].C.sum()
    for st in hist[1:]:
        assert abs(st.C.sum() - s0) <= 1e-12 * s0


def test_minimal_model_without_flow_keeps_solute(cavity_run):
    """Minimal model (Sec. 2: no solute diffusion in the liquid, D_l = 0): with
    the melt at rest the solute system reduces to I/dt and C^{n+1} = C^n
    exactly, whatever g_l; with D_l > 0 the same state does redistribute
    solute (so the check discriminates)."""
    case = _small(3)
    st = _state_from_random(case, 8)
    g = oracle.Grid(case)
    rest = [np.zeros_like(v) for v in st.vel]
    for Dl, moves in ((0.0, False), (case["alloy"]["Dl"], True)):
        c2 = dict(case, alloy=dict(case["alloy"], Dl=Dl))
        C = oracle.solve_system(oracle.assemble_solute(g, rest, st.gl, st.C, c2))
        if moves:
            assert np.abs(C - st.C).max() > 1e-9 * np.abs(st.C).max()
        else:
            assert np.abs(C - st.C).max() <= 1e-13 * np.abs(st.C).max()


def test_energy_balance(cavity_run):
    """Sum of T + (L/c_p) g changes only by the Robin wall flux (Eq. 3.12 + 3.13)."""
    case, g, hist, infos = cavity_run
    al = case["alloy"]
    A = al["L"] / al["cp"]
    hc, Text = case["robin"]["x-"]
    U = 1.0 / (1.0 / hc + g.h[0] / (2.0 * al["k"]))
    coef = U / (al["rho"] * al["cp"] * g.h[0])
    for n in range(len(infos)):
        e0 = (hist[n].T + A * hist[n].gl).sum()
        e1 = (hist[n + 1].T + A * hist[n + 1].gl).sum()
        loss = case["dt"] * coef * (infos[n]["Tstar"][0, :, 0] - Text).sum()
        assert abs((e1 - e0) + loss) <= 1e-12 * abs(e0)


def test_projection_divergence_free(cavity_run):
    case, g, hist, _ = cavity_run
    for st in hist[1:]:
        assert np.abs(oracle.divergence(g, st.vel)).max() < 1e-10


def test_phase_bounds(cavity_run):
    _, _, hist, _ = cavity_run
    for st in hist:
        assert st.gl.min() >= 0.0 and st.gl.max() <= 1.0
    assert hist[-1].gl.min() < 1.0   # the mush actually formed


def test_cooled_wall_downflow(cavity_run):
    """Thermal buoyancy drives fluid down along the cooled (left) wall (Sec. 5, Example 1)."""
    case, g, hist, _ = cavity_run
    v = hist[-1].v[0]
    assert v[1:-1, 0].mean() < 0.0 and v[1:-1, 0].min() < -1e-5


def test_hydrostatic_rest():
    """Uniform T and C, no cooling: the buoyancy vanishes (up to the rounding
    of k_p + (1 - k_p) in C_l) and the melt stays at rest."""
    case = _cavity(robin={}, noise=0.0)
    g = oracle.Grid(case)
    st = oracle.initial_state(case, np.full(g.cells, case["T0"]), np.full(g.cells, case["alloy"]["C0"]))
    for _ in range(5):
        st = oracle.step(g, st, case)
    for k in ("u", "v"):
        assert np.abs(getattr(st, k)).max() < 1e-15
    assert np.all(np.abs(st.T - case["T0"]) < 1e-10)


def test_free_slip_mirror_symmetry():
    """Free-slip side walls keep the x-mirror symmetry of the cavity."""
    base = dict(nx=12, ny=8)
    A = cases.cavity_2d(robin={"x-": (400.0, 298.0)}, slip=("x-", "x+", "y-", "y+"), **base)
    B = cases.cavity_2d(robin={"x+": (400.0, 298.0)}, slip=("x-", "x+", "y-", "y+"), **base)
    f = cases.initial_fields(A)
    g = oracle.Grid(A)
    sa = oracle.initial_state(A, f["T"] - 0.5, f["C"])
    sb = oracle.initial_state(B, f["T"][:, :, ::-1] - 0.5, f["C"])
    for _ in range(10):
        sa = oracle.step(g, sa, A)
        sb = oracle.step(g, sb, B)
    flip = lambda x: x[:, :, ::-1]
    vscale = max(np.abs(x).max() for x in sa.vel)
    assert np.abs(flip(sb.v) - sa.v).max() < 1e-11 * vscale and np.abs(-flip(sb.u) - sa.u).max() < 1e-11 * vscale
    assert _rel(flip(sb.T), sa.T) < 1e-12


@pytest.mark.parametrize("dim", [2, 3])
def test_mirror_symmetry(dim):
    """Cooling the right wall instead of the left, with the initial noise
    mirrored in x, mirrors every field (u changes sign)."""
    if dim == 2:
        kw = dict(nx=12, ny=8)
        mk = lambda robin: cases.cavity_2d(robin=robin, **kw)
    else:
        mk = lambda robin: cases.box_3d(8, 6, 5, robin=robin)
    A = mk({"x-": (400.0, 298.0)})
    B = mk({"x+": (400.0, 298.0)})
    f = cases.initial_fields(A)
    ga = oracle.Grid(A)
    sa = oracle.initial_state(A, f["T"] - 0.5, f["C"])
    sb = oracle.initial_state(B, f["T"][:, :, ::-1] - 0.5, f["C"])
    for _ in range(15):
        sa = oracle.step(ga, sa, A)
        sb = oracle.step(ga, sb, B)
    flip = lambda x: x[:, :, ::-1]
    for k in ("T", "C", "gl", "p"):
        assert _rel(flip(getattr(sb, k)), getattr(sa, k)) < 1e-11, k
    vscale = max(np.abs(x).max() for x in sa.vel)   # velocities relative to the flow speed
    for x, y in ((sb.v, sa.v), (sb.w, sa.w), (-sb.u, sa.u)):
        assert np.abs(flip(x) - y).max() < 1e-11 * vscale
    assert np.abs(sa.u).max() > 1e-6


# ---------------------------------------------------------------- closed forms

def _slab(nx, dt, **alloy_kw):
    al = cases.sn_pb_alloy()
    al.update(betaT=0.0, betaC=0.0, Dl=0.0)
    al.update(alloy_kw)
    return cases.make_case(2, nx, 1, 1, 0.1, 0.002, 1.0, dt, alloy=al, noise=0.0)


def _robin_error(nx, dt, t_end=2.0, hc=5000.0):
    case = _slab(nx, dt)
    case["robin"] = {"x-": (hc, 550.0)}
    case["T0"] = 600.0
    st = oracle.run(case, int(round(t_end / dt)))
    g = oracle.Grid(case)
    al = case["alloy"]
    alpha = al["k"] / (al["rho"] * al["cp"])
    x = (np.arange(nx) + 0.5) * g.h[0]
    exact = cf.robin_semi_infinite(x, t_end, alpha, hc / al["k"], 600.0, 550.0)
    assert np.all(st.gl == 1.0) and np.abs(st.u).max() == 0.0
    return np.abs(st.T[0, 0] - exact).max() / 50.0


def test_robin_conduction_closed_form():
    """Pure conduction with a convective wall against Carslaw & Jaeger's
    semi-infinite solution: small error, first-order convergence in (h, dt)."""
    e1 = _robin_error(100, 0.02)
    e2 = _robin_error(200, 0.01)
    assert e2 < 5e-3
    order = np.log2(e1 / e2)
    assert 0.7 < order < 1.6, order


def _linear_wall_error(nx, dt, t_end=2.0, rate=-20.0):
    case = _slab(nx, dt)
    case["robin"] = {}
    case["dirichlet"] = {"x-": (600.0, rate)}
    case["T0"] = 600.0
    st = oracle.run(case, int(round(t_end / dt)))
    g = oracle.Grid(case)
    al = case["alloy"]
    alpha = al["k"] / (al["rho"] * al["cp"])
    x = (np.arange(nx) + 0.5) * g.h[0]
    exact = cf.linear_wall_semi_infinite(x, t_end, alpha, 600.0, rate)
    assert np.all(st.gl == 1.0)
    return np.abs(st.T[0, 0] - exact).max() / (abs(rate) * t_end)


def test_linearly_cooled_wall_closed_form():
    """Example 2's wall temperature falling linearly in time against Carslaw &
    Jaeger's semi-infinite solution; first-order convergence in (h, dt)."""
    e1 = _linear_wall_error(100, 0.02)
    e2 = _linear_wall_error(200, 0.01)
    assert e2 < 2e-2
    assert 0.6 < np.log2(e1 / e2) < 1.8, (e1, e2)


def _stefan_front(nx, dt, t_end):
    al = cases.sn_pb_alloy()
    case = _slab(nx, dt, C0=al["Ce"])
    Te = al["Tm"] + al["m"] * al["Ce"]
    case["T0"] = Te + 10.0
    case["robin"] = {"x-": (1e8, Te - 100.0)}
    st = oracle.run(case, int(round(t_end / dt)))
    g = oracle.Grid(case)
    solid = ((1.0 - st.gl[0, 0]) * g.h[0]).sum()
    alpha = al["k"] / (al["rho"] * al["cp"])
    St = al["cp"] * 100.0 / al["L"]
    return solid, cf.neumann_front(t_end, alpha, St, 10.0 / 100.0)


def test_stefan_neumann_closed_form():
    """Isothermal (eutectic-composition) solidification from a chilled wall:
    the solidified thickness follows the two-phase Neumann solution
    X = 2 lambda sqrt(alpha t), converging as the grid and step refine."""
    s1, x1 = _stefan_front(100, 0.02, 4.0)
    s2, x2 = _stefan_front(200, 0.01, 4.0)
    assert abs(s2 - x2) / x2 < 0.03
    assert abs(s2 - x2) < abs(s1 - x1)


def _mms_error(n, nsteps, t_end=0.5):
    """Manufactured solution of the temperature transport equation with a
    source (the S_Phi of Eq. 3.26) and a discretely divergence-free flow."""
    lx = ly = 0.01
    case = cases.make_case(2, n, n, 1, lx, ly, 1.0, t_end / nsteps, robin={})
    g = oracle.Grid(case)
    alpha = case["alloy"]["k"] / (case["alloy"]["rho"] * case["alloy"]["cp"])
    U0 = 0.01 * lx / np.pi
    kx, ky = np.pi / lx, np.pi / ly
    psi = lambda x, y: U0 * np.sin(kx * x) * np.sin(ky * y)
    xf = np.arange(n + 1) * g.h[0]
    yf = np.arange(n + 1) * g.h[1]
    xc = (np.arange(n) + 0.5) * g.h[0]
    yc = (np.arange(n) + 0.5) * g.h[1]
    u = ((psi(xf[None, :], yf[1:, None]) - psi(xf[None, :], yf[:-1, None])) / g.h[1])[None]
    v = (-(psi(xf[None, 1:], yf[:, None]) - psi(xf[None, :-1], yf[:, None])) / g.h[0])[None]
    vel = [u, v, np.zeros(g.faces(2))]
    assert np.abs(oracle.divergence(g, vel)).max() < 1e-12
    Y, X = np.meshgrid(yc, xc, indexing="ij")
    exact = lambda t: (1.0 + np.exp(-t) * np.cos(kx * X) * np.cos(ky * Y))[None]
    ux = U0 * ky * np.sin(kx * X) * np.cos(ky * Y)
    vy = -U0 * kx * np.cos(kx * X) * np.sin(ky * Y)

    def source(t):
        e = np.exp(-t)
        phit = -e * np.cos(kx * X) * np.cos(ky * Y)
        phix = -e * kx * np.sin(kx * X) * np.cos(ky * Y)
        phiy = -e * ky * np.cos(kx * X) * np.sin(ky * Y)
        lap = -e * (kx * kx + ky * ky) * np.cos(kx * X) * np.cos(ky * Y)
        return (phit + ux * phix + vy * phiy - alpha * lap)[None]

    T = exact(0.0)
    dt = case["dt"]
    for s in range(nsteps):
        sysT = oracle.assemble_temperature(g, vel, T, case, source=source((s + 1) * dt))
        T = oracle.solve_system(sysT)
    return np.abs(T - exact(t_end)).max()


def test_manufactured_advection_diffusion_first_order():
    e1 = _mms_error(16, 10)
    e2 = _mms_error(32, 20)
    e3 = _mms_error(64, 40)
    assert e3 < e2 < e1
    assert np.log2(e2 / e3) > 0.7


# ---------------------------------------------------------------- Darcy drag (Eq. 2.8 in Eq. 3.3)

@pytest.mark.parametrize("g", [0.5, 0.8, 0.95])
def test_darcy_damping_of_uniform_flow_closed_form(g):
    """A uniform x-velocity U in a uniform mushy zone (g_l = g), with no
    pressure gradient and the gravity along z, keeps convection and diffusion
    in balance away from the walls, so the implicit drag alone acts:
    u* (1/dt + nu K^-1) = U / dt, i.e. u* = U / (1 + dt nu K^-1) with
    K^-1 = (1 - g)^2 / (K0 (g^3 + eps)). The wall rows' influence decays by
    ~dt nu / h^2 (~1e-4 here) per cell, so faces four cells in meet the closed
    form to rounding. A dropped or sign-flipped drag, or a drag on the wrong
    face average, fails by orders of magnitude (dt nu K^-1 = 7.9, 0.31, 0.012).
    Along x the x-walls' disturbance is carried by the upwind convection and
    decays only by ~U dt / h (~0.02) per cell, so the check keeps to the middle
    of the x range, more than eight cells from either x-wall."""
    case = cases.box_3d(24, 16, 16)
    al = case["alloy"]
    grid = oracle.Grid(case)
    assert grid.vert == 2
    U = 0.01
    u = np.zeros(grid.faces(0))                   # (z, y, x) order
    u[..., 1:-1] = U                              # interior x-faces; the walls hold 0
    st = State([u, np.zeros(grid.faces(1)), np.zeros(grid.faces(2))], np.zeros(grid.cells),
               np.full(grid.cells, case["T0"]), np.full(grid.cells, al["C0"]), np.full(grid.cells, g),
               np.full(grid.cells, al["C0"]), np.full(grid.cells, al["kp"] * al["C0"]))
    sysm = oracle.assemble_momentum(grid, st, case, 0)
    ustar = oracle.solve_system(sysm, x0=st.vel[0], method="direct", rtol=1e-14).reshape(grid.faces(0))
    nu = al["mu"] / al["rho"]
    kinv = (1.0 - g) ** 2 / (al["K0"] * (g ** 3 + al["darcy_eps"]))
    expect = U / (1.0 + case["dt"] * nu * kinv)
    core = ustar[4:-4, 4:-4, 10:16]
    assert np.abs(core - expect).max() <= 1e-13 * expect, (np.abs(core - expect).max(), expect)
    # and the drag matters: the undamped value is far off
    assert abs(U - expect) > 1e-2 * U


# ---------------------------------------------------------------- Boussinesq force (Eq. 2.9 in Eq. 3.3)

@pytest.mark.parametrize("dT,dC,g", [(2.0, 0.0, 1.0), (0.0, 0.5, 1.0), (1.5, -0.3, 0.8)])
def test_buoyancy_of_a_resting_melt_closed_form(dT, dC, g):
    """A resting melt (u = 0, p = 0) with uniform T = T_ref + dT and
    C_l = C_ref + dC feels f = g (1 - beta_T dT - beta_c dC) with g pointing
    down; the constant part is hydrostatic, so the intermediate vertical
    velocity away from the walls is w* = dt |g| (beta_T dT + beta_c dC) /
    (1 + dt nu K^-1): a warmer melt (beta_T > 0) rises and a melt richer in
    the heavier component (beta_c < 0 here) sinks; the horizontal components
    stay at rest. The wall rows' influence decays by ~dt nu / h^2 per cell."""
    case = cases.box_3d(24, 16, 16)
    al = case["alloy"]
    grid = oracle.Grid(case)
    assert grid.vert == 2 and al["betaT"] > 0 and al["betaC"] < 0 and al["gravity"] > 0
    zero = [np.zeros(grid.faces(a)) for a in range(3)]
    Cl = al["C0"] + dC
    st = State(zero, np.zeros(grid.cells), np.full(grid.cells, case["T0"] + dT), np.full(grid.cells, al["C0"]),
               np.full(grid.cells, g), np.full(grid.cells, Cl), np.full(grid.cells, al["kp"] * Cl))
    out = []
    for a in range(3):
        sysm = oracle.assemble_momentum(grid, st, case, a)
        out.append(oracle.solve_system(sysm, x0=st.vel[a], method="direct", rtol=1e-14).reshape(grid.faces(a)))
    nu = al["mu"] / al["rho"]
    kinv = (1.0 - g) ** 2 / (al["K0"] * (g ** 3 + al["darcy_eps"]))
    expect = case["dt"] * al["gravity"] * (al["betaT"] * dT + al["betaC"] * dC) / (1.0 + case["dt"] * nu * kinv)
    core = out[2][4:-4, 4:-4, 4:-4]
    assert np.abs(core - expect).max() <= 1e-12 * abs(expect), (np.abs(core - expect).max(), expect)
    if dC == 0.0:
        assert expect > 0                         # warmer than the reference: rises
    if dT == 0.0:
        assert expect < 0                         # richer in the heavier component: sinks
    assert np.abs(out[0]).max() == 0.0 and np.abs(out[1]).max() == 0.0


# ---------------------------------------------------------------- pressure gradient (Eq. 3.3, explicit -grad p^n / rho)

@pytest.mark.parametrize("axis", [0, 1])
def test_linear_pressure_accelerates_a_resting_liquid(axis):
    """A resting liquid (g_l = 1, so no drag; T and C_l at their reference
    values, so no buoyancy) under the linear pressure p^n = G x_axis takes
    u*_axis = -dt G / rho away from the walls: the face difference of p
    across one cell is G h exactly, and the other components stay at rest.
    A wrong sign, a missing 1/rho or 1/h, or a gradient on the wrong axis
    fails it."""
    case = cases.box_3d(24, 16, 16)
    al = case["alloy"]
    grid = oracle.Grid(case)
    G = 250.0                                     # Pa/m
    # cell centres along the axis; cells are (z, y, x) ordered
    n = grid.n[axis]
    xc = (np.arange(n) + 0.5) * grid.h[axis]
    shape = [1, 1, 1]
    shape[2 - axis] = n
    p = np.broadcast_to(G * xc.reshape(shape), grid.cells).copy()
    zero = [np.zeros(grid.faces(a)) for a in range(3)]
    st = State(zero, p, np.full(grid.cells, case["T0"]), np.full(grid.cells, al["C0"]),
               np.full(grid.cells, 1.0), np.full(grid.cells, al["C0"]), np.full(grid.cells, al["kp"] * al["C0"]))
    out = []
    for a in range(3):
        sysm = oracle.assemble_momentum(grid, st, case, a)
        out.append(oracle.solve_system(sysm, x0=st.vel[a], method="direct", rtol=1e-14).reshape(grid.faces(a)))
    expect = -case["dt"] * G / al["rho"]
    core = out[axis][4:-4, 4:-4, 4:-4]
    assert np.abs(core - expect).max() <= 1e-12 * abs(expect), (np.abs(core - expect).max(), expect)
    for a in range(3):
        if a != axis:
            assert np.abs(out[a]).max() == 0.0

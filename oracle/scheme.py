"""Vectorised FP64 statement of one time step of the scheme (Algorithm 1, Sec. 4).

TEST INFRASTRUCTURE ONLY (see the package docstring): never imported by the
product path.

Conventions (Sec. 3, "Spatial discretization", Eq. 3.20-3.25)
---------------------------------------------------------------
* Paper axes a = 0, 1, 2 are x, y, z. numpy arrays are shaped (nz, ny, nx)
  so x is fastest, matching the lexicographic unknown ordering of Eq. 4.2;
  paper axis a is numpy axis 2 - a.
* Cell-centred fields (the set E^c): p, T, C, g_l, C_l, C_s.
* Face velocities on the staggered sets: u on x-faces (E^we), shape
  (nz, ny, nx+1); v on y-faces (E^sn), shape (nz, ny+1, nx); w on z-faces,
  shape (nz+1, ny, nx). Faces 0 and n_a along their own axis are walls.
* 2D runs have nz = 1, no z terms at all and a w array of zeros.
* The vertical axis is y in 2D and z in 3D.

Linear systems are stored as seven DIA planes on the grid of their unknowns
(Eq. 4.1): 'P' (the main diagonal A_0), 'W'/'E' (offsets -1/+1 along x),
'S'/'N' (along y), 'B'/'T' (along z), plus the right-hand side 'b'. Row r of
the matrix reads  P[r] x[r] + W[r] x[r-1] + E[r] x[r+1] + S[r] x[r-m_x] + ...
A plane holds 0 wherever the neighbour is not an unknown of the system.

Readings of points the paper leaves open:
* flux-form upwind convection everywhere (Eq. 3.28-3.29), with the advecting
  velocity u^n in the momentum step and u^{n+1} in the C and T steps;
* advecting velocities on staggered control-volume faces are arithmetic
  means of the two nearest face velocities; cell quantities on faces
  (g_l, K^{-1}, T, C_l) are arithmetic means of the two adjacent cells;
* no-slip walls: the wall-normal velocity is 0 (wall faces are identity rows
  with zero right-hand side, and their coupling to interior rows is dropped
  because their value is the boundary datum 0); tangential components use a
  ghost value equal to minus the interior value, i.e. 2*nu/h^2 on the diagonal;
* the solute operator is column-scaled: (I/dt + (A_con - A_lap) A_g) C = C^n/dt
  (Eq. 3.10 with C_l = A_g C substituted into the convection and diffusion of
  C_l; Eq. 3.10 prints the product in the other order);
* the Boussinesq force keeps only its variable part,
  f_vert = g (beta_T (T - T_ref) + beta_C (C_l - C_ref)) (Eq. 2.9 without the
  constant hydrostatic term, which the pressure absorbs);
* the permeability is K = K0 g^3/(1-g)^2 (Eq. 2.8 with K0 in place of
  lambda_2^2/180) and K^{-1} = (1-g)^2 / (K0 (g^3 + eps));
* cooled walls: heat flux U (T_P - T_ext) with U = 1/(1/h + dx/(2k)) for a
  Robin wall and U = 2k/dx with T_ext = T_w(t^{n+1}) for a Dirichlet wall;
* free-slip walls (Example 2) use the ghost +u_P: no shear on the wall;
* the larger root of Eq. 3.16, clamped to [0, 1]; the eutectic plateau holds
  T = T_e while liquid remains (Sec. 3 after Eq. 3.17, Table 1);
* pressure-correction gauge: the right-hand side of Eq. 3.4 has its mean
  removed and the correction is returned with zero mean.
"""
import numpy as np

PLANES = ("P", "W", "E", "S", "N", "B", "T")
# (axis, side) -> plane name; side 0 = back (west/south/bottom), 1 = front
_NB = {(0, 0): "W", (0, 1): "E", (1, 0): "S", (1, 1): "N", (2, 0): "B", (2, 1): "T"}


# ----------------------------------------------------------------- helpers

def _sl(arr, a, start, stop):
    """Slice ``arr`` along paper axis ``a``."""
    idx = [slice(None)] * 3
    idx[2 - a] = slice(start, stop)
    return arr[tuple(idx)]


def _pad(arr, a):
    """Zero-pad ``arr`` by one entry on both ends of paper axis ``a``."""
    w = [(0, 0)] * 3
    w[2 - a] = (1, 1)
    return np.pad(arr, w)


def _index(shape, a):
    """Integer index along paper axis ``a`` broadcast to ``shape``."""
    s = [1, 1, 1]
    s[2 - a] = shape[2 - a]
    return np.broadcast_to(np.arange(shape[2 - a]).reshape(s), shape)


def _cells_to_faces(x, a, n_a):
    """Arithmetic mean of the two cells adjacent to each face along axis a.
    Wall faces (index 0 and n_a) get 0."""
    xp = _pad(x, a)
    fm = 0.5 * (_sl(xp, a, 0, n_a + 1) + _sl(xp, a, 1, n_a + 2))
    f = _index(fm.shape, a)
    return np.where((f >= 1) & (f <= n_a - 1), fm, 0.0)


# ----------------------------------------------------------------- grid / state

class Grid:
    """Uniform structured grid x_i = i h_x, h = l/n (Eq. 3.20-3.21)."""

    def __init__(self, case):
        self.dim = int(case["dim"])
        nz = int(case["nz"]) if self.dim == 3 else 1
        self.n = (int(case["nx"]), int(case["ny"]), nz)
        self.l = (float(case["lx"]), float(case["ly"]), float(case["lz"]) if self.dim == 3 else 1.0)
        self.h = tuple(self.l[a] / self.n[a] for a in range(3))
        self.vert = 1 if self.dim == 2 else 2
        self.cells = (self.n[2], self.n[1], self.n[0])
        self.ncell = self.n[0] * self.n[1] * self.n[2]
        self.volume = self.h[0] * self.h[1] * (self.h[2] if self.dim == 3 else 1.0)

    def faces(self, a):
        s = list(self.cells)
        s[2 - a] += 1
        return tuple(s)

    def key(self):
        return (self.dim,) + self.n + self.l


class State:
    """Fields at time level n: face velocities ``vel = [u, v, w]``, pressure
    ``p``, temperature ``T``, mixture concentration ``C``, liquid fraction
    ``gl``, liquid and solid concentrations ``Cl`` and ``Cs``."""

    FIELDS = ("u", "v", "w", "p", "T", "C", "gl", "Cl", "Cs")

    def __init__(self, vel, p, T, C, gl, Cl, Cs, t=0.0):
        self.t = float(t)
        self.vel = [np.array(v, dtype=np.float64) for v in vel]
        self.p, self.T, self.C = (np.array(x, dtype=np.float64) for x in (p, T, C))
        self.gl, self.Cl, self.Cs = (np.array(x, dtype=np.float64) for x in (gl, Cl, Cs))

    u = property(lambda s: s.vel[0])
    v = property(lambda s: s.vel[1])
    w = property(lambda s: s.vel[2])

    def as_dict(self):
        return {k: getattr(self, k) for k in self.FIELDS}

    def copy(self):
        return State(self.vel, self.p, self.T, self.C, self.gl, self.Cl, self.Cs, self.t)


# ----------------------------------------------------------------- model relations

def liquidus(C, al):
    """Liquidus temperature T_l = T_m + m C of the linearised phase diagram (Eq. 2.20, Eq. 3.14)."""
    return al["Tm"] + al["m"] * C


def equilibrium_fraction(T, C, al):
    """Liquid fraction in equilibrium with (T, C): 1 at or above the liquidus,
    otherwise Eq. 3.15 solved for g_l and clamped to [0, 1]. (Eq. 3.15 alone
    changes branch above T_m, where the melt is liquid.)"""
    kp = al["kp"]
    Tl = liquidus(C, al)
    g = 1.0 - (T - Tl) / ((1.0 - kp) * (T - al["Tm"]))
    return np.where(T >= Tl, 1.0, np.clip(g, 0.0, 1.0))


def liquid_concentration(C, gl, al):
    """C_l = C / (1 + (1 - g_l)(k_p - 1)) (Eq. 3.18), capped at the eutectic
    concentration when the alloy has one."""
    Cl = C / (1.0 + (1.0 - gl) * (al["kp"] - 1.0))
    if al.get("Ce") is not None:
        Cl = np.minimum(Cl, al["Ce"])
    return Cl


def inverse_permeability(gl, al):
    """K^{-1} from the Carman-Kozeny law K = K0 g^3 / (1 - g)^2 (Eq. 2.8),
    regularised as (1 - g)^2 / (K0 (g^3 + eps))."""
    return (1.0 - gl) ** 2 / (al["K0"] * (gl ** 3 + al["darcy_eps"]))


def initial_state(case, T, C):
    """Quiescent start: u = p = 0, given T and C; g_l from the lever rule in
    equilibrium (Eq. 3.15), C_l and C_s from Eq. 3.18-3.19."""
    g = Grid(case)
    al = case["alloy"]
    T = np.asarray(T, dtype=np.float64).reshape(g.cells)
    C = np.asarray(C, dtype=np.float64).reshape(g.cells)
    gl = equilibrium_fraction(T, C, al)
    Cl = liquid_concentration(C, gl, al)
    vel = [np.zeros(g.faces(a)) for a in range(3)]
    return State(vel, np.zeros(g.cells), T, C, gl, Cl, al["kp"] * Cl)


# ----------------------------------------------------------------- assembly (vectorised, Sec. 4)

def conv_diff_coeffs(shape, dim, h, F, D, has):
    """Row coefficients of the upwind-convection / central-diffusion operator
    of the general form Eq. 3.26, by the vectorised method (Eq. 4.3-4.4).

    For each axis a < dim and side s (0 = back, 1 = front) of each control
    volume: ``F[(a, s)]`` is the advecting velocity normal to that face,
    ``D[(a, s)]`` the diffusion coefficient multiplying (Phi_P - Phi_nb), and
    ``has[(a, s)]`` whether the neighbour is an unknown of the same system
    (otherwise its value is the boundary datum 0 and the coupling drops).

    Per axis the convection tuple is
    [-max(F_b, 0); max(F_f, 0) - min(F_b, 0); min(F_f, 0)] / h and the
    diffusion tuple (with the sign of -div(D grad)) is
    [-D_b; D_b + D_f; -D_f] / h^2.
    Returns the main diagonal and a dict of neighbour planes."""
    P = np.zeros(shape)
    nb = {name: np.zeros(shape) for name in _NB.values()}
    for a in range(dim):
        ha = h[a]
        Fb, Ff = F[(a, 0)], F[(a, 1)]
        Db, Df = D[(a, 0)], D[(a, 1)]
        P = P + (np.maximum(Ff, 0.0) - np.minimum(Fb, 0.0)) / ha + (Db + Df) / ha ** 2
        back = -np.maximum(Fb, 0.0) / ha - Db / ha ** 2
        front = np.minimum(Ff, 0.0) / ha - Df / ha ** 2
        nb[_NB[(a, 0)]] = np.where(has[(a, 0)], back, 0.0)
        nb[_NB[(a, 1)]] = np.where(has[(a, 1)], front, 0.0)
    return P, nb


def assemble_momentum(grid, st, case, a, Kinv=None):
    """System for the intermediate velocity component ``a`` (Eq. 3.3, momentum
    form Eq. 2.7): transient 1/dt, implicit upwind convection advected by u^n,
    implicit diffusion nu = mu/rho, implicit Darcy nu K^{-1} (Eq. 2.8),
    explicit -grad(p^n)/rho and the Boussinesq force (Eq. 2.9) on the
    vertical component."""
    al = case["alloy"]
    dt, rho = case["dt"], al["rho"]
    nu = al["mu"] / rho
    if Kinv is None:
        Kinv = inverse_permeability(st.gl, al)
    shape = grid.faces(a)
    na = grid.n[a]
    f = _index(shape, a)
    interior = (f >= 1) & (f <= na - 1)
    F, D, has = {}, {}, {}
    for d in range(grid.dim):
        if d == a:
            vp = _pad(st.vel[a], a)
            own = _sl(vp, a, 1, na + 2)
            F[(d, 0)] = 0.5 * (_sl(vp, a, 0, na + 1) + own)
            F[(d, 1)] = 0.5 * (own + _sl(vp, a, 2, na + 3))
            has[(d, 0)] = f - 1 >= 1
            has[(d, 1)] = f + 1 <= na - 1
            D[(d, 0)] = np.full(shape, nu)
            D[(d, 1)] = np.full(shape, nu)
        else:
            nd = grid.n[d]
            vdp = _pad(st.vel[d], a)
            lo = _sl(vdp, a, 0, na + 1)   # the cell behind the face along a
            hi = _sl(vdp, a, 1, na + 2)   # the cell in front of it
            F[(d, 0)] = 0.5 * (_sl(lo, d, 0, nd) + _sl(hi, d, 0, nd))
            F[(d, 1)] = 0.5 * (_sl(lo, d, 1, nd + 1) + _sl(hi, d, 1, nd + 1))
            j = _index(shape, d)
            has[(d, 0)] = j >= 1
            has[(d, 1)] = j <= nd - 2
            # beyond a wall the ghost is -u_P (no-slip: 2 nu/h^2 on the diagonal)
            # or +u_P (free-slip: no shear, nothing on the diagonal)
            wb = 0.0 if _slip(case, d, 0) else 2.0 * nu
            wf = 0.0 if _slip(case, d, 1) else 2.0 * nu
            D[(d, 0)] = np.where(j >= 1, nu, wb)
            D[(d, 1)] = np.where(j <= nd - 2, nu, wf)
    P, nb = conv_diff_coeffs(shape, grid.dim, grid.h, F, D, has)
    Kp = _pad(Kinv, a)
    Kface = 0.5 * (_sl(Kp, a, 0, na + 1) + _sl(Kp, a, 1, na + 2))
    P = P + 1.0 / dt + nu * Kface
    pp = _pad(st.p, a)
    dpdx = (_sl(pp, a, 1, na + 2) - _sl(pp, a, 0, na + 1)) / grid.h[a]
    b = st.vel[a] / dt - dpdx / rho
    if a == grid.vert:
        Tp, Cp = _pad(st.T, a), _pad(st.Cl, a)
        Tf = 0.5 * (_sl(Tp, a, 0, na + 1) + _sl(Tp, a, 1, na + 2))
        Cf = 0.5 * (_sl(Cp, a, 0, na + 1) + _sl(Cp, a, 1, na + 2))
        b = b + al["gravity"] * (al["betaT"] * (Tf - case["T0"]) + al["betaC"] * (Cf - al["C0"]))
    out = {"P": np.where(interior, P, 1.0), "b": np.where(interior, b, 0.0)}
    for name, plane in nb.items():
        out[name] = np.where(interior, plane, 0.0)
    return out


def assemble_scalar(grid, vel, Dface):
    """Convection-diffusion rows on cells (Eq. 3.26 without transient and
    source): advecting velocities are the face velocities themselves;
    ``Dface[a]`` holds the diffusion coefficient on the faces along axis a
    (0 on walls: zero flux there)."""
    shape = grid.cells
    F, D, has = {}, {}, {}
    for a in range(grid.dim):
        na = grid.n[a]
        i = _index(shape, a)
        F[(a, 0)] = _sl(vel[a], a, 0, na)
        F[(a, 1)] = _sl(vel[a], a, 1, na + 1)
        D[(a, 0)] = _sl(Dface[a], a, 0, na)
        D[(a, 1)] = _sl(Dface[a], a, 1, na + 1)
        has[(a, 0)] = i >= 1
        has[(a, 1)] = i <= na - 2
    return conv_diff_coeffs(shape, grid.dim, grid.h, F, D, has)


def assemble_solute(grid, vel, gl_n, C_n, case):
    """Matrix-based solute system (Eq. 3.6-3.10): (I/dt + (A_con - A_lap) A_g) C^{n+1}
    = C^n/dt with A_g = diag(1 / (1 - (1 - k_p)(1 - g_l^n))) (Eq. 3.8), upwind
    convection by u^{n+1} and diffusivity g_l^n D_l on faces. A_g scales the
    columns of the convection-diffusion operator."""
    al = case["alloy"]
    Dface = [_cells_to_faces(gl_n, a, grid.n[a]) * al["Dl"] for a in range(grid.dim)]
    P, nb = assemble_scalar(grid, vel, Dface)
    Ag = 1.0 / (1.0 - (1.0 - al["kp"]) * (1.0 - gl_n))
    out = {"P": 1.0 / case["dt"] + P * Ag, "b": C_n / case["dt"]}
    for a in range(3):
        for s in (0, 1):
            name = _NB[(a, s)]
            if a >= grid.dim:
                out[name] = nb[name]
                continue
            Agp = _pad(Ag, a)
            na = grid.n[a]
            Ag_nb = _sl(Agp, a, 0, na) if s == 0 else _sl(Agp, a, 2, na + 2)
            out[name] = nb[name] * Ag_nb
    return out


_FACE = {"x-": (0, 0), "x+": (0, 1), "y-": (1, 0), "y+": (1, 1), "z-": (2, 0), "z+": (2, 1)}


def _slip(case, a, s):
    """True if the wall on side s of axis a is free-slip."""
    return any(_FACE[f] == (a, s) for f in case.get("slip", ()))


def thermal_walls(case, grid, t):
    """[(axis, side, U, T_ext)] for every cooled wall at time t: a Robin wall
    has U = 1/(1/h + dx/(2k)) (film and half cell in series) and a fixed T_ext;
    a Dirichlet wall has U = 2k/dx (the half cell alone) and the wall
    temperature T_w(t) = T_w0 + rate t (Example 2's linear cooling)."""
    k = case["alloy"]["k"]
    out = []
    for face, (hc, Text) in case.get("robin", {}).items():
        a, s = _FACE[face]
        if a < grid.dim:
            out.append((a, s, 1.0 / (1.0 / hc + grid.h[a] / (2.0 * k)), float(Text)))
    for face, (Tw0, rate) in case.get("dirichlet", {}).items():
        a, s = _FACE[face]
        if a < grid.dim:
            out.append((a, s, 2.0 * k / grid.h[a], float(Tw0) + float(rate) * t))
    return out


def assemble_temperature(grid, vel, T_n, case, source=None, t=None):
    """First energy split step (Eq. 3.12): (T* - T^n)/dt + div(u^{n+1} T*) =
    div(k/(rho c_p) grad T*), with the cooled walls of ``thermal_walls`` at
    the new time level ``t`` (default dt) and zero flux elsewhere.
    ``source`` (optional, per cell) is the S_Phi of Eq. 3.26, used only by
    manufactured-solution tests."""
    if t is None:
        t = case["dt"]
    al = case["alloy"]
    alpha = al["k"] / (al["rho"] * al["cp"])
    Dface = []
    for a in range(grid.dim):
        f = _index(grid.faces(a), a)
        Dface.append(np.where((f >= 1) & (f <= grid.n[a] - 1), alpha, 0.0))
    P, nb = assemble_scalar(grid, vel, Dface)
    P = P + 1.0 / case["dt"]
    b = T_n / case["dt"]
    if source is not None:
        b = b + source
    for a, s, U, Text in thermal_walls(case, grid, t):
        coef = U / (al["rho"] * al["cp"] * grid.h[a])
        i = _index(grid.cells, a)
        wall = (i == 0) if s == 0 else (i == grid.n[a] - 1)
        P = P + np.where(wall, coef, 0.0)
        b = b + np.where(wall, coef * Text, 0.0)
    out = {"P": P, "b": b}
    out.update(nb)
    return out


def poisson_matrix(grid):
    """Planes of A = -L, the negative discrete Laplacian on cells with
    homogeneous Neumann walls (Eq. 3.4 discretised by Eq. 3.27 with D = 1).
    A is symmetric positive semi-definite with the constants as null space."""
    shape = grid.cells
    D, F, has = {}, {}, {}
    for a in range(grid.dim):
        i = _index(shape, a)
        has[(a, 0)] = i >= 1
        has[(a, 1)] = i <= grid.n[a] - 2
        D[(a, 0)] = np.where(has[(a, 0)], 1.0, 0.0)
        D[(a, 1)] = np.where(has[(a, 1)], 1.0, 0.0)
        F[(a, 0)] = F[(a, 1)] = np.zeros(shape)
    P, nb = conv_diff_coeffs(shape, grid.dim, grid.h, F, D, has)
    out = {"P": P}
    out.update(nb)
    return out


def divergence(grid, vel):
    """Discrete divergence on cells: sum_a (u_a[front face] - u_a[back face]) / h_a."""
    d = np.zeros(grid.cells)
    for a in range(grid.dim):
        na = grid.n[a]
        d = d + (_sl(vel[a], a, 1, na + 1) - _sl(vel[a], a, 0, na)) / grid.h[a]
    return d


def poisson_rhs(grid, ustar, case):
    """Right-hand side of A p' = b with A = -L (Eq. 3.4): b = -(rho/dt) div u*,
    with its mean removed so that the singular Neumann system is consistent."""
    b = -(case["alloy"]["rho"] / case["dt"]) * divergence(grid, ustar)
    return b - b.mean()


def project(grid, ustar, pc, case):
    """Velocity correction (Eq. 3.5): u^{n+1} = u* - (dt/rho) grad p' on the
    interior faces; wall faces stay 0."""
    k = case["dt"] / case["alloy"]["rho"]
    out = []
    for a in range(3):
        if a >= grid.dim:
            out.append(np.zeros(grid.faces(a)))
            continue
        na = grid.n[a]
        pp = _pad(pc, a)
        grad = (_sl(pp, a, 1, na + 2) - _sl(pp, a, 0, na + 1)) / grid.h[a]
        f = _index(grid.faces(a), a)
        out.append(np.where((f >= 1) & (f <= na - 1), ustar[a] - k * grad, 0.0))
    return out


# ----------------------------------------------------------------- lever rule (Eq. 3.13-3.19)

def lever_update(Tstar, gl_n, C_new, al):
    """Second energy split step and phase update, pointwise.

    The latent-heat correction T^{n+1} = T* - (L/c_p)(g^{n+1} - g^n) (Eq. 3.13)
    combined with the lever relation (Eq. 3.15) at the liquidus T_l(C^{n+1})
    (Eq. 3.14) gives a g^2 + b g + c = 0 (Eq. 3.16) with the coefficients of
    Eq. 3.17. The larger root is taken and clamped to [0, 1]; T^{n+1} follows
    from Eq. 3.13. Below the eutectic temperature T_e = T_m + m C_e, while
    liquid remains, the cell is held at T_e and the fraction absorbs the
    energy (isothermal eutectic solidification). C_l and C_s follow from
    Eq. 3.18-3.19.

    Returns (T, g_l, C_l, C_s)."""
    kp, Tm, L, cp = al["kp"], al["Tm"], al["L"], al["cp"]
    Tl = liquidus(C_new, al)
    a = 1.0 - kp
    b = kp - gl_n * (1.0 - kp) + (cp / L) * (1.0 - kp) * (Tm - Tstar)
    c = -(gl_n + (cp / L) * Tstar) * kp + (cp / L) * (Tl - (1.0 - kp) * Tm)
    disc = np.maximum(b * b - 4.0 * a * c, 0.0)
    g = (-b + np.sqrt(disc)) / (2.0 * a)
    g = np.clip(g, 0.0, 1.0)
    T = Tstar - (L / cp) * (g - gl_n)
    if al.get("Ce") is not None:
        Te = liquidus(al["Ce"], al)
        eut = (T < Te) & (g > 0.0)
        g_e = gl_n - (cp / L) * (Te - Tstar)
        T_e = np.where(g_e >= 0.0, Te, Tstar + (L / cp) * gl_n)
        g = np.where(eut, np.maximum(g_e, 0.0), g)
        T = np.where(eut, T_e, T)
    Cl = liquid_concentration(C_new, g, al)
    return T, g, Cl, kp * Cl


# ----------------------------------------------------------------- sparse view

def sparse_from_planes(planes):
    """CSR matrix of a DIA system (Eq. 4.1). Checks that no plane couples a
    row to a point outside the grid (so no coupling wraps around a row)."""
    import scipy.sparse as sp
    shape = planes["P"].shape
    mz, my, mx = shape
    n = mx * my * mz
    k, j, i = np.unravel_index(np.arange(n), shape)
    offs = {"P": (0, None), "W": (-1, i >= 1), "E": (1, i <= mx - 2), "S": (-mx, j >= 1),
            "N": (mx, j <= my - 2), "B": (-mx * my, k >= 1), "T": (mx * my, k <= mz - 2)}
    rows, cols, vals = [], [], []
    for name, (off, ok) in offs.items():
        a = planes[name].ravel()
        r = np.nonzero(a)[0]
        if ok is not None and not ok[r].all():
            raise ValueError("plane %s couples a row to a point outside the grid" % name)
        rows.append(r)
        cols.append(r + off)
        vals.append(a[r])
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))


# ----------------------------------------------------------------- Algorithm 1

def step(grid, st, case, method="auto", info=None):
    """One time step n -> n+1 in the order of Algorithm 1:
    1 intermediate velocity (Eq. 3.3); 2 pressure correction (Eq. 3.4);
    3 projection (Eq. 3.5); 4 solute (Eq. 3.10); 5 liquidus (Eq. 3.14);
    6 intermediate temperature (Eq. 3.12); 7 latent-heat correction and
    liquid fraction (Eq. 3.13, 3.16-3.17); 8 phase concentrations (Eq. 3.18-3.19).

    ``info``, if a dict, receives the intermediate fields (u*, p', T*)."""
    from .solve import solve_system, solve_poisson
    al = case["alloy"]
    tol_t = min(float(case.get("tol_t", 1e-12)), 1e-13)
    tol_p = min(float(case.get("tol_p", 1e-10)), 1e-13)
    Kinv = inverse_permeability(st.gl, al)
    ustar = []
    for a in range(3):
        if a < grid.dim:
            sysm = assemble_momentum(grid, st, case, a, Kinv)
            ustar.append(solve_system(sysm, x0=st.vel[a], method=method, rtol=tol_t))
        else:
            ustar.append(np.zeros(grid.faces(a)))
    bp = poisson_rhs(grid, ustar, case)
    pc = solve_poisson(grid, bp, method=method, rtol=tol_p)
    vel = project(grid, ustar, pc, case)
    p = st.p + pc
    sysc = assemble_solute(grid, vel, st.gl, st.C, case)
    C = solve_system(sysc, x0=st.C, method=method, rtol=tol_t)
    t_new = st.t + case["dt"]
    syst = assemble_temperature(grid, vel, st.T, case, t=t_new)
    Tstar = solve_system(syst, x0=st.T, method=method, rtol=tol_t)
    T, gl, Cl, Cs = lever_update(Tstar, st.gl, C, al)
    if info is not None:
        info.update(ustar=ustar, pc=pc, Tstar=Tstar, sysc=sysc, syst=syst)
    return State(vel, p, T, C, gl, Cl, Cs, t_new)


def run(case, nsteps, T=None, C=None, method="auto"):
    """Initial state from (T, C) (or uniform T0, C0) and ``nsteps`` steps."""
    grid = Grid(case)
    if T is None:
        T = np.full(grid.cells, case["T0"])
    if C is None:
        C = np.full(grid.cells, case["alloy"]["C0"])
    st = initial_state(case, T, C)
    for _ in range(nsteps):
        st = step(grid, st, case, method=method)
    return st

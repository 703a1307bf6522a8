"""Forward (equation-based) matrix assembly by residual probing (Sec. 4,
"Forward method", Eq. 4.5-4.7).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The discrete equation of each unknown is coded straight from its fluxes
(Eq. 4.6): upwind fluxes by the case form of Eq. 3.29, central diffusion
(Eq. 3.27), ghost values for walls. With r = 0 - Eq(Phi) = b - A Phi
(Eq. 4.5): b = -Eq(0), and A's entries follow from residuals at trial vectors
that are 1 on one colour of a 3-colouring along each axis (3^dim probes),
because the seven stencil points of any row carry seven distinct colours.
The paper states that this yields the vectorised matrix up to rounding;
the tests use that as a pin of ``scheme``'s vectorised assembly.

Pure-Python loops over rows: for small grids only.
"""
import itertools
import numpy as np

from .scheme import Grid, inverse_permeability, liquid_concentration

_OFFS = {"P": (0, 0, 0), "W": (-1, 0, 0), "E": (1, 0, 0), "S": (0, -1, 0), "N": (0, 1, 0),
         "B": (0, 0, -1), "T": (0, 0, 1)}


def _get(arr, i, j, k):
    """Value at paper index (i, j, k) of an array shaped (z, y, x)."""
    return arr[k, j, i]


def _e(a):
    e = [0, 0, 0]
    e[a] = 1
    return e


def _add(idx, e, s=1):
    return (idx[0] + s * e[0], idx[1] + s * e[1], idx[2] + s * e[2])


def _slip_wall(case, a, side):
    names = {("x-"): (0, 0), "x+": (0, 1), "y-": (1, 0), "y+": (1, 1), "z-": (2, 0), "z+": (2, 1)}
    return any(names[f] == (a, side) for f in case.get("slip", ()))


def _upwind_flux(F, phi_back, phi_front):
    """(Phi F) on a face with Phi_back behind and Phi_front in front (Eq. 3.29)."""
    return (phi_back if F >= 0.0 else phi_front) * F


def momentum_eq(grid, st, case, a, phi):
    """Eq(phi) for component ``a`` of the intermediate velocity (Eq. 3.3) at
    every face. Wall faces carry the equation phi - 0."""
    al = case["alloy"]
    dt, rho, nu = case["dt"], al["rho"], al["mu"] / al["rho"]
    Kinv = inverse_permeability(st.gl, al)
    n = grid.n
    shape = grid.faces(a)
    ea = _e(a)
    out = np.zeros(shape)
    na = n[a]
    dims = [n[0] + (a == 0), n[1] + (a == 1), n[2] + (a == 2)]
    for k in range(dims[2]):
        for j in range(dims[1]):
            for i in range(dims[0]):
                idx = (i, j, k)
                P = _get(phi, *idx)
                if idx[a] == 0 or idx[a] == na:
                    out[k, j, i] = P
                    continue
                c_lo, c_hi = _add(idx, ea, -1), idx       # the two cells sharing this face
                r = (P - _get(st.vel[a], *idx)) / dt
                for d in range(grid.dim):
                    ed = _e(d)
                    h = grid.h[d]
                    if d == a:
                        Uf = 0.5 * (_get(st.vel[a], *idx) + _get(st.vel[a], *_add(idx, ea)))
                        Ub = 0.5 * (_get(st.vel[a], *_add(idx, ea, -1)) + _get(st.vel[a], *idx))
                        fi, bi = _add(idx, ea), _add(idx, ea, -1)
                        # wall faces hold the boundary datum 0
                        Pf = 0.0 if fi[a] == na else _get(phi, *fi)
                        Pb = 0.0 if bi[a] == 0 else _get(phi, *bi)
                    else:
                        Uf = 0.5 * (_get(st.vel[d], *_add(c_lo, ed)) + _get(st.vel[d], *_add(c_hi, ed)))
                        Ub = 0.5 * (_get(st.vel[d], *c_lo) + _get(st.vel[d], *c_hi))
                        # ghost beyond a wall: minus the interior value (no-slip) or
                        # the interior value itself (free-slip)
                        gf = P if _slip_wall(case, d, 1) else -P
                        gb = P if _slip_wall(case, d, 0) else -P
                        Pf = _get(phi, *_add(idx, ed)) if idx[d] + 1 <= n[d] - 1 else gf
                        Pb = _get(phi, *_add(idx, ed, -1)) if idx[d] - 1 >= 0 else gb
                    r += (_upwind_flux(Uf, P, Pf) - _upwind_flux(Ub, Pb, P)) / h
                    r -= nu * ((Pf - P) - (P - Pb)) / h ** 2
                r += nu * 0.5 * (_get(Kinv, *c_lo) + _get(Kinv, *c_hi)) * P
                r += (_get(st.p, *c_hi) - _get(st.p, *c_lo)) / (grid.h[a] * rho)
                if a == grid.vert:
                    Tf = 0.5 * (_get(st.T, *c_lo) + _get(st.T, *c_hi))
                    Cf = 0.5 * (_get(st.Cl, *c_lo) + _get(st.Cl, *c_hi))
                    r -= al["gravity"] * (al["betaT"] * (Tf - case["T0"]) + al["betaC"] * (Cf - al["C0"]))
                out[k, j, i] = r
    return out


def _cell_eq(grid, vel, phi, phi_n, dt, D, field_of, robin):
    """Eq(phi) of a cell-centred transport equation: transient, upwind
    convection of ``field_of(phi)`` by the face velocities, central diffusion
    with face coefficient D(a, idx_lo, idx_hi) (0 at walls) and Robin wall
    terms given as [(a, side, coef, T_ext)] (flux coef (phi_P - T_ext))."""
    n = grid.n
    out = np.zeros(grid.cells)
    q = field_of(phi)
    for k in range(n[2]):
        for j in range(n[1]):
            for i in range(n[0]):
                idx = (i, j, k)
                P = _get(q, *idx)
                r = (_get(phi, *idx) - _get(phi_n, *idx)) / dt
                for a in range(grid.dim):
                    ea = _e(a)
                    h = grid.h[a]
                    Uf = _get(vel[a], *_add(idx, ea))
                    Ub = _get(vel[a], *idx)
                    has_f = idx[a] + 1 <= n[a] - 1
                    has_b = idx[a] - 1 >= 0
                    Qf = _get(q, *_add(idx, ea)) if has_f else 0.0
                    Qb = _get(q, *_add(idx, ea, -1)) if has_b else 0.0
                    r += (_upwind_flux(Uf, P, Qf) - _upwind_flux(Ub, Qb, P)) / h
                    Df = D(a, idx, _add(idx, ea)) if has_f else 0.0
                    Db = D(a, _add(idx, ea, -1), idx) if has_b else 0.0
                    r -= (Df * (Qf - P) - Db * (P - Qb)) / h ** 2
                for a, s, coef, Text in robin:
                    if (s == 0 and idx[a] == 0) or (s == 1 and idx[a] == n[a] - 1):
                        r += coef * (_get(phi, *idx) - Text)
                out[k, j, i] = r
    return out


def solute_eq(grid, vel, gl_n, C_n, case, C):
    """Eq(C) of the solute step (Eq. 3.7 with C_l^{n+1} = A_g C^{n+1}, Eq. 3.8)."""
    al = case["alloy"]

    def to_cl(c):
        return c / (1.0 - (1.0 - al["kp"]) * (1.0 - gl_n))

    def D(a, lo, hi):
        return al["Dl"] * 0.5 * (_get(gl_n, *lo) + _get(gl_n, *hi))

    return _cell_eq(grid, vel, C, C_n, case["dt"], D, to_cl, [])


def temperature_eq(grid, vel, T_n, case, T, t=None):
    """Eq(T*) of the first energy step (Eq. 3.12) with its cooled walls: the
    wall flux is written from the wall's own definition (film plus half cell
    for Robin, the half cell to the prescribed wall temperature for Dirichlet)."""
    al = case["alloy"]
    k = al["k"]
    t = case["dt"] if t is None else t
    alpha = k / (al["rho"] * al["cp"])
    names = {"x-": (0, 0), "x+": (0, 1), "y-": (1, 0), "y+": (1, 1), "z-": (2, 0), "z+": (2, 1)}
    robin = []
    for face, (hc, Text) in case.get("robin", {}).items():
        a, s = names[face]
        if a < grid.dim:
            dx = grid.h[a]
            robin.append((a, s, 1.0 / ((1.0 / hc + dx / (2.0 * k)) * al["rho"] * al["cp"] * dx), Text))
    for face, (Tw0, rate) in case.get("dirichlet", {}).items():
        a, s = names[face]
        if a < grid.dim:
            dx = grid.h[a]
            robin.append((a, s, k / (0.5 * dx) / (al["rho"] * al["cp"] * dx), Tw0 + rate * t))
    return _cell_eq(grid, vel, T, T_n, case["dt"], lambda a, lo, hi: alpha, lambda t: t, robin)


def poisson_eq(grid, p):
    """Eq(p) = -L p with homogeneous Neumann walls (Eq. 3.4, left-hand side, negated)."""
    zero = [np.zeros(grid.faces(a)) for a in range(3)]
    return _cell_eq(grid, zero, p, p, np.inf, lambda a, lo, hi: 1.0, lambda t: t, [])


def forward_assemble(grid, eq, shape):
    """Planes and right-hand side of the system whose residual is
    r = 0 - eq(Phi), by 3^dim colour probes (Eq. 4.5-4.7)."""
    base = eq(np.zeros(shape))
    out = {"b": -base}
    for name in _OFFS:
        out[name] = np.zeros(shape)
    mz, my, mx = shape
    k, j, i = np.meshgrid(np.arange(mz), np.arange(my), np.arange(mx), indexing="ij")
    colours = list(itertools.product(range(3), range(3), range(3) if grid.dim == 3 else range(1)))
    resid = {}
    for c in colours:
        trial = ((i % 3 == c[0]) & (j % 3 == c[1]) & (k % 3 == c[2] if grid.dim == 3 else True)).astype(np.float64)
        resid[c] = eq(trial) - base
    for name, (di, dj, dk) in _OFFS.items():
        ni, nj, nk = i + di, j + dj, k + dk
        inside = (ni >= 0) & (ni < mx) & (nj >= 0) & (nj < my) & (nk >= 0) & (nk < mz)
        for c in colours:
            sel = inside & (ni % 3 == c[0]) & (nj % 3 == c[1])
            if grid.dim == 3:
                sel &= (nk % 3 == c[2])
            out[name][sel] = resid[c][sel]
    return out


def forward_momentum(grid, st, case, a):
    return forward_assemble(grid, lambda phi: momentum_eq(grid, st, case, a, phi), grid.faces(a))


def forward_solute(grid, vel, gl_n, C_n, case):
    return forward_assemble(grid, lambda c: solute_eq(grid, vel, gl_n, C_n, case, c), grid.cells)


def forward_temperature(grid, vel, T_n, case, t=None):
    return forward_assemble(grid, lambda T: temperature_eq(grid, vel, T_n, case, T, t), grid.cells)


def forward_poisson(grid):
    planes = forward_assemble(grid, lambda p: poisson_eq(grid, p), grid.cells)
    planes.pop("b")
    return planes

"""Workload definitions and seeded synthetic initial fields.

This module is the only code shared by the CUDA path and the CPU oracle. It
holds plain data (grid sizes, domain extents, alloy properties, cooling
conditions, time step, solver tolerances) and draws the seeded initial
temperature noise. It holds none of the scheme's arithmetic: no liquidus, no
lever rule, no assembly. Each side derives everything else from these inputs.

A case is a plain ``dict``:

``dim``                 2 or 3 (2D runs use ``nz == 1`` and have no w field)
``nx, ny, nz``          cell counts; x is fastest in memory, then y, then z
``lx, ly, lz``          domain extents in metres (``lz`` unused in 2D)
``dt``                  time step in seconds
``alloy``               dict of material data (see :func:`sn_pb_alloy`)
``robin``               dict face -> (h [W/m^2K], T_ext [K]); faces not listed
                        in ``robin`` or ``dirichlet`` are adiabatic. Faces are
                        ``x-, x+, y-, y+, z-, z+``.
``dirichlet``           dict face -> (T_w0 [K], rate [K/s]): wall held at
                        T_w(t) = T_w0 + rate t
``slip``                faces that are free-slip (the others are no-slip)
``perturb``             None, or a factor applied to C on the central
                        vertical line (Example 2 seeds freckles with 1.0001)
``T0``                  nominal initial temperature [K]; also the Boussinesq
                        reference temperature
``noise``               half-width of the uniform initial temperature noise [K]
``seed``                seed of the noise generator (numpy PCG64)
``tol_p, tol_t``        relative residual tolerances (2-norm) of the pressure
                        and transport solves
``max_it_p, max_it_t``  iteration caps of those solves
``precond_p``           pressure solver of the CUDA path: "mg" (multigrid-preconditioned CG),
                        "jacobi" (Jacobi-preconditioned CG) or "dct" (refinement around the
                        cosine-transform inverse)
``steps``               number of time steps the workload runs

The vertical axis is y in 2D and z in 3D; gravity points along minus that
axis. All walls are rigid and impermeable.
"""
import numpy as np

FACES = ("x-", "x+", "y-", "y+", "z-", "z+")


def sn_pb_alloy():
    """Sn-Pb-like binary alloy of the 2D cavity workload (C in wt% Pb)."""
    return dict(
        Tm=505.0,        # melting point at C = 0 [K]
        m=-1.286,        # liquidus slope [K / wt%]
        kp=0.0656,       # partition coefficient C_s / C_l
        C0=5.0,          # nominal concentration [wt%]
        rho=7000.0,      # density [kg/m^3]
        k=55.0,          # thermal conductivity [W/mK]
        cp=200.0,        # specific heat [J/kgK]
        L=6.1e4,         # latent heat [J/kg]
        mu=1.0e-3,       # liquid dynamic viscosity [Pa s]
        Dl=3.0e-9,       # liquid solute diffusivity [m^2/s]
        betaT=6.0e-5,    # thermal expansion [1/K]
        betaC=-5.3e-3,   # solutal expansion [1/wt%]
        K0=3.6e-10,      # Carman-Kozeny prefactor [m^2]
        Ce=38.1,         # eutectic concentration [wt%]; None disables the branch
        gravity=9.81,    # [m/s^2]
        darcy_eps=1.0e-6,  # regularisation of g_l^3 in the inverse permeability
    )


def fe_c_alloy():
    """Fe-C-like alloy of the large 3D ingot workload (no eutectic branch)."""
    a = sn_pb_alloy()
    a.update(Tm=1811.0, m=-78.0, kp=0.34, C0=0.45, rho=7200.0, k=30.0, cp=700.0, L=2.7e5, Dl=2.0e-8, Ce=None)
    return a


def make_case(dim, nx, ny, nz, lx, ly, lz, dt, alloy=None, robin=None, T0=499.0, noise=1.0e-3, seed=0,
              tol_p=1.0e-10, tol_t=1.0e-12, max_it_p=20000, max_it_t=2000, steps=100, precond_p="dct",
              dirichlet=None, slip=(), perturb=None):
    if dim == 2:
        nz, lz = 1, 1.0
    return dict(dim=dim, nx=nx, ny=ny, nz=nz, lx=lx, ly=ly, lz=lz, dt=dt,
                alloy=dict(alloy if alloy is not None else sn_pb_alloy()),
                robin=dict(robin if robin is not None else {"x-": (400.0, 298.0)}),
                dirichlet=dict(dirichlet or {}), slip=tuple(slip), perturb=perturb,
                T0=T0, noise=noise, seed=seed, tol_p=tol_p, tol_t=tol_t,
                max_it_p=max_it_p, max_it_t=max_it_t, steps=steps, precond_p=precond_p)


def cavity_2d(nx=50, ny=30, **kw):
    """2D 0.10 m x 0.06 m cavity, Sn-Pb-like alloy, left wall cooled (h = 400 to 298 K), dt = 0.01 s."""
    kw.setdefault("steps", 300)
    return make_case(2, nx, ny, 1, 0.10, 0.06, 1.0, 0.01, **kw)


def box_3d(nx=128, ny=96, nz=96, **kw):
    """3D 0.10 x 0.06 x 0.06 m box, same alloy and cooling as the 2D cavity; 200 steps."""
    kw.setdefault("steps", 200)
    kw.setdefault("seed", 1)
    return make_case(3, nx, ny, nz, 0.10, 0.06, 0.06, 0.01, **kw)


def ingot_3d(nx=384, ny=256, nz=256, **kw):
    """Large 3D 0.2 x 0.1 x 0.1 m ingot, Fe-C-like alloy cooled from the bottom (h = 800 to 298 K).

    The workload states no initial temperature: 1776.4 K is taken, about
    half a kelvin above the liquidus of the nominal composition, like the
    superheat of the cavity workload."""
    kw.setdefault("steps", 100)
    kw.setdefault("seed", 4)
    kw.setdefault("robin", {"z-": (800.0, 298.0)})
    kw.setdefault("T0", 1776.4)
    return make_case(3, nx, ny, nz, 0.2, 0.1, 0.1, 0.01, alloy=fe_c_alloy(), **kw)


def pb_sn_alloy():
    """Pb-48%Sn alloy of Example 2 (Table 1; C in wt% Sn, temperatures in K)."""
    a = sn_pb_alloy()
    a.update(Tm=327.5 + 273.15, m=-2.334, kp=0.307, C0=48.0, rho=9000.0, k=50.0, cp=200.0, L=5.35e4,
             betaT=1.0e-4, betaC=4.5e-3, Ce=61.9)
    return a


def freckle_2d(nx=30, ny=90, slip=False, **kw):
    """Example 2 in 2D: Pb-48%Sn in a cavity of aspect ratio nx:ny (1 mm
    cells), cooled from the bottom by a wall temperature
    falling linearly from 216 C at 0.05 K/s, the top held adiabatic here,
    side walls no-slip (or free-slip), C raised by 1e-4 relative on the
    central vertical line, dt = 0.01 s. The initial melt is at 216 C."""
    kw.setdefault("steps", 100)
    kw.setdefault("seed", 5)
    h = 1.0e-3
    walls = ("x-", "x+") if slip else ()
    return make_case(2, nx, ny, 1, nx * h, ny * h, 1.0, 0.01, alloy=pb_sn_alloy(), robin={},
                     dirichlet={"y-": (216.0 + 273.15, -0.05)}, slip=walls, T0=216.0 + 273.15,
                     perturb=1.0001, **kw)


def cell_shape(case):
    """numpy shape (nz, ny, nx) of a cell-centred field."""
    return (case["nz"], case["ny"], case["nx"])


def initial_fields(case):
    """Seeded initial fields: T = T0 + U(-noise, noise) per cell, C = C0, u = p = 0.

    Returns float64 arrays of shape (nz, ny, nx), x fastest."""
    rng = np.random.Generator(np.random.PCG64(case["seed"]))
    shape = cell_shape(case)
    T = case["T0"] + rng.uniform(-case["noise"], case["noise"], size=shape)
    C = np.full(shape, case["alloy"]["C0"], dtype=np.float64)
    if case.get("perturb"):
        nx, ny = case["nx"], case["ny"]
        if case["dim"] == 2:
            C[:, :, nx // 2] *= case["perturb"]
        else:
            C[:, ny // 2, nx // 2] *= case["perturb"]
    return dict(T=np.ascontiguousarray(T, dtype=np.float64), C=C)


def random_state(case, seed, vel_scale=1e-3):
    """Seeded random mid-run state for kernel-level checks: face velocities,
    pressure, temperature around T0, concentration around C0 and liquid
    fractions in [0, 1] (a quarter of the cells exactly 0 or 1).

    The velocity is not divergence-free; the assembly and solver kernels do
    not need it to be."""
    rng = np.random.Generator(np.random.PCG64(seed))
    nz, ny, nx = cell_shape(case)
    a = case["alloy"]
    out = dict(
        u=rng.uniform(-vel_scale, vel_scale, size=(nz, ny, nx + 1)),
        v=rng.uniform(-vel_scale, vel_scale, size=(nz, ny + 1, nx)),
        w=rng.uniform(-vel_scale, vel_scale, size=(nz + 1, ny, nx)) if case["dim"] == 3 else np.zeros((nz + 1, ny, nx)),
        p=rng.uniform(-1.0, 1.0, size=(nz, ny, nx)),
        T=case["T0"] + rng.uniform(-2.0, 0.5, size=(nz, ny, nx)),
        C=a["C0"] * (1.0 + rng.uniform(-0.2, 0.2, size=(nz, ny, nx))),
    )
    g = rng.uniform(0.0, 1.0, size=(nz, ny, nx))
    sel = rng.uniform(size=g.shape)
    g[sel < 0.125] = 0.0
    g[sel > 0.875] = 1.0
    out["gl"] = g
    out["Cl"] = out["C"] * (1.0 + rng.uniform(0.0, 0.5, size=g.shape))
    # walls carry zero normal velocity
    out["u"][:, :, 0] = out["u"][:, :, -1] = 0.0
    out["v"][:, 0, :] = out["v"][:, -1, :] = 0.0
    out["w"][0] = out["w"][-1] = 0.0
    return {k: np.ascontiguousarray(v, dtype=np.float64) for k, v in out.items()}


# ---------------------------------------------------------------- batched and served workloads

BATCH_2D = ((64, 64), (96, 64), (128, 64), (128, 96), (128, 128), (192, 96), (192, 128), (256, 128), (64, 96),
            (64, 128), (96, 128))
BATCH_3D_EDGE = (32, 48, 64, 80, 96)


def batch_cases(n=64, seed=2, steps=100):
    """Independent cavities for the batched workload: half 2D, half 3D, x/y
    aspect ratio drawn in [0.5, 2] (the grid closest to it from 64x64..256x128
    in 2D, 32^3..96^3 in 3D, square cells, 0.06 m high), C0 ~ U[2, 15] wt%,
    left-wall Robin cooling with h ~ U[100, 1000] W/m^2K to 298 K, mixed
    precision tolerances of the 3D box workload. Initial temperature 503 K
    (above the liquidus of every drawn composition), seeded noise."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for q in range(n):
        dim = 2 if rng.uniform() < 0.5 else 3
        aspect = rng.uniform(0.5, 2.0)
        C0 = rng.uniform(2.0, 15.0)
        h = rng.uniform(100.0, 1000.0)
        alloy = sn_pb_alloy()
        alloy["C0"] = C0
        if dim == 2:
            nx, ny = min(BATCH_2D, key=lambda g: abs(g[0] / g[1] - aspect))
            nz = 1
        else:
            ny = nz = int(rng.choice(BATCH_3D_EDGE))
            nx = min(BATCH_3D_EDGE, key=lambda e: abs(e / ny - aspect))
        hy = 0.06 / ny
        out.append(make_case(dim, nx, ny, nz, nx * hy, 0.06, nz * hy, 0.01, alloy=alloy,
                             robin={"x-": (h, 298.0)}, T0=503.0, seed=1000 * seed + q, steps=steps))
    return out


SERVE_GRIDS = ((32, 32, 32), (64, 64, 64), (96, 96, 96), (128, 96, 96), (192, 192, 192))


def serving_requests(n=1000, rate=20.0, seed=3, steps=500, grids=SERVE_GRIDS):
    """Simulation requests of the serving workload: Poisson arrivals (mean
    `rate` per second), 3D grid drawn uniformly from `grids` (0.06 m edge at
    the smallest grid spacing of the box), C0 ~ U[2, 15] wt%, h ~ U[100, 1000],
    bottom or side cooling 50/50, `steps` steps each. Returns a list of
    (arrival_time_s, case)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = 0.0
    out = []
    for q in range(n):
        t += rng.exponential(1.0 / rate)
        nx, ny, nz = grids[int(rng.integers(len(grids)))]
        C0 = rng.uniform(2.0, 15.0)
        h = rng.uniform(100.0, 1000.0)
        face = "z-" if rng.uniform() < 0.5 else "x-"
        alloy = sn_pb_alloy()
        alloy["C0"] = C0
        hh = 0.06 / max(nx, ny, nz)
        out.append((t, make_case(3, nx, ny, nz, nx * hh, ny * hh, nz * hh, 0.01, alloy=alloy, robin={face: (h, 298.0)},
                                 T0=503.0, seed=10000 * seed + q, steps=steps)))
    return out

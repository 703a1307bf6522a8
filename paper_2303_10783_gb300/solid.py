"""Thin ctypes binding of libsolid (include/solid.h).

Argument marshalling only: every stage of the time step runs in the
library's CUDA kernels. PyTorch provides the device workspace and the
stream. Importing this module does not load the library; :func:`load` does,
and raises if the compiled library is missing (there is no fallback)."""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsolid.so")

# status codes, enums (mirror include/solid.h)
SS_OK, SS_EINVAL, SS_ENOMEM, SS_ENOTCONV, SS_ENAN, SS_ECUDA, SS_ESTATE, SS_ETIMEOUT = range(8)
STATUS_NAMES = {0: "SS_OK", 1: "SS_EINVAL", 2: "SS_ENOMEM", 3: "SS_ENOTCONV", 4: "SS_ENAN", 5: "SS_ECUDA",
                6: "SS_ESTATE", 7: "SS_ETIMEOUT"}
SS_FP64, SS_MIXED = 0, 1
SS_PRECOND_MG, SS_PRECOND_JACOBI, SS_PRECOND_DCT = 0, 1, 2
SS_TC_AUTO, SS_TC_ON, SS_TC_OFF = 0, 1, 2
SS_ADIABATIC, SS_ROBIN, SS_DIRICHLET = 0, 1, 2
SS_NOSLIP, SS_FREESLIP = 0, 1
FIELDS = ("u", "v", "w", "p", "T", "C", "gl", "Cl", "Cs")
FIELD_ID = {name: i for i, name in enumerate(FIELDS)}
SYSTEMS = ("u", "v", "w", "p", "C", "T")
SYS_ID = {name: i for i, name in enumerate(SYSTEMS)}
FACE_ID = {"x-": 0, "x+": 1, "y-": 2, "y+": 3, "z-": 4, "z+": 5}
PLANE_NAMES = ("P", "W", "E", "S", "N", "B", "T", "b", "x")


class Grid(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("lx", ctypes.c_double), ("ly", ctypes.c_double), ("lz", ctypes.c_double),
                ("dt", ctypes.c_double), ("precision", ctypes.c_int),
                ("tol_p", ctypes.c_double), ("tol_t", ctypes.c_double),
                ("max_it_p", ctypes.c_int), ("max_it_t", ctypes.c_int), ("precond_p", ctypes.c_int)]


class Alloy(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in ("Tm", "m", "kp", "C0", "rho", "k", "cp", "L", "mu", "Dl", "betaT",
                                               "betaC", "K0", "Ce", "gravity", "darcy_eps", "Tref")]


class BC(ctypes.Structure):
    _fields_ = [("thermal", ctypes.c_int), ("h", ctypes.c_double), ("Text", ctypes.c_double),
                ("dTdt", ctypes.c_double), ("flow", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_longlong), ("iters", ctypes.c_int * 6), ("refinements", ctypes.c_int * 6),
                ("relres", ctypes.c_double * 6), ("status", ctypes.c_int), ("jacobi", ctypes.c_int * 6)]


PROF_NAMES = (tuple("assemble_" + s for s in SYSTEMS) + tuple("solve_" + s for s in SYSTEMS) +
              ("project", "lever", "presolve_T"))


class Profile(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double * 15), ("launches", ctypes.c_longlong * 15), ("kernels", ctypes.c_longlong),
                ("iters", ctypes.c_longlong * 6), ("presolve_sweeps", ctypes.c_longlong),
                ("jacobi", ctypes.c_longlong * 6)]


class SolidError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


_lib = None


def _declare(lib):
    P = ctypes.c_void_p
    sig = {
        "ss_workspace_bytes": [ctypes.POINTER(Grid), ctypes.POINTER(ctypes.c_size_t)],
        "ss_create_case": [ctypes.POINTER(Grid), P, ctypes.c_size_t, P, ctypes.POINTER(P)],
        "ss_set_alloy": [P, ctypes.POINTER(Alloy)],
        "ss_set_boundary": [P, ctypes.c_int, ctypes.POINTER(BC)],
        "ss_step": [P, ctypes.c_int],
        "ss_step_graph": [P, ctypes.c_int],
        "ss_sync": [P],
        "ss_get_fields": [P, ctypes.c_uint, ctypes.POINTER(P), ctypes.c_int],
        "ss_set_fields": [P, ctypes.c_uint, ctypes.POINTER(P), ctypes.c_int],
        "ss_equilibrate": [P],
        "ss_get_stats": [P, ctypes.POINTER(Stats)],
        "ss_set_time": [P, ctypes.c_double],
        "ss_set_block_cap": [P, ctypes.c_int],
        "ss_set_tensor_cores": [P, ctypes.c_int],
        "ss_get_time": [P, ctypes.POINTER(ctypes.c_double)],
        "ss_destroy": [P],
        "ss_assemble": [P, ctypes.c_int],
        "ss_solve": [P, ctypes.c_int],
        "ss_get_system": [P, ctypes.c_int, ctypes.POINTER(P), ctypes.c_int],
        "ss_get_system_f32": [P, ctypes.c_int, ctypes.POINTER(P), ctypes.c_int],
        "ss_assemble_forward": [P, ctypes.c_int],
        "ss_convert_f64_to_f32": [P, P, ctypes.c_longlong, P],
        "ss_project": [P],
        "ss_lever": [P],
        "ss_set_profiling": [P, ctypes.c_int],
        "ss_get_profile": [P, ctypes.POINTER(Profile)],
        "ss_batch_workspace_bytes": [ctypes.POINTER(P), ctypes.c_int, ctypes.POINTER(ctypes.c_size_t)],
        "ss_batch_create": [ctypes.POINTER(P), ctypes.c_int, P, ctypes.c_size_t, P, ctypes.POINTER(P)],
        "ss_batch_set_schedule": [P, ctypes.c_double, ctypes.c_int],
        "ss_batch_get_teams": [P, ctypes.POINTER(ctypes.c_int)],
        "ss_batch_step": [P, ctypes.c_int],
        "ss_batch_sync": [P, ctypes.POINTER(ctypes.c_longlong)],
        "ss_batch_destroy": [P],
        "ss_set_wait_limit": [P, ctypes.c_longlong],
        "ss_wait_selftest": [P],
        "ss_tc_selftest": [P, P, P, P, ctypes.c_int, ctypes.c_int, ctypes.c_int],
        "ss_poisson_solve_noalloc": [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                     ctypes.c_double, ctypes.c_double, P, P, ctypes.c_double, ctypes.c_int,
                                     ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double), P],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    lib.ss_last_error.argtypes = []
    lib.ss_last_error.restype = ctypes.c_char_p
    return lib


def load(path=LIB_PATH):
    """Load libsolid.so (built by ``paper_2303_10783_gb300._build.build``)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError("libsolid.so is not built (%s); run __graft_entry__.build()" % path)
        _lib = _declare(ctypes.CDLL(path))
    return _lib


def check(status, allow=()):
    if status != SS_OK and status not in allow:
        raise SolidError(status, load().ss_last_error().decode())
    return status


def grid_struct(case, precision=SS_FP64):
    return Grid(case["dim"], case["nx"], case["ny"], case["nz"] if case["dim"] == 3 else 1,
                case["lx"], case["ly"], case["lz"], case["dt"], precision,
                case["tol_p"], case["tol_t"], case["max_it_p"], case["max_it_t"],
                {"mg": SS_PRECOND_MG, "jacobi": SS_PRECOND_JACOBI,
                 "dct": SS_PRECOND_DCT}[case.get("precond_p", "dct")])


def alloy_struct(case):
    a = case["alloy"]
    return Alloy(a["Tm"], a["m"], a["kp"], a["C0"], a["rho"], a["k"], a["cp"], a["L"], a["mu"], a["Dl"],
                 a["betaT"], a["betaC"], a["K0"], a["Ce"] if a.get("Ce") is not None else -1.0,
                 a["gravity"], a["darcy_eps"], case["T0"])


def workspace_bytes(case, precision=SS_FP64):
    n = ctypes.c_size_t(0)
    g = grid_struct(case, precision)
    check(load().ss_workspace_bytes(ctypes.byref(g), ctypes.byref(n)))
    return n.value


class Case:
    """One simulation case on the current CUDA device.

    ``case`` is a dict from :mod:`paper_2303_10783_gb300.cases`. The device
    workspace is a torch uint8 tensor owned by this object."""

    def __init__(self, case, precision=SS_FP64, stream=None):
        import torch
        self.lib = load()
        self.case = case
        self.dim = case["dim"]
        nx, ny, nz = case["nx"], case["ny"], case["nz"] if case["dim"] == 3 else 1
        self.shapes = {"u": (nz, ny, nx + 1), "v": (nz, ny + 1, nx), "w": (nz + 1, ny, nx)}
        for k in ("p", "T", "C", "gl", "Cl", "Cs"):
            self.shapes[k] = (nz, ny, nx)
        self.sys_shapes = {"u": self.shapes["u"], "v": self.shapes["v"], "w": self.shapes["w"]}
        for k in ("p", "C", "T"):
            self.sys_shapes[k] = (nz, ny, nx)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        g = grid_struct(case, precision)
        nbytes = workspace_bytes(case, precision)
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        h = ctypes.c_void_p()
        check(self.lib.ss_create_case(ctypes.byref(g), ctypes.c_void_p(self.workspace.data_ptr()), nbytes,
                                      ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h)))
        self.h = h
        al = alloy_struct(case)
        check(self.lib.ss_set_alloy(self.h, ctypes.byref(al)))
        for face in FACE_ID:
            if FACE_ID[face] // 2 >= self.dim:
                continue
            flow = SS_FREESLIP if face in case.get("slip", ()) else SS_NOSLIP
            if face in case["robin"]:
                hc, Text = case["robin"][face]
                self.set_boundary(face, SS_ROBIN, hc, Text, flow=flow)
            elif face in case.get("dirichlet", {}):
                Tw0, rate = case["dirichlet"][face]
                self.set_boundary(face, SS_DIRICHLET, 0.0, Tw0, rate, flow=flow)
            elif flow != SS_NOSLIP:
                self.set_boundary(face, SS_ADIABATIC, flow=flow)

    # -- C-ABI calls, same names
    def set_boundary(self, face, thermal, h=0.0, Text=0.0, dTdt=0.0, flow=SS_NOSLIP):
        bc = BC(thermal, h, Text, dTdt, flow)
        check(self.lib.ss_set_boundary(self.h, FACE_ID[face] if isinstance(face, str) else face, ctypes.byref(bc)))

    def set_block_cap(self, max_blocks):
        """At most ``max_blocks`` blocks per cooperative solver launch (0: no cap)."""
        check(self.lib.ss_set_block_cap(self.h, int(max_blocks)))

    def set_tensor_cores(self, mode):
        """Where the FP32 transforms form their products: "auto", "on" or "off"
        (or SS_TC_AUTO / SS_TC_ON / SS_TC_OFF)."""
        mode = {"auto": SS_TC_AUTO, "on": SS_TC_ON, "off": SS_TC_OFF}.get(mode, mode)
        check(self.lib.ss_set_tensor_cores(self.h, int(mode)))

    def set_wait_limit(self, polls):
        """Polls per device-side wait before it gives up (0: the default, about a second)."""
        check(self.lib.ss_set_wait_limit(self.h, int(polls)))

    def wait_selftest(self):
        """Enqueue a wait that nothing completes; the next sync reports SS_ETIMEOUT."""
        check(self.lib.ss_wait_selftest(self.h))

    def tc_selftest(self, a_ptr, b_ptr, d_ptr, n, k, transposed=False):
        """Enqueue d = a b^T (a: 128 x k, b: n x k, d: 128 x n; FP32 row-major
        device pointers, a and b stored transposed when asked) on the
        tensor-core path of the transform solvers."""
        check(self.lib.ss_tc_selftest(self.h, a_ptr, b_ptr, d_ptr, int(n), int(k), 1 if transposed else 0))

    def set_time(self, t):
        check(self.lib.ss_set_time(self.h, float(t)))

    def get_time(self):
        t = ctypes.c_double(0.0)
        check(self.lib.ss_get_time(self.h, ctypes.byref(t)))
        return t.value

    def step(self, n=1):
        check(self.lib.ss_step(self.h, n))

    def step_graph(self, n=1):
        check(self.lib.ss_step_graph(self.h, n))

    def sync(self, allow=()):
        return check(self.lib.ss_sync(self.h), allow)

    def equilibrate(self):
        check(self.lib.ss_equilibrate(self.h))

    def set_fields(self, fields):
        """``fields``: dict name -> numpy array (host) or CUDA tensor (device), float64, C-contiguous.
        Host sources are copied before the call returns; device sources are
        copied in stream order (after the caller's current stream's earlier
        work, before its later work)."""
        import torch
        mask = 0
        ptrs = (ctypes.c_void_p * 9)()
        keep = []
        on_dev = None
        for name, arr in fields.items():
            i = FIELD_ID[name]
            if name == "w" and self.dim != 3:
                continue
            if isinstance(arr, torch.Tensor):
                dev = True
                t = arr.to(dtype=torch.float64).contiguous()
                keep.append(t)
                ptrs[i] = t.data_ptr()
            else:
                dev = False
                a = np.ascontiguousarray(arr, dtype=np.float64)
                if a.size != int(np.prod(self.shapes[name])):
                    raise ValueError("field %s has %d values, expected shape %s" % (name, a.size, self.shapes[name]))
                keep.append(a)
                ptrs[i] = a.ctypes.data
            if on_dev is not None and on_dev != dev:
                raise ValueError("mix of host and device sources")
            on_dev = dev
            mask |= 1 << i
        if on_dev:
            # device sources: stream-ordered both ways, no host wait. The case's
            # stream waits for the caller's current stream (which produced the
            # sources), the caller's later work waits for the copies, and the
            # allocator keeps converted temporaries until the case's stream is done
            cur = torch.cuda.current_stream()
            self.stream.wait_stream(cur)
            check(self.lib.ss_set_fields(self.h, mask, ptrs, 1))
            for t in keep:
                t.record_stream(self.stream)
            cur.wait_stream(self.stream)
        else:
            check(self.lib.ss_set_fields(self.h, mask, ptrs, 0))

    def initialize(self, T, C):
        """Seeded initial fields: set T and C, then the equilibrium g_l, C_l, C_s."""
        self.set_fields({"T": T, "C": C})
        self.equilibrate()

    def get_fields(self, names=FIELDS, device=False, out=None):
        """Dict name -> numpy array (or CUDA tensor when ``device``) of the
        current fields; ``out`` may supply the destination arrays (e.g. pinned).
        Host copies wait for the case's stream; device copies are ordered
        before the caller's current stream's later work."""
        import torch
        names = [n for n in names if not (n == "w" and self.dim != 3)]
        ptrs = (ctypes.c_void_p * 9)()
        res = {}
        mask = 0
        for name in names:
            i = FIELD_ID[name]
            if out is not None and name in out:
                t = out[name]
                ptrs[i] = t.data_ptr() if isinstance(t, torch.Tensor) else t.ctypes.data
            elif device:
                t = torch.empty(self.shapes[name], dtype=torch.float64, device="cuda")
                ptrs[i] = t.data_ptr()
            else:
                t = np.empty(self.shapes[name], dtype=np.float64)
                ptrs[i] = t.ctypes.data
            res[name] = t
            mask |= 1 << i
        check(self.lib.ss_get_fields(self.h, mask, ptrs, int(device)))
        if device:
            # device copies are stream-ordered on the case's stream: order the
            # caller's current stream after them (no host wait)
            torch.cuda.current_stream().wait_stream(self.stream)
        if self.dim != 3 and not device and out is None:
            res.setdefault("w", np.zeros(self.shapes["w"]))
        return res

    def assemble(self, sys):
        check(self.lib.ss_assemble(self.h, SYS_ID[sys]))

    def solve(self, sys, allow=()):
        return check(self.lib.ss_solve(self.h, SYS_ID[sys]), allow)

    def get_system(self, sys):
        """Dict of the system's planes P, W, E, S, N, B, T, right-hand side b and solution x (numpy)."""
        shape = self.sys_shapes[sys]
        ptrs = (ctypes.c_void_p * 9)()
        out = {}
        for q, name in enumerate(PLANE_NAMES):
            if sys == "p" and q < 7:
                continue
            a = np.empty(shape, dtype=np.float64)
            ptrs[q] = a.ctypes.data
            out[name] = a
        check(self.lib.ss_get_system(self.h, SYS_ID[sys], ptrs, 0))
        return out

    def assemble_forward(self, sys):
        """Forward (residual-probing) assembly of ``sys``, a validation mode of assemble."""
        check(self.lib.ss_assemble_forward(self.h, SYS_ID[sys]))

    def get_system_f32(self, sys):
        """Dict of the FP32 planes P, W, E, S, N, B, T and inverse diagonal "idiag" (mixed cases)."""
        shape = self.sys_shapes[sys]
        ptrs = (ctypes.c_void_p * 8)()
        out = {}
        for q, name in enumerate(PLANE_NAMES[:7] + ("idiag",)):
            a = np.empty(shape, dtype=np.float32)
            ptrs[q] = a.ctypes.data
            out[name] = a
        check(self.lib.ss_get_system_f32(self.h, SYS_ID[sys], ptrs, 0))
        return out

    def project(self):
        check(self.lib.ss_project(self.h))

    def lever(self):
        check(self.lib.ss_lever(self.h))

    def stats(self, allow=(SS_ENOTCONV,)):
        s = Stats()
        st = check(self.lib.ss_get_stats(self.h, ctypes.byref(s)), allow)
        return dict(steps=s.steps, status=st,
                    iters={k: s.iters[i] for i, k in enumerate(SYSTEMS)},
                    refinements={k: s.refinements[i] for i, k in enumerate(SYSTEMS)},
                    relres={k: s.relres[i] for i, k in enumerate(SYSTEMS)},
                    jacobi={k: s.jacobi[i] for i, k in enumerate(SYSTEMS)})

    def set_profiling(self, on=True):
        check(self.lib.ss_set_profiling(self.h, int(bool(on))))

    def get_profile(self):
        """Accumulated ms and kernel launches per stage since the previous call."""
        p = Profile()
        check(self.lib.ss_get_profile(self.h, ctypes.byref(p)))
        return dict(ms={k: p.ms[i] for i, k in enumerate(PROF_NAMES)},
                    launches={k: p.launches[i] for i, k in enumerate(PROF_NAMES)}, kernels=p.kernels,
                    iters={k: p.iters[i] for i, k in enumerate(SYSTEMS)}, presolve_sweeps=p.presolve_sweeps,
                    jacobi={k: p.jacobi[i] for i, k in enumerate(SYSTEMS)})

    def close(self):
        if getattr(self, "h", None):
            self.lib.ss_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def convert_f64_to_f32(src):
    """The library's FP64 -> FP32 plane rounding applied to a CUDA float64 tensor."""
    import torch
    src = src.contiguous()
    dst = torch.empty(src.shape, dtype=torch.float32, device=src.device)
    check(load().ss_convert_f64_to_f32(ctypes.c_void_p(src.data_ptr()), ctypes.c_void_p(dst.data_ptr()),
                                       src.numel(), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)))
    return dst


class PackedBatch:
    """ss_batch: many cases stepped with one launch per stage (see include/solid.h).
    ``members`` are :class:`Case` objects (SS_MIXED, "dct" pressure solver);
    the batch's tables live in a torch uint8 workspace owned by this object."""

    def __init__(self, members, stream=None):
        import torch
        self.lib = load()
        self.members = list(members)
        n = len(self.members)
        arr = (ctypes.c_void_p * n)(*[m.h.value for m in self.members])
        nb = ctypes.c_size_t(0)
        check(self.lib.ss_batch_workspace_bytes(arr, n, ctypes.byref(nb)))
        self.stream = stream if stream is not None else torch.cuda.Stream()
        self.workspace = torch.empty(max(nb.value, 256), dtype=torch.uint8, device="cuda")
        h = ctypes.c_void_p()
        check(self.lib.ss_batch_create(arr, n, ctypes.c_void_p(self.workspace.data_ptr()), nb.value,
                                       ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h)))
        self.h = h

    def set_schedule(self, gamma, tile_rows):
        check(self.lib.ss_batch_set_schedule(self.h, float(gamma), int(tile_rows)))

    def teams(self):
        out = (ctypes.c_int * len(self.members))()
        check(self.lib.ss_batch_get_teams(self.h, out))
        return list(out)

    def step(self, n=1):
        check(self.lib.ss_batch_step(self.h, int(n)))

    def sync(self, allow=()):
        """Wait for the batch; returns (worst sticky status, kernels launched so far)."""
        k = ctypes.c_longlong(0)
        st = check(self.lib.ss_batch_sync(self.h, ctypes.byref(k)), allow)
        return st, k.value

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self.lib.ss_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

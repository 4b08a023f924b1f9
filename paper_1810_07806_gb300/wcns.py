"""Thin ctypes binding of libwcns (include/wcns.h): argument marshalling only.

Every step of the scheme runs in the library's CUDA kernels.  Arrays are
torch tensors on the CUDA device (PyTorch provides device memory and
streams); pointers and the current stream are passed through the C ABI.
Loading fails loudly when the library has not been built.
"""
import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libwcns.so")

OK, ERR_INVALID, ERR_NOMEM, ERR_NONPHYSICAL, ERR_TIMEOUT, ERR_BUSY, ERR_CUDA = range(7)
BC_TRANSMISSIVE, BC_PERIODIC, BC_REFLECTING, BC_FIXED = 0, 1, 2, 3
FLUX_ROE, FLUX_VANLEER, FLUX_AUSM = 0, 1, 2
DIFF_MD6, DIFF_HWCNS, DIFF_MND = 0, 1, 2
FP64, FP32 = 0, 1
W_TENO, W_JS, W_LINEAR, W_Z = 0, 1, 2, 3
SCALAR_ADVECTION, SCALAR_BURGERS = 0, 1


class WcnsError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("wcns status %d: %s" % (status, msg))
        self.status = status


class Grid(C.Structure):
    _fields_ = [("ndim", C.c_int), ("n", C.c_int * 3), ("lo", C.c_double * 3), ("hi", C.c_double * 3),
                ("bc", (C.c_int * 2) * 3), ("bc_state", ((C.c_double * 5) * 2) * 3), ("gravity", C.c_double * 3)]


class SchemeParams(C.Structure):
    _fields_ = [("flux", C.c_int), ("diff", C.c_int), ("weights", C.c_int), ("C", C.c_double),
                ("eps", C.c_double), ("CT", C.c_double), ("q", C.c_int), ("characteristic", C.c_int),
                ("precision", C.c_int), ("cfl", C.c_double), ("entropy_fix", C.c_int),
                ("eps_js", C.c_double)]


_lib = None


def lib():
    """Load libwcns.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libwcns.so is not built: run __graft_entry__.build() or "
                               "python -m paper_1810_07806_gb300.build")
        L = C.CDLL(LIB_PATH)
        vp, sz = C.c_void_p, C.c_size_t
        L.wcns_last_error.restype = C.c_char_p
        L.wcns_version.restype = C.c_char_p
        L.wcns_default_params.argtypes = [C.POINTER(SchemeParams)]
        L.wcns_create.argtypes = [C.POINTER(Grid), C.c_double, C.POINTER(SchemeParams), C.POINTER(vp)]
        L.wcns_destroy.argtypes = [vp]
        L.wcns_handle_bytes.argtypes = [vp]
        L.wcns_handle_bytes.restype = sz
        L.wcns_flags_bytes.argtypes = [vp]
        L.wcns_flags_bytes.restype = sz
        L.wcns_rhs.argtypes = [vp, vp, vp, vp, vp]
        L.wcns_step_rk3.argtypes = [vp, vp, C.c_double, C.POINTER(C.c_double), vp]
        L.wcns_advance.argtypes = [vp, vp, C.c_double, C.c_int, C.c_int, C.POINTER(C.c_double),
                                   C.POINTER(C.c_int), vp]
        L.wcns_conserved.argtypes = [vp, vp, C.POINTER(C.c_double), vp]
        L.wcns_cfl_dt.argtypes = [vp, vp, C.POINTER(C.c_double), vp]
        L.wcns_fallback_count.argtypes = [vp, C.POINTER(C.c_longlong), C.c_int, vp]
        L.wcns_profile.argtypes = [vp, C.c_int]
        L.wcns_profile_read.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(C.c_longlong)]
        L.wcns_launches_per_step.argtypes = [vp, C.c_int]
        L.wcns_launches_per_step.restype = C.c_int
        for f in ("wcns_create", "wcns_destroy", "wcns_rhs", "wcns_step_rk3", "wcns_advance",
                  "wcns_conserved", "wcns_cfl_dt", "wcns_fallback_count", "wcns_profile",
                  "wcns_profile_read"):
            getattr(L, f).restype = C.c_int
        _lib = L
    return _lib


def check(status):
    if status != OK:
        raise WcnsError(status, lib().wcns_last_error().decode())


def check_physical(status):
    """Like check(), but WCNS_ERR_NONPHYSICAL (the call completed; some faces
    used first-order values) is returned as True instead of raised."""
    if status == ERR_NONPHYSICAL:
        return True
    check(status)
    return False


def default_params(**kw):
    p = SchemeParams()
    lib().wcns_default_params(C.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def make_grid(ndim, n, lo, hi, periodic, bc_lo=None, bc_hi=None, bc_state=None, gravity=None):
    """periodic axes wrap; other axes are transmissive unless bc_lo / bc_hi
    give a kind per axis (BC_REFLECTING, BC_FIXED with bc_state[axis][side]
    the conserved state).  gravity: body force per unit mass."""
    g = Grid()
    g.ndim = ndim
    for a in range(3):
        g.n[a] = int(n[a]) if a < ndim else 1
        g.lo[a] = float(lo[a]) if a < ndim else 0.0
        g.hi[a] = float(hi[a]) if a < ndim else 1.0
        kind = BC_PERIODIC if (a < ndim and periodic[a]) else BC_TRANSMISSIVE
        g.bc[a][0] = kind
        g.bc[a][1] = kind
        if a < ndim and not periodic[a]:
            if bc_lo is not None and bc_lo[a] in (BC_REFLECTING, BC_FIXED):
                g.bc[a][0] = bc_lo[a]
            if bc_hi is not None and bc_hi[a] in (BC_REFLECTING, BC_FIXED):
                g.bc[a][1] = bc_hi[a]
        if bc_state is not None and a < len(bc_state) and bc_state[a] is not None:
            for sd in range(2):
                st = bc_state[a][sd]
                if st is not None:
                    for v in range(len(st)):
                        g.bc_state[a][sd][v] = float(st[v])
        g.gravity[a] = float(gravity[a]) if (gravity is not None and a < len(gravity)) else 0.0
    return g


def grid_of(pb):
    """The wcns_grid of an inputs.Problem (boundary kinds, fixed states, gravity)."""
    return make_grid(pb.ndim, pb.n, pb.lo, pb.hi, pb.periodic, getattr(pb, "bc_lo", None),
                     getattr(pb, "bc_hi", None), getattr(pb, "bc_state", None), getattr(pb, "gravity", None))


def _stream(stream):
    if stream is not None:
        return C.c_void_p(stream)
    import torch
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    return C.c_void_p(t.data_ptr())


class Solver:
    """One grid + scheme on the current CUDA device (a wcns_handle)."""

    def __init__(self, ndim, n, lo, hi, periodic, gamma=1.4, grid=None, **params):
        self.ndim = ndim
        self.n = tuple(int(v) for v in n[:ndim])
        self.nv = ndim + 2
        self.params = default_params(**params)
        self.grid = grid if grid is not None else make_grid(ndim, n, lo, hi, periodic)
        h = C.c_void_p()
        check(lib().wcns_create(C.byref(self.grid), gamma, C.byref(self.params), C.byref(h)))
        self.h = h
        # set when a synchronising step or advance reported first-order faces
        self.nonphysical = False

    @classmethod
    def for_problem(cls, pb, **params):
        return cls(pb.ndim, pb.n, pb.lo, pb.hi, pb.periodic, pb.gamma, grid=grid_of(pb), **params)

    def close(self):
        if getattr(self, "h", None):
            check(lib().wcns_destroy(self.h))
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle_bytes(self):
        return lib().wcns_handle_bytes(self.h)

    @property
    def flags_bytes(self):
        return lib().wcns_flags_bytes(self.h)

    def rhs(self, U, L, flags=None, stream=None):
        check(lib().wcns_rhs(self.h, _ptr(U), _ptr(L), _ptr(flags) if flags is not None else None,
                             _stream(stream)))

    def step(self, U, dt=0.0, want_dt=False, stream=None):
        d = C.c_double()
        st = lib().wcns_step_rk3(self.h, _ptr(U), float(dt), C.byref(d) if want_dt else None,
                                 _stream(stream))
        self.nonphysical |= check_physical(st)
        return d.value if want_dt else None

    def step_host(self, U_host, nsteps=1, stream=None):
        """wcns_step_rk3_host: nsteps CFL steps of a host FP64 state (a numpy
        array or a CPU torch tensor, pinned for speed), copied in and out by
        the library."""
        L = lib()
        L.wcns_step_rk3_host.argtypes = [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]
        L.wcns_step_rk3_host.restype = C.c_int
        ptr = U_host.ctypes.data if hasattr(U_host, "ctypes") else U_host.data_ptr()
        st = L.wcns_step_rk3_host(self.h, C.c_void_p(ptr), int(nsteps), _stream(stream))
        self.nonphysical |= check_physical(st)

    def advance(self, U, t_end, max_steps=10 ** 9, check_every=64, stream=None):
        """Returns (t reached, steps); sets self.nonphysical when faces fell
        back to first-order values during the run."""
        t = C.c_double()
        s = C.c_int()
        st = lib().wcns_advance(self.h, _ptr(U), float(t_end), int(min(max_steps, 2 ** 31 - 1)),
                                int(check_every), C.byref(t), C.byref(s), _stream(stream))
        self.nonphysical |= check_physical(st)
        return t.value, s.value

    def conserved(self, U, stream=None):
        out = (C.c_double * self.nv)()
        check(lib().wcns_conserved(self.h, _ptr(U), out, _stream(stream)))
        return list(out)

    def cfl_dt(self, U, stream=None):
        d = C.c_double()
        check(lib().wcns_cfl_dt(self.h, _ptr(U), C.byref(d), _stream(stream)))
        return d.value

    def fallback_count(self, reset=False, stream=None):
        c = C.c_longlong()
        check(lib().wcns_fallback_count(self.h, C.byref(c), int(reset), _stream(stream)))
        return c.value

    def profile(self, enable=True):
        check(lib().wcns_profile(self.h, int(enable)))

    def profile_read(self):
        ms = C.c_double()
        n = C.c_longlong()
        check(lib().wcns_profile_read(self.h, C.byref(ms), C.byref(n)))
        return ms.value, n.value

    def autotune(self, U, stream=None):
        """Pick the fastest tile configuration of each direction's FP32 sweep
        for this grid (returns the configuration per direction)."""
        L = lib()
        L.wcns_autotune.argtypes = [C.c_void_p, C.c_void_p, C.POINTER(C.c_int), C.c_void_p]
        L.wcns_autotune.restype = C.c_int
        out = (C.c_int * 3)()
        check(L.wcns_autotune(self.h, _ptr(U), out, _stream(stream)))
        return list(out)[: self.ndim]

    def tile_config(self, cfg=None):
        L = lib()
        L.wcns_tile_config.argtypes = [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_int)]
        L.wcns_tile_config.restype = C.c_int
        get = (C.c_int * 3)()
        st = (C.c_int * 3)(*(list(cfg) + [0, 0, 0])[:3]) if cfg is not None else None
        check(L.wcns_tile_config(self.h, st, get))
        return list(get)[: self.ndim]

    def launches_per_step(self, cfl_step=True):
        return lib().wcns_launches_per_step(self.h, int(cfl_step))


def step_rk3_noalloc(grid, gamma, params, U, dt=0.0, want_dt=False, stream=None):
    """wcns_step_rk3_noalloc: one FP64 RK3 step using the library's static
    device buffer instead of a handle (for callers that cannot allocate)."""
    L = lib()
    fn = L.wcns_step_rk3_noalloc
    fn.argtypes = [C.POINTER(Grid), C.c_double, C.POINTER(SchemeParams), C.c_void_p, C.c_double,
                   C.POINTER(C.c_double), C.c_void_p]
    fn.restype = C.c_int
    d = C.c_double()
    check(fn(C.byref(grid), float(gamma), C.byref(params), _ptr(U), float(dt),
             C.byref(d) if want_dt else None, _stream(stream)))
    return d.value if want_dt else None


def alu_probe(kind, stream=None):
    """wcns_alu_probe: TFLOP/s of FMA chains on every SM (0: FP32, 1: packed
    FP32, 2: FP64)."""
    L = lib()
    L.wcns_alu_probe.argtypes = [C.c_int, C.POINTER(C.c_double), C.c_void_p]
    L.wcns_alu_probe.restype = C.c_int
    t = C.c_double()
    check(L.wcns_alu_probe(int(kind), C.byref(t), _stream(stream)))
    return t.value


def _scalar_lines(u):
    if u.dim() == 1:
        return 1, u.shape[0], u.shape[0]
    if u.dim() != 2 or u.stride(1) != 1:
        raise ValueError("u must be (n,) or (count, n) with unit stride along n")
    return u.shape[0], u.shape[1], u.stride(0)


def _scalar_fns():
    L = lib()
    vp = C.c_void_p
    L.wcns_scalar_max_nodes.restype = C.c_int
    L.wcns_scalar_rhs.argtypes = [C.c_int, C.POINTER(SchemeParams), C.c_int, C.c_double, C.c_int, vp,
                                  C.c_longlong, vp, vp]
    L.wcns_scalar_run.argtypes = [C.c_int, C.POINTER(SchemeParams), C.c_int, C.c_double, C.c_double,
                                  C.c_int, C.c_int, vp, C.c_longlong, vp]
    L.wcns_scalar_rhs.restype = C.c_int
    L.wcns_scalar_run.restype = C.c_int
    return L


def scalar_max_nodes():
    """Largest line the scalar solver accepts on the current device."""
    return _scalar_fns().wcns_scalar_max_nodes()


def scalar_rhs(kind, u, h, L=None, stream=None, **params):
    """wcns_scalar_rhs: L = -f'(u) (Eq. 6 flux, Eq. 3 derivative) for each
    periodic line of u, a float64 CUDA tensor of shape (n,) or (count, n)."""
    count, n, ld = _scalar_lines(u)
    if L is None:
        L = u.new_empty(u.shape)
    if L.shape != u.shape or L.stride() != u.stride():
        raise ValueError("L must have the layout of u")
    p = default_params(**params)
    check(_scalar_fns().wcns_scalar_rhs(int(kind), C.byref(p), n, float(h), count, _ptr(u), ld, _ptr(L),
                                        _stream(stream)))
    return L


def scalar_run(kind, u, h, t_end, nsteps, stream=None, **params):
    """wcns_scalar_run: nsteps SSP-RK3 steps of size t_end / nsteps on each
    periodic line of u (float64 CUDA tensor (n,) or (count, n)), in place."""
    count, n, ld = _scalar_lines(u)
    p = default_params(**params)
    check(_scalar_fns().wcns_scalar_run(int(kind), C.byref(p), n, float(h), float(t_end), int(nsteps), count,
                                        _ptr(u), ld, _stream(stream)))
    return u


class Batch:
    """A wcns_batch: many independent grids of one dimension and precision
    advanced together (per-instance sizes, boundary rules, time steps and
    end times)."""

    def __init__(self, ndim, max_nodes, max_instances, gamma=1.4, **params):
        L = lib()
        L.wcns_batch_create.argtypes = [C.c_int, C.c_double, C.POINTER(SchemeParams), C.c_longlong, C.c_int,
                                        C.POINTER(C.c_void_p)]
        L.wcns_batch_destroy.argtypes = [C.c_void_p]
        L.wcns_batch_bytes.argtypes = [C.c_void_p]
        L.wcns_batch_bytes.restype = C.c_size_t
        L.wcns_batch_add.argtypes = [C.c_void_p, C.POINTER(Grid), C.c_void_p, C.c_int, C.c_double,
                                     C.POINTER(C.c_int), C.c_void_p]
        L.wcns_batch_remove.argtypes = [C.c_void_p, C.c_int]
        L.wcns_batch_step.argtypes = [C.c_void_p, C.c_int, C.POINTER(C.c_int), C.c_void_p]
        L.wcns_batch_run.argtypes = [C.c_void_p, C.c_int, C.c_int, C.POINTER(C.c_int), C.c_void_p]
        L.wcns_batch_read.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.POINTER(C.c_double),
                                      C.POINTER(C.c_int), C.c_void_p]
        for f in ("wcns_batch_create", "wcns_batch_destroy", "wcns_batch_add", "wcns_batch_remove",
                  "wcns_batch_step", "wcns_batch_run", "wcns_batch_read"):
            getattr(L, f).restype = C.c_int
        self.ndim = ndim
        self.nv = ndim + 2
        self.params = default_params(**params)
        h = C.c_void_p()
        check(L.wcns_batch_create(ndim, gamma, C.byref(self.params), int(max_nodes), int(max_instances), C.byref(h)))
        self.h = h
        self.grids = {}
        self.nonphysical = {}   # slot -> True when its read reported first-order faces

    def close(self):
        if getattr(self, "h", None):
            check(lib().wcns_batch_destroy(self.h))
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def nbytes(self):
        return lib().wcns_batch_bytes(self.h)

    def add(self, pb, U0=None, t_end=None, stream=None):
        """Add a Problem (inputs.Problem); U0: a CUDA tensor or a numpy array
        (defaults to pb.U0).  Returns the slot."""
        import numpy as np
        g = grid_of(pb)
        U0 = pb.U0 if U0 is None else U0
        slot = C.c_int()
        if isinstance(U0, np.ndarray):
            U0 = np.ascontiguousarray(U0, dtype=np.float64)
            check(lib().wcns_batch_add(self.h, C.byref(g), U0.ctypes.data_as(C.c_void_p), 0,
                                       float(pb.t_end if t_end is None else t_end), C.byref(slot), _stream(stream)))
        else:
            check(lib().wcns_batch_add(self.h, C.byref(g), _ptr(U0), 1,
                                       float(pb.t_end if t_end is None else t_end), C.byref(slot), _stream(stream)))
        self.grids[slot.value] = (pb.ndim, tuple(pb.n))
        return slot.value

    def remove(self, slot):
        check(lib().wcns_batch_remove(self.h, int(slot)))
        self.grids.pop(slot, None)

    def step(self, nsteps=1, stream=None):
        a = C.c_int()
        check(lib().wcns_batch_step(self.h, int(nsteps), C.byref(a), _stream(stream)))
        return a.value

    def launch_mode(self, mode):
        """0: one CTA per tile (tile table); 1: persistent CTAs taking tiles
        from a device counter."""
        L = lib()
        L.wcns_batch_launch_mode.argtypes = [C.c_void_p, C.c_int]
        L.wcns_batch_launch_mode.restype = C.c_int
        check(L.wcns_batch_launch_mode(self.h, int(mode)))

    def autotune(self, steps=5, stream=None):
        """Time both launch forms on the current instances, keep the faster
        (state unchanged).  Returns (mode kept, [ms per step of each form])."""
        L = lib()
        L.wcns_batch_autotune.argtypes = [C.c_void_p, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_double),
                                          C.c_void_p]
        L.wcns_batch_autotune.restype = C.c_int
        m = C.c_int()
        ms = (C.c_double * 2)()
        check(L.wcns_batch_autotune(self.h, int(steps), C.byref(m), ms, _stream(stream)))
        return m.value, [ms[0], ms[1]]

    def run(self, max_steps=10 ** 9, check_every=32, stream=None):
        s = C.c_int()
        check(lib().wcns_batch_run(self.h, int(min(max_steps, 2 ** 31 - 1)), int(check_every), C.byref(s),
                                   _stream(stream)))
        return s.value

    def read(self, slot, out=None, stream=None):
        """Returns (U as a numpy array or the given CUDA tensor, t, steps)."""
        import numpy as np
        t = C.c_double()
        st = C.c_int()
        nd, n = self.grids[slot]
        shape = (nd + 2,) + tuple(reversed(n))
        if out is None:
            host = np.empty(shape, dtype=np.float64)
            r = lib().wcns_batch_read(self.h, int(slot), host.ctypes.data_as(C.c_void_p), 0, C.byref(t),
                                      C.byref(st), _stream(stream))
            out = host
        else:
            r = lib().wcns_batch_read(self.h, int(slot), _ptr(out), 1, C.byref(t), C.byref(st), _stream(stream))
        self.nonphysical[slot] = check_physical(r)
        return out, t.value, st.value


class Request(C.Structure):
    _fields_ = [("grid", Grid), ("gamma", C.c_double), ("params", SchemeParams),
                ("U0", C.POINTER(C.c_double)), ("t_end", C.c_double), ("tag", C.c_uint64)]


class Result(C.Structure):
    _fields_ = [("ticket", C.c_uint64), ("tag", C.c_uint64), ("status", C.c_int), ("ndim", C.c_int),
                ("n", C.c_int * 3), ("precision", C.c_int), ("t", C.c_double), ("steps", C.c_int),
                ("U", C.POINTER(C.c_double)), ("t_submit", C.c_double), ("t_admit", C.c_double),
                ("t_done", C.c_double)]


class ServerConfig(C.Structure):
    _fields_ = [("hbm_budget_bytes", C.c_size_t), ("max_instances_per_class", C.c_int),
                ("max_nodes_per_class", C.c_longlong), ("steps_per_tick", C.c_int)]


class ServerStats(C.Structure):
    _fields_ = [("queued", C.c_int), ("max_queue", C.c_int), ("max_running", C.c_int),
                ("admitted", C.c_longlong), ("completed", C.c_longlong), ("ticks", C.c_longlong),
                ("steps", C.c_longlong), ("bytes_reserved", C.c_size_t)]


class Server:
    """A wcns_server: continuous batching of solve requests on the current
    CUDA device.  submit() queues a problem; poll() returns finished ones as
    dicts with the final state (numpy), time, steps and timestamps."""

    def __init__(self, hbm_budget_bytes=8 << 30, max_instances_per_class=256, max_nodes_per_class=0,
                 steps_per_tick=16):
        L = lib()
        L.wcns_server_default_config.argtypes = [C.POINTER(ServerConfig)]
        L.wcns_server_create.argtypes = [C.POINTER(ServerConfig), C.POINTER(C.c_void_p)]
        L.wcns_server_destroy.argtypes = [C.c_void_p]
        L.wcns_batch_submit.argtypes = [C.c_void_p, C.POINTER(Request), C.POINTER(C.c_uint64)]
        L.wcns_serve_poll.argtypes = [C.c_void_p, C.POINTER(Result), C.c_int, C.POINTER(C.c_int), C.c_int]
        L.wcns_result_free.argtypes = [C.POINTER(Result)]
        L.wcns_server_stats.argtypes = [C.c_void_p, C.POINTER(ServerStats)]
        for f in ("wcns_server_create", "wcns_server_destroy", "wcns_batch_submit", "wcns_serve_poll",
                  "wcns_server_stats"):
            getattr(L, f).restype = C.c_int
        cfg = ServerConfig(int(hbm_budget_bytes), int(max_instances_per_class), int(max_nodes_per_class),
                           int(steps_per_tick))
        h = C.c_void_p()
        check(L.wcns_server_create(C.byref(cfg), C.byref(h)))
        self.h = h
        self.shapes = {}

    def close(self):
        if getattr(self, "h", None):
            check(lib().wcns_server_destroy(self.h))
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, pb, tag=0, t_end=None, **params):
        import numpy as np
        U0 = np.ascontiguousarray(pb.U0, dtype=np.float64)
        req = Request()
        req.grid = grid_of(pb)
        req.gamma = pb.gamma
        req.params = default_params(**params)
        req.U0 = U0.ctypes.data_as(C.POINTER(C.c_double))
        req.t_end = float(pb.t_end if t_end is None else t_end)
        req.tag = int(tag)
        ticket = C.c_uint64()
        check(lib().wcns_batch_submit(self.h, C.byref(req), C.byref(ticket)))
        self.shapes[ticket.value] = (pb.ndim + 2,) + tuple(reversed(pb.n[:pb.ndim]))
        return ticket.value

    def poll(self, max_results=64, timeout_us=0):
        import numpy as np
        arr = (Result * max_results)()
        n = C.c_int()
        st = lib().wcns_serve_poll(self.h, arr, max_results, C.byref(n), int(timeout_us))
        if st not in (OK, ERR_TIMEOUT):
            check(st)
        out = []
        for k in range(n.value):
            r = arr[k]
            shape = self.shapes.pop(r.ticket, None)
            U = None
            if r.U and shape is not None:
                U = np.ctypeslib.as_array(r.U, shape=(int(np.prod(shape)),)).reshape(shape).copy()
            out.append(dict(ticket=r.ticket, tag=r.tag, status=r.status, t=r.t, steps=r.steps, U=U,
                            t_submit=r.t_submit, t_admit=r.t_admit, t_done=r.t_done, precision=r.precision))
            lib().wcns_result_free(C.byref(arr[k]))
        return out

    def stats(self):
        s = ServerStats()
        check(lib().wcns_server_stats(self.h, C.byref(s)))
        return {f: getattr(s, f) for f, _ in ServerStats._fields_}

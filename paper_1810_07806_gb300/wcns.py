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
BC_TRANSMISSIVE, BC_PERIODIC = 0, 1
FLUX_ROE, FLUX_VANLEER = 0, 1
FP64, FP32 = 0, 1


class WcnsError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("wcns status %d: %s" % (status, msg))
        self.status = status


class Grid(C.Structure):
    _fields_ = [("ndim", C.c_int), ("n", C.c_int * 3), ("lo", C.c_double * 3), ("hi", C.c_double * 3),
                ("bc", (C.c_int * 2) * 3)]


class SchemeParams(C.Structure):
    _fields_ = [("flux", C.c_int), ("diff", C.c_int), ("weights", C.c_int), ("C", C.c_double),
                ("eps", C.c_double), ("CT", C.c_double), ("q", C.c_int), ("characteristic", C.c_int),
                ("precision", C.c_int), ("cfl", C.c_double), ("entropy_fix", C.c_int)]


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


def default_params(**kw):
    p = SchemeParams()
    lib().wcns_default_params(C.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def make_grid(ndim, n, lo, hi, periodic):
    g = Grid()
    g.ndim = ndim
    for a in range(3):
        g.n[a] = int(n[a]) if a < ndim else 1
        g.lo[a] = float(lo[a]) if a < ndim else 0.0
        g.hi[a] = float(hi[a]) if a < ndim else 1.0
        kind = BC_PERIODIC if (a < ndim and periodic[a]) else BC_TRANSMISSIVE
        g.bc[a][0] = kind
        g.bc[a][1] = kind
    return g


def _stream(stream):
    if stream is not None:
        return C.c_void_p(stream)
    import torch
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    return C.c_void_p(t.data_ptr())


class Solver:
    """One grid + scheme on the current CUDA device (a wcns_handle)."""

    def __init__(self, ndim, n, lo, hi, periodic, gamma=1.4, **params):
        self.ndim = ndim
        self.n = tuple(int(v) for v in n[:ndim])
        self.nv = ndim + 2
        self.params = default_params(**params)
        self.grid = make_grid(ndim, n, lo, hi, periodic)
        h = C.c_void_p()
        check(lib().wcns_create(C.byref(self.grid), gamma, C.byref(self.params), C.byref(h)))
        self.h = h

    @classmethod
    def for_problem(cls, pb, **params):
        return cls(pb.ndim, pb.n, pb.lo, pb.hi, pb.periodic, pb.gamma, **params)

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
        check(lib().wcns_step_rk3(self.h, _ptr(U), float(dt), C.byref(d) if want_dt else None,
                                  _stream(stream)))
        return d.value if want_dt else None

    def advance(self, U, t_end, max_steps=10 ** 9, check_every=64, stream=None):
        t = C.c_double()
        s = C.c_int()
        check(lib().wcns_advance(self.h, _ptr(U), float(t_end), int(min(max_steps, 2 ** 31 - 1)),
                                 int(check_every), C.byref(t), C.byref(s), _stream(stream)))
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

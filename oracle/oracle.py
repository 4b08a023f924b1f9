"""ctypes wrapper around the C oracle (liboracle.so).

TEST INFRASTRUCTURE ONLY: only the test suite, the package smoke check and
the benchmark's CPU-baseline leg may import this module.  Arrays are numpy
float64, SoA layout U[var][z][y][x] (x fastest).
"""
import ctypes as C
import numpy as np

from . import build as _build

FLUX_ROE, FLUX_VANLEER, FLUX_AUSM = 0, 1, 2
DIFF_MD, DIFF_HWCNS, DIFF_MND = 0, 1, 2
BC_AUTO, BC_REFLECT, BC_FIXED = 0, 2, 3
W_TENO, W_JS, W_LINEAR, W_Z = 0, 1, 2, 3

_dp = C.POINTER(C.c_double)
_u8p = C.POINTER(C.c_uint8)


class OraCfg(C.Structure):
    _fields_ = [
        ("ndim", C.c_int), ("n", C.c_int * 3), ("h", C.c_double * 3), ("periodic", C.c_int * 3),
        ("gamma", C.c_double), ("flux", C.c_int), ("weights", C.c_int),
        ("C", C.c_double), ("eps", C.c_double), ("CT", C.c_double), ("q", C.c_int),
        ("eps_js", C.c_double), ("characteristic", C.c_int), ("diff", C.c_int),
        ("bc_lo", C.c_int * 3), ("bc_hi", C.c_int * 3), ("bc_state", ((C.c_double * 5) * 2) * 3),
        ("gravity", C.c_double * 3),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(_build.build())
        L = _lib
        L.ora_interp_left.restype = C.c_double
        L.ora_interp_left.argtypes = [C.POINTER(OraCfg), _dp, C.c_int, C.POINTER(C.c_int), _dp, _dp]
        L.ora_teno_chi.restype = C.c_int
        L.ora_teno_chi.argtypes = [C.POINTER(OraCfg), _dp, _dp, _dp, _dp]
        L.ora_md_coeffs.argtypes = [_dp]
        L.ora_phys_flux.argtypes = [C.c_int, C.c_int, C.c_double, _dp, _dp]
        L.ora_roe_eigen.argtypes = [C.c_int, C.c_int, C.c_double, _dp, _dp, _dp, _dp, _dp]
        L.ora_roe_flux.argtypes = [C.c_int, C.c_int, C.c_double, _dp, _dp, _dp]
        L.ora_vanleer_half.argtypes = [C.c_int, C.c_int, C.c_double, _dp, C.c_int, _dp]
        L.ora_ausm_flux.argtypes = [C.c_int, C.c_int, C.c_double, _dp, _dp, _dp]
        L.ora_ausm_split.argtypes = [C.c_double, C.c_double, C.c_int, _dp, _dp]
        L.ora_diff_coeffs.argtypes = [C.c_int, _dp]
        L.ora_flags_offset.restype = C.c_long
        L.ora_flags_offset.argtypes = [C.POINTER(OraCfg), C.c_int]
        L.ora_flags_size.restype = C.c_long
        L.ora_flags_size.argtypes = [C.POINTER(OraCfg)]
        L.ora_euler_rhs.restype = C.c_long
        L.ora_euler_rhs.argtypes = [C.POINTER(OraCfg), _dp, _dp, _u8p, _dp, _dp]
        L.ora_euler_rhs_at.restype = C.c_long
        L.ora_euler_rhs_at.argtypes = [C.POINTER(OraCfg), _dp, C.c_long, C.POINTER(C.c_long), _dp]
        L.ora_euler_rhs_lines.restype = C.c_long
        L.ora_euler_rhs_lines.argtypes = [C.POINTER(OraCfg), _dp, _dp, C.c_int, C.c_long, C.c_long]
        L.ora_cfl_dt.restype = C.c_double
        L.ora_cfl_dt.argtypes = [C.POINTER(OraCfg), _dp, C.c_double]
        L.ora_rk3_step.restype = C.c_long
        L.ora_rk3_step.argtypes = [C.POINTER(OraCfg), _dp, C.c_double]
        L.ora_euler_run.restype = C.c_long
        L.ora_euler_run.argtypes = [C.POINTER(OraCfg), _dp, C.c_double, C.c_double, C.c_int,
                                    _dp, C.POINTER(C.c_int)]
        L.ora_conserved.argtypes = [C.POINTER(OraCfg), _dp, _dp]
        L.ora_scalar_rhs.argtypes = [C.POINTER(OraCfg), C.c_int, C.c_int, C.c_double, _dp, _dp]
        L.ora_scalar_run.argtypes = [C.POINTER(OraCfg), C.c_int, C.c_int, C.c_double, C.c_double,
                                     C.c_int, _dp]
    return _lib


def _p(a):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_dp)


def make_cfg(ndim=1, n=(1, 1, 1), h=(1.0, 1.0, 1.0), periodic=(0, 0, 0), gamma=1.4,
             flux=FLUX_ROE, weights=W_TENO, C_=1.0, eps=1e-40, CT=1e-5, q=6, eps_js=1e-6,
             characteristic=1, diff=DIFF_MD, bc_lo=(0, 0, 0), bc_hi=(0, 0, 0), bc_state=None,
             gravity=(0.0, 0.0, 0.0)):
    """Scheme constants default to the paper's: C = 1, eps = 1e-40, q = 6 (Eq. 16),
    C_T = 1e-5 (Sec. 2.3), JS eps = 1e-6 (Eq. 14), MD differencing (Eq. 3).
    bc_lo / bc_hi: BC_AUTO (periodic flag), BC_REFLECT or BC_FIXED per axis;
    bc_state[axis][side] = conserved state of a FIXED side; gravity = body
    force per unit mass."""
    c = OraCfg()
    c.ndim = ndim
    for a in range(3):
        c.n[a] = int(n[a]) if a < len(n) else 1
        c.h[a] = float(h[a]) if a < len(h) else 1.0
        c.periodic[a] = int(periodic[a]) if a < len(periodic) else 0
    c.gamma, c.flux, c.weights = gamma, flux, weights
    c.C, c.eps, c.CT, c.q, c.eps_js, c.characteristic = C_, eps, CT, q, eps_js, characteristic
    c.diff = diff
    for a in range(3):
        c.bc_lo[a] = int(bc_lo[a]) if a < len(bc_lo) else 0
        c.bc_hi[a] = int(bc_hi[a]) if a < len(bc_hi) else 0
        c.gravity[a] = float(gravity[a]) if a < len(gravity) else 0.0
        if bc_state is not None and a < len(bc_state):
            for side in range(2):
                st = bc_state[a][side]
                if st is not None:
                    for v in range(len(st)):
                        c.bc_state[a][side][v] = float(st[v])
    return c


def interp_left(cfg, s, force_flags=-1):
    s = np.ascontiguousarray(s, dtype=np.float64)
    fl = C.c_int()
    m = C.c_double()
    ld = C.c_double()
    u = lib().ora_interp_left(C.byref(cfg), _p(s), int(force_flags), C.byref(fl), C.byref(m), C.byref(ld))
    return u, fl.value, m.value, ld.value


def teno_chi(cfg, s):
    s = np.ascontiguousarray(s, dtype=np.float64)
    chi = np.zeros(3)
    chil = np.zeros(3)
    beta = np.zeros(3)
    fl = lib().ora_teno_chi(C.byref(cfg), _p(s), _p(chi), _p(chil), _p(beta))
    return fl, chi, chil, beta


def md_coeffs():
    a = np.zeros(3)
    lib().ora_md_coeffs(_p(a))
    return a


def diff_coeffs(diff):
    """Coefficients of Eq. 3, 4 or 5 as the oracle uses them."""
    a = np.zeros(3)
    lib().ora_diff_coeffs(int(diff), _p(a))
    return a


def ausm_flux(nd, d, gamma, UL, UR):
    F = np.zeros(nd + 2)
    lib().ora_ausm_flux(nd, d, gamma, _p(np.ascontiguousarray(UL, dtype=np.float64)),
                        _p(np.ascontiguousarray(UR, dtype=np.float64)), _p(F))
    return F


def ausm_split(M, p, sign):
    """(M^+-, p^+-) of one side (sign = +1 or -1)."""
    Ms, ps = C.c_double(), C.c_double()
    lib().ora_ausm_split(float(M), float(p), int(sign), C.byref(Ms), C.byref(ps))
    return Ms.value, ps.value


def phys_flux(nd, d, gamma, U):
    U = np.ascontiguousarray(U, dtype=np.float64)
    F = np.zeros(nd + 2)
    lib().ora_phys_flux(nd, d, gamma, _p(U), _p(F))
    return F


def roe_eigen(nd, d, gamma, Ua, Ub):
    nv = nd + 2
    Ua = np.ascontiguousarray(Ua, dtype=np.float64)
    Ub = np.ascontiguousarray(Ub, dtype=np.float64)
    R = np.zeros((nv, nv))
    L = np.zeros((nv, nv))
    lam = np.zeros(nv)
    lib().ora_roe_eigen(nd, d, gamma, _p(Ua), _p(Ub), _p(R), _p(L), _p(lam))
    return R, L, lam


def roe_flux(nd, d, gamma, UL, UR):
    F = np.zeros(nd + 2)
    lib().ora_roe_flux(nd, d, gamma, _p(np.ascontiguousarray(UL, dtype=np.float64)),
                       _p(np.ascontiguousarray(UR, dtype=np.float64)), _p(F))
    return F


def vanleer_half(nd, d, gamma, U, sign):
    F = np.zeros(nd + 2)
    lib().ora_vanleer_half(nd, d, gamma, _p(np.ascontiguousarray(U, dtype=np.float64)), int(sign), _p(F))
    return F


def flags_size(cfg):
    return lib().ora_flags_size(C.byref(cfg))


def flags_offset(cfg, d):
    return lib().ora_flags_offset(C.byref(cfg), d)


def euler_rhs(cfg, U, want_flags=False):
    """Returns (L, flags or None, margin or None, fallback_faces, chi_literal_dev)."""
    U = np.ascontiguousarray(U, dtype=np.float64)
    L = np.empty_like(U)
    fl = mg = None
    fp = C.cast(None, _u8p)
    mp = C.cast(None, _dp)
    if want_flags:
        sz = flags_size(cfg)
        fl = np.zeros(sz, dtype=np.uint8)
        mg = np.zeros(sz, dtype=np.float64)
        fp = fl.ctypes.data_as(_u8p)
        mp = _p(mg)
    ld = C.c_double()
    np_ = lib().ora_euler_rhs(C.byref(cfg), _p(U), _p(L), fp, mp, C.byref(ld))
    return L, fl, mg, np_, ld.value


def euler_rhs_at(cfg, U, idx):
    """RHS at the flattened node indices idx (x fastest): array [nv, len(idx)]."""
    U = np.ascontiguousarray(U, dtype=np.float64)
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    out = np.zeros((cfg.ndim + 2, idx.size))
    lib().ora_euler_rhs_at(C.byref(cfg), _p(U), idx.size, idx.ctypes.data_as(C.POINTER(C.c_long)), _p(out))
    return out


def euler_rhs_lines(cfg, U, L, d, line_lo, line_hi):
    """Add direction-d contributions of lines [line_lo, line_hi) into L (in place)."""
    return lib().ora_euler_rhs_lines(C.byref(cfg), _p(U), _p(L), d, line_lo, line_hi)


def cfl_dt(cfg, U, cfl):
    return lib().ora_cfl_dt(C.byref(cfg), _p(np.ascontiguousarray(U, dtype=np.float64)), cfl)


def rk3_step(cfg, U, dt):
    """In place on U (float64, contiguous). Returns fallback face count."""
    return lib().ora_rk3_step(C.byref(cfg), _p(U), dt)


def euler_run(cfg, U, cfl, t_end, max_steps=10 ** 9):
    """In place on U. Returns (t, steps, fallback faces)."""
    t = C.c_double()
    s = C.c_int()
    np_ = lib().ora_euler_run(C.byref(cfg), _p(U), cfl, t_end, int(max_steps), C.byref(t), C.byref(s))
    return t.value, s.value, np_


def conserved(cfg, U):
    out = np.zeros(cfg.ndim + 2)
    lib().ora_conserved(C.byref(cfg), _p(np.ascontiguousarray(U, dtype=np.float64)), _p(out))
    return out


def scalar_rhs(cfg, kind, u, h):
    u = np.ascontiguousarray(u, dtype=np.float64)
    L = np.empty_like(u)
    lib().ora_scalar_rhs(C.byref(cfg), kind, u.size, h, _p(u), _p(L))
    return L


def scalar_run(cfg, kind, u, h, t_end, nsteps):
    u = np.array(u, dtype=np.float64)
    lib().ora_scalar_run(C.byref(cfg), kind, u.size, h, t_end, int(nsteps), _p(u))
    return u

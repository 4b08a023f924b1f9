"""Pins of the oracle's Rayleigh-Taylor ingredients (Sec. 3.9): reflecting
walls, fixed-state boundaries and the body-force source (0, 0, rho, rho v).

The paper shows the flow only as figures, so each ingredient is pinned by
what the physics and the discretisation fix: hydrostatic balance (which
fixes the sign and size of the source against the pressure gradient),
conservation of mass, tangential momentum and energy between reflecting
walls, mirror symmetry of the configuration about x = 1/8, exact rest
states, and the source of a uniform state.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1810_07806_gb300 import inputs


def ora_cfg(pb, flux=O.FLUX_ROE, **kw):
    oc = lambda k: k if k in (O.BC_REFLECT, O.BC_FIXED) else O.BC_AUTO
    return O.make_cfg(ndim=pb.ndim, n=pb.n, h=pb.h, periodic=pb.periodic, gamma=pb.gamma, flux=flux,
                      bc_lo=tuple(oc(k) for k in pb.bc_lo), bc_hi=tuple(oc(k) for k in pb.bc_hi),
                      bc_state=pb.bc_state, gravity=pb.gravity, **kw)


def _with(pb, U=None, **kw):
    out = inputs.Problem(**{**pb.__dict__, **kw})
    if U is not None:
        out.U0 = np.ascontiguousarray(U)
    return out


@pytest.mark.parametrize("flux", [O.FLUX_ROE, O.FLUX_VANLEER, O.FLUX_AUSM])
def test_hydrostatic_layers_are_in_balance_away_from_interface_and_ends(flux):
    """Without the perturbation the two layers are hydrostatic: dp/dy = rho g.
    Pressure, density and energy are linear (or constant) in y within a
    layer, the interpolation and Eq. 3 are exact for them, so the RHS
    vanishes to round-off except near the interface and the fixed ends.  A
    source of the wrong sign or size leaves 2 rho there."""
    pb = inputs.rayleigh_taylor(8, amp=0.0)
    L = O.euler_rhs(ora_cfg(pb, flux), pb.U0)[0]
    ny = pb.n[1]
    rows = [j for j in range(ny) if 6 <= j < ny - 6 and abs(j - ny // 2) >= 6]
    assert len(rows) > 0
    assert np.max(np.abs(L[:, rows, :])) <= 1e-12
    # near the fixed ends the constant ghost states are not hydrostatic
    assert np.max(np.abs(L[2, :3, :])) > 1e-3


def test_source_of_a_uniform_state():
    """Uniform state, periodic box, g = (0.3, -0.7): L = (0, rho g, rho u.g)."""
    g = (0.3, -0.7)
    n = (9, 7)
    U = inputs.prim_to_cons(np.full((7, 9), 1.7), [np.full((7, 9), 0.4), np.full((7, 9), -0.25)],
                            np.full((7, 9), 0.9), 1.4)
    cfg = O.make_cfg(ndim=2, n=n, h=(0.1, 0.2), periodic=(1, 1), gravity=g)
    L = O.euler_rhs(cfg, U)[0]
    assert np.all(L[0] == 0.0)
    assert np.allclose(L[1], 1.7 * 0.3, rtol=1e-15, atol=0)
    assert np.allclose(L[2], -1.7 * 0.7, rtol=1e-15, atol=0)
    assert np.allclose(L[3], 1.7 * (0.4 * 0.3 + 0.25 * 0.7), rtol=1e-14, atol=0)


def test_rest_states_between_walls_and_fixed_ends_are_exact():
    """A fluid at rest equal to both fixed states, between reflecting walls,
    without gravity: every ghost equals the interior, the RHS is zero."""
    pb = inputs.rayleigh_taylor(8)
    st = inputs.prim_to_cons(np.array(1.3), [np.array(0.0), np.array(0.0)], np.array(0.8), pb.gamma)
    U = np.empty_like(pb.U0)
    for v in range(4):
        U[v] = st[v]
    rest = _with(pb, U, bc_state=((None, None), (tuple(st), tuple(st)), (None, None)),
                 gravity=(0.0, 0.0, 0.0))
    for flux in (O.FLUX_ROE, O.FLUX_VANLEER, O.FLUX_AUSM):
        L = O.euler_rhs(ora_cfg(rest, flux), U)[0]
        assert np.max(np.abs(L)) <= 1e-15


def test_reflecting_walls_conserve_mass_tangential_momentum_and_energy():
    """Reflecting x walls, periodic y: the wall face carries no mass, no
    tangential momentum and no energy (the normal velocity there is zero by
    symmetry), so those totals stay constant; the normal momentum does not
    (the walls push)."""
    rng = np.random.default_rng(3)
    nx, ny = 24, 20
    x = (np.arange(nx) + 0.5) / nx
    y = np.arange(ny) / ny
    Y, X = np.meshgrid(y, x, indexing="ij")
    rho = 1 + 0.3 * np.sin(2 * np.pi * X + 1) * np.cos(2 * np.pi * Y)
    u = 0.3 * np.sin(2 * np.pi * Y + rng.uniform())
    v = 0.2 * np.cos(2 * np.pi * X)
    p = 1 + 0.2 * np.cos(2 * np.pi * (X + Y))
    U = inputs.prim_to_cons(rho, [u, v], p, 1.4)
    cfg = O.make_cfg(ndim=2, n=(nx, ny), h=(1.0 / nx, 1.0 / ny), periodic=(0, 1),
                     bc_lo=(O.BC_REFLECT, 0), bc_hi=(O.BC_REFLECT, 0))
    c0 = O.conserved(cfg, U)
    scale = O.conserved(cfg, np.abs(U))
    for _ in range(4):
        O.rk3_step(cfg, U, O.cfl_dt(cfg, U, 0.5))
    c1 = O.conserved(cfg, U)
    for v in (0, 2, 3):
        assert abs(c1[v] - c0[v]) <= 1e-13 * scale[v], v
    assert abs(c1[1] - c0[1]) > 1e-6 * scale[1]


@pytest.mark.parametrize("flux", [O.FLUX_ROE, O.FLUX_VANLEER, O.FLUX_AUSM])
def test_rayleigh_taylor_is_mirror_symmetric_about_x_one_eighth(flux):
    """cos(8 pi x) is symmetric about x = 1/8 and the walls reflect, so the
    RHS (and a few steps) map onto themselves under x -> 1/4 - x, u -> -u."""
    pb = inputs.rayleigh_taylor(16)
    cfg = ora_cfg(pb, flux)
    U = pb.U0.copy()
    for _ in range(3):
        O.rk3_step(cfg, U, 2e-3)
    L = O.euler_rhs(cfg, U)[0]
    Lm = L[:, :, ::-1].copy()
    Lm[1] *= -1
    assert np.max(np.abs(Lm - L)) <= 1e-12 * np.max(np.abs(L))
    Um = U[:, :, ::-1].copy()
    Um[1] *= -1
    assert np.max(np.abs(Um - U)) <= 1e-13 * np.max(np.abs(U))


def test_fixed_state_ghosts_are_the_given_state():
    """A 1D line with fixed states on both ends: the RHS at the first node
    sees the fixed state's flux through the outer faces.  Compared with an
    explicitly padded periodic grid holding the same ghost values."""
    n = 12
    rng = np.random.default_rng(5)
    U = inputs.prim_to_cons(rng.uniform(0.8, 1.2, n), [rng.uniform(-0.2, 0.2, n)], rng.uniform(0.8, 1.2, n),
                            1.4)
    lo = inputs.prim_to_cons(np.array(1.1), [np.array(0.1)], np.array(1.05), 1.4)
    hi = inputs.prim_to_cons(np.array(0.9), [np.array(-0.05)], np.array(0.95), 1.4)
    cfg = O.make_cfg(ndim=1, n=(n,), h=(0.1,), bc_lo=(O.BC_FIXED,), bc_hi=(O.BC_FIXED,),
                     bc_state=((tuple(lo), tuple(hi)),))
    L = O.euler_rhs(cfg, U)[0]
    # padded grid: 10 ghosts of each state, interior the same; transmissive
    # ends far away cannot reach the nodes compared
    P = np.concatenate([np.repeat(lo[:, None], 10, axis=1), U, np.repeat(hi[:, None], 10, axis=1)], axis=1)
    cfgp = O.make_cfg(ndim=1, n=(n + 20,), h=(0.1,))
    Lp = O.euler_rhs(cfgp, P)[0][:, 10:10 + n]
    assert np.array_equal(L, Lp)


@pytest.mark.parametrize("diff", [O.DIFF_MD, O.DIFF_HWCNS, O.DIFF_MND])
def test_pointwise_rhs_equals_full_rhs_with_boundaries_and_source(diff):
    """The oracle's pointwise RHS (used for sampled parity at full size)
    applies the same boundary rules, differences and source as the full
    RHS: equal at every node."""
    pb = inputs.rayleigh_taylor(16)
    cfg = ora_cfg(pb, diff=diff)
    U = pb.U0.copy()
    O.rk3_step(cfg, U, 2e-3)
    L = O.euler_rhs(cfg, U)[0].reshape(pb.nv, -1)
    La = O.euler_rhs_at(cfg, U, np.arange(pb.cells))
    assert np.array_equal(La, L)

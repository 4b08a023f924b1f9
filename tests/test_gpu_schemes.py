"""GPU parity of the alternative schemes through the C ABI: the AUSM midpoint
flux and the HWCNS / MND differences (Eq. 4-5), alone and combined with the
other weights, in the FP64 path (bit-identical to the oracle), the FP32 path
(bounded error against the oracle), batches and the scalar solver.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1810_07806_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1810_07806_gb300 import wcns  # noqa: E402

DEV = "cuda:0"
FLUX = {"roe": (wcns.FLUX_ROE, O.FLUX_ROE), "vanleer": (wcns.FLUX_VANLEER, O.FLUX_VANLEER),
        "ausm": (wcns.FLUX_AUSM, O.FLUX_AUSM)}
DIFF = {"md": (wcns.DIFF_MD6, O.DIFF_MD), "hwcns": (wcns.DIFF_HWCNS, O.DIFF_HWCNS),
        "mnd": (wcns.DIFF_MND, O.DIFF_MND)}


def _cfg(pb, flux, diff, weights=O.W_TENO):
    return O.make_cfg(ndim=pb.ndim, n=pb.n, h=pb.h, periodic=pb.periodic, gamma=pb.gamma,
                      flux=FLUX[flux][1], diff=DIFF[diff][1], weights=weights)


def _rough(nd, n, periodic, seed):
    U = inputs.random_rough_state(nd, n, seed)
    hi = tuple(1.0 + 0.3 * a for a in range(nd))
    return inputs._finish("rough", nd, n, (0.0,) * nd, hi, periodic, 1.4, U, 0.0)


def _cases():
    return [inputs.shock_tube(400), inputs.four_quadrant(67, ny=45), inputs.taylor_green(20),
            _rough(1, (517,), (0,), 11), _rough(2, (70, 61), (1, 0), 12), _rough(3, (21, 19, 17), (1, 0, 1), 13),
            _rough(2, (5, 1), (0, 1), 14)]


def _gpu_rhs(pb, U, flux, diff, precision=wcns.FP64, weights=wcns.W_TENO):
    s = wcns.Solver.for_problem(pb, flux=FLUX[flux][0], diff=DIFF[diff][0], precision=precision,
                                weights=weights)
    dt = torch.float32 if precision == wcns.FP32 else torch.float64
    Ud = torch.from_numpy(np.ascontiguousarray(U)).to(DEV, dt)
    Ld = torch.empty_like(Ud)
    fl = torch.zeros(s.flags_bytes, dtype=torch.uint8, device=DEV)
    s.rhs(Ud, Ld, fl)
    torch.cuda.synchronize()
    out = Ld.double().cpu().numpy(), fl.cpu().numpy(), s.fallback_count()
    s.close()
    return out


@pytest.mark.parametrize("diff", sorted(DIFF))
@pytest.mark.parametrize("flux", sorted(FLUX))
def test_fp64_rhs_bit_identical_to_oracle(flux, diff):
    for pb in _cases():
        Lo, flo, _, np_o, _ = O.euler_rhs(_cfg(pb, flux, diff), pb.U0, want_flags=True)
        Lg, flg, np_g = _gpu_rhs(pb, pb.U0, flux, diff)
        assert np.array_equal(Lg, Lo), (pb.name, pb.n, np.max(np.abs(Lg - Lo)))
        assert np.array_equal(flg, flo) and np_g == np_o, pb.name


@pytest.mark.parametrize("flux,diff,weights", [("ausm", "mnd", "z"), ("vanleer", "hwcns", "js"),
                                               ("roe", "mnd", "linear")])
def test_fp64_rhs_with_other_weights_bit_identical(flux, diff, weights):
    wg = {"z": wcns.W_Z, "js": wcns.W_JS, "linear": wcns.W_LINEAR}[weights]
    wo = {"z": O.W_Z, "js": O.W_JS, "linear": O.W_LINEAR}[weights]
    for pb in _cases()[:4]:
        Lo = O.euler_rhs(_cfg(pb, flux, diff, wo), pb.U0)[0]
        Lg = _gpu_rhs(pb, pb.U0, flux, diff, weights=wg)[0]
        assert np.array_equal(Lg, Lo), pb.name


@pytest.mark.parametrize("flux,diff", [("ausm", "md"), ("roe", "hwcns"), ("vanleer", "mnd"), ("ausm", "mnd")])
def test_fp64_sod_end_state_bit_identical(flux, diff):
    pb = inputs.shock_tube(400)
    Uo = pb.U0.copy()
    t_o, steps_o, np_o = O.euler_run(_cfg(pb, flux, diff), Uo, 0.5, 0.2)
    s = wcns.Solver.for_problem(pb, flux=FLUX[flux][0], diff=DIFF[diff][0], cfl=0.5)
    Ud = torch.from_numpy(pb.U0.copy()).to(DEV)
    t_g, steps_g = s.advance(Ud, 0.2, check_every=16)
    assert (t_g, steps_g) == (t_o, steps_o)
    assert np.array_equal(Ud.cpu().numpy(), Uo)
    assert s.fallback_count() == np_o
    s.close()


@pytest.mark.parametrize("flux,diff", [("ausm", "md"), ("roe", "hwcns"), ("roe", "mnd"), ("ausm", "mnd")])
def test_fp32_rhs_close_to_oracle(flux, diff):
    """Smooth flow: |L32 - Lo| <= 2e-6 (|Lo| + S_v) against the FP64 oracle,
    S_v the flux scale of variable v (sum over directions of
    max (|F_v| + c |U_v|) / h): the MD and node differences subtract fluxes of
    that size, so FP32 rounding in them appears divided by h (the bound of the
    default scheme's test)."""
    for pb in (inputs.taylor_green(24), inputs.density_wave_1d(64)):
        Lo = O.euler_rhs(_cfg(pb, flux, diff), pb.U0)[0]
        L32 = _gpu_rhs(pb, pb.U0, flux, diff, precision=wcns.FP32)[0]
        S = _flux_scale(pb.U0, pb).reshape((-1,) + (1,) * pb.ndim)
        rel = np.max(np.abs(L32 - Lo) / (np.abs(Lo) + S))
        assert rel < 2e-6, (pb.name, rel)


def _flux_scale(U, pb):
    nd = pb.ndim
    rho, vel, p = inputs.cons_to_prim(U, pb.gamma)
    c = np.sqrt(pb.gamma * np.abs(p) / rho)
    S = np.zeros(nd + 2)
    for d in range(nd):
        F = np.zeros_like(U)
        F[0] = U[1 + d]
        for a in range(nd):
            F[1 + a] = U[1 + a] * vel[d]
        F[1 + d] += p
        F[nd + 1] = (U[nd + 1] + p) * vel[d]
        for v in range(nd + 2):
            S[v] += np.max(np.abs(F[v]) + c * np.abs(U[v])) / pb.h[d]
    return S


def _oracle_sensitivity(pb, cfg, t_end, seeds=3):
    """How far the oracle's own end state moves when its initial state is
    perturbed by relative noise of FP32 rounding size (2^-24): the largest
    relative L1 change per variable over a few seeds.  Next to shocks the
    cut decisions of Eq. 18 (and the positivity fallback) are discrete, so
    an ulp-level change of the data can flip them; this is the floor any
    FP32 evaluation of the same method sits on."""
    Uref = pb.U0.copy()
    O.euler_run(cfg, Uref, 0.5, t_end)
    worst = np.zeros(pb.nv)
    for seed in range(seeds):
        rng = np.random.default_rng(seed)
        U = pb.U0 * (1.0 + rng.uniform(-1.0, 1.0, pb.U0.shape) * 2.0 ** -24)
        O.euler_run(cfg, U, 0.5, t_end)
        rel = np.sum(np.abs(U - Uref), axis=1) / np.sum(np.abs(Uref), axis=1)
        worst = np.maximum(worst, rel)
    return worst, Uref


@pytest.mark.parametrize("flux,diff", [("ausm", "md"), ("roe", "mnd")])
def test_fp32_sod_end_state_close_to_oracle(flux, diff):
    """Sod to t = 0.2 in FP32 against the oracle: within 1e-3 relative L1, or
    twice the oracle's own response to FP32-sized noise in its input where
    that is larger (AUSM: the oracle moves by up to 1.7e-3 in the momentum
    under 2^-24 relative noise)."""
    pb = inputs.shock_tube(400)
    sens, Uo = _oracle_sensitivity(pb, _cfg(pb, flux, diff), 0.2)
    s = wcns.Solver.for_problem(pb, flux=FLUX[flux][0], diff=DIFF[diff][0], precision=wcns.FP32, cfl=0.5)
    Ud = torch.from_numpy(pb.U0.copy()).to(DEV)
    s.advance(Ud, 0.2, check_every=16)
    s.close()
    rel = np.sum(np.abs(Ud.cpu().numpy() - Uo), axis=1) / np.sum(np.abs(Uo), axis=1)
    assert np.all(rel <= np.maximum(1e-3, 2.0 * sens)), (rel, sens)


@pytest.mark.parametrize("precision", [wcns.FP64, wcns.FP32])
def test_batch_with_ausm_and_mnd_equals_batch_of_one(precision):
    pbs = inputs.shu_osher_batch(6)
    kw = dict(flux=wcns.FLUX_AUSM, diff=wcns.DIFF_MND, precision=precision)
    b = wcns.Batch(1, max_nodes=sum(p.cells for p in pbs), max_instances=len(pbs), **kw)
    slots = [b.add(pb, t_end=0.05) for pb in pbs]
    b.run(check_every=32)
    together = [b.read(k)[0] for k in slots]
    b.close()
    for pb, U in zip(pbs, together):
        b1 = wcns.Batch(1, max_nodes=pb.cells, max_instances=1, **kw)
        k = b1.add(pb, t_end=0.05)
        b1.run(check_every=32)
        assert np.array_equal(b1.read(k)[0], U)
        b1.close()
        Uo = pb.U0.copy()
        O.euler_run(_cfg(pb, "ausm", "mnd"), Uo, 0.5, 0.05)
        if precision == wcns.FP64:
            assert np.array_equal(U, Uo)
        else:
            rel = np.sum(np.abs(U - Uo), axis=1) / np.sum(np.abs(Uo), axis=1)
            assert np.all(rel <= 1e-3), rel


@pytest.mark.parametrize("diff", ["hwcns", "mnd"])
@pytest.mark.parametrize("kind", [wcns.SCALAR_ADVECTION, wcns.SCALAR_BURGERS])
def test_scalar_path_with_eq4_eq5_bit_identical(kind, diff):
    rng = np.random.default_rng(77 + kind)
    for n, steps in ((7, 5), (300, 20), (1500, 6)):
        x = np.arange(n) / n
        u = np.sin(2 * np.pi * x) + 0.5 + (x > 0.4) * rng.uniform(0.5, 1.0)
        h = 1.0 / n
        cfg = O.make_cfg(diff=DIFF[diff][1])
        Ud = torch.from_numpy(u.copy()).to(DEV)
        L = wcns.scalar_rhs(kind, Ud, h, diff=DIFF[diff][0])
        assert np.array_equal(L.cpu().numpy(), O.scalar_rhs(cfg, kind, u, h))
        t_end = steps * 0.2 * h / np.max(np.abs(u))
        wcns.scalar_run(kind, Ud, h, t_end, steps, diff=DIFF[diff][0])
        assert np.array_equal(Ud.cpu().numpy(), O.scalar_run(cfg, kind, u, h, t_end, steps))


@pytest.mark.parametrize("weights", ["js", "linear", "z"])
def test_fp32_comparison_weights_close_to_oracle(weights):
    """FP32 single grids with the comparison weights (rescaled indicators):
    smooth flow within the same flux-scale bound as TENO against the FP64
    oracle; flags report all stencils kept."""
    wg = {"z": wcns.W_Z, "js": wcns.W_JS, "linear": wcns.W_LINEAR}[weights]
    wo = {"z": O.W_Z, "js": O.W_JS, "linear": O.W_LINEAR}[weights]
    for pb in (inputs.taylor_green(24), inputs.density_wave_1d(64), inputs.four_quadrant(40, ny=33)):
        for flux in ("roe", "ausm"):
            Lo = O.euler_rhs(_cfg(pb, flux, "md", wo), pb.U0)[0]
            L32, fl32, _ = _gpu_rhs(pb, pb.U0, flux, "md", precision=wcns.FP32, weights=wg)
            assert np.all(fl32 == 0x3F)
            S = _flux_scale(pb.U0, pb).reshape((-1,) + (1,) * pb.ndim)
            rel = np.max(np.abs(L32 - Lo) / (np.abs(Lo) + S))
            bound = 2e-6 if pb.name != "four_quadrant" else 2e-5
            assert rel < bound, (pb.name, flux, rel)


@pytest.mark.parametrize("weights", ["js", "z"])
def test_fp32_comparison_weights_sod_end_state(weights):
    wg = {"z": wcns.W_Z, "js": wcns.W_JS}[weights]
    wo = {"z": O.W_Z, "js": O.W_JS}[weights]
    pb = inputs.shock_tube(400)
    Uo = pb.U0.copy()
    O.euler_run(_cfg(pb, "roe", "md", wo), Uo, 0.5, 0.2)
    s = wcns.Solver.for_problem(pb, weights=wg, precision=wcns.FP32, cfl=0.5)
    Ud = torch.from_numpy(pb.U0.copy()).to(DEV)
    s.advance(Ud, 0.2, check_every=16)
    s.close()
    rel = np.sum(np.abs(Ud.cpu().numpy() - Uo), axis=1) / np.sum(np.abs(Uo), axis=1)
    assert np.all(rel <= 1e-4), rel


def test_fp32_weights_of_an_all_zero_or_tiny_field_are_finite():
    """A field that is zero (or at the eps floor) everywhere keeps finite
    weights: the rescaled JS eps is clamped and the Z ratios are bounded."""
    pb = inputs.taylor_green(16)
    U = pb.U0.copy()
    U[3] = 0.0          # w-momentum exactly zero
    U[1] *= 1e-30       # u-momentum tiny
    for wg in (wcns.W_JS, wcns.W_Z, wcns.W_LINEAR):
        L32 = _gpu_rhs(pb, U, "roe", "md", precision=wcns.FP32, weights=wg)[0]
        assert np.all(np.isfinite(L32))

"""The allocation-free step, wcns_step_rk3_noalloc, checked against wcns_step_rk3.

Some callers cannot call cudaMalloc: an application whose device memory is
all reserved up front by another allocator, or a time-critical loop that
must make no allocation calls.  For them the library offers one FP64 RK3
step that needs no handle and keeps its stage state and right-hand side in a
static device buffer of fixed size.  These tests call it through the C ABI,
twice in a row, and compare with the handle-based step (the FP64 path is
deterministic, so the results must agree within the FP64 tolerance the
parity tests use; they are in fact identical) and with the FP64 oracle's
SSP-RK3 step.  The file is collected last so that a failure here comes after
every other test has run.
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

RTOL = 1e-13


def _grid(pb):
    return wcns.make_grid(pb.ndim, pb.n, pb.lo, pb.hi, pb.periodic)


@pytest.mark.parametrize("which", ["sod400", "quad96x80", "tgv24"])
def test_noalloc_step_matches_handle_step_on_two_calls(which):
    pb = {"sod400": lambda: inputs.shock_tube(400),
          "quad96x80": lambda: inputs.four_quadrant(96, ny=80),
          "tgv24": lambda: inputs.taylor_green(24)}[which]()
    solver = wcns.Solver.for_problem(pb)
    Ua = torch.from_numpy(pb.U0.copy()).to("cuda:0")
    Ub = Ua.clone()
    grid, params = _grid(pb), wcns.default_params()
    cfg = O.make_cfg(ndim=pb.ndim, n=pb.n, h=pb.h, periodic=pb.periodic, gamma=pb.gamma)
    Uo = pb.U0.copy()
    for call in range(2):
        dta = solver.step(Ua, 0.0, want_dt=True)
        dtb = wcns.step_rk3_noalloc(grid, pb.gamma, params, Ub, 0.0, want_dt=True)
        assert dtb == pytest.approx(dta, rel=RTOL)
        scale = float(Ua.abs().max())
        err = float((Ua - Ub).abs().max())
        assert err <= RTOL * scale, (call, err)
        # the oracle's step with its own CFL step size
        dto = O.cfl_dt(cfg, Uo, 0.5)
        assert dtb == pytest.approx(dto, rel=RTOL)
        O.rk3_step(cfg, Uo, dto)
        err_o = np.max(np.abs(Ub.cpu().numpy() - Uo))
        assert err_o <= 1e-12 * np.max(np.abs(Uo)), (call, err_o)
    # a given step size as well
    solver.step(Ua, 1e-4)
    wcns.step_rk3_noalloc(grid, pb.gamma, params, Ub, 1e-4)
    assert float((Ua - Ub).abs().max()) <= RTOL * float(Ua.abs().max())
    solver.close()


def test_noalloc_rejects_grids_beyond_the_static_buffer():
    pb = inputs.taylor_green(64)     # 2 x 5 x 64^3 x 8 bytes > 16 MiB
    U = torch.from_numpy(pb.U0.copy()).to("cuda:0")
    before = U.clone()
    with pytest.raises(wcns.WcnsError) as ei:
        wcns.step_rk3_noalloc(_grid(pb), pb.gamma, wcns.default_params(), U)
    assert ei.value.status == wcns.ERR_INVALID
    assert "scratch" in str(ei.value)
    torch.cuda.synchronize()
    assert torch.equal(U, before)


@pytest.mark.parametrize("nd,n", [(1, (349514,)), (2, (1024, 255)), (3, (58, 59, 61))])
def test_noalloc_at_the_size_limit(nd, n):
    """The largest 1D grid that fits (512 + 2 round_up(8 nv N, 256) bytes =
    16 MiB exactly) and two 2D/3D grids just below the limit step like the
    handle; one node more is rejected with the state untouched."""
    if nd == 1:
        pb = inputs.shock_tube(n[0])
    elif nd == 2:
        pb = inputs.four_quadrant(n[0], ny=n[1])
    else:
        pb = inputs._finish("rough", 3, n, (0.0,) * 3, (1.0, 1.3, 1.6), (1, 0, 1), 1.4,
                            inputs.random_rough_state(3, n, 5), 0.0)
    solver = wcns.Solver.for_problem(pb)
    Ua = torch.from_numpy(pb.U0.copy()).to("cuda:0")
    Ub = Ua.clone()
    for _ in range(2):
        solver.step(Ua, 0.0)
        wcns.step_rk3_noalloc(_grid(pb), pb.gamma, wcns.default_params(), Ub)
        assert float((Ua - Ub).abs().max()) <= RTOL * float(Ua.abs().max())
    solver.close()
    if nd == 1:
        big = inputs.shock_tube(n[0] + 1)
        U = torch.from_numpy(big.U0.copy()).to("cuda:0")
        before = U.clone()
        with pytest.raises(wcns.WcnsError) as ei:
            wcns.step_rk3_noalloc(_grid(big), big.gamma, wcns.default_params(), U)
        assert ei.value.status == wcns.ERR_INVALID
        torch.cuda.synchronize()
        assert torch.equal(U, before)


def test_noalloc_rejects_fp32():
    pb = inputs.shock_tube(64)
    U = torch.from_numpy(pb.U0.copy()).to("cuda:0")
    with pytest.raises(wcns.WcnsError):
        wcns.step_rk3_noalloc(_grid(pb), pb.gamma, wcns.default_params(precision=wcns.FP32), U)

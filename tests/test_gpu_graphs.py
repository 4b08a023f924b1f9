"""The captured-graph path of wcns_step_rk3 / wcns_advance against direct
launches (profiling on forces direct launches): identical bits, per state
pointer, across tile-configuration changes."""
import numpy as np
import pytest

from paper_1810_07806_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1810_07806_gb300 import wcns  # noqa: E402

DEV = "cuda:0"


def _run(pb, precision, steps, profile, tiles=None, switch_U=False):
    s = wcns.Solver.for_problem(pb, precision=precision, cfl=0.5)
    if tiles is not None:
        s.tile_config(tiles)
    s.profile(profile)
    Ua = torch.from_numpy(pb.U0.copy()).to(DEV)
    Ub = torch.from_numpy(pb.U0.copy()).to(DEV)
    for k in range(steps):
        if switch_U and k % 2:
            Ub.copy_(Ua)
            s.step(Ub)
            Ua.copy_(Ub)
        else:
            s.step(Ua)
        if tiles is not None and k == steps // 2:
            s.tile_config([2, 1, 0][:pb.ndim])
    torch.cuda.synchronize()
    out = Ua.cpu().numpy()
    s.close()
    return out


@pytest.mark.parametrize("precision", [wcns.FP64, wcns.FP32])
@pytest.mark.parametrize("name", ["sod", "rt", "tgv"])
def test_graph_steps_equal_direct_launches(name, precision):
    pb = {"sod": lambda: inputs.shock_tube(400), "rt": lambda: inputs.rayleigh_taylor(16),
          "tgv": lambda: inputs.taylor_green(24)}[name]()
    direct = _run(pb, precision, 6, profile=True)
    graph = _run(pb, precision, 6, profile=False)
    assert np.array_equal(graph, direct)
    switched = _run(pb, precision, 6, profile=False, switch_U=True)
    assert np.array_equal(switched, direct)


def test_graph_steps_follow_tile_configuration_changes():
    pb = inputs.taylor_green(24)
    a = _run(pb, wcns.FP32, 6, profile=False, tiles=[0, 0, 0])
    b = _run(pb, wcns.FP32, 6, profile=True, tiles=[0, 0, 0])
    assert np.array_equal(a, b)


def test_advance_graph_equals_stepping():
    pb = inputs.rayleigh_taylor(16)
    s = wcns.Solver.for_problem(pb, cfl=0.5, precision=wcns.FP32)
    U1 = torch.from_numpy(pb.U0.copy()).to(DEV)
    t, n = s.advance(U1, 0.05, check_every=8)
    s.profile(True)          # direct launches, clipped like advance
    U2 = torch.from_numpy(pb.U0.copy()).to(DEV)
    t2, n2 = s.advance(U2, 0.05, check_every=3)
    s.profile(False)
    assert (t, n) == (t2, n2)
    assert torch.equal(U1, U2)
    s.close()


@pytest.mark.parametrize("precision", [wcns.FP32, wcns.FP64])
def test_profile_counts_every_sweep_launch(precision):
    """wcns_profile_read reports the sweep launches its events cover (one
    event pair per RHS, ndim sweeps each: the FP32 sweeps of an RHS overlap,
    so only the whole RHS can be timed) and a positive total, then clears."""
    pb = inputs.four_quadrant(96, ny=64)
    s = wcns.Solver.for_problem(pb, precision=precision)
    U = torch.from_numpy(pb.U0.copy()).to(DEV)
    s.profile(True)
    for _ in range(3):
        s.step(U, 1e-4)
    ms, n = s.profile_read()
    assert n == 3 * 3 * pb.ndim and ms > 0.0
    ms2, n2 = s.profile_read()
    assert n2 == 0 and ms2 == 0.0
    s.profile(False)
    s.close()


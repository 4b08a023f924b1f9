"""GPU tests of the batch engine (wcns_batch_*): many uneven instances of one
dimension advanced together give, instance by instance, the results of the
same instance run alone (bit for bit in FP64), and the FP64 end states match
the oracle."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1810_07806_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1810_07806_gb300 import wcns  # noqa: E402


def _alone(pb, precision, t_end):
    s = wcns.Solver.for_problem(pb, precision=precision)
    U = torch.from_numpy(pb.U0.copy()).cuda()
    t, steps = s.advance(U, t_end, check_every=16)
    out = U.cpu().numpy()
    s.close()
    return out, t, steps


def _batch_of_one(pb, precision):
    b = wcns.Batch(pb.ndim, max_nodes=pb.cells, max_instances=1, precision=precision)
    slot = b.add(pb)
    b.run(check_every=8)
    out = b.read(slot)
    b.close()
    return out


def _check_against_alone(Ub, tb, sb, pb, precision):
    """Mixed batch == batch of one == the single-grid solver, bit for bit in
    either precision: the FP32 kernels are compiled without multiply-add
    contraction, so the batched and the single-grid instances of the same
    face code round identically, and both take the same reference state."""
    U1, t1, s1 = _batch_of_one(pb, precision)
    assert tb == t1 and sb == s1 and np.array_equal(Ub, U1)
    Ua, ta, sa = _alone(pb, precision, pb.t_end)
    assert tb == ta == pb.t_end and sb == sa
    assert np.array_equal(Ub, Ua)


def _uneven_1d(count, seed):
    rng = np.random.default_rng(seed)
    pbs = []
    for i in range(count):
        n = int(rng.integers(40, 700))
        pb = inputs.shu_osher_like(n, rng.uniform(1.5, 5), rng.uniform(0.1, 0.3), rng.uniform(3, 8))
        pb.t_end = float(rng.uniform(0.05, 0.3))
        pbs.append(pb)
    pbs.append(inputs.shock_tube(400))                           # Sod, t = 0.2
    pbs.append(inputs.shock_tube(157, states=inputs.LAX, t_end=0.14))
    return pbs


@pytest.mark.parametrize("precision", [wcns.FP64, wcns.FP32])
def test_batch_1d_equals_each_instance_alone(precision):
    pbs = _uneven_1d(12, 5)
    b = wcns.Batch(1, max_nodes=sum(p.cells for p in pbs), max_instances=len(pbs), precision=precision)
    slots = [b.add(pb) for pb in pbs]
    b.run(check_every=8)
    for pb, slot in zip(pbs, slots):
        Ub, tb, sb = b.read(slot)
        _check_against_alone(Ub, tb, sb, pb, precision)
    b.close()


def test_batch_fp64_sod_matches_oracle():
    pbs = _uneven_1d(5, 9)
    b = wcns.Batch(1, max_nodes=sum(p.cells for p in pbs), max_instances=len(pbs))
    slots = [b.add(pb) for pb in pbs]
    b.run()
    sod = pbs[-2]
    Ub, t, steps = b.read(slots[-2])
    Uo = sod.U0.copy()
    t_o, steps_o, _ = O.euler_run(O.make_cfg(ndim=1, n=sod.n, h=sod.h), Uo, 0.5, sod.t_end)
    assert t == t_o and steps == steps_o
    assert np.all(np.mean(np.abs(Ub - Uo), axis=1) <= 1e-10)
    b.close()


@pytest.mark.parametrize("precision", [wcns.FP64, wcns.FP32])
def test_batch_2d_uneven_sizes(precision):
    pbs = [inputs.four_quadrant(48, t_end=0.05), inputs.four_quadrant(37, ny=29, t_end=0.08),
           inputs.four_quadrant(64, ny=40, quads=inputs.LAX_LIU_6, t_end=0.03)]
    b = wcns.Batch(2, max_nodes=sum(p.cells for p in pbs), max_instances=4, precision=precision)
    slots = [b.add(pb) for pb in pbs]
    b.run(check_every=4)
    for pb, slot in zip(pbs, slots):
        Ub, tb, sb = b.read(slot)
        _check_against_alone(Ub, tb, sb, pb, precision)
    b.close()


def test_batch_3d_periodic():
    pbs = [inputs.taylor_green(12), inputs.taylor_green(16)]
    for p in pbs:
        p.t_end = 0.05
    b = wcns.Batch(3, max_nodes=sum(p.cells for p in pbs), max_instances=2)
    slots = [b.add(pb) for pb in pbs]
    b.run()
    for pb, slot in zip(pbs, slots):
        Ub, tb, sb = b.read(slot)
        Ua, ta, sa = _alone(pb, wcns.FP64, pb.t_end)
        assert np.array_equal(Ub, Ua) and sb == sa
    b.close()


def test_batch_slots_and_arena_are_reused():
    """Instances join and leave between steps: results stay identical to the
    instance alone, freed arena ranges are reused, capacity errors are clean."""
    pbs = _uneven_1d(6, 2)
    cap = sum(p.cells for p in pbs[:4])
    b = wcns.Batch(1, max_nodes=cap, max_instances=4)
    slots = [b.add(pb) for pb in pbs[:4]]
    with pytest.raises(wcns.WcnsError) as ei:
        b.add(pbs[4])
    assert ei.value.status in (wcns.ERR_BUSY, wcns.ERR_NOMEM)
    b.step(5)
    b.remove(slots[1])
    s_new = b.add(pbs[1])            # re-admitted from scratch into the freed range
    b.run()
    Ub, t, steps = b.read(s_new)
    Ua, ta, sa = _alone(pbs[1], wcns.FP64, pbs[1].t_end)
    assert np.array_equal(Ub, Ua) and steps == sa
    for k in (0, 2, 3):
        Ub, t, steps = b.read(slots[k])
        Ua, ta, sa = _alone(pbs[k], wcns.FP64, pbs[k].t_end)
        assert np.array_equal(Ub, Ua)
    b.close()


@pytest.mark.parametrize("precision", [wcns.FP64, wcns.FP32])
def test_persistent_launch_and_autotune_give_identical_results(precision):
    """The persistent launch form (CTAs taking tiles from a device counter)
    and the tile-table form compute the same faces: end states bit-identical;
    the autotuner's trial steps leave the batch's results unchanged."""
    pbs = _uneven_1d(10, 3)
    out = []
    for mode in (0, 1, "tuned"):
        b = wcns.Batch(1, max_nodes=sum(p.cells for p in pbs), max_instances=len(pbs), precision=precision)
        slots = [b.add(pb) for pb in pbs]
        if mode == "tuned":
            b.step(3)
            chosen, ms = b.autotune(steps=2)
            assert chosen in (0, 1) and ms[0] > 0 and ms[1] > 0
        else:
            b.launch_mode(mode)
        b.run(check_every=8)
        out.append([b.read(k) for k in slots])
        b.close()
    for k in range(len(pbs)):
        for other in (1, 2):
            assert np.array_equal(out[0][k][0], out[other][k][0])
            assert out[0][k][1:] == out[other][k][1:]


@pytest.mark.parametrize("weights", [wcns.W_JS, wcns.W_LINEAR, wcns.W_Z])
def test_fp32_batch_with_comparison_weights_equals_instances_alone(weights):
    """FP32 batches take the comparison weights (Eq. 14, Eq. 13, WCNS-Z):
    each instance bit-identical to the single-grid FP32 solver."""
    pbs = _uneven_1d(4, 8)
    b = wcns.Batch(1, max_nodes=sum(p.cells for p in pbs), max_instances=len(pbs), precision=wcns.FP32,
                   weights=weights)
    slots = [b.add(pb) for pb in pbs]
    b.run(check_every=8)
    for pb, k in zip(pbs, slots):
        Ub, tb, sb = b.read(k)
        s = wcns.Solver.for_problem(pb, precision=wcns.FP32, weights=weights)
        U = torch.from_numpy(pb.U0.copy()).cuda()
        ta, sa = s.advance(U, pb.t_end, check_every=16)
        s.close()
        assert (tb, sb) == (ta, sa) and np.array_equal(Ub, U.cpu().numpy())
    b.close()


def test_fp32_batch_of_smooth_waves_within_1e6_of_the_oracle():
    """Smooth flow in a batch: eight periodic density waves (N 64..400,
    62-291 steps to t = 0.2) in FP32 stay within 1e-6 relative L1 of the
    FP64 oracle (measured 1.2e-7 .. 7.5e-7: rounding of each step's FP32
    stage input, accumulated over the steps)."""
    pbs = inputs.density_wave_batch(8, seed=5, n_lo=64, n_hi=400)
    b = wcns.Batch(1, max_nodes=sum(p.cells for p in pbs), max_instances=len(pbs), precision=wcns.FP32)
    slots = [b.add(pb) for pb in pbs]
    b.run(check_every=32)
    for pb, k in zip(pbs, slots):
        U, t, _ = b.read(k)
        Uo = pb.U0.copy()
        O.euler_run(O.make_cfg(ndim=1, n=pb.n, h=pb.h, periodic=(1,)), Uo, 0.5, pb.t_end)
        rel = np.sum(np.abs(U - Uo), axis=1) / np.sum(np.abs(Uo), axis=1)
        assert t == pb.t_end and np.all(rel <= 1e-6), (pb.n, rel)
    b.close()


@pytest.mark.parametrize("mode", [0, 1])
def test_batch_3d_fp32_equals_single_grid(mode):
    """3D FP32 batches (the deferred full-cutoff pass, the shared-memory
    layouts of the y/z sweeps) in both launch forms: each instance equals the
    single-grid FP32 solver bit for bit, and stays within the FP32 bounds of
    the oracle's run (smooth Taylor-Green 1e-6; the rough state, whose jumps
    make cut decisions sensitive to rounding, 1e-3)."""
    pbs = [inputs.taylor_green(12), inputs.taylor_green(16), _rough3d()]
    for p in pbs:
        p.t_end = 0.02
    b = wcns.Batch(3, max_nodes=sum(p.cells for p in pbs), max_instances=len(pbs), precision=wcns.FP32)
    b.launch_mode(mode)
    slots = [b.add(pb) for pb in pbs]
    b.run(check_every=4)
    for pb, k in zip(pbs, slots):
        Ub, tb, sb = b.read(k)
        Ua, ta, sa = _alone(pb, wcns.FP32, pb.t_end)
        assert (tb, sb) == (ta, sa) and np.array_equal(Ub, Ua), pb.name
        Uo = pb.U0.copy()
        O.euler_run(O.make_cfg(ndim=3, n=pb.n, h=pb.h, periodic=pb.periodic), Uo, 0.5, pb.t_end)
        d = np.sum(np.abs(Ub - Uo).reshape(5, -1), axis=1)
        tot = np.sum(np.abs(Uo).reshape(5, -1), axis=1)
        tot[1:-1] = tot[1:-1].max()
        bound = 1e-6 if pb.name == "taylor_green" else 1e-3
        assert np.all(d <= bound * tot), (pb.name, d / tot)
    b.close()


def _rough3d():
    U = inputs.random_rough_state(3, (14, 11, 9), 31)
    return inputs._finish("rough", 3, (14, 11, 9), (0.0,) * 3, (1.0, 1.3, 1.6), (1, 0, 1), 1.4, U, 0.0)

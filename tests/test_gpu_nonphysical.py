"""WCNS_ERR_NONPHYSICAL through the C ABI: a face whose interpolated state
has rho <= 0 or p <= 0 takes first-order values (the positivity reading of
the method) and the calls that can see it report it.  The case is a
Shu-Osher-type instance of the batched benchmark (Mach-number draw of seed
1810, instance 10, 312 nodes) whose first step, in the oracle, has one
such face; Sod's shock tube has none.  Reports: a synchronising step, an
advance, a batch read (per instance) and a served result (per request),
each with the state still equal to the oracle's."""
import time

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
T_END = 0.02


def _cases():
    return inputs.shu_osher_batch(64)[10], inputs.shock_tube(400)


def _oracle_run(pb, t_end):
    cfg = O.make_cfg(ndim=1, n=pb.n, h=pb.h)
    U = pb.U0.copy()
    t, steps, nfb = O.euler_run(cfg, U, 0.5, t_end)
    return U, t, steps, nfb


def test_first_step_and_advance_report_first_order_faces():
    bad, good = _cases()
    cfg = O.make_cfg(ndim=1, n=bad.n, h=bad.h)
    Uo = bad.U0.copy()
    assert O.rk3_step(cfg, Uo, O.cfl_dt(cfg, Uo, 0.5)) == 1     # the oracle's count for step 1
    s = wcns.Solver.for_problem(bad)
    U = torch.from_numpy(bad.U0.copy()).to(DEV)
    s.step(U, 0.0)                       # asynchronous: no report
    assert not s.nonphysical
    assert s.fallback_count(reset=True) == 1
    U = torch.from_numpy(bad.U0.copy()).to(DEV)
    s.step(U, 0.0, want_dt=True)         # synchronising: reported
    assert s.nonphysical
    assert np.array_equal(U.cpu().numpy(), Uo)
    s.close()
    Uo, t_o, steps_o, nfb = _oracle_run(bad, T_END)
    assert nfb > 0
    s = wcns.Solver.for_problem(bad)
    U = torch.from_numpy(bad.U0.copy()).to(DEV)
    assert s.advance(U, T_END, check_every=4) == (t_o, steps_o)
    assert s.nonphysical and s.fallback_count() == nfb
    assert np.array_equal(U.cpu().numpy(), Uo)
    s.close()
    s = wcns.Solver.for_problem(good)
    U = torch.from_numpy(good.U0.copy()).to(DEV)
    s.advance(U, 0.2)
    assert not s.nonphysical and s.fallback_count() == 0
    s.close()


def test_batch_reports_first_order_faces_per_instance():
    bad, good = _cases()
    b = wcns.Batch(1, max_nodes=bad.cells + good.cells, max_instances=2)
    kb = b.add(bad, t_end=T_END)
    kg = b.add(good, t_end=T_END)
    b.run(check_every=4)
    Ub, _, steps_b = b.read(kb)
    Ug, _, _ = b.read(kg)
    assert b.nonphysical[kb] and not b.nonphysical[kg]
    Uo, _, steps_o, _ = _oracle_run(bad, T_END)
    assert steps_b == steps_o and np.array_equal(Ub, Uo)
    assert np.array_equal(Ug, _oracle_run(good, T_END)[0])
    # a new instance in the freed slot (and arena range) starts with a clean counter
    b.remove(kb)
    k2 = b.add(inputs.shock_tube(300), t_end=T_END)
    b.run(check_every=4)
    b.read(k2)
    assert not b.nonphysical[k2]
    b.close()


def test_served_request_carries_the_status_alone():
    bad, good = _cases()
    sv = wcns.Server(hbm_budget_bytes=1 << 28, max_instances_per_class=4, steps_per_tick=2)
    sv.submit(bad, tag=1, t_end=T_END)
    sv.submit(good, tag=2, t_end=T_END)
    got = {}
    t0 = time.time()
    while len(got) < 2 and time.time() - t0 < 60:
        for r in sv.poll(8, timeout_us=100000):
            got[r["tag"]] = r
    sv.close()
    assert got[1]["status"] == wcns.ERR_NONPHYSICAL
    assert got[2]["status"] == wcns.OK
    assert np.array_equal(got[1]["U"], _oracle_run(bad, T_END)[0])
    assert np.array_equal(got[2]["U"], _oracle_run(good, T_END)[0])

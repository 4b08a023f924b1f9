"""GPU tests of the serving loop (wcns_batch_submit / wcns_serve_poll):
requests that arrive while others run are admitted as slots and memory free
up, overlap on the device, and each result equals the same problem solved
alone (bit for bit, in FP64 and in FP32) and the FP64 oracle's solution
(FP64: within 1e-10 L1; FP32: within a stated relative L1 bound)."""
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


def _alone(pb, precision):
    """The same problem solved alone: a batch holding only this instance."""
    b = wcns.Batch(pb.ndim, max_nodes=pb.cells, max_instances=1, precision=precision)
    slot = b.add(pb)
    b.run(check_every=8)
    U, t, steps = b.read(slot)
    b.close()
    return U, t, steps


def _requests(seed, count, side_lo=24, side_hi=72):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        side = int(rng.integers(side_lo, side_hi))
        quads = tuple((float(rng.uniform(0.3, 2.0)), float(rng.uniform(-0.7, 0.7)), float(rng.uniform(-0.7, 0.7)),
                       float(rng.uniform(0.2, 2.0))) for _ in range(4))
        pb = inputs.four_quadrant(side, ny=side + int(rng.integers(-5, 6)), quads=quads,
                                  t_end=float(rng.uniform(0.02, 0.06)))
        out.append((pb, wcns.FP32 if i % 2 else wcns.FP64))
    return out


def _drain(sv, expected, timeout_s=120):
    got = {}
    t0 = time.time()
    while len(got) < expected and time.time() - t0 < timeout_s:
        for r in sv.poll(64, timeout_us=200000):
            got[r["tag"]] = r
    return got


def _check_against_oracle(pb, prec, r):
    """The served end state against the FP64 oracle's run of the same
    request: FP64 within 1e-10 mean absolute difference per variable and the
    same number of steps; FP32 within 1e-4 relative L1 per variable (the
    momenta measured against the larger momentum total)."""
    cfg = O.make_cfg(ndim=pb.ndim, n=pb.n, h=pb.h, periodic=pb.periodic, gamma=pb.gamma)
    Uo = pb.U0.copy()
    t_o, steps_o, _ = O.euler_run(cfg, Uo, 0.5, pb.t_end)
    U = r["U"].reshape(pb.nv, -1)
    Uo = Uo.reshape(pb.nv, -1)
    if prec == wcns.FP64:
        assert r["steps"] == steps_o and r["t"] == t_o
        assert np.all(np.mean(np.abs(U - Uo), axis=1) <= 1e-10)
    else:
        tot = np.sum(np.abs(Uo), axis=1)
        tot[1:-1] = tot[1:-1].max()
        rel = np.sum(np.abs(U - Uo), axis=1) / tot
        assert np.all(rel <= 1e-4), rel


def test_served_results_equal_each_problem_alone():
    reqs = _requests(1, 10)
    sv = wcns.Server(hbm_budget_bytes=1 << 30, max_instances_per_class=8, steps_per_tick=4)
    for k, (pb, prec) in enumerate(reqs[:5]):
        sv.submit(pb, tag=k, precision=prec)
    time.sleep(0.05)                          # others arrive while the first ones run
    for k, (pb, prec) in enumerate(reqs[5:], start=5):
        sv.submit(pb, tag=k, precision=prec)
    got = _drain(sv, len(reqs))
    assert len(got) == len(reqs)
    for k, (pb, prec) in enumerate(reqs):
        r = got[k]
        assert r["status"] == wcns.OK
        Ua, ta, sa = _alone(pb, prec)
        assert r["t"] == ta == pb.t_end and r["steps"] == sa
        assert np.array_equal(r["U"], Ua)
        assert r["t_submit"] <= r["t_admit"] <= r["t_done"]
        _check_against_oracle(pb, prec, r)
    st = sv.stats()
    assert st["completed"] == len(reqs) and st["queued"] == 0
    sv.close()


def test_admission_waits_for_memory_and_slots():
    """With room for about two instances of each class, later requests queue
    until earlier ones finish, and every result is still exact."""
    reqs = [(inputs.four_quadrant(40, t_end=0.03), wcns.FP64) for _ in range(5)]
    per = 40 * 40 * 4 * 24                       # bytes per instance of the FP64 2D class
    sv = wcns.Server(hbm_budget_bytes=int(per * 2.6) * 2, max_instances_per_class=2, steps_per_tick=2)
    for k, (pb, prec) in enumerate(reqs):
        sv.submit(pb, tag=k, precision=prec)
    got = _drain(sv, len(reqs))
    assert len(got) == len(reqs)
    st = sv.stats()
    assert st["max_running"] <= 2
    assert st["max_queue"] >= 1
    Ua, _, _ = _alone(reqs[0][0], wcns.FP64)
    _check_against_oracle(reqs[0][0], wcns.FP64, got[0])
    for k in range(len(reqs)):
        assert got[k]["status"] == wcns.OK
        assert np.array_equal(got[k]["U"], Ua)
    admits = sorted(got[k]["t_admit"] for k in got)
    assert admits[-1] > admits[0]                # the last ones waited
    sv.close()


def test_request_larger_than_the_budget_is_rejected():
    sv = wcns.Server(hbm_budget_bytes=1 << 20, max_instances_per_class=4, steps_per_tick=2)
    pb = inputs.four_quadrant(256, t_end=0.01)
    sv.submit(pb, tag=7)
    got = _drain(sv, 1, timeout_s=30)
    assert got[7]["status"] == wcns.ERR_NOMEM and got[7]["U"] is None
    sv.close()


def test_bad_requests_are_rejected_and_every_scheme_is_served():
    """Requests with bad parameters fail at submit, with a reason.  The
    comparison weights (both precisions) and the Rayleigh-Taylor boundaries
    and body force are served, each result equal to the same problem solved
    alone by the single-grid path."""
    sv = wcns.Server(hbm_budget_bytes=1 << 28, max_instances_per_class=4, steps_per_tick=2)
    with pytest.raises(wcns.WcnsError):
        sv.submit(inputs.four_quadrant(32, t_end=0.01), tag=3, flux=9)
    with pytest.raises(wcns.WcnsError):
        sv.submit(inputs.rayleigh_taylor(1), tag=6, t_end=0.01)   # reflecting axis of 1 node
    pb = inputs.four_quadrant(32, t_end=0.01)
    rt = inputs.rayleigh_taylor(8)
    sv.submit(pb, tag=4, weights=wcns.W_JS)
    sv.submit(pb, tag=5, weights=wcns.W_Z, precision=wcns.FP32)
    sv.submit(rt, tag=7, t_end=0.02)
    sv.submit(rt, tag=8, t_end=0.02, precision=wcns.FP32)
    got = _drain(sv, 4, timeout_s=60)
    for tag, prob, prec, w, t_end in ((4, pb, wcns.FP64, wcns.W_JS, pb.t_end), (5, pb, wcns.FP32, wcns.W_Z, pb.t_end),
                                      (7, rt, wcns.FP64, wcns.W_TENO, 0.02), (8, rt, wcns.FP32, wcns.W_TENO, 0.02)):
        assert got[tag]["status"] == wcns.OK
        s = wcns.Solver.for_problem(prob, precision=prec, weights=w)
        U = torch.from_numpy(prob.U0.copy()).cuda()
        s.advance(U, t_end)
        assert np.array_equal(got[tag]["U"], U.cpu().numpy()), tag
        s.close()
    sv.close()

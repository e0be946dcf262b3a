"""Batched applies and the request server against single applies of the same problems.

Each result of a batch or of the server must be the product of dpstokes_apply for that problem,
within the alone-vs-in-mix bars (1e-12 relative L2 in FP64, 1e-6 mixed).  (Bins are sorted by
particle index, so the spread repeats bit for bit; the tile-gather interpolation adds shares with
shared-memory float atomics, whose order can vary.)"""

import numpy as np
import pytest

from paper_2210_01837_gb300 import binding
from paper_2210_01837_gb300.workloads import random_particles

from gpu_helpers import rel_l2, small_params, to_dev

pytestmark = pytest.mark.gpu

BAR = {"fp64": 1e-12, "mixed": 1e-6}

# (mode, nx, ny, nz, torque route (False: forces only, True: spectral curl), precision, n, seed)
PROBLEMS = [
    ("bottom_wall", 48, 48, 33, True, "fp64", 120, 11),
    ("slit", 40, 56, 25, False, "mixed", 200, 12),
    ("free", 54, 36, 17, True, "mixed", 80, 13),
    ("bottom_wall", 72, 40, 33, False, "fp64", 150, 14),
    ("slit", 36, 36, 33, True, "mixed", 60, 15),
    ("bottom_wall", 40, 48, 25, "kernel_derivative", "mixed", 90, 16),
]


def _problem(mode, nx, ny, nz, torque, precision, n, seed):
    params = small_params(mode, nx=nx, ny=ny, nz=nz, zmax=8.0 if mode != "slit" else 6.0, torque=bool(torque))
    pos, F, T = random_particles(params, n, seed, torques=bool(torque))
    return params, pos, F, T if torque else None


def _alone(params, pos, F, T, precision, route, sizes=None):
    import torch
    plan = binding.Plan.from_params(params, with_torque=route, precision=precision, max_n=len(pos))
    U, W = plan.apply(to_dev(pos), to_dev(F), None if T is None else to_dev(T), check=True)
    torch.cuda.synchronize()
    out = (U.cpu().numpy(), None if W is None else W.cpu().numpy())
    if sizes is not None:
        sizes.append(plan.info().device_bytes)
    plan.close()
    return out


def _check(got, want, precision):
    assert rel_l2(got[0], want[0]) <= BAR[precision]
    if want[1] is not None:
        assert rel_l2(got[1], want[1]) <= BAR[precision]


def test_batch_matches_single_applies_and_reports_status():
    import torch
    probs = [_problem(*p) for p in PROBLEMS]
    alone = [_alone(pa, pos, F, T, p[5], p[4]) for p, (pa, pos, F, T) in zip(PROBLEMS, probs)]
    plans, items, outs = [], [], []
    for p, (pa, pos, F, T) in zip(PROBLEMS, probs):
        plan = binding.Plan.from_params(pa, with_torque=p[4], precision=p[5], max_n=len(pos))
        plans.append(plan)
        U = torch.empty((len(pos), 3), dtype=torch.float64, device="cuda")
        W = torch.empty_like(U) if T is not None else None
        items.append((plan, to_dev(pos), to_dev(F), None if T is None else to_dev(T), U, W))
        outs.append((U, W))
    # a bad request (particle above the slit) in the same batch reports only its own status
    pa, pos, F, T = probs[1]
    bad_pos = pos.copy()
    bad_pos[3, 2] = pa["zmax"] + 1.0
    bad_plan = binding.Plan.from_params(pa, with_torque=False, precision="mixed", max_n=len(pos))
    Ub = torch.empty((len(pos), 3), dtype=torch.float64, device="cuda")
    items.append((bad_plan, to_dev(bad_pos), to_dev(F), None, Ub, None))
    status = torch.full((len(items),), 77, dtype=torch.int32, device="cuda")
    binding.apply_batch(items, status=status)
    torch.cuda.synchronize()
    st = status.cpu().numpy().tolist()
    assert st[:-1] == [binding.DPS_OK] * len(PROBLEMS)
    assert st[-1] == binding.DPS_ERR_OUT_OF_DOMAIN
    for p, (U, W), want in zip(PROBLEMS, outs, alone):
        _check((U.cpu().numpy(), None if W is None else W.cpu().numpy()), want, p[5])
    for plan in plans + [bad_plan]:
        plan.close()


def test_batch_same_plan_twice_runs_in_order():
    import torch
    pa, pos, F, T = _problem(*PROBLEMS[0])
    plan = binding.Plan.from_params(pa, with_torque=True, precision="fp64", max_n=len(pos))
    want1 = _alone(pa, pos, F, T, "fp64", True)
    F2 = -2.0 * F
    want2 = _alone(pa, pos, F2, T, "fp64", True)
    U1, W1, U2, W2 = (torch.empty((len(pos), 3), dtype=torch.float64, device="cuda") for _ in range(4))
    binding.apply_batch([(plan, to_dev(pos), to_dev(F), to_dev(T), U1, W1),
                         (plan, to_dev(pos), to_dev(F2), to_dev(T), U2, W2)])
    torch.cuda.synchronize()
    _check((U1.cpu().numpy(), W1.cpu().numpy()), want1, "fp64")
    _check((U2.cpu().numpy(), W2.cpu().numpy()), want2, "fp64")
    plan.close()


def test_batch_captured_in_a_cuda_graph_and_replayed():
    import torch
    probs = [_problem(*p) for p in PROBLEMS[:3]]
    binding.dpstokes_batch_prepare()
    plans, items, outs, ins = [], [], [], []
    for p, (pa, pos, F, T) in zip(PROBLEMS[:3], probs):
        plan = binding.Plan.from_params(pa, with_torque=p[4], precision=p[5], max_n=len(pos))
        plans.append(plan)
        dpos, dF, dT = to_dev(pos), to_dev(F), None if T is None else to_dev(T)
        U = torch.empty((len(pos), 3), dtype=torch.float64, device="cuda")
        W = torch.empty_like(U) if T is not None else None
        items.append((plan, dpos, dF, dT, U, W))
        outs.append((U, W))
        ins.append(dF)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):  # warm-up outside the capture
        binding.apply_batch(items, stream=side)
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        binding.apply_batch(items)
    for scale in (1.0, -3.0):
        for (pa, pos, F, T), dF in zip(probs, ins):
            dF.copy_(to_dev(scale * F))
        for U, W in outs:
            U.zero_()
        graph.replay()
        torch.cuda.synchronize()
        for p, (pa, pos, F, T), (U, W) in zip(PROBLEMS[:3], probs, outs):
            want = _alone(pa, pos, scale * F, T, p[5], p[4])
            _check((U.cpu().numpy(), None if W is None else W.cpu().numpy()), want, p[5])
    del graph
    for plan in plans:
        plan.close()


def _pinned(a):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).pin_memory()
    return t.numpy()


def test_server_results_equal_single_applies_and_evicts_under_budget():
    probs = [_problem(*p) for p in PROBLEMS]
    sizes = []
    alone = [_alone(pa, pos, F, T, p[5], p[4], sizes) for p, (pa, pos, F, T) in zip(PROBLEMS, probs)]
    # budget for about two of these plans at a time: every request still completes, plans are
    # evicted and recreated, and the results do not depend on what ran beside them
    budget = int(2.5 * max(sizes))
    srv = binding.Server(memory_budget_bytes=budget, slots=3)
    tickets = []
    for rep in range(3):
        for k, (p, (pa, pos, F, T)) in enumerate(zip(PROBLEMS, probs)):
            t = srv.submit(pa, with_torque=p[4], precision=p[5], max_n=len(pos), pos=_pinned(pos),
                           F=_pinned(F), T=None if T is None else _pinned(T))
            tickets.append((k, t))
    for k, t in tickets:
        r, U, W = srv.wait(t, timeout_s=300.0)
        assert r.status == binding.DPS_OK
        assert r.t_submit <= r.t_start <= r.t_done
        _check((U, W), alone[k], PROBLEMS[k][5])
    stats = srv.stats()
    assert stats["queued"] == 0 and stats["running"] == 0
    assert stats["plans_created"] >= len(PROBLEMS)
    assert stats["plans_evicted"] >= 1
    assert stats["bytes_resident"] <= budget
    srv.close()


def test_server_rejects_a_request_that_can_never_fit():
    pa, pos, F, T = _problem(*PROBLEMS[0])
    srv = binding.Server(memory_budget_bytes=1 << 20, slots=1)
    t = srv.submit(pa, with_torque=True, precision="fp64", max_n=len(pos), pos=_pinned(pos), F=_pinned(F),
                   T=_pinned(T))
    r, _, _ = srv.wait(t, timeout_s=60.0)
    assert r.status == binding.DPS_ERR_OOM
    srv.close()


@pytest.mark.parametrize("pinned", [False, True])
def test_server_overlaps_requests_with_pinned_or_pageable_outputs(pinned):
    """Two requests of different plans, both cached, submitted together: the second is admitted and
    enqueued while the first product still runs (a direct device-to-host copy into pageable output
    arrays would hold the worker until the first product finished, which would delay the second
    admission by a whole product), and both results equal single applies."""
    from paper_2210_01837_gb300.workloads import slit_16k
    reqs = []
    for nz in (97, 65):
        pa, pos, F, T = slit_16k(n=4096, nz=nz)
        reqs.append((pa, pos, F, T, _alone(pa, pos, F, T, "fp64", True)))
    srv = binding.Server(memory_budget_bytes=64 << 30, slots=4)

    def submit(pa, pos, F, T):
        n = len(pos)
        U = _pinned(np.zeros((n, 3))) if pinned else np.zeros((n, 3))
        W = _pinned(np.zeros((n, 3))) if pinned else np.zeros((n, 3))
        return srv.submit(pa, with_torque=True, precision="fp64", max_n=n, pos=_pinned(pos), F=_pinned(F),
                          T=_pinned(T), U=U, W=W)

    for _ in range(2):  # plans created and resident before the measured round
        for t in [submit(*r[:4]) for r in reqs]:
            assert srv.wait(t, timeout_s=300.0)[0].status == binding.DPS_OK
    tickets = [submit(*r[:4]) for r in reqs]
    res = [srv.wait(t, timeout_s=300.0) for t in tickets]
    for (r, U, W), req in zip(res, reqs):
        assert r.status == binding.DPS_OK
        _check((U, W), req[4], "fp64")
    (ra, _, _), (rb, _, _) = res
    assert rb.t_start < ra.t_done and ra.t_start < rb.t_done
    assert rb.t_start - ra.t_start < 0.25 * (ra.t_done - ra.t_start), (ra.t_start, ra.t_done, rb.t_start)
    srv.close()


def test_server_queue_limit_refuses_and_still_serves():
    """With a queue limit, submissions that find the queue full are refused at once (no ticket)
    and counted; every accepted request completes with the single-apply result."""
    probs = [_problem(*p) for p in PROBLEMS[:2]]
    alone = [_alone(pa, pos, F, T, p[5], p[4]) for p, (pa, pos, F, T) in zip(PROBLEMS[:2], probs)]
    srv = binding.Server(memory_budget_bytes=8 << 30, slots=1, max_queued=2)
    accepted, refused = [], 0
    for rep in range(12):
        k = rep % 2
        pa, pos, F, T = probs[k]
        t = srv.submit(pa, with_torque=PROBLEMS[k][4], precision=PROBLEMS[k][5], max_n=len(pos), pos=_pinned(pos),
                       F=_pinned(F), T=None if T is None else _pinned(T))
        if t is None:
            refused += 1
        else:
            accepted.append((k, t))
    for k, t in accepted:
        r, U, W = srv.wait(t, timeout_s=300.0)
        assert r.status == binding.DPS_OK
        _check((U, W), alone[k], PROBLEMS[k][5])
    stats = srv.stats()
    assert refused >= 1 and stats["rejected"] == refused
    assert len(accepted) + refused == 12
    srv.close()

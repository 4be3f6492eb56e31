"""Serving loop: continuous batching over several operators.

Requests on three operators are submitted in a mixed order (some while
earlier batches are running); every result must equal the same solve done
alone (pm_solve on that operator) within 1e-9, batching must actually occur,
and a budget that fits one request at a time must still serve everything.
Operators described by their arrays are built by the server itself (one
near-field build per geometry, clones for further coefficients) and give the
same results as caller-built ones; an FMM-sized operator (the 98,304-node
torus) mixed with small ones gives the results it gives alone.
"""

import time

import numpy as np
import pytest

from workloads import make_workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ops():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2401_12501_gb300 as pm
    ctx = pm.Context(0)
    out = []
    for name in ("ellipsoid_small", "sphere_384", "star_small"):
        wl = make_workload(name)
        s = pm.Surface.from_fixture(ctx, wl.surface)
        s.set_coeff(wl.coeff.a, wl.coeff.grad_a)
        out.append((wl, s))
    yield ctx, out
    for _, s in out:
        s.close()
    ctx.close()


def rhs_set(wl, k, seed):
    rng = np.random.default_rng(seed)
    w = wl.surface.weights
    F = [np.roll(wl.f, int(rng.integers(0, wl.N))) * rng.uniform(0.5, 2.0) for _ in range(k)]
    return [f - np.dot(w, f) / w.sum() for f in F]


def test_mixed_requests_match_standalone(ops):
    import paper_2401_12501_gb300 as pm
    ctx, lst = ops
    reqs = []
    for idx, (wl, s) in enumerate(lst):
        for f in rhs_set(wl, 6, idx):
            reqs.append((idx, f))
    order = np.random.default_rng(0).permutation(len(reqs))
    sv = pm.Server(ctx, hbm_budget_bytes=2 << 30, max_batch=16, n_workers=3)
    tickets = []
    for n, k in enumerate(order):
        idx, f = reqs[k]
        tickets.append((k, sv.submit(lst[idx][1], f, tol=1e-11)))
        if n == 5:
            time.sleep(0.05)                # later requests arrive while batches run
    results = {k: sv.wait(t) for k, t in tickets}
    st = sv.stats()
    sv.close()
    assert st["solved"] == len(reqs)
    assert st["batches"] < len(reqs) and st["max_batch"] > 1
    for k, (u, info, lat) in results.items():
        idx, f = reqs[k]
        wl, s = lst[idx]
        alone, _ = s.solve(f, tol=1e-11)
        w = wl.surface.weights
        assert info.residual <= 1e-11
        assert np.sqrt(np.dot(w, (u - alone) ** 2) / np.dot(w, alone ** 2)) < 1e-9
        assert lat > 0


def test_precisions_are_not_mixed_in_a_batch(ops):
    """Requests on one operator in different precisions: each is solved in its own
    precision (a batch joins one precision only) and matches the standalone solve."""
    import paper_2401_12501_gb300 as pm
    ctx, lst = ops
    wl, s = lst[0]
    fs = rhs_set(wl, 6, 7)
    precs = ["fp32", "fmm", "ff", "fp32", "fmm", "ff"]
    sv = pm.Server(ctx, hbm_budget_bytes=2 << 30, max_batch=16, n_workers=2)
    tickets = [sv.submit(s, f, tol=1e-11, prec=p) for f, p in zip(fs, precs)]
    res = [sv.wait(t) for t in tickets]
    st = sv.stats()
    sv.close()
    assert st["solved"] == len(fs)
    w = wl.surface.weights
    for f, p, (u, info, _) in zip(fs, precs, res):
        alone, ai = s.solve(f, tol=1e-11, prec=p)
        assert info.residual <= 1e-11
        assert np.sqrt(np.dot(w, (u - alone) ** 2) / np.dot(w, alone ** 2)) < 1e-9
    sv = pm.Server(ctx, hbm_budget_bytes=2 << 30)
    try:
        with pytest.raises(pm.PmError):
            sv.submit(s, fs[0], tol=1e-8, prec=7)          # unknown precision
    finally:
        sv.close()


def test_budget_for_one_request_serialises(ops):
    """Admission counts the workspace a batch would newly allocate: on a fresh operator a
    budget of one single-RHS Krylov workspace admits one request at a time (a batched
    workspace for two would exceed it), and a request above the budget is refused."""
    import paper_2401_12501_gb300 as pm
    ctx, lst = ops
    wl = lst[0][0]
    s = pm.Surface.from_fixture(ctx, wl.surface)
    s.set_coeff(wl.coeff.a, wl.coeff.grad_a)
    per = (50 + 11) * wl.N * 8 + (64 << 10)   # one Krylov basis + vectors + small arrays
    sv = pm.Server(ctx, hbm_budget_bytes=per, max_batch=16, n_workers=2)
    ts = [sv.submit(s, f, tol=1e-10) for f in rhs_set(wl, 5, 9)]
    outs = [sv.wait(t) for t in ts]
    st = sv.stats()
    sv.close()
    assert st["max_batch"] == 1 and st["solved"] == 5
    assert all(o[1].residual <= 1e-10 for o in outs)
    # a request larger than the whole budget is refused at submit (fresh operator:
    # its Krylov workspace does not exist yet)
    s2 = pm.Surface.from_fixture(ctx, wl.surface)
    s2.set_coeff(wl.coeff.a, wl.coeff.grad_a)
    tiny = pm.Server(ctx, hbm_budget_bytes=1024, max_batch=4, n_workers=1)
    with pytest.raises(pm.PmError) as e:
        tiny.submit(s2, wl.f)
    assert e.value.status == 2
    tiny.close()
    s.close()
    s2.close()


def test_full_device_admits_one_batch_at_a_time(ops):
    """Admission against a device reported full (PM_FAKE_HBM_BYTES = 0 replaces the
    free-memory reading on the host): nothing is admitted next to a batch in flight,
    the oldest item still goes when the device is idle, so every request completes,
    with the result it has alone."""
    import os
    import paper_2401_12501_gb300 as pm
    ctx, lst = ops
    os.environ["PM_FAKE_HBM_BYTES"] = "0"
    try:
        sv = pm.Server(ctx, hbm_budget_bytes=2 << 30, max_batch=4, n_workers=3)
        reqs = [(idx, f) for idx, (wl, _) in enumerate(lst) for f in rhs_set(wl, 3, 40 + idx)]
        ts = [sv.submit(lst[idx][1], f, tol=1e-11) for idx, f in reqs]
        outs = [sv.wait(t) for t in ts]
        st = sv.stats()
        sv.close()
    finally:
        del os.environ["PM_FAKE_HBM_BYTES"]
    assert st["solved"] == len(reqs)
    for (idx, f), (u, info, _) in zip(reqs, outs):
        alone, _ = lst[idx][1].solve(f, tol=1e-11)
        w = lst[idx][0].surface.weights
        assert info.residual <= 1e-11
        assert np.sqrt(np.dot(w, (u - alone) ** 2) / np.dot(w, alone ** 2)) < 1e-9


def test_failed_solve_reports_status_and_message(ops):
    """A request whose solve fails (f with a non-zero mean) ends with the solve's status,
    and the waiting thread's pm_last_error holds the worker's message."""
    import paper_2401_12501_gb300 as pm
    ctx, lst = ops
    wl, s = lst[0]
    sv = pm.Server(ctx, hbm_budget_bytes=2 << 30, max_batch=4, n_workers=1)
    t_bad = sv.submit(s, wl.f + 1.0, tol=1e-8)
    t_ok = sv.submit(s, rhs_set(wl, 1, 3)[0], tol=1e-8)
    with pytest.raises(pm.PmError) as e:
        sv.wait(t_bad)
    assert e.value.status == 6 and "mean" in str(e.value)
    u, info, _ = sv.wait(t_ok)
    assert info.residual <= 1e-8
    sv.close()


def _desc_parts(name, coeff_seed=None):
    from workloads import smooth_random_coefficient
    wl = make_workload(name)
    co = wl.coeff if coeff_seed is None else smooth_random_coefficient(wl.surface, coeff_seed)
    return wl, co


def test_described_operators_built_by_the_server(ops):
    """Two geometries, two coefficients on one of them: three operators, two near-field
    builds and one clone; results equal caller-built operators' solves; a request on
    a resident operator spends no build time; a second waiter on a ticket is refused."""
    import threading
    import paper_2401_12501_gb300 as pm
    ctx, _ = ops
    wl_a, co_a0 = _desc_parts("ellipsoid_9600")
    _, co_a1 = _desc_parts("ellipsoid_9600", coeff_seed=3)
    wl_b, co_b = _desc_parts("star_small")
    sv = pm.Server(ctx, hbm_budget_bytes=8 << 30, max_batch=8, n_workers=2)
    jobs = [(11, 0, wl_a, co_a0), (11, 1, wl_a, co_a1), (12, 0, wl_b, co_b)]
    fs = {k: rhs_set(j[2], 3, 20 + k) for k, j in enumerate(jobs)}
    first = sv.submit_desc(11, 0, wl_a.surface, co_a0.a, co_a0.grad_a, fs[0][0], tol=1e-10)
    # a second thread may not wait on a ticket another thread is waiting on (the
    # first request waits for the ~1 s near-field build of its geometry)
    got = {}
    th = threading.Thread(target=lambda: got.setdefault("r", sv.wait_ex(first)))
    th.start()
    time.sleep(0.15)
    with pytest.raises(pm.PmError) as e:
        sv.wait(first, timeout_ms=0)
    assert e.value.status == 1 and "already waiting" in str(e.value)
    th.join()
    tickets = []
    for k, (gid, cid, wl, co) in enumerate(jobs):
        for r, f in enumerate(fs[k]):
            if k == 0 and r == 0:
                continue
            tickets.append((k, r, sv.submit_desc(gid, cid, wl.surface, co.a, co.grad_a, f,
                                                 tol=1e-10)))
    res = {(k, r): sv.wait_ex(t) for k, r, t in tickets}
    res[(0, 0)] = got["r"]
    st = sv.stats()
    sv.close()
    assert st["builds"] == 3 and st["operators"] == 3
    assert got["r"][2]["build_s"] > 0.05                    # waited for the near-field build
    for k, (gid, cid, wl, co) in enumerate(jobs):
        s = pm.Surface.from_fixture(ctx, wl.surface)
        s.set_coeff(co.a, co.grad_a)
        w = wl.surface.weights
        for r, f in enumerate(fs[k]):
            u, info, tm = res[(k, r)]
            alone, _ = s.solve(f, tol=1e-10)
            assert info.residual <= 1e-10
            assert np.sqrt(np.dot(w, (u - alone) ** 2) / np.dot(w, alone ** 2)) < 1e-9
            assert tm["latency_s"] >= tm["solve_s"] >= 0
        s.close()


def test_fmm_sized_operator_in_the_mix(ops):
    """Requests on the 98,304-node torus (FMM applies, float-float refinement) mixed with
    requests on small operators: each result equals its operator's standalone solve."""
    import paper_2401_12501_gb300 as pm
    ctx, lst = ops
    wl_t = make_workload("torus_98304")
    big = pm.Surface.from_fixture(ctx, wl_t.surface)
    big.set_coeff(wl_t.coeff.a, wl_t.coeff.grad_a)
    reqs = [(big, wl_t, f, "fmm") for f in rhs_set(wl_t, 3, 31)]
    for idx, (wl, s) in enumerate(lst):
        reqs += [(s, wl, f, "fp32") for f in rhs_set(wl, 3, 40 + idx)]
    order = np.random.default_rng(5).permutation(len(reqs))
    sv = pm.Server(ctx, hbm_budget_bytes=16 << 30, max_batch=8, n_workers=3)
    tickets = [(k, sv.submit(reqs[k][0], reqs[k][2], tol=1e-10, prec=reqs[k][3])) for k in order]
    res = {k: sv.wait(t) for k, t in tickets}
    sv.close()
    for k, (s, wl, f, prec) in enumerate(reqs):
        u, info, _ = res[k]
        alone, _ = s.solve(f, tol=1e-10, prec=prec)
        w = wl.surface.weights
        assert info.residual <= 1e-10
        assert np.sqrt(np.dot(w, (u - alone) ** 2) / np.dot(w, alone ** 2)) < 1e-9
    big.close()

"""Serving loop: continuous batching over several operators.

Requests on three operators are submitted in a mixed order (some while
earlier batches are running); every result must equal the same solve done
alone (pm_solve on that operator) within 1e-9, batching must actually occur,
and a budget that fits one request at a time must still serve everything.
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
    import paper_2401_12501_gb300 as pm
    ctx, lst = ops
    wl, s = lst[0]
    per = (50 + 11) * wl.N * 8
    sv = pm.Server(ctx, hbm_budget_bytes=per, max_batch=16, n_workers=2)
    ts = [sv.submit(s, f, tol=1e-10) for f in rhs_set(wl, 5, 9)]
    outs = [sv.wait(t) for t in ts]
    st = sv.stats()
    sv.close()
    assert st["max_batch"] == 1 and st["solved"] == 5
    assert all(o[1].residual <= 1e-10 for o in outs)
    # a request larger than the whole budget is refused at submit
    tiny = pm.Server(ctx, hbm_budget_bytes=1024, max_batch=4, n_workers=1)
    with pytest.raises(pm.PmError) as e:
        tiny.submit(s, wl.f)
    assert e.value.status == 2
    tiny.close()

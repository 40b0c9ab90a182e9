"""The continuous-batching server: requests admitted by free device memory, batched into
the persistent kernel on several streams. Each served result must be bitwise identical to
the same request solved alone by the batched kernel, and match the FP64 oracle."""
import time

import numpy as np
import pytest

import oracle
from paper_0912_2572_gb300 import inputs
from conftest import to_dev, to_host

pytestmark = pytest.mark.gpu


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def requests(count, seed, mlo=300, mhi=40000, ns=(16, 32, 64, 128)):
    g = inputs.rng(seed)
    out = []
    for q in range(count):
        n = int(g.choice(ns))
        m = max(int(np.exp(g.uniform(np.log(mlo), np.log(mhi)))), n)
        k = int(g.integers(1, 9)) if n < 128 else 0
        A = inputs.graded(m, n, 4.0, seed_g=seed * 1000 + q, seed_v=seed * 1000 + q + 1)
        B = inputs.gaussian(m, k, seed * 1000 + q + 500) if k else None
        out.append((A, B))
    return out


def serve(reqs, chain_tiles=8, **kw):
    import paper_0912_2572_gb300 as ts
    res = {}
    with ts.Server(chain_tiles=chain_tiles, **kw) as srv:
        outs = {}
        for A, B in reqs:
            item = {"A": to_dev(A)}
            if B is not None:
                item["B"] = to_dev(B)
            t, out = srv.submit(item)
            outs[t] = out
        done = []
        deadline = time.time() + 120
        while len(done) < len(reqs) and time.time() < deadline:
            done += srv.poll()
            time.sleep(0.001)
        stats = srv.stats()
    assert len(done) == len(reqs)
    for t, lat, st in done:
        R, X = outs[t]
        res[t] = (st, lat, to_host(R), to_host(X) if X is not None else None)
    return res, stats


def alone(A, B, chain_tiles=8):
    import paper_0912_2572_gb300 as ts
    item = {"A": to_dev(A)}
    if B is not None:
        item["B"] = to_dev(B)
    (R, X), = ts.batch_solve([item], chain_tiles=chain_tiles)
    return to_host(R), to_host(X) if X is not None else None


def test_served_equals_alone_and_oracle(cuda_lib):
    reqs = requests(48, 1)
    res, stats = serve(reqs, max_batch=16, streams=2)
    assert stats["completed"] == len(reqs) and stats["bytes_in_flight"] == 0
    assert stats["batches"] >= 3
    for t, (A, B) in enumerate(reqs):
        st, lat, R, X = res[t]
        assert st == 0 and lat > 0
        R1, X1 = alone(A, B)
        assert np.array_equal(R, R1)
        if B is not None:
            assert np.array_equal(X, X1)
        if t % 6 == 0:
            assert rel(R, oracle.r_factor(A)) <= 1e-12
            if B is not None:
                assert rel(X, oracle.lstsq(A, B)) <= 1e-10


def test_admission_by_memory_budget(cuda_lib):
    """A budget that holds one request at a time forces batches of one; each still runs."""
    reqs = requests(6, 2, mlo=20000, mhi=30000, ns=(32,))
    res, stats = serve(reqs, max_bytes=1, max_batch=64, streams=3)
    assert stats["max_batch"] == 1 and stats["batches"] == len(reqs)
    for t, (A, B) in enumerate(reqs):
        st, _, R, X = res[t]
        assert st == 0
        assert np.array_equal(R, alone(A, B)[0])


def test_server_reports_singular_and_rejects_bad_items(cuda_lib):
    import paper_0912_2572_gb300 as ts
    A = inputs.gaussian(3000, 8, 9)
    A[:, 5] = 0.0
    B = inputs.gaussian(3000, 1, 10)
    good = requests(3, 3, ns=(16,))
    res, _ = serve(good[:1] + [(A, B)] + good[1:], max_batch=8)
    assert [res[t][0] for t in range(4)] == [0, 4, 0, 0]
    with ts.Server() as srv:
        bad = {"A": to_dev(inputs.gaussian(200, 8, 1)), "B": to_dev(inputs.gaussian(200, 140, 2))}  # n + k > 144
        with pytest.raises(ts.TSQRError) as e:
            srv.submit(bad)
        assert e.value.status == 1
        assert srv.stats()["submitted"] == 0


def test_server_drain_and_destroy_finish_everything(cuda_lib):
    import paper_0912_2572_gb300 as ts
    reqs = requests(20, 4, mhi=5000)
    srv = ts.Server(max_batch=4, streams=2)
    keep = [srv.submit({"A": to_dev(A), **({"B": to_dev(B)} if B is not None else {})}) for A, B in reqs]
    srv.drain()
    assert srv.stats()["completed"] == len(reqs)
    assert len(srv.poll()) == len(reqs)
    srv.close()
    assert keep


def test_concurrent_submitters(cuda_lib):
    """Two host threads submit at once; every ticket completes once and every result is
    bitwise the request solved alone."""
    import threading
    import paper_0912_2572_gb300 as ts
    reqs = requests(24, 5, mhi=20000)
    dev = [({"A": to_dev(A), **({"B": to_dev(B)} if B is not None else {})}) for A, B in reqs]
    outs = {}
    lock = threading.Lock()
    with ts.Server(max_batch=8, streams=2, chain_tiles=8) as srv:
        def worker(part):
            for i in part:
                t, out = srv.submit(dev[i])
                with lock:
                    outs[t] = (i, out)
        th = [threading.Thread(target=worker, args=(range(k, len(dev), 2),)) for k in range(2)]
        for t in th:
            t.start()
        for t in th:
            t.join()
        srv.drain()
        done = srv.poll()
    assert sorted(t for t, _, _ in done) == sorted(outs) and len(done) == len(reqs)
    assert all(st == 0 for _, _, st in done)
    for t, (i, (R, X)) in outs.items():
        A, B = reqs[i]
        R1, X1 = alone(A, B)
        assert np.array_equal(to_host(R), R1)
        if B is not None:
            assert np.array_equal(to_host(X), X1)


def mixed_requests(count, seed, mlo=1000, mhi=200_000, ns=(16, 32, 64, 128)):
    """Served least-squares requests shaped like the served workload: m log-uniform, n from
    {16, 32, 64, 128}, k from 1..8 (n = 128 included), kappa log-uniform in [1, 1e4],
    b = A x_true + 1e-6 N(0, 1)."""
    g = inputs.rng(seed)
    out = []
    for q in range(count):
        n = int(ns[q % len(ns)])
        m = max(int(np.exp(g.uniform(np.log(mlo), np.log(mhi)))), n)
        k = int(g.integers(1, 9))
        dec = float(g.uniform(0.0, 4.0))
        A = inputs.graded(m, n, dec, seed_g=seed * 1000 + q, seed_v=seed * 1000 + q + 1)
        B, _ = inputs.lstsq_rhs(A, k, 1e-6, seed * 1000 + q + 500)
        out.append((A, B))
    return out


@pytest.mark.parametrize("prec_name", ["MIXED", "AUTO"])
def test_served_mixed_and_auto_match_oracle(cuda_lib, prec_name):
    """The served mixed-precision path (FP32 leaves, FP64 tree, FP64 refinement) and the
    AUTO policy, through the server's multi-stream batches and refinement launches: every
    X is bitwise the request solved alone with the same precision, and within 1e-10 of the
    FP64 oracle, for kappa up to 1e4, n up to 128 with right-hand sides, and one request of
    a million rows."""
    import paper_0912_2572_gb300 as ts
    prec = getattr(ts, prec_name)
    reqs = mixed_requests(48, 7 if prec_name == "MIXED" else 8)
    A1 = inputs.graded(1_000_000, 32, 4.0, seed_g=70, seed_v=71)
    B1, _ = inputs.lstsq_rhs(A1, 2, 1e-6, 72)
    reqs.append((A1, B1))
    dev = [({"A": to_dev(A), "B": to_dev(B), "prec": prec, "want_r": False}) for A, B in reqs]
    outs = {}
    with ts.Server(max_batch=16, streams=2, chain_tiles=8) as srv:
        for i, it in enumerate(dev):
            t, out = srv.submit(it)
            outs[t] = (i, out)
        srv.drain()
        done = srv.poll()
        stats = srv.stats()
    assert len(done) == len(reqs) and all(st == 0 for _, _, st in done)
    assert stats["batches"] >= 3
    for t, (i, (_, X)) in outs.items():
        A, B = reqs[i]
        Xs = to_host(X)
        (_, Xa), = ts.batch_solve([{"A": dev[i]["A"], "B": dev[i]["B"], "prec": prec, "want_r": False}],
                                  chain_tiles=8)
        assert np.array_equal(Xs, to_host(Xa)), f"request {i}: served != alone"
        err = rel(Xs, oracle.lstsq(A, B))
        assert err <= 1e-10, f"request {i} (m={A.shape[0]}, n={A.shape[1]}, k={B.shape[1]}): {err:.2e}"


def test_server_survives_a_failed_batch_allocation(cuda_lib):
    """Host-side failure injection (no GPU fault): the library's next device allocation
    fails as if the device were out of memory. The batch that hits it reports
    TSQR_ERR_OOM for each of its requests, nothing is left in flight, and the server goes
    on serving: every other request completes and equals the request solved alone."""
    import paper_0912_2572_gb300 as ts
    lib = cuda_lib
    reqs = requests(12, 6, mhi=5000, ns=(16, 32))
    dev = [({"A": to_dev(A), **({"B": to_dev(B)} if B is not None else {})}) for A, B in reqs]
    outs = {}
    try:
        assert lib.tsqr_debug_fail_allocations(1) == 0
        with ts.Server(max_batch=4, streams=1, chain_tiles=8) as srv:
            for i, it in enumerate(dev):
                t, out = srv.submit(it)
                outs[t] = (i, out)
            srv.drain()
            done = srv.poll()
            stats = srv.stats()
    finally:
        lib.tsqr_debug_fail_allocations(0)
    assert len(done) == len(reqs) and stats["bytes_in_flight"] == 0
    st = {t: s for t, _, s in done}
    assert set(st.values()) <= {0, 2} and 1 <= list(st.values()).count(2) <= 4
    assert list(st.values()).count(0) >= len(reqs) - 4
    for t, (i, (R, X)) in outs.items():
        if st[t] != 0:
            continue
        A, B = reqs[i]
        R1, X1 = alone(A, B)
        assert np.array_equal(to_host(R), R1)
        if B is not None:
            assert np.array_equal(to_host(X), X1)


def test_admission_follows_live_free_memory(cuda_lib):
    """Without a budget the server admits by the device memory free at admission time:
    its stats report that figure (positive, at most the device's memory)."""
    import torch
    import paper_0912_2572_gb300 as ts
    reqs = requests(4, 8, mhi=3000, ns=(16,))
    with ts.Server(max_batch=8, streams=2) as srv:
        for A, B in reqs:
            srv.submit({"A": to_dev(A), **({"B": to_dev(B)} if B is not None else {})})
        srv.drain()
        stats = srv.stats()
    total = torch.cuda.get_device_properties(0).total_memory
    assert 0 < stats["budget_bytes"] <= total

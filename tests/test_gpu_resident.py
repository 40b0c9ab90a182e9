"""The resident server: requests admitted into one persistent kernel that is already
running (a ring in device memory the host appends to while the kernel claims from it;
refinement steps of mixed requests queued by the kernel itself). Every served result must
be bitwise the request solved alone by tsqr_batch_solve and match the FP64 oracle."""
import time

import numpy as np
import pytest

import oracle
from paper_0912_2572_gb300 import inputs
from conftest import to_dev, to_host
from test_gpu_server import mixed_requests, rel, requests

pytestmark = pytest.mark.gpu


def _item(A, B, prec=None, want_r=True):
    import paper_0912_2572_gb300 as ts
    it = {"A": to_dev(A), "want_r": want_r, "prec": ts.FP64 if prec is None else prec}
    if B is not None:
        it["B"] = to_dev(B)
    return it


def _alone(it, chain_tiles):
    import paper_0912_2572_gb300 as ts
    (R, X), = ts.batch_solve([dict(it)], chain_tiles=chain_tiles)
    return (to_host(R) if R is not None else None), (to_host(X) if X is not None else None)


def _serve(srv, items, gap_s=0.0):
    outs = {}
    for i, it in enumerate(items):
        t, out = srv.submit(it)
        outs[t] = (i, out)
        if gap_s:
            time.sleep(gap_s)
    srv.drain()
    done = srv.poll()
    assert sorted(t for t, _, _ in done) == sorted(outs)
    return outs, {t: (lat, st) for t, lat, st in done}


@pytest.mark.parametrize("prec_name", ["FP64", "MIXED", "AUTO"])
def test_resident_equals_alone_and_oracle(cuda_lib, prec_name):
    """Served requests of the served workload's shape (m log-uniform, n in {16, 32, 64, 128}
    with 1..8 right-hand sides, kappa up to 1e4): X bitwise the request alone, within 1e-10
    of the FP64 oracle; FP64 requests also R bitwise alone and within 1e-12 of the oracle.
    FP64 requests with n = 128 need one CTA per SM (their tile is wider than half an SM's
    shared memory), so the FP64 case runs the kernel at one CTA per SM."""
    import paper_0912_2572_gb300 as ts
    prec = getattr(ts, prec_name)
    reqs = mixed_requests(24, {"FP64": 21, "MIXED": 22, "AUTO": 23}[prec_name], mhi=120_000)
    items = [_item(A, B, prec, want_r=(prec_name == "FP64")) for A, B in reqs]
    cps = 1 if prec_name == "FP64" else 2
    with ts.Server(resident=True, chain_tiles=8, ctas_per_sm=cps, idle_us=50_000) as srv:
        outs, done = _serve(srv, items)
        stats = srv.stats()
    assert all(st == 0 for _, st in done.values())
    assert stats["completed"] == len(reqs) and stats["bytes_in_flight"] == 0 and stats["launches"] >= 1
    for t, (i, (R, X)) in outs.items():
        A, B = reqs[i]
        R1, X1 = _alone(items[i], 8)
        assert np.array_equal(to_host(X), X1), f"request {i}: served X != alone"
        assert rel(to_host(X), oracle.lstsq(A, B)) <= 1e-10
        if prec_name == "FP64":
            assert np.array_equal(to_host(R), R1)
            if i % 4 == 0:
                assert rel(to_host(R), oracle.r_factor(A)) <= 1e-12


def test_resident_admits_into_the_running_kernel(cuda_lib):
    """A long request keeps the kernel busy while more arrive one by one: all of them are
    admitted into that one launch (one launch in the stats) and each equals the request
    solved alone."""
    import paper_0912_2572_gb300 as ts
    big = inputs.graded(1_000_000, 64, 3.0, seed_g=31, seed_v=32)
    Bb, _ = inputs.lstsq_rhs(big, 2, 1e-6, 33)
    reqs = [(big, Bb)] + mixed_requests(12, 24, mhi=30_000, ns=(16, 32, 64))
    items = [_item(A, B, ts.MIXED, want_r=False) for A, B in reqs]
    with ts.Server(resident=True, chain_tiles=8, idle_us=500_000) as srv:
        outs, done = _serve(srv, items, gap_s=0.0005)
        stats = srv.stats()
    assert stats["launches"] == 1, stats
    assert stats["max_in_flight"] >= 2
    assert all(st == 0 for _, st in done.values())
    for t, (i, (_, X)) in outs.items():
        assert np.array_equal(to_host(X), _alone(items[i], 8)[1]), f"request {i}"


def test_resident_relaunches_after_idle(cuda_lib):
    """With a short idle time the kernel ends between two bursts and is launched again;
    the second burst is served correctly by the new launch."""
    import paper_0912_2572_gb300 as ts
    reqs = mixed_requests(8, 25, mhi=20_000, ns=(16, 32))
    items = [_item(A, B, ts.MIXED, want_r=False) for A, B in reqs]
    with ts.Server(resident=True, chain_tiles=8, idle_us=200) as srv:
        outs1, done1 = _serve(srv, items[:4])
        time.sleep(0.2)
        outs2, done2 = _serve(srv, items[4:])
        stats = srv.stats()
    assert stats["launches"] >= 2 and stats["completed"] == len(items)
    for outs, off in ((outs1, 0), (outs2, 4)):
        for t, (i, (_, X)) in outs.items():
            A, B = reqs[off + i]
            assert np.array_equal(to_host(X), _alone(items[off + i], 8)[1])
            assert rel(to_host(X), oracle.lstsq(A, B)) <= 1e-10


def test_resident_refuses_what_it_cannot_run(cuda_lib):
    """At two CTAs per SM an FP64 request of 128 + 8 columns needs more shared memory than a
    CTA has: submit refuses it (TSQR_ERR_UNSUPPORTED), nothing is queued. Invalid items
    are refused as on the launching server."""
    import paper_0912_2572_gb300 as ts
    A = inputs.gaussian(2000, 128, 41)
    B = inputs.gaussian(2000, 8, 42)
    with ts.Server(resident=True, ctas_per_sm=2) as srv:
        with pytest.raises(ts.TSQRError) as e:
            srv.submit(_item(A, B))
        assert e.value.status == 6
        bad = {"A": to_dev(inputs.gaussian(200, 8, 1)), "B": to_dev(inputs.gaussian(200, 140, 2))}
        with pytest.raises(ts.TSQRError) as e:
            srv.submit(bad)
        assert e.value.status == 1
        assert srv.stats()["submitted"] == 0


def test_resident_singular_and_failure_injection(cuda_lib):
    """A request with a zero column reports TSQR_ERR_SINGULAR; a request whose admission
    hits an injected allocation failure reports TSQR_ERR_OOM; the rest complete and equal
    the request solved alone."""
    import paper_0912_2572_gb300 as ts
    lib = cuda_lib
    A0 = inputs.gaussian(3000, 8, 9)
    A0[:, 5] = 0.0
    B0 = inputs.gaussian(3000, 1, 10)
    reqs = requests(6, 26, mhi=5000, ns=(16, 32))
    items = [_item(A0, B0)] + [_item(A, B) for A, B in reqs]
    try:
        assert lib.tsqr_debug_fail_allocations(0) == 0
        with ts.Server(resident=True, chain_tiles=8, idle_us=20_000) as srv:
            srv.submit(items[0])
            srv.drain()
            (_, _, st0), = srv.poll()
            lib.tsqr_debug_fail_allocations(1)
            outs, done = _serve(srv, items[1:])
            stats = srv.stats()
    finally:
        lib.tsqr_debug_fail_allocations(0)
    assert st0 == 4
    sts = [st for _, st in done.values()]
    assert sts.count(2) == 1 and sts.count(0) == len(sts) - 1
    assert stats["bytes_in_flight"] == 0
    for t, (i, (R, X)) in outs.items():
        if done[t][1] != 0:
            continue
        R1, X1 = _alone(items[1 + i], 8)
        assert np.array_equal(to_host(R), R1)
        if X1 is not None:
            assert np.array_equal(to_host(X), X1)


def test_resident_rings_wrap_around(cuda_lib):
    """Rings of 16 entries (the test hook): 40 FP64 and mixed requests of a few chain jobs
    and refinement tasks each wrap both rings several times; admission waits for room in
    them; every result equals the request solved alone. A request with more chain jobs than
    a ring holds is refused at submission."""
    import paper_0912_2572_gb300 as ts
    lib = cuda_lib
    reqs = mixed_requests(40, 27, mlo=2000, mhi=20_000, ns=(16, 32, 64))
    items = [_item(A, B, ts.MIXED if i % 2 else ts.FP64, want_r=False) for i, (A, B) in enumerate(reqs)]
    try:
        assert lib.tsqr_debug_resident_ring_entries(16) == 0
        assert lib.tsqr_debug_resident_ring_entries(24) == 1  # not a power of two
        with ts.Server(resident=True, chain_tiles=8, idle_us=2_000) as srv:
            outs, done = _serve(srv, items)
            big = inputs.gaussian(200_000, 16, 28)
            with pytest.raises(ts.TSQRError) as e:
                srv.submit(_item(big, None, ts.MIXED, want_r=True))
            assert e.value.status == 6
            stats = srv.stats()
    finally:
        lib.tsqr_debug_resident_ring_entries(0)
    assert all(st == 0 for _, st in done.values())
    assert stats["completed"] == len(items) and stats["bytes_in_flight"] == 0
    for t, (i, (_, X)) in outs.items():
        assert np.array_equal(to_host(X), _alone(items[i], 8)[1]), f"request {i}"
        if i % 8 == 0:
            A, B = reqs[i]
            assert rel(to_host(X), oracle.lstsq(A, B)) <= 1e-10

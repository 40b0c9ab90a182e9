"""The library's autotuners (tsqr_batch_autotune, tsqr_factor_autotune): they time their
candidates on the caller's data and return one of them; the configuration they return
must give results that match the oracle."""
import numpy as np
import pytest

import oracle
from paper_0912_2572_gb300 import inputs
from conftest import to_dev, to_host

pytestmark = pytest.mark.gpu


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_batch_autotune_returns_the_fastest_candidate(cuda_lib):
    import paper_0912_2572_gb300 as ts
    g = inputs.rng(31)
    host, dev = [], []
    for q in range(48):
        m = int(np.exp(g.uniform(np.log(300), np.log(30000))))
        n = int(g.choice([8, 16, 32, 64]))
        A = inputs.gaussian(max(m, n), n, 3100 + q)
        host.append(A)
        dev.append({"A": to_dev(A), "prec": q & 1})
    L, ar, table = ts.batch_autotune(dev, sample=32)
    assert (L, ar) in ts.BATCH_TUNE_CANDIDATES
    assert sorted(table) == sorted(ts.BATCH_TUNE_CANDIDATES)
    assert all(t > 0 for t in table.values())
    assert table[(L, ar)] == min(table.values())
    outs, st = ts.batch_solve(dev, chain_tiles=L, arity=ar, status=True)
    assert st == [0] * len(dev)
    for q, (A, (R, _)) in enumerate(zip(host, outs)):
        assert rel(to_host(R), oracle.r_factor(A)) <= (1e-12 if q % 2 == 0 else 1e-5)


def test_factor_autotune_configuration_matches_oracle(cuda_lib):
    import paper_0912_2572_gb300 as ts
    m, n = 200_000, 16
    A = inputs.graded(m, n, 4.0, seed_g=41, seed_v=42)
    Ad = to_dev(A)
    before = Ad.clone()
    cfg = ts.factor_autotune(Ad)
    assert bool((Ad == before).all())  # A is not modified
    tile = ts.plan_describe(m, n, 1 << 20)["tile_rows"]
    assert cfg["leaf_h"] in (tile, 4 * tile, 16 * tile)
    assert cfg["arity"] in (0, 2, 4) and cfg["ms"] > 0
    assert cfg["arity"] != 0 or not cfg["two_level"]
    F = ts.factor(Ad, leaf_h=cfg["leaf_h"], arity=cfg["arity"], two_level=cfg["two_level"])
    R = to_host(F.R)
    F.free()
    assert rel(R, oracle.r_factor(A)) <= 1e-12


def test_factor_autotune_small_matrix(cuda_lib):
    """A matrix of at most one tile per SM also tries the flat tree (one chain)."""
    import paper_0912_2572_gb300 as ts
    m, n = 20_000, 16
    A = inputs.gaussian(m, n, 77)
    Ad = to_dev(A)
    cfg = ts.factor_autotune(Ad)
    assert cfg["ms"] > 0 and cfg["arity"] in (0, 2, 4)
    F = ts.factor(Ad, leaf_h=cfg["leaf_h"], arity=cfg["arity"], two_level=cfg["two_level"])
    R = to_host(F.R)
    F.free()
    assert rel(R, oracle.r_factor(A)) <= 1e-12

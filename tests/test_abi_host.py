"""Host-side checks of the C ABI (no GPU): the library loads and exports every symbol the
public header declares, argument errors are reported before any CUDA work, and the
planner builds the leaf partition and reduction tree of paper §2.3 (k-ary, flat, and
the two-level tree) correctly."""
import ctypes
import math

import pytest

from paper_0912_2572_gb300 import _lib, build

# a GB300-like device description: 152 SMs, 228 KiB shared memory per SM
GB300 = dict(sms=152, smem=233472, reserved=1024, optin=232448)


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _lib.load()


def test_every_declared_symbol_is_exported(lib):
    names = _lib.declared_functions()
    assert {"tsqr_factor", "tsqr_apply_qt", "tsqr_apply_q", "tsqr_form_q", "tsqr_lstsq",
            "tsqr_free"} <= set(names)
    missing = [n for n in names if not hasattr(lib, n)]
    assert missing == []


def test_strerror(lib):
    assert lib.tsqr_strerror(0) == b"success"
    assert lib.tsqr_strerror(1) == b"invalid argument"
    assert lib.tsqr_strerror(4) == b"R is singular"


FAKE = 4096  # a non-null address that must never be dereferenced by argument checks


@pytest.mark.parametrize("kw,why", [
    (dict(A=0), "A is NULL"),
    (dict(n=0), "n=0"),
    (dict(n=129), "n=129"),
    (dict(m=10, n=11, leaf_h=11), "m=10 < n"),
    (dict(lda=99), "lda=99"),
    (dict(leaf_h=8), "leaf_h=8 < n"),
    (dict(arity=1), "arity=1"),
    (dict(arity=17), "arity=17"),
    (dict(F=False), "F is NULL"),
    (dict(ldr=3), "ldr=3"),
    (dict(flags=8), "unknown flags"),
    (dict(prec=7), "unknown prec"),
])
def test_factor_argument_errors(lib, kw, why):
    a = dict(A=FAKE, m=100, n=16, lda=100, leaf_h=32, arity=2, prec=0, flags=0, F=True, ldr=16)
    a.update(kw)
    h = ctypes.c_void_p()
    st = lib.tsqr_factor(a["A"], a["m"], a["n"], a["lda"], a["leaf_h"], a["arity"], a["prec"], a["flags"],
                         None, ctypes.byref(h) if a["F"] else None, FAKE, a["ldr"])
    assert st == 1
    assert why.split()[0] in lib.tsqr_last_error().decode()
    assert not h.value


@pytest.mark.parametrize("kw,why", [
    (dict(A=0), "A is NULL"),
    (dict(n=4097, m=5000, lda=5000), "n=4097"),
    (dict(m=100, n=101, lda=101), "m=100 < n"),
    (dict(lda=99), "lda=99"),
    (dict(panel=129), "panel=129"),
    (dict(panel=-1), "panel=-1"),
    (dict(leaf_h=63), "leaf_h=63 < panel"),
    (dict(arity=17), "arity=17"),
    (dict(F=False), "F is NULL"),
    (dict(ldr=199), "ldr=199"),
    (dict(flags=8), "unknown flags"),
])
def test_caqr_argument_errors(lib, kw, why):
    """tsqr_caqr (CAQR for wide matrices, paper §2.4) rejects bad arguments on the host."""
    a = dict(A=FAKE, m=1000, n=200, lda=1000, panel=0, leaf_h=64, arity=2, flags=0, F=True, ldr=200)
    a.update(kw)
    h = ctypes.c_void_p()
    st = lib.tsqr_caqr(a["A"], a["m"], a["n"], a["lda"], a["panel"], a["leaf_h"], a["arity"], a["flags"], None,
                       ctypes.byref(h) if a["F"] else None, FAKE, a["ldr"])
    assert st == 1
    assert why.split()[0] in lib.tsqr_last_error().decode()
    assert not h.value


def test_wide_least_squares_arguments(lib):
    """tsqr_lstsq with n > 128 goes through CAQR: FP64 only, same argument checks."""
    assert lib.tsqr_lstsq(FAKE, 1000, 200, 1000, FAKE, 1000, 1, FAKE, 200, 256, 2, 1, 0, 0, None, None) == 6
    assert lib.tsqr_lstsq(FAKE, 1000, 200, 1000, FAKE, 1000, 0, FAKE, 200, 256, 2, 0, 0, 0, None, None) == 1
    assert lib.tsqr_lstsq(FAKE, 1000, 200, 1000, FAKE, 1000, 1, FAKE, 199, 256, 2, 0, 0, 0, None, None) == 1
    assert lib.tsqr_lstsq(FAKE, 1000, 200, 1000, FAKE, 1000, 1, FAKE, 200, 32, 2, 0, 0, 0, None, None) == 1


def test_factor_mixed_is_unsupported(lib):
    h = ctypes.c_void_p()
    st = lib.tsqr_factor(FAKE, 100, 16, 100, 32, 2, 1, 0, None, ctypes.byref(h), FAKE, 16)
    assert st == 6


def test_other_entry_points_reject_null(lib):
    assert lib.tsqr_apply_qt(None, FAKE, 10, 1, None) == 1
    assert lib.tsqr_apply_q(None, FAKE, 10, 1, None) == 1
    assert lib.tsqr_form_q(None, FAKE, 10, None) == 1
    assert lib.tsqr_free(None) == 0
    assert lib.tsqr_factors_info(None, None) == 1
    # least squares: k outside [1, 64], null X, bad ldx
    assert lib.tsqr_lstsq(FAKE, 100, 8, 100, FAKE, 100, 0, FAKE, 8, 32, 2, 0, 0, 0, None, None) == 1
    assert lib.tsqr_lstsq(FAKE, 100, 8, 100, FAKE, 100, 65, FAKE, 8, 32, 2, 0, 0, 0, None, None) == 1
    assert lib.tsqr_lstsq(FAKE, 100, 8, 100, FAKE, 100, 1, None, 8, 32, 2, 0, 0, 0, None, None) == 1
    assert lib.tsqr_lstsq(FAKE, 100, 8, 100, FAKE, 100, 1, FAKE, 7, 32, 2, 0, 0, 0, None, None) == 1


def describe(lib, m, n, h, arity, flags, nc=None, dev=GB300):
    nc = n if nc is None else nc
    out = (ctypes.c_int64 * 8)()
    st = lib.tsqr_plan_describe(m, n, nc, h, arity, flags, dev["sms"], dev["smem"], dev["reserved"],
                                dev["optin"], out, None, 0, None, 0)
    assert st == 0, lib.tsqr_last_error()
    ntiles, njobs = out[5], out[4]
    tiles = (ctypes.c_int64 * (5 * ntiles))()
    jobs = (ctypes.c_int64 * (4 * njobs))()
    st = lib.tsqr_plan_describe(m, n, nc, h, arity, flags, dev["sms"], dev["smem"], dev["reserved"],
                                dev["optin"], out, tiles, ntiles, jobs, njobs)
    assert st == 0
    info = dict(zip(["m", "n", "leaves", "tile_rows", "jobs", "tiles", "launches", "cps"], list(out)))
    T = [tuple(tiles[5 * t:5 * t + 5]) for t in range(ntiles)]
    J = [tuple(jobs[4 * j:4 * j + 4]) for j in range(njobs)]
    return info, T, J


def check_plan(m, n, h, arity, flags, info, T, J):
    P = max(1, m // h)
    assert info["leaves"] == P
    th = info["tile_rows"]
    assert n <= th <= 512
    # launch 0: the chains cover every row exactly once, tiles in row order per job
    chain_jobs = [j for j in J if j[3] == 0]
    covered = []
    for piv, tb, tc, _ in chain_jobs:
        tl = T[tb:tb + tc]
        assert tl[0][2] == 0 and tl[0][0] == piv and tl[0][1] >= n  # leaf QR first, >= n rows
        assert all(t[2] == 1 for t in tl[1:])                      # then triangle-on-tile
        for r0, rows, kind, job, launch in tl:
            assert 1 <= rows <= th
            covered.append((r0, r0 + rows))
    covered.sort()
    assert covered[0][0] == 0 and covered[-1][1] == m
    assert all(a[1] == b[0] for a, b in zip(covered, covered[1:]))
    # the tree: every chain result is merged into the root (row 0) exactly once
    sets = {j[0]: {j[0]} for j in chain_jobs}
    nlaunch = max(j[3] for j in J)
    for lvl in range(1, nlaunch + 1):
        for piv, tb, tc, launch in (j for j in J if j[3] == lvl):
            assert tc >= 1 and (arity == 0 or tc <= arity - 1)
            for r0, rows, kind, job, _ in T[tb:tb + tc]:
                assert kind == 2 and rows == n
                assert r0 in sets and piv in sets and r0 != piv
                sets[piv] |= sets.pop(r0)
    assert list(sets) == [0] and sets[0] == {j[0] for j in chain_jobs}
    return chain_jobs, nlaunch


@pytest.mark.parametrize("m,n,h,arity", [(4096, 16, 256, 2), (4096, 16, 256, 4), (4096, 16, 256, 0),
                                         (10000, 7, 100, 3), (1000, 64, 64, 2), (130, 128, 128, 2),
                                         (2049, 1, 1, 2), (64, 64, 64, 2), (4_194_304, 64, 208, 2)])
def test_pure_trees(lib, m, n, h, arity):
    """A k-ary tree over P leaves has ceil(log_k P) sequential levels of n x n
    triangle-on-triangle combines: for the binary tree this is the paper's message count
    log2(P) for R only, each level adding one 2/3 n^3 combine to the critical path
    (Table 1; Table 2 doubles both when Q is formed)."""
    info, T, J = describe(lib, m, n, h, arity, 0)
    chain_jobs, nlaunch = check_plan(m, n, h, arity, 0, info, T, J)
    P = max(1, m // h)
    if arity == 0:
        assert len(chain_jobs) == 1 and nlaunch == 0
    else:
        assert len(chain_jobs) == P
        assert nlaunch == (0 if P == 1 else math.ceil(math.log(P, arity) - 1e-9))


@pytest.mark.parametrize("m,n,h,arity", [(4_194_304, 64, 208, 2), (4_194_304, 64, 208, 4),
                                         (4_194_304, 64, 1024, 0), (16_777_216, 32, 512, 2),
                                         (5000, 64, 208, 2)])
def test_two_level_tree(lib, m, n, h, arity):
    info, T, J = describe(lib, m, n, h, arity, 2)
    chain_jobs, _ = check_plan(m, n, h, arity, 2, info, T, J)
    P = max(1, m // h)
    G = min(P, GB300["sms"] * info["cps"] * 4)
    assert len(chain_jobs) == G
    sizes = [sum(1 for t in T[tb:tb + tc]) for _, tb, tc, _ in chain_jobs]
    # balanced chains: leaf counts differ by at most one, and the last leaf (which takes
    # the remainder rows) may need one more tile
    assert max(sizes) - min(sizes) <= 2 * math.ceil(h / info["tile_rows"])


def test_tile_capacity_choice(lib):
    # n = 64: three CTAs per SM fit a 144-row tile (>= 2n rows, so the third CTA is taken);
    # n = 96: a three-CTA tile would hold 96 rows < 2n, so two CTAs with 144 rows;
    # n = 128 needs one CTA per SM
    info, _, _ = describe(lib, 100_000, 64, 1024, 2, 2)
    assert info["cps"] == 3 and info["tile_rows"] == 144
    info, _, _ = describe(lib, 100_000, 96, 1024, 2, 2)
    assert info["cps"] == 2 and info["tile_rows"] == 144
    info, _, _ = describe(lib, 100_000, 128, 1024, 2, 2)
    assert info["cps"] == 1 and info["tile_rows"] >= 128
    # the fused least-squares factorization sees n + k columns
    info, _, _ = describe(lib, 100_000, 64, 1024, 2, 2, nc=72)
    assert info["cps"] == 3 and info["tile_rows"] == 128
    # the leaf height caps the tile
    info, _, _ = describe(lib, 100_000, 16, 100, 2, 0)
    assert info["tile_rows"] == 100
    # small widths: the three-CTA plan with 512-row tiles, the apply kernels' cap
    info, _, _ = describe(lib, 1_000_000, 8, 1024, 2, 2)
    assert info["cps"] == 3 and info["tile_rows"] == 512


def test_server_entry_points_reject_bad_arguments(lib):
    h = ctypes.c_void_p()
    assert lib.tsqr_server_create(0, 0, 2, 0, 0, ctypes.byref(h)) == 1      # max_batch < 1
    assert lib.tsqr_server_create(0, 16, 0, 0, 0, ctypes.byref(h)) == 1     # no stream
    assert lib.tsqr_server_create(0, 16, 17, 0, 0, ctypes.byref(h)) == 1    # too many streams
    assert lib.tsqr_server_create(0, 16, 2, -1, 0, ctypes.byref(h)) == 1    # chain_tiles < 0
    assert lib.tsqr_server_create(0, 16, 2, 0, 3, ctypes.byref(h)) == 1     # ctas_per_sm > 2
    assert lib.tsqr_server_create(0, 16, 2, 0, 0, None) == 1
    # the resident server: bad chain_tiles, ctas_per_sm, idle_us or output, before any CUDA call
    assert lib.tsqr_server_create_resident(0, -1, 0, 1000, ctypes.byref(h)) == 1
    assert lib.tsqr_server_create_resident(0, 0, 3, 1000, ctypes.byref(h)) == 1
    assert lib.tsqr_server_create_resident(0, 0, 0, -1, ctypes.byref(h)) == 1
    assert lib.tsqr_server_create_resident(0, 0, 0, 1000, None) == 1
    # its ring-size test hook: powers of two from 16, or 0 for the default
    for bad in (1, 8, 24, 100, -16):
        assert lib.tsqr_debug_resident_ring_entries(bad) == 1
    assert lib.tsqr_debug_resident_ring_entries(64) == 0
    assert lib.tsqr_debug_resident_ring_entries(0) == 0
    assert not h.value
    c = ctypes.c_int32(0)
    assert lib.tsqr_server_submit(None, None, None) == 1
    assert lib.tsqr_server_poll(None, 4, None, None, None, ctypes.byref(c)) == 1
    assert lib.tsqr_server_drain(None) == 1
    assert lib.tsqr_server_stats(None, None) == 1
    assert lib.tsqr_server_destroy(None) == 0


def test_factor_qt_rejects_bad_arguments(lib):
    h = ctypes.c_void_p()
    ptr = ctypes.c_void_p(256)
    assert lib.tsqr_factor_qt(ptr, 100, 4, 100, None, 100, 1, 16, 2, 0, 0, None, ctypes.byref(h), None, 4) == 1
    assert lib.tsqr_factor_qt(ptr, 100, 4, 100, ptr, 100, 0, 16, 2, 0, 0, None, ctypes.byref(h), None, 4) == 1
    assert lib.tsqr_factor_qt(ptr, 100, 4, 100, ptr, 99, 1, 16, 2, 0, 0, None, ctypes.byref(h), None, 4) == 1
    assert lib.tsqr_factor_qt(ptr, 100, 4, 100, ptr, 100, 1, 16, 2, 0, 1, None, ctypes.byref(h), None, 4) == 1
    assert lib.tsqr_factor_qt(None, 100, 4, 100, ptr, 100, 1, 16, 2, 0, 0, None, ctypes.byref(h), None, 4) == 1
    assert not h.value


def test_orthonormalize_rejects_bad_arguments(lib):
    ptr = ctypes.c_void_p(256)
    f = lib.tsqr_orthonormalize
    assert f(ptr, 100, 4, 100, None, 100, None, 4, 16, 2, 0, 0, None) == 1     # Q NULL
    assert f(ptr, 100, 4, 100, ptr, 99, None, 4, 16, 2, 0, 0, None) == 1       # ldq < m
    assert f(ptr, 100, 4, 100, ptr, 100, None, 4, 16, 2, 0, 1, None) == 1      # INPLACE
    assert f(None, 100, 4, 100, ptr, 100, None, 4, 16, 2, 0, 0, None) == 1     # A NULL
    assert f(ptr, 100, 4, 100, ptr, 100, ptr, 3, 16, 2, 0, 0, None) == 1       # ldr < n
    assert f(ptr, 3, 4, 3, ptr, 3, None, 4, 16, 2, 0, 0, None) == 1            # m < n
    assert f(ptr, 100, 4, 100, ptr, 100, None, 4, 16, 2, 1, 0, None) == 6      # MIXED


def test_autotuners_reject_bad_arguments(lib):
    L, a, f = ctypes.c_int32(0), ctypes.c_int32(0), ctypes.c_int32(0)
    item = _lib.BatchItem()                   # A = NULL: an invalid item
    item.m, item.n, item.lda = 100, 4, 100
    assert lib.tsqr_batch_autotune(None, 1, 0, None, ctypes.byref(L), ctypes.byref(a), None) == 1
    assert lib.tsqr_batch_autotune(ctypes.byref(item), 0, 0, None, ctypes.byref(L), ctypes.byref(a), None) == 1
    assert lib.tsqr_batch_autotune(ctypes.byref(item), 1, 0, None, ctypes.byref(L), ctypes.byref(a), None) == 1
    assert lib.tsqr_factor_autotune(None, 100, 4, 100, None, ctypes.byref(L), ctypes.byref(a), ctypes.byref(f),
                                    None) == 1
    assert lib.tsqr_factor_autotune(ctypes.c_void_p(256), 100, 4, 100, None, None, ctypes.byref(a),
                                    ctypes.byref(f), None) == 1
    assert lib.tsqr_factor_autotune(ctypes.c_void_p(256), 3, 4, 100, None, ctypes.byref(L), ctypes.byref(a),
                                    ctypes.byref(f), None) == 1   # m < n


def test_batch_plan_entry_points_reject_bad_arguments(lib):
    h = ctypes.c_void_p()
    assert lib.tsqr_batch_plan_create(None, 1, 0, 0, ctypes.byref(h)) == 1
    assert lib.tsqr_batch_plan_create(None, 0, 0, 0, ctypes.byref(h)) == 1
    assert lib.tsqr_batch_plan_create(None, 1, 0, 0, None) == 1
    assert not h.value
    assert lib.tsqr_batch_plan_run(None, None) == 1
    assert lib.tsqr_batch_plan_results(None, None, None) == 1
    assert lib.tsqr_batch_plan_destroy(None) == 0


def clusters(lib, m, n, h, flags, nc=None, dev=GB300):
    nc = n if nc is None else nc
    out = (ctypes.c_int64 * 2)()
    st = lib.tsqr_plan_clusters(m, n, nc, h, flags, dev["sms"], dev["smem"], dev["reserved"], dev["optin"], out,
                                None, 0, None, 0)
    assert st == 0, lib.tsqr_last_error()
    nl, ns = out[0], out[1]
    L = (ctypes.c_int32 * max(1, 4 * nl))()
    S = (ctypes.c_int32 * max(1, 3 * ns))()
    assert lib.tsqr_plan_clusters(m, n, nc, h, flags, dev["sms"], dev["smem"], dev["reserved"], dev["optin"], out,
                                  L, nl, S, ns) == 0
    return [tuple(L[4 * q:4 * q + 4]) for q in range(nl)], [tuple(S[3 * q:3 * q + 3]) for q in range(ns)]


@pytest.mark.parametrize("m,n,h,flags", [
    (4_194_304, 64, 144, 2), (1 << 20, 16, 64, 2), (100_000, 32, 64, 0), (5000, 64, 64, 0),
    (3000, 16, 100, 0), (640, 64, 64, 0), (200, 8, 64, 0), (4096, 16, 256, 0), (1 << 20, 65, 144, 2),
])
def test_cluster_schedule_simulated(lib, m, n, h, flags):
    """Host simulation of the TSQR_CLUSTER schedule against the binary tree of
    tsqr_plan_describe: every combine job runs exactly once, in the launch that covers its
    level; a slot's in-cluster children are the jobs that produced its pivot and tile
    triangles (same rows), with a lower rank (the pipeline's waits point down the tree, so
    no CTA waits on itself or in a cycle); out-of-cluster children were finished by an
    earlier launch. Replaying the launches in order reduces every chain into the root."""
    info, T, J = describe(lib, m, n, h, 2, flags | 4)  # TSQR_CLUSTER: the same jobs, fewer launches
    launches, slots = clusters(lib, m, n, h, flags)
    nlevels = max(j[3] for j in J)
    if nlevels == 0:
        assert launches == [] and slots == []
        return
    # levels too wide for one wave of clusters stay one launch each; the rest go in threes
    base = launches[0][2] - 1
    assert 0 <= base < nlevels and len(launches) == (nlevels - base + 2) // 3
    chains = sum(1 for j in J if j[3] == 0)
    width = -(-chains // 2 ** base)
    assert -(-width // 8) * 8 <= GB300["sms"] * (2 if n > 64 else 3)  # the first cluster launch is one wave
    assert info["launches"] == 1 + base + len(launches) + 1  # chains, plain levels, clusters, sign fix
    seen = set()
    done_before = {j[0]: True for j in J if j[3] <= base}  # pivot row -> its triangle is final
    for sb, ncl, lo, hi in launches:
        assert 1 <= lo <= hi <= nlevels and hi - lo <= 2
        final_here = {}
        for c in range(ncl):
            cl = slots[sb + 8 * c: sb + 8 * c + 8]
            for rank, (job, c0, c1) in enumerate(cl):
                if job < 0:
                    assert c0 == -1 and c1 == -1
                    continue
                piv, tb, tc, lvl = J[job]
                assert lo <= lvl <= hi and job not in seen
                seen.add(job)
                assert tc == 1
                trow = T[tb][0]
                for ch, row in ((c0, piv), (c1, trow)):
                    if ch < 0:
                        assert done_before.get(row), "an external child must be final before the launch"
                    else:
                        assert 0 <= ch < rank
                        cj = cl[ch][0]
                        assert cj >= 0 and J[cj][0] == row and J[cj][3] < lvl
                final_here[piv] = True
        done_before.update(final_here)
    assert seen == {i for i, j in enumerate(J) if j[3] > base}


def test_cluster_flag_ignored_when_it_cannot_fit(lib):
    """n = 128 triangles do not fit one CTA's shared memory twice: no cluster schedule, the
    plain per-level launches stay."""
    launches, slots = clusters(lib, 1 << 20, 128, 128, 2)
    assert launches == [] and slots == []


def batch_jobs(lib, items, chain_tiles=8, arity=2, dev=GB300):
    arr = (_lib.BatchItem * len(items))()
    for q, (m, n, k, prec) in enumerate(items):
        arr[q].A, arr[q].m, arr[q].n, arr[q].lda = FAKE, m, n, m
        arr[q].B, arr[q].ldb, arr[q].k = (FAKE if k else None), m, k
        arr[q].R, arr[q].ldr, arr[q].X, arr[q].ldx, arr[q].prec = FAKE, n, (FAKE if k else None), n, prec
    out = (ctypes.c_int64 * 4)()
    st = lib.tsqr_batch_describe(arr, len(items), chain_tiles, arity, dev["sms"], dev["smem"], dev["reserved"],
                                 dev["optin"], out, None, 0)
    assert st == 0, lib.tsqr_last_error()
    nj = out[1]
    J = (ctypes.c_int64 * (7 * nj))()
    assert lib.tsqr_batch_describe(arr, len(items), chain_tiles, arity, dev["sms"], dev["smem"], dev["reserved"],
                                   dev["optin"], out, J, nj) == 0
    return out[0], [tuple(J[7 * j:7 * j + 7]) for j in range(nj)]


@pytest.mark.parametrize("chain_tiles,arity", [(8, 2), (2, 4), (32, 2), (1, 16)])
def test_batch_job_table_simulated(lib, chain_tiles, arity):
    """Host simulation of the persistent batched kernel's protocol on its real job table:
    CTAs finish chain jobs in an arbitrary order; a finished job arrives at its parent's
    counter and the last child to arrive runs the parent. Every job must run exactly once
    and only after all of its children, every item's root must be reached exactly once,
    and a node's child count must equal the jobs that name it as parent. Several random
    completion orders are replayed."""
    import random
    g = random.Random(chain_tiles * 31 + arity)
    items = []
    for q in range(40):
        n = g.choice([1, 8, 16, 33, 64, 100, 128])
        m = max(n, int(2 ** g.uniform(8, 17)))
        prec = g.choice([0, 1])
        k = g.choice([0, 0, 3]) if n <= 100 else 0
        items.append((m, n, k, prec))
    nchains, J = batch_jobs(lib, items, chain_tiles, arity)
    nj = len(J)
    assert 0 < nchains <= nj
    kids = [0] * nj
    for j, (inst, parent, nchild, *_rest) in enumerate(J):
        assert -1 <= parent < nj and parent != j
        if parent >= 0:
            assert parent >= nchains, "a chain job is never a parent"
            assert J[parent][0] == inst, "a parent belongs to the same item"
            kids[parent] += 1
    for j in range(nchains, nj):
        assert J[j][2] == kids[j] >= 2, f"node {j}: child count {J[j][2]} vs {kids[j]}"
    assert all(J[j][2] == 0 for j in range(nchains))
    roots = [j for j in range(nj) if J[j][1] < 0]
    assert sorted(J[r][0] for r in roots) == list(range(len(items)))
    for _ in range(5):
        order = list(range(nchains))
        g.shuffle(order)
        ran = [0] * nj
        arrivals = [0] * nj
        finished_items = []
        for c in order:               # each CTA runs a chain, then climbs while it arrives last
            jb = c
            while True:
                assert ran[jb] == 0 and arrivals[jb] == J[jb][2]
                ran[jb] += 1
                parent = J[jb][1]
                if parent < 0:
                    finished_items.append(J[jb][0])
                    break
                arrivals[parent] += 1
                if arrivals[parent] < J[parent][2]:
                    break
                jb = parent
        assert ran == [1] * nj
        assert sorted(finished_items) == list(range(len(items)))

"""Host model of the tile-pair schedule that applies Q^T or Q to one column (paper §2.3: the
implicit Q is applied tile by tile along a flat chain or tree node, each tile's reflectors in
order). The GPU kernel deals a job's tiles alternately to the two half-warps of a warp, half
1 one reflector step behind half 0, and keeps the pivot entries in two buffers (tile q reads
buffer q mod 2 and writes the other). This model runs that schedule step by step in numpy:
in each warp step both halves read the state as it was before the step and write after it.
The checks are that (1) no address one half writes in a step is read or written by the other
half in that step, (2) no pivot entry is read and rewritten in the same step, and (3) the
result equals plain sequential application. Planted schedule errors (no lag, one pivot buffer)
must fail (1)-(3)."""
import numpy as np
import pytest

GEQRT, TSQRT, TTQRT = 0, 1, 2


def refl_rows(kind, j, ht, off):
    """Tail rows [lo, hi) of reflector j in a tile (GEQRT: below the diagonal; TSQRT: every
    row; TTQRT: the rows of the child's triangle at or above row j)."""
    if kind == GEQRT:
        return j + 1, ht
    if kind == TSQRT:
        return 0, ht
    return 0, min(max(j + 1 - off, 0), ht)


def sequential(tiles, n, b, V, tau, scl, trans):
    """Every tile in processing order, every reflector in order; the head entry of reflector
    j is row j of a leaf tile (GEQRT) or entry j of the job's pivot vector."""
    b = b.copy()
    piv = b[:n].copy()
    order = range(len(tiles)) if trans else range(len(tiles) - 1, -1, -1)
    for tt in order:
        row0, nrows, kind, off, refl = tiles[tt]
        x = b[row0:row0 + nrows].copy()
        ge = kind == GEQRT
        if ge:
            x[:n] = piv
        for j in (range(n) if trans else range(n - 1, -1, -1)):
            lo, hi = refl_rows(kind, j, nrows, off)
            v = V[row0 + lo:row0 + hi, j]
            head = x[j] if ge else piv[j]
            w = head + scl[refl + j] * float(v @ x[lo:hi])
            x[lo:hi] -= tau[refl + j] * scl[refl + j] * w * v
            if ge:
                x[j] = head - tau[refl + j] * w
            else:
                piv[j] = head - tau[refl + j] * w
        if ge:
            piv = x[:n].copy()
            b[row0 + n:row0 + nrows] = x[n:]
        else:
            b[row0:row0 + nrows] = x
    b[:n] = piv
    return b


def tile_pairs(tiles, n, b, V, tau, scl, trans, lag=1, two_buffers=True):
    """The kernel's schedule; returns (result, conflicts)."""
    b = b.copy()
    nt = len(tiles)
    mem = {("P", 0, j): b[j] for j in range(n)}
    usteps = [((nt - h + 1) >> 1) * n for h in (0, 1)]
    T = max(((nt + 1) >> 1) * n, (nt >> 1) * n + lag)
    td, pin, pout = [None, None], [0, 0], [1, 1]
    conflicts = 0

    def position(u, h):
        q = 2 * (u // n) + h
        return q, (q if trans else nt - 1 - q)

    def refl_of(u):
        return u % n if trans else n - 1 - u % n

    def commit(R, W):
        nonlocal conflicts
        for h in (0, 1):
            if set(W[h]) & (R[1 - h] | set(W[1 - h])):
                conflicts += 1
            if any(k[0] == "P" and k in R[h] for k in W[h]):
                conflicts += 1
        for h in (0, 1):
            for k, v in W[h].items():
                if k[0] == "B":
                    b[k[1]] = v
                else:
                    mem[k] = v

    for t in range(T + 1):
        # staging: the half's previous tile leaves, its next tile arrives
        R, W = [set(), set()], [{}, {}]
        for h in (0, 1):
            u = t - h * lag
            up = u - 1
            if 0 <= up < usteps[h] and up % n == n - 1:
                row0, nrows, kind, off, refl = td[h]
                for i in range(nrows):
                    if kind == GEQRT and i < n:
                        if not trans:
                            R[h].add(("T", h, i))
                            W[h][("P", pout[h], i)] = mem[("T", h, i)]
                    else:
                        R[h].add(("T", h, i))
                        W[h][("B", row0 + i)] = mem[("T", h, i)]
            if t < T and 0 <= u < usteps[h] and u % n == 0:
                q, tt = position(u, h)
                td[h] = tiles[tt]
                pin[h], pout[h] = (q & 1, (q + 1) & 1) if two_buffers else (0, 0)
                row0, nrows, kind, off, refl = td[h]
                for i in range(nrows):
                    if kind == GEQRT and i < n:
                        if trans:
                            R[h].add(("P", pin[h], i))
                            W[h][("T", h, i)] = mem[("P", pin[h], i)]
                    else:
                        W[h][("T", h, i)] = b[row0 + i]
        commit(R, W)
        if t == T:
            break
        # one reflector per active half
        R, W = [set(), set()], [{}, {}]
        for h in (0, 1):
            u = t - h * lag
            if not 0 <= u < usteps[h]:
                continue
            row0, nrows, kind, off, refl = td[h]
            j, ge = refl_of(u), kind == GEQRT
            lo, hi = refl_rows(kind, j, nrows, off)
            dot = 0.0
            for i in range(lo, hi):
                R[h].add(("T", h, i))
                dot += V[row0 + i, j] * mem[("T", h, i)]
            hk = ("T", h, j) if (ge and trans) else ("P", pin[h], j)
            R[h].add(hk)
            w = mem[hk] + scl[refl + j] * dot
            for i in range(lo, hi):
                W[h][("T", h, i)] = mem[("T", h, i)] - tau[refl + j] * scl[refl + j] * w * V[row0 + i, j]
            new_head = mem[hk] - tau[refl + j] * w
            W[h][("T", h, j) if (ge and not trans) else ("P", pout[h], j)] = new_head
        commit(R, W)
    final = (nt & 1) if two_buffers else 0
    for j in range(n):
        b[j] = mem[("P", final, j)]
    return b, conflicts


def chain(n, nt, h, ragged):
    """A flat chain: a leaf tile (its first n rows are the pivot rows) then nt - 1 tiles."""
    tiles, row = [], 0
    for q in range(nt):
        nr = max(1, h // 3) if (ragged and q == nt - 1 and q > 0) else h
        tiles.append((row, nr, GEQRT if q == 0 else TSQRT, 0, q * n))
        row += nr
    return tiles, row


def tree_node(n, nt, piece):
    """A tree node: pivot triangle at rows 0..n-1, then the children's triangles in pieces."""
    tiles, row, k = [], n, 0
    while len(tiles) < nt:
        for o in range(0, n, piece):
            tiles.append((row + o, min(piece, n - o), TTQRT, o, k * n))
            k += 1
        row += n
    return tiles[:nt], row


def cases():
    rng = np.random.default_rng(11)
    for n in (2, 3, 5, 8):
        for nt in (1, 2, 3, 4, 7):
            for form in ("chain", "ragged", "node", "pieces"):
                if form in ("chain", "ragged"):
                    tiles, m = chain(n, nt, n + int(rng.integers(0, 9)), form == "ragged")
                else:
                    tiles, m = tree_node(n, nt, n if form == "node" else max(1, n // 2))
                V = rng.standard_normal((m, n))
                nref = (len(tiles) + 8) * n
                tau, scl = rng.uniform(0.5, 1.5, nref), rng.uniform(-1, 1, nref)
                yield tiles, n, rng.standard_normal(m), V, tau, scl


@pytest.mark.parametrize("trans", [1, 0])
def test_tile_pair_schedule_matches_sequential(trans):
    worst, count = 0.0, 0
    for tiles, n, b, V, tau, scl in cases():
        ref = sequential(tiles, n, b, V, tau, scl, trans)
        got, conflicts = tile_pairs(tiles, n, b, V, tau, scl, trans)
        assert conflicts == 0
        worst = max(worst, np.max(np.abs(got - ref)) / max(1.0, np.max(np.abs(ref))))
        count += 1
    assert count == 80
    assert worst <= 1e-13


@pytest.mark.parametrize("mutant", ["no_lag", "one_buffer"])
def test_tile_pair_schedule_mutants_fail(mutant):
    bad = 0
    for tiles, n, b, V, tau, scl in cases():
        for trans in (1, 0):
            ref = sequential(tiles, n, b, V, tau, scl, trans)
            try:
                got, conflicts = tile_pairs(tiles, n, b, V, tau, scl, trans, lag=0 if mutant == "no_lag" else 1,
                                            two_buffers=mutant != "one_buffer")
            except KeyError:  # read of a pivot entry nobody wrote
                bad += 1
                continue
            if conflicts or np.max(np.abs(got - ref)) > 1e-13 * max(1.0, np.max(np.abs(ref))):
                bad += 1
    assert bad > 0

"""Host model of the resident server's work protocol (the kernel k_resident and the worker
that feeds it). The worker writes an admitted request's chain entries into one of two host
rings (short requests, of few chain jobs, into ring 0) and only then advances that ring's
`tail`; a CTA claims an entry by compare-and-swap on `head` (device ring first, by
compare-and-swap on `dhead`, then ring 0, then ring 1) after reading `tail`, and runs the job while
counted `busy`. The job that ends a request's factorization, or the last task of a
refinement step, reserves the next step's tasks on the device ring (`dtail`) and releases
each entry afterwards; a claimer waits for the release. A CTA that finds nothing to claim
for long enough ends the launch (`quit`) if no CTA is busy and both rings are empty;
entries not yet claimed stay in the rings, and the worker launches the kernel again
whenever requests are in flight and no launch is running.

The model runs CTAs and the worker as generators under random schedules, with a short idle
limit so that launches end and restart between admissions, and checks that every request
completes, that every chain job and refinement task runs exactly once with the data that
was published for it, and that a request's refinement steps run after its factorization
and in order. Planted mistakes must fail: a claim past `tail`, a claimer that does not wait
for the release of a device-ring entry, a claim that is not one atomic step, and a worker
that does not launch again after a launch has ended."""
import random

import pytest


SMALL = 3  # requests of at most this many chain jobs go to ring 0


class State:
    def __init__(self, reqs):
        self.ring = [[], []]    # host rings: entries (req, chain); None until written
        self.tail = [0, 0]
        self.head = [0, 0]
        self.dring = []         # device ring: (req, step, task) once released, None while reserved
        self.dhead = 0
        self.busy = 0
        self.quit = False
        self.reqs = reqs        # req -> dict(chains, steps, tasks)
        self.ran_chain = {}
        self.ran_task = {}
        self.chains_left = {r: c["chains"] for r, c in reqs.items()}
        self.tasks_left = {}
        self.step = {r: -1 for r in reqs}
        self.done = set()
        self.errors = []


def cta(st, idle_limit, mistakes):
    empty = 0
    while True:
        if st.quit:
            return
        if st.dhead < len(st.dring):  # refinement tasks first
            idx = st.dhead
            if "nonatomic_claim" in mistakes:
                yield
            st.dhead = idx + 1
            st.busy += 1
            if "no_release_wait" not in mistakes:
                while st.dring[idx] is None:
                    yield
            entry = st.dring[idx]
            if entry is None:
                st.errors.append("device-ring entry read before its release")
                st.busy -= 1
                continue
            yield from run_task(st, *entry)
            empty = 0
            continue
        claimed = False
        for c in (0, 1):
            limit = len(st.ring[c]) if "read_before_tail" in mistakes else st.tail[c]
            if st.head[c] >= limit:
                continue
            idx = st.head[c]
            if "nonatomic_claim" in mistakes:
                yield
            st.head[c] = idx + 1
            st.busy += 1
            entry = st.ring[c][idx]
            claimed = True
            if entry is None:
                st.errors.append("host-ring entry read before it was written")
                st.busy -= 1
                break
            yield from run_chain(st, *entry)
            empty = 0
            break
        if claimed:
            continue
        empty += 1
        if (empty >= idle_limit and st.busy == 0 and st.dhead == len(st.dring) and st.head[0] == st.tail[0]
                and st.head[1] == st.tail[1]):
            st.quit = True
            return
        yield


def reserve(st, req, step):
    n = st.reqs[req]["tasks"]
    base = len(st.dring)
    st.dring.extend([None] * n)  # dtail advanced; entries not yet written
    st.tasks_left[(req, step)] = n
    for t in range(n):
        yield
        st.dring[base + t] = (req, step, t)  # released


def run_chain(st, req, chain):
    key = (req, chain)
    st.ran_chain[key] = st.ran_chain.get(key, 0) + 1
    yield
    st.chains_left[req] -= 1
    if st.chains_left[req] == 0:  # the root of the request's tree
        if st.reqs[req]["steps"] == 0:
            st.done.add(req)
        else:
            st.step[req] = 0
            yield from reserve(st, req, 0)
    st.busy -= 1  # after the reservation and the releases


def run_task(st, req, step, task):
    key = (req, step, task)
    st.ran_task[key] = st.ran_task.get(key, 0) + 1
    if st.chains_left[req] != 0 or st.step[req] != step:
        st.errors.append(f"task {key} out of order")
    yield
    st.tasks_left[(req, step)] -= 1
    if st.tasks_left[(req, step)] == 0:  # the last task of the step decides
        if step + 1 < st.reqs[req]["steps"]:
            st.step[req] = step + 1
            yield from reserve(st, req, step + 1)
        else:
            st.done.add(req)
    st.busy -= 1


def run(nreq=12, ctas=6, idle_limit=3, mistakes=(), seed=0, max_ticks=200_000):
    rng = random.Random(seed)
    reqs = {r: {"chains": rng.randint(1, 6), "steps": rng.choice([0, 1, 2, 3]), "tasks": rng.randint(1, 4)}
            for r in range(nreq)}
    st = State(reqs)
    pending = list(range(nreq))
    writing = []  # ring slots the worker is still writing
    admitted = 0
    launches = 0
    progs = []
    for _ in range(max_ticks):
        # the worker: write a request's entries one per tick, then advance its ring's tail
        if writing:
            c, i, entry = writing.pop(0)
            st.ring[c][i] = entry
            if not writing:
                st.tail[c] = len(st.ring[c])
        elif pending and rng.random() < 0.05:
            r = pending.pop(0)
            admitted += 1
            c = 0 if reqs[r]["chains"] <= SMALL else 1
            for j in range(reqs[r]["chains"]):
                st.ring[c].append(None)
                writing.append((c, len(st.ring[c]) - 1, (r, j)))
        # a launch whenever requests are in flight and none runs
        if not progs and len(st.done) < admitted and ("no_relaunch" not in mistakes or launches == 0):
            st.quit = False
            progs = [cta(st, idle_limit, set(mistakes)) for _ in range(ctas)]
            launches += 1
        if not pending and not writing and len(st.done) == len(reqs) and not progs:
            break
        if progs:
            p = rng.choice(progs)
            try:
                next(p)
            except StopIteration:
                progs.remove(p)
    return st, launches


def ok(st):
    return (not st.errors and st.done == set(st.reqs)
            and all(v == 1 for v in st.ran_chain.values())
            and len(st.ran_chain) == sum(r["chains"] for r in st.reqs.values())
            and all(v == 1 for v in st.ran_task.values())
            and len(st.ran_task) == sum(r["steps"] * r["tasks"] for r in st.reqs.values()))


@pytest.mark.parametrize("seed", range(10))
def test_every_job_runs_once_and_every_request_completes(seed):
    st, launches = run(seed=seed)
    assert not st.errors, st.errors[:3]
    assert ok(st), f"incomplete: {sorted(set(st.reqs) - st.done)}"


def test_launches_end_and_restart():
    # the short idle limit ends launches between admissions; the work still completes
    runs = [run(seed=seed, idle_limit=2) for seed in range(10)]
    assert all(ok(st) for st, _ in runs)
    assert max(launches for _, launches in runs) >= 3


@pytest.mark.parametrize("mistake", ["read_before_tail", "no_release_wait", "nonatomic_claim", "no_relaunch"])
def test_planted_mistakes_are_caught(mistake):
    caught = sum(not ok(run(seed=seed, mistakes=(mistake,))[0]) for seed in range(20))
    assert caught > 0

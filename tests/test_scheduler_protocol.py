"""Host-side model of the persistent step kernel's scheduler protocol
(CPU only).

The kernel's protocol (csrc/wavefront.cuh, csrc/gol_api.cu) is restated here
step by step and run under random interleavings of many simulated warps,
with sequentially consistent memory: units on a wrapping grid of row blocks
and tiles (at most 8 neighbours each), countdown join counters per pass
parity that a unit restores when it starts its next pass, two queue rings
(critical passes, whose unit still has at least a given share of the longest
chain ahead, and the others) whose slots are handed out only by atomic
tickets, a warp holding at most one ticket of each ring until its slot
fills, a warp whose critical ticket is still unfilled waiting for it alone
for a bounded time (counted here in the warp's own steps) before it takes or
serves other-ring work, and the first critical passes dealt to warps by
index.  Every run must execute every pass exactly once, never start a pass
before its neighbours finished the previous one, never overflow a ring, and
end.
"""
import random

import pytest

INF = 1 << 62


def make_units(boards, K=3):
    """boards: (row blocks, tiles, segment height).  Units of a board are
    consecutive; neighbours: the 8 around on the wrapping grid, minus self."""
    units = []
    for b, (nb, nt, H) in enumerate(boards):
        first = len(units)
        for i in range(nb):
            for t in range(nt):
                me = first + i * nt + t
                nbs = []
                for a in (-1, 0, 1):
                    for d in (-1, 0, 1):
                        v = first + ((i + a) % nb) * nt + (t + d) % nt
                        if v != me and v not in nbs:
                            nbs.append(v)
                units.append({"board": b, "cost": H + 2 * K, "nb": nbs})
    return units


def plan_rings(units, npass, permille):
    """Critical threshold, critical ring size, critical first passes and the
    launch order (critical first passes, then the others)."""
    maxchain = max([1] + [npass[u["board"]] * u["cost"] for u in units])
    thr = max(1, (maxchain * permille + 999) // 1000) if permille > 0 else INF
    hi_cap = hi_init = 0
    for u in units:
        np_, cost = npass[u["board"]], u["cost"]
        need = np_ + 1 if thr == INF else (thr + cost - 1) // cost
        hi_cap += max(0, min(np_, np_ + 1 - need))
        hi_init += np_ * cost >= thr
    crit = [npass[u["board"]] * u["cost"] >= thr for u in units]
    order = [i for i in range(len(units)) if crit[i]] + [i for i in range(len(units)) if not crit[i]]
    return thr, hi_cap, hi_init, order


def run(units, npass, nwarps, permille, seed, crit_wait=0):
    """crit_wait: how many of its own steps a warp holding an unfilled
    critical ticket waits for it alone (INF: without limit)."""
    rng = random.Random(seed)
    n = len(units)
    thr, hi_cap, hi_init, order = plan_rings(units, npass, permille)
    total = sum(npass[u["board"]] for u in units)
    lo_cap = total - hi_cap
    ring = [-1] * total
    for i in range(total):
        if i < hi_cap:
            if i < hi_init:
                ring[i] = order[i]
        elif i - hi_cap < n - hi_init:
            ring[i] = order[hi_init + (i - hi_cap)]
    q = [min(hi_init, nwarps), hi_init, 0, n - hi_init]   # critical head/tail, other tickets/tail
    join = [[len(u["nb"]) + 1] * 2 for u in units]
    next_pass = [1] * n
    state = {"done": 0}
    ran = set()
    finished = {}

    def enqueue(v, rem):
        hi = rem >= thr
        k = 1 if hi else 3
        slot = q[k]
        q[k] += 1
        yield
        base, cap = (0, hi_cap) if hi else (hi_cap, lo_cap)
        assert slot < cap, "ring overflow"
        ring[base + slot] = v
        yield

    def ticket_unit(tk):
        if 0 <= tk[0] < hi_cap and ring[tk[0]] >= 0:
            v, tk[0] = ring[tk[0]], -1
            return v
        if 0 <= tk[1] < lo_cap and ring[hi_cap + tk[1]] >= 0:
            v, tk[1] = ring[hi_cap + tk[1]], -1
            return v
        return -1

    def warp(w):
        u = ring[w] if w < min(hi_init, nwarps) else -1
        p, tk = 1, [-1, -1]
        clock = {"now": 0, "tk0": 0}          # the warp's own steps; when it took tk[0]
        while True:
            if u < 0:
                spin = 0
                while True:
                    clock["now"] += 1
                    waiting = 0 <= tk[0] < hi_cap and clock["now"] - clock["tk0"] < crit_wait
                    if waiting:
                        v = ring[tk[0]]
                        if v >= 0:
                            tk[0] = -1
                    else:
                        v = ticket_unit(tk)
                    if v >= 0:
                        break
                    if tk[0] < 0 and hi_cap > 0 and spin % 8 == 0:
                        head, tail = q[0], q[1]
                        yield
                        if head < tail:
                            tk[0] = q[0]
                            q[0] += 1
                            clock["tk0"] = clock["now"]
                            yield
                            spin += 1
                            continue
                    if tk[1] < 0 and not waiting:
                        tk[1] = q[2]
                        q[2] += 1
                        yield
                        spin += 1
                        continue
                    if state["done"] >= total:
                        return
                    spin += 1
                    yield
                u, p = v, next_pass[v]
                yield
            # run pass p of u
            clock["now"] += 1
            assert (u, p) not in ran, "a pass ran twice"
            for x in units[u]["nb"]:
                assert finished.get(x, 0) >= p - 1, "a pass started before a neighbour's previous pass"
                assert finished.get(x, 0) <= p, "a neighbour ran more than one pass ahead"
            ran.add((u, p))
            if p > 1:
                join[u][(p - 1) & 1] = len(units[u]["nb"]) + 1
            yield
            finished[u] = p
            state["done"] += 1
            np_, cost = npass[units[u]["board"]], units[u]["cost"]
            nxt = -1
            if p < np_:
                if not units[u]["nb"]:
                    nxt = u
                else:
                    ready = []
                    for x in [u] + units[u]["nb"]:
                        join[x][p & 1] -= 1
                        if join[x][p & 1] == 0:
                            ready.append(x)
                        yield
                    if ready:
                        nxt = ready[0]
                        for x in ready[1:]:
                            next_pass[x] = p + 1
                            yield from enqueue(x, (np_ - p) * cost)
            take = -1
            if nxt >= 0 and (tk[0] >= 0 or tk[1] >= 0):
                take = ticket_unit(tk)
                if take >= 0:
                    next_pass[nxt] = p + 1
                    yield from enqueue(nxt, (np_ - p) * cost)
            if take >= 0:
                u, p = take, next_pass[take]
            elif nxt >= 0:
                u, p = nxt, p + 1
            else:
                u = -1

    gens = [warp(w) for w in range(nwarps)]
    live = list(range(nwarps))
    steps = 0
    while live:
        steps += 1
        if steps >= 3_000_000:
            raise RuntimeError("no progress (deadlock or livelock)")
        i = rng.randrange(len(live))
        try:
            next(gens[live[i]])
        except StopIteration:
            live.pop(i)
    assert len(ran) == total, "some passes never ran"


@pytest.mark.parametrize("permille", [0, 1, 250, 750, 1000])
def test_two_ring_ticket_protocol(permille):
    for seed in range(150):
        r = random.Random(1000 * permille + seed)
        nboards = r.randint(1, 6)
        boards = [(r.randint(1, 4), r.randint(1, 3), r.randint(1, 20)) for _ in range(nboards)]
        npass = [r.randint(1, 9) for _ in range(nboards)]
        run(make_units(boards), npass, r.randint(2, 10), permille, seed)


@pytest.mark.parametrize("crit_wait", [1, 6, 40])
def test_bounded_wait_for_a_critical_ticket(crit_wait):
    for seed in range(120):
        r = random.Random(7000 + 100 * crit_wait + seed)
        nboards = r.randint(1, 6)
        boards = [(r.randint(1, 4), r.randint(1, 3), r.randint(1, 20)) for _ in range(nboards)]
        npass = [r.randint(1, 9) for _ in range(nboards)]
        run(make_units(boards), npass, r.randint(2, 10), r.choice([250, 500, 750]), seed, crit_wait)


def test_unbounded_wait_for_a_critical_ticket_can_stall():
    # why the kernel's wait has a time limit: warps holding critical tickets
    # that no queued pass will fill, waiting without limit, leave the queued
    # other-ring passes to nobody
    stalled = 0
    for seed in range(60):
        r = random.Random(9000 + seed)
        boards = [(r.randint(2, 4), r.randint(1, 3), r.randint(1, 20)) for _ in range(r.randint(2, 6))]
        npass = [r.randint(2, 9) for _ in range(len(boards))]
        try:
            run(make_units(boards), npass, r.randint(2, 6), 500, seed, INF)
        except RuntimeError:
            stalled += 1
    assert stalled > 0


def test_join_counters_two_parities_suffice():
    # a unit may never be more than one pass ahead of a neighbour, so the
    # counter of pass q and of pass q + 2 share a slot safely
    for seed in range(100):
        r = random.Random(seed)
        boards = [(r.randint(2, 5), r.randint(1, 4), 8)]
        run(make_units(boards), [12], r.randint(2, 12), 0, seed)

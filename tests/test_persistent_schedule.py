"""Host checks of the persistent step kernel's work lists, as the library itself builds them
(lbm_debug_persist_plan: host code, no device).  For each list the tests check, without
reusing the planner's row-to-chunk rule:
- the odd steps' list is the even steps' list in another order, starting (for a single
  instance) from its middle chunk row;
- every pair of items of consecutive steps of one instance where the later one reads rows
  the earlier one writes, or writes rows the earlier one reads, is covered: the later
  item's dependencies hold the earlier item's chunk, and a chunk's `strips` is the number
  of its items;
- the queue protocol of sweep2_persist_kernel ends for any number of CTAs: items taken in
  order, each CTA holding its current item and the next, waiting (after releasing its
  finished item) until its dependency chunks have completed all strips of the previous
  steps, with random item durations."""
import ctypes
import heapq
import random

import numpy as np
import pytest

from paper_1211_6932_gb300 import _lib


def plan(shapes, threads, rows):
    L = _lib.lib()
    n = len(shapes)
    arr = lambda k: (ctypes.c_int * n)(*[s[k] for s in shapes])  # noqa: E731
    nx, ny, walls = arr(0), arr(1), arr(2)
    ni = ctypes.c_int()
    rc = L.lbm_debug_persist_plan(n, nx, ny, walls, threads, rows, ctypes.byref(ni), None, None)
    if rc == 1:
        return None
    assert rc == 0
    m = ni.value
    items = (ctypes.c_int * (10 * m))()
    links = (ctypes.c_int * (12 * m))()
    assert L.lbm_debug_persist_plan(n, nx, ny, walls, threads, rows, ctypes.byref(ni), items,
                                    links) == 0
    return (np.frombuffer(items, dtype=np.int32).reshape(2, m, 5),
            np.frombuffer(links, dtype=np.int32).reshape(2, m, 6))


def rows_read(shape, y0, y1):
    nx, ny, walls = shape
    return {min(max(r, 0), ny - 1) if walls else r % ny for r in range(y0 - 2, y1 + 2)}


CASES = [
    ([(600, 250, 0)], 128, 16),           # strips, periodic
    ([(300, 97, 1)], 96, 12),             # walls, a one-row last chunk
    ([(257, 37, 0)], 128, 12),            # odd width, a one-row last chunk
    ([(200, 64, 0)], 128, 2),             # full width, two-row chunks
    ([(40, 3, 0)], 128, 8),               # one chunk
    ([(200, 64, 0), (400, 40, 0), (130, 67, 1)], 128, 8),  # several instances
    # strip instances, then full-width ones: one list, as a batch's persistent launch
    ([(400, 40, 0), (300, 97, 1), (200, 64, 0), (64, 200, 0), (5, 3, 0)], 128, 12),
]


@pytest.mark.parametrize("shapes,threads,rows", CASES)
def test_lists_cover_every_cross_step_hazard(shapes, threads, rows):
    items, links = plan(shapes, threads, rows)
    key = lambda a: sorted(map(tuple, a.tolist()))  # noqa: E731
    assert key(items[0]) == key(items[1])
    if len(shapes) == 1:
        nch = -(-shapes[0][1] // rows)
        assert items[1][0][2] == (nch // 2) * rows  # the odd list starts mid-instance
    for par in (0, 1):
        strips = {}
        for (inst, x0, y0, y1, d), ln in zip(items[par], links[par]):
            strips.setdefault(ln[0], set()).add(x0)
        for ln in links[par]:
            assert ln[1] == len(strips[ln[0]])
        prev_items, prev_links = items[1 - par], links[1 - par]
        for (inst, x0, y0, y1, d), ln in zip(items[par], links[par]):
            sh = shapes[inst]
            rd, wr = rows_read(sh, y0, y1), set(range(y0, y1))
            deps = set(ln[2:6].tolist())
            for (i2, _, a0, a1, _), l2 in zip(prev_items, prev_links):
                if i2 != inst:
                    continue
                if rd & set(range(a0, a1)) or wr & rows_read(sh, a0, a1):
                    assert l2[0] in deps, (inst, y0, y1, a0, a1, deps)


def run_queue(items, links, G, steps, seed):
    """Event simulation of the kernel's queue protocol; True if every item finishes."""
    m = items.shape[1]
    total = steps * m
    n_chunks = int(links[:, :, 0].max()) + 1
    done = [0] * n_chunks
    rnd = random.Random(seed)

    def link(q):
        t, k = divmod(q, m)
        return t, links[t & 1][k]

    def met(q):
        t, ln = link(q)
        return t == 0 or all(done[d] >= ln[1] * t for d in ln[2:6])

    nxt = 0
    ctas = []
    events = []
    seq = 0
    for c in range(G):
        ctas.append({"next": nxt, "cur": None, "release": None, "dep_ok": False})
        nxt += 1
        heapq.heappush(events, (0.0, seq, c, "boundary"))
        seq += 1
    waiting, finished = set(), 0
    while events:
        now, _, c, kind = heapq.heappop(events)
        S = cta = ctas[c]
        if kind == "boundary":
            q = S["next"]
            if q >= total or not (S["dep_ok"] or met(q)):
                if S["release"] is not None:  # release before any wait or exit
                    done[S["release"]] += 1
                    S["release"] = None
                if q < total:
                    waiting.add(c)
            else:
                S["cur"] = q
                dur = rnd.uniform(0.5, 1.5)
                for dt, k in ((0.01, "start"), (0.3 * dur, "row4"), (dur, "finish")):
                    heapq.heappush(events, (now + dt, seq, c, k))
                    seq += 1
        elif kind == "start":  # first rows issued: release the previous item, take the next
            if S["release"] is not None:
                done[S["release"]] += 1
                S["release"] = None
            S["next"], S["dep_ok"] = nxt, False
            nxt += 1
        elif kind == "row4":
            S["dep_ok"] = S["next"] < total and met(S["next"])
        else:  # finish
            S["release"] = int(link(S["cur"])[1][0])
            finished += 1
            heapq.heappush(events, (now, seq, c, "boundary"))
            seq += 1
        for w in list(waiting):
            if met(ctas[w]["next"]):
                waiting.discard(w)
                ctas[w]["dep_ok"] = True
                heapq.heappush(events, (now, seq, w, "boundary"))
                seq += 1
        del cta
    return finished == total and not waiting


@pytest.mark.parametrize("shapes,threads,rows", CASES)
def test_queue_protocol_always_ends(shapes, threads, rows):
    items, links = plan(shapes, threads, rows)
    m = items.shape[1]
    for G in sorted({1, 2, 7, max(1, m // 2), m + 3}):
        for seed in range(3):
            assert run_queue(items, links, G, steps=6, seed=seed), (G, seed)


def test_one_row_chunks_are_refused():
    assert plan([(100, 33, 0)], 128, 1) is None
    assert plan([(100, 33, 0)], 128, 2) is not None

"""A lockstep CPU model of the 32-walker protocol with parked paths (test
infrastructure): a design considered for the walker kernel, not built.

The protocol of tests/walker_protocol_model.py binds one walk to each lane for
its whole life, so a lane whose walk waits on another walker's path idles.
Here a tree has P path slots served by L lanes (P >= L).  A lane whose slot has
confirmed a wait (two iterations on the same foreign path) parks the slot and
binds another: first a slot whose wait cycle was found (it must pop), then a
parked slot whose target changed (it must re-read), then a fresh start.
Parked slots learn of a change of their target at the end of the iteration in
which it happens (an idealised notification: the count is a bound on what a
kernel could get).  Claims, loops, cycle pops (over all slots, every 4th
iteration) and commits are those of the 32-walker protocol with slots in place
of lanes, so by cycle popping the model must give sequential Wilson's tree and
step count for every P and L.

    python tests/walker_park_model.py 60 32:32 32:64 32:256   # grid side, L:P ...
"""
from __future__ import annotations

import sys

import numpy as np

IDLE, WALK, WAIT, POPSET, POP, COUNT, COMMIT = range(7)


def walk_tree_parked(g, r, seed, sample, sorder, lanes=32, slots=64, max_iter=10 ** 8):
    import oracle as O

    n = g.n
    L, P = lanes, slots
    nxt = np.zeros(n, dtype=np.int64)
    cnt = np.zeros(n, dtype=np.int64)
    owned = np.zeros(n, dtype=bool)
    owner = np.full(n, -1, dtype=np.int64)     # owning slot
    intree = np.zeros(n, dtype=bool)
    depth = np.zeros(n, dtype=np.int64)
    intree[r] = True
    nxt[r] = -1
    ph = [IDLE] * P
    busy = [False] * P        # the slot holds a start (with or without a path)
    has_path = [False] * P
    s = [-1] * P
    c = [-1] * P
    x = [-1] * P
    u = [-1] * P
    pcur = [-1] * P
    pend = [-1] * P
    prew = [-1] * P
    cc = [0] * P
    ln = [0] * P
    ii = [0] * P
    dh = [0] * P
    mypos = [0] * P
    confirmed = [False] * P   # WAIT seen on two consecutive reads
    parked = [False] * P
    recheck = [False] * P
    bound = [-1] * L          # lane -> slot
    lane_of = [-1] * P
    steps = 0
    next_start = 0
    pos = 1
    order = np.full(n, -1)
    order[0] = r
    for it in range(max_iter):
        # ---- park confirmed waits, then bind free lanes
        for lane in range(L):
            k = bound[lane]
            if k >= 0 and P > L and ph[k] == WAIT and confirmed[k]:
                parked[k] = True
                bound[lane] = -1
                lane_of[k] = -1
        for lane in range(L):
            if bound[lane] >= 0:
                continue
            pick = -1
            for k in range(P):
                if lane_of[k] < 0 and busy[k] and ph[k] == POPSET:
                    pick = k
                    break
            if pick < 0:
                for k in range(P):
                    if lane_of[k] < 0 and busy[k] and parked[k] and recheck[k]:
                        pick = k
                        break
            if pick < 0 and next_start < n:
                for k in range(P):
                    if not busy[k]:
                        pick = k
                        busy[k] = True
                        has_path[k] = False
                        s[k] = int(sorder[next_start])
                        next_start += 1
                        ph[k] = IDLE
                        break
            if pick >= 0:
                bound[lane] = pick
                lane_of[pick] = lane
                parked[pick] = False
                recheck[pick] = False
                confirmed[pick] = False
        if next_start >= n and not any(busy):
            break
        # ---- act: departures and the vertex each bound lane reads
        ld = [-1] * L
        for lane in range(L):
            k = bound[lane]
            if k < 0:
                continue
            p = ph[k]
            if p == WALK:
                kk = O.bounded(seed, c[k], cc[k], sample, 0, int(g.deg[c[k]]))
                v = int(g.col[g.row_off[c[k]] + kk])
                nxt[c[k]] = v
                cnt[c[k]] = cc[k] + 1
                cc[k] += 1
                steps += 1
                x[k] = v
                ld[lane] = v
            elif p == IDLE:
                ld[lane] = s[k]
            elif p == WAIT:
                ld[lane] = x[k]
            elif p == POPSET:
                ld[lane] = prew[k]
            elif p == POP:
                ld[lane] = pcur[k]
            elif p in (COUNT, COMMIT):
                ld[lane] = u[k]
        snap = {}
        for lane in range(L):
            v = ld[lane]
            if v >= 0:
                snap[lane] = (bool(intree[v]), bool(owned[v]) and not intree[v],
                              int(owner[v]), int(nxt[v]), int(cnt[v]), int(depth[v]))
        was_wait = {lane: bound[lane] >= 0 and ph[bound[lane]] == WAIT for lane in range(L)}
        may = {lane: bound[lane] >= 0 and ph[bound[lane]] in (IDLE, WALK, WAIT)
               for lane in range(L)}
        want = {lane: may[lane] and ld[lane] >= 0 and not snap[lane][0] and not snap[lane][1]
                for lane in range(L)}
        winner = {}
        for lane in range(L):
            if want[lane] and ld[lane] not in winner:
                winner[ld[lane]] = lane
        fin = [False] * P
        for lane in range(L):
            v = ld[lane]
            if v < 0:
                continue
            k = bound[lane]
            in_tree, own, own_slot, wn, wc, wd = snap[lane]
            p = ph[k]
            if want[lane]:
                if winner[v] == lane:  # claim a free vertex
                    owned[v] = True
                    owner[v] = k
                    if not has_path[k]:
                        s[k] = v
                    has_path[k] = True
                    c[k] = v
                    cc[k] = wc
                    ph[k] = WALK
                else:
                    if p == IDLE:
                        has_path[k] = False
                    x[k] = v
                    ph[k] = WAIT
                    confirmed[k] = False
            elif may[lane]:
                if in_tree:
                    if not has_path[k]:
                        busy[k] = False
                        ph[k] = IDLE
                        bound[lane] = -1
                        lane_of[k] = -1
                    else:
                        ph[k] = COUNT
                        u[k] = s[k]
                        ln[k] = 0
                elif own_slot == k:  # loop on the own path
                    prew[k] = v
                    cc[k] = wc
                    pcur[k] = wn
                    pend[k] = c[k]
                    ph[k] = POP
                else:
                    if p == IDLE:
                        has_path[k] = False
                    confirmed[k] = was_wait[lane] and x[k] == v
                    x[k] = v
                    ph[k] = WAIT
            elif p == POPSET:
                cc[k] = wc
                if prew[k] == c[k]:
                    ph[k] = WALK
                else:
                    pcur[k] = wn
                    pend[k] = c[k]
                    ph[k] = POP
            elif p == POP:
                owned[v] = False
                owner[v] = -1
                if v == pend[k]:
                    c[k] = prew[k]
                    ph[k] = WALK
                else:
                    pcur[k] = wn
            elif p == COUNT:
                if in_tree:
                    dh[k] = wd
                    fin[k] = True
                else:
                    ln[k] += 1
                    u[k] = wn
                    assert ln[k] <= n
            elif p == COMMIT:
                d = dh[k] + ln[k] - ii[k]
                intree[v] = True
                depth[v] = d
                owned[v] = False
                owner[v] = -1
                order[mypos[k] + ln[k] - 1 - ii[k]] = v
                ii[k] += 1
                u[k] = wn
                if ii[k] == ln[k]:
                    busy[k] = False
                    has_path[k] = False
                    ph[k] = IDLE
                    bound[lane] = -1
                    lane_of[k] = -1
        # order positions of finished paths: exclusive scan in slot order
        acc = 0
        for k in range(P):
            if fin[k]:
                mypos[k] = pos + acc
                acc += ln[k]
                ph[k] = COMMIT
                u[k] = s[k]
                ii[k] = 0
        pos += acc
        # parked slots whose target changed re-read it (idealised notification)
        for k in range(P):
            if parked[k] and ph[k] == WAIT and not recheck[k]:
                v = x[k]
                if intree[v] or not owned[v]:
                    recheck[k] = True
        # cycles of confirmed waits over all slots, every 4th iteration
        if it % 4 != 0:
            continue
        succ = [-1] * P
        for k in range(P):
            if busy[k] and ph[k] == WAIT and confirmed[k] and has_path[k]:
                v = x[k]
                if owned[v] and not intree[v] and owner[v] != k:
                    succ[k] = int(owner[v])
        if sum(1 for q in succ if q >= 0) < 2:
            continue
        on = [False] * P
        for k in range(P):
            y = k
            for _ in range(P):
                y = succ[y] if y >= 0 else -1
                if y == k:
                    on[k] = True
                    break
        entry = {}
        for k in range(P):
            if on[k]:
                pred = [j for j in range(P) if on[j] and succ[j] == k]
                assert len(pred) == 1
                entry[k] = x[pred[0]]
        for k, v in entry.items():
            prew[k] = v
            ph[k] = POPSET
            confirmed[k] = False
            recheck[k] = False
    else:
        raise RuntimeError("iteration cap")
    assert intree.all() and pos == n
    parent = nxt.copy()
    parent[r] = -1
    return parent.astype(np.int32), steps, depth, order, it


def main(side: int, specs):
    import oracle as O
    from paper_2511_16356_gb300 import synth as S

    g = S.grid_perturbed(side, side, 0.25, 1)
    t0 = O.tau0(g)
    sorder = np.random.default_rng(0).permutation(g.n)
    ref = O.tree(g, t0, 5, 0)
    for spec in specs:
        lanes, slots = (int(a) for a in spec.split(":"))
        parent, steps, _, _, it = walk_tree_parked(g, t0.r, 5, 0, sorder, lanes, slots)
        assert np.array_equal(parent, ref.parent) and steps == ref.steps
        print(f"{side}x{side} grid: {lanes} lanes, {slots} slots: {it} iterations, "
              f"{steps / it:.2f} departures per iteration", flush=True)


if __name__ == "__main__":
    import os

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    main(int(sys.argv[1]), sys.argv[2:] or ["32:32", "32:64"])

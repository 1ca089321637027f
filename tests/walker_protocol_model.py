"""A lockstep CPU model of the 32-walker Wilson protocol of the device kernel
(test infrastructure): L walkers of one tree advance one action per iteration;
claims of the same free vertex go to the lowest lane; closing a loop on the
own path frees the loop and re-departs from its entry (whose departure count
is kept); a walker whose arrow points into another walker's live path waits;
confirmed waits that close a cycle among walkers are popped (searched every
4th iteration, as the kernel does); a path that reaches the tree is counted,
given order positions by an exclusive scan over the finishing lanes, and
committed parent first.

The departure of u on its k-th visit uses the oracle's bounded Philox draw, so
by cycle popping the model must reproduce the oracle's sequential tree, step
count and depths for every start order and walker count.  It documents and
checks the protocol's design on the CPU; it is not the device code.
"""
import numpy as np

IDLE, WALK, WAIT, POPSET, POP, COUNT, COMMIT, DONE = range(8)


def walk_tree(g, r, seed, sample, sorder, lanes=32, max_iter=10 ** 7, phases=None):
    """phases: optional list of 8 counters, incremented per lane-iteration
    spent in each phase (IDLE .. DONE)."""
    import oracle as O

    n = g.n
    nxt = np.zeros(n, dtype=np.int64)
    cnt = np.zeros(n, dtype=np.int64)
    owned = np.zeros(n, dtype=bool)
    owner = np.full(n, -1, dtype=np.int64)
    intree = np.zeros(n, dtype=bool)
    depth = np.zeros(n, dtype=np.int64)
    intree[r] = True
    nxt[r] = -1
    L = lanes
    ph = [IDLE] * L
    has_path = [False] * L
    s = [-1] * L
    c = [-1] * L
    x = [-1] * L
    u = [-1] * L
    pcur = [-1] * L
    pend = [-1] * L
    prew = [-1] * L
    cc = [0] * L
    ln = [0] * L
    ii = [0] * L
    dh = [0] * L
    mypos = [0] * L
    steps = 0
    next_start = 0
    pos = 1
    order = np.full(n, -1)
    order[0] = r
    for it in range(max_iter):
        # start vertices for idle lanes, in lane order
        idle = [lane for lane in range(L) if ph[lane] == IDLE]
        for rank, lane in enumerate(idle):
            q = next_start + rank
            if q < n:
                s[lane] = int(sorder[q])
            else:
                ph[lane] = DONE
            has_path[lane] = False
        next_start += len(idle)
        if all(p == DONE for p in ph):
            break
        # act: departures and the vertex each lane reads
        if phases is not None:
            for p in ph:
                phases[p] += 1
        ld = [-1] * L
        for lane in range(L):
            p = ph[lane]
            if p == WALK:
                k = O.bounded(seed, c[lane], cc[lane], sample, 0, int(g.deg[c[lane]]))
                v = int(g.col[g.row_off[c[lane]] + k])
                nxt[c[lane]] = v
                cnt[c[lane]] = cc[lane] + 1
                cc[lane] += 1
                steps += 1
                x[lane] = v
                ld[lane] = v
            elif p == IDLE:
                ld[lane] = s[lane]
            elif p == WAIT:
                ld[lane] = x[lane]
            elif p == POPSET:
                ld[lane] = prew[lane]
            elif p == POP:
                ld[lane] = pcur[lane]
            elif p in (COUNT, COMMIT):
                ld[lane] = u[lane]
        snap = {}
        for lane in range(L):
            v = ld[lane]
            if v >= 0:
                snap[lane] = (bool(intree[v]), bool(owned[v]) and not intree[v],
                              int(owner[v]), int(nxt[v]), int(cnt[v]), int(depth[v]))
        was_wait = [p == WAIT for p in ph]
        may = [p in (IDLE, WALK, WAIT) for p in ph]
        want = [may[lane] and ld[lane] >= 0 and not snap[lane][0] and not snap[lane][1]
                for lane in range(L)]
        winner = {}
        for lane in range(L):
            if want[lane] and ld[lane] not in winner:
                winner[ld[lane]] = lane
        fin = [False] * L
        for lane in range(L):
            v = ld[lane]
            if v < 0:
                continue
            in_tree, own, own_lane, wn, wc, wd = snap[lane]
            p = ph[lane]
            if want[lane]:
                if winner[v] == lane:  # claim a free vertex
                    owned[v] = True
                    owner[v] = lane
                    if not has_path[lane]:
                        s[lane] = v
                    has_path[lane] = True
                    c[lane] = v
                    cc[lane] = wc
                    ph[lane] = WALK
                else:
                    if p == IDLE:
                        has_path[lane] = False
                    x[lane] = v
                    ph[lane] = WAIT
            elif may[lane]:
                if in_tree:
                    if not has_path[lane]:
                        ph[lane] = IDLE
                    else:
                        ph[lane] = COUNT
                        u[lane] = s[lane]
                        ln[lane] = 0
                elif own_lane == lane:  # loop on the own path
                    prew[lane] = v
                    cc[lane] = wc
                    pcur[lane] = wn
                    pend[lane] = c[lane]
                    ph[lane] = POP
                else:
                    if p == IDLE:
                        has_path[lane] = False
                    x[lane] = v
                    ph[lane] = WAIT
            elif p == POPSET:
                cc[lane] = wc
                if prew[lane] == c[lane]:
                    ph[lane] = WALK
                else:
                    pcur[lane] = wn
                    pend[lane] = c[lane]
                    ph[lane] = POP
            elif p == POP:
                owned[v] = False
                owner[v] = -1
                if v == pend[lane]:
                    c[lane] = prew[lane]
                    ph[lane] = WALK
                else:
                    pcur[lane] = wn
            elif p == COUNT:
                if in_tree:
                    dh[lane] = wd
                    fin[lane] = True
                else:
                    ln[lane] += 1
                    u[lane] = wn
                    assert ln[lane] <= n
            elif p == COMMIT:
                d = dh[lane] + ln[lane] - ii[lane]
                intree[v] = True
                depth[v] = d
                owned[v] = False
                owner[v] = -1
                order[mypos[lane] + ln[lane] - 1 - ii[lane]] = v
                ii[lane] += 1
                u[lane] = wn
                if ii[lane] == ln[lane]:
                    ph[lane] = IDLE
        # order positions of finished paths: exclusive scan in lane order
        acc = 0
        for lane in range(L):
            if fin[lane]:
                mypos[lane] = pos + acc
                acc += ln[lane]
                ph[lane] = COMMIT
                u[lane] = s[lane]
                ii[lane] = 0
        pos += acc
        # cycles of confirmed waits, every 4th iteration
        if it % 4 != 0:
            continue
        succ = [-1] * L
        for lane in range(L):
            v = ld[lane]
            if v >= 0 and was_wait[lane] and ph[lane] == WAIT and has_path[lane]:
                _, own, own_lane, _, _, _ = snap[lane]
                if own and own_lane != lane:
                    succ[lane] = own_lane
        if sum(1 for q in succ if q >= 0) < 2:
            continue
        on = [False] * L
        for lane in range(L):
            y = lane
            for _ in range(L):
                y = succ[y] if y >= 0 else -1
                if y == lane:
                    on[lane] = True
                    break
        entry = {}
        for lane in range(L):
            if on[lane]:
                pred = [j for j in range(L) if on[j] and succ[j] == lane]
                assert len(pred) == 1
                entry[lane] = x[pred[0]]
        for lane, v in entry.items():
            prew[lane] = v
            ph[lane] = POPSET
    else:
        raise RuntimeError("iteration cap")
    assert intree.all() and pos == n
    parent = nxt.copy()
    parent[r] = -1
    return parent.astype(np.int32), steps, depth, order, it

"""Ticket legality with split-K and fused tiles, by the oracle's checker.

A split-K output region has S tiles: partials 0..S-2 store partial sums and
partial S-1 finishes the region.  The oracle's checker wants each region
written exactly once, so it runs once per partial index k with partial k
standing in as the region's writer (partial S-1 for nodes split fewer ways):
its reads are checked against their producers and its consumers must start
after it.  Then every partial must
have ended before its region's finishing partial started.

A tile of a fused group (the library's fusion map: kernel -> the kernel whose
tiles compute it, or -1) -- a GEMM with elementwise kernels in its epilogue,
or an add computing the adds that feed it -- stands for one tile of each
kernel of the group on the same region.  Tickets are scaled by 8 and the
group's tiles placed in dependency order between the tile's start and end
tickets, the last one ending at the tile's end.  The start ticket of such a
tile is drawn after all its waits, so every operand of the group must have
been released before it.

A tile of a merged GEMM (the library's merge map: kernel -> (the sibling
whose tiles compute it, its first column in that GEMM's output)) covers the
summed width of its siblings: it stands for one tile of each sibling whose
columns it covers, on its share of them, with the same tickets."""
import numpy as np

import oracle


def _groups(w, fused):
    """head -> the kernels its tiles compute (itself included) in dependency order."""
    members = {}
    for v, h in enumerate(fused or []):
        if h >= 0:
            members.setdefault(h, []).append(v)
    groups = {}
    for h, ms in members.items():
        left, order = [h] + ms, []
        while left:
            outs = {w.nodes[u].out for u in left}
            ready = [v for v in left if not ({w.nodes[v].a, w.nodes[v].b} & outs - {w.nodes[v].out})]
            assert ready, f"fused kernels of {h} form a cycle"
            order.append(ready[0])
            left.remove(ready[0])
        groups[h] = order
    return groups


def expand_fused(w, tiles5, split, start, end, fused):
    groups = _groups(w, fused)
    T, S, st, en = [], [], [], []
    for i, t in enumerate(np.asarray(tiles5, np.int64)):
        s8, e8 = 8 * int(start[i]), 8 * int(end[i])
        node = int(t[0])
        sp = int(split[i])
        partial = (sp & 0xFF) and (sp >> 8) < (sp & 0xFF) - 1
        group = groups.get(node)
        if not group or partial:  # a split partial computes the GEMM alone
            T.append(t); S.append(sp); st.append(s8); en.append(e8)
            continue
        for j, m in enumerate(group):
            T.append(np.array([m, t[1], t[2], t[3], t[4]]))
            S.append(sp if m == node else 0)
            st.append(s8 + 2 * j)
            en.append(s8 + 2 * j + 1 if j + 1 < len(group) else e8)
    return (np.array(T, np.int32).reshape(-1, 5), np.array(S, np.int32), np.array(st, np.uint64),
            np.array(en, np.uint64))


def expand_merged(w, tiles5, split, start, end, merges):
    leader, off = merges
    members = {}
    for v, h in enumerate(leader):
        if h >= 0:
            members.setdefault(h, []).append(v)
    T, S, st, en = [], [], [], []
    for i, t in enumerate(np.asarray(tiles5, np.int64)):
        node = int(t[0])
        if node not in members:
            T.append(t); S.append(split[i]); st.append(start[i]); en.append(end[i])
            continue
        for m in members[node]:
            lo, hi = int(off[m]), int(off[m]) + w.buffers[w.nodes[m].out].cols
            c0, c1 = max(int(t[3]), lo), min(int(t[4]), hi)
            if c0 < c1:
                T.append(np.array([m, t[1], t[2], c0 - lo, c1 - lo]))
                S.append(split[i]); st.append(start[i]); en.append(end[i])
    return (np.array(T, np.int32).reshape(-1, 5), np.array(S, np.int32), np.array(st, np.int64),
            np.array(en, np.int64))


def check(w, tiles5, split, start, end, fused=None, merges=None):
    tiles5 = np.asarray(tiles5, np.int32)
    split = np.asarray(split, np.int32)
    start = np.asarray(start, np.int64)
    end = np.asarray(end, np.int64)
    if merges is not None and any(h >= 0 for h in merges[0]):
        tiles5, split, start, end = expand_merged(w, tiles5, split, start, end, merges)
    if fused is not None and any(h >= 0 for h in fused):
        tiles5, split, start, end = expand_fused(w, tiles5, split, start, end, fused)
    assert end.max(initial=0) < 2 ** 32, "tickets out of range"
    start = start.astype(np.uint32)
    end = end.astype(np.uint32)
    S = split & 0xFF
    idx = split >> 8
    assert ((S == 0) | (idx < S)).all()
    for k in sorted(set(idx[S > 0].tolist())) or [0]:
        # nodes split fewer ways than k + 1 stand in with their finishing partials
        keep = (S == 0) | (idx == np.minimum(k, S - 1))
        rc, bu, bv = oracle.check_trace(w, tiles5[keep], start[keep], end[keep])
        assert rc == 0, f"illegal trace (partial index {k}): code {rc}, tiles {bu} -> {bv}"
    fin = {}
    for i in np.nonzero((S > 0) & (idx == S - 1))[0]:
        fin[tuple(tiles5[i, [0, 1, 3]])] = i
    for i in np.nonzero((S > 0) & (idx < S - 1))[0]:
        f = fin[tuple(tiles5[i, [0, 1, 3]])]
        assert end[i] < start[f], f"partial tile {i} ends after its finishing tile {f} starts"

"""Ticket legality with split-K and fused tiles, by the oracle's checker.

A split-K output region has S tiles: partials 0..S-2 store partial sums and
partial S-1 finishes the region.  The oracle's checker wants each region
written exactly once, so it runs once per partial index k with partial k
standing in as the region's writer (partial S-1 for nodes split fewer ways):
its reads are checked against their producers and its consumers must start
after it.  Then every partial must
have ended before its region's finishing partial started.

A tile of a GEMM with fused elementwise kernels (the library's fusion map:
kernel -> the GEMM that computes it, or -1) stands for one tile of each kernel
of its chain on the same region.  Tickets are scaled by 8 and the chain's
tiles placed in chain order between the tile's start and end tickets: the
GEMM's right after the start, each fused kernel's after the previous one's,
the last one ending at the tile's end.  The start ticket of such a tile is
drawn after the waits of its epilogue, so each fused kernel's other operand
must have been released before it."""
import numpy as np

import oracle


def _chains(w, fused):
    """head GEMM -> its fused kernels in chain order (each reads the previous output)."""
    members = {}
    for v, h in enumerate(fused or []):
        if h >= 0:
            members.setdefault(h, []).append(v)
    chains = {}
    for h, ms in members.items():
        prev, order, left = w.nodes[h].out, [], list(ms)
        while left:
            nxt = [v for v in left if prev in (w.nodes[v].a, w.nodes[v].b)]
            assert len(nxt) == 1, f"fused kernels of {h} do not form a chain"
            order.append(nxt[0])
            left.remove(nxt[0])
            prev = w.nodes[nxt[0]].out
        chains[h] = order
    return chains


def expand_fused(w, tiles5, split, start, end, fused):
    chains = _chains(w, fused)
    T, S, st, en = [], [], [], []
    for i, t in enumerate(np.asarray(tiles5, np.int64)):
        s8, e8 = 8 * int(start[i]), 8 * int(end[i])
        node = int(t[0])
        sp = int(split[i])
        partial = (sp & 0xFF) and (sp >> 8) < (sp & 0xFF) - 1
        chain = chains.get(node, [])
        if not chain or partial:
            T.append(t); S.append(sp); st.append(s8); en.append(e8)
            continue
        T.append(t); S.append(sp); st.append(s8); en.append(s8 + 1)
        for j, m in enumerate(chain):
            T.append(np.array([m, t[1], t[2], t[3], t[4]]))
            S.append(0)
            st.append(s8 + 2 * (j + 1))
            en.append(s8 + 2 * (j + 1) + 1 if j + 1 < len(chain) else e8)
    return (np.array(T, np.int32).reshape(-1, 5), np.array(S, np.int32), np.array(st, np.uint64),
            np.array(en, np.uint64))


def check(w, tiles5, split, start, end, fused=None):
    tiles5 = np.asarray(tiles5, np.int32)
    split = np.asarray(split, np.int32)
    start = np.asarray(start, np.int64)
    end = np.asarray(end, np.int64)
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

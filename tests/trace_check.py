"""Ticket legality with split-K tiles, by the oracle's checker.

A split-K output region has S tiles: partials 0..S-2 store partial sums and
partial S-1 finishes the region.  The oracle's checker wants each region
written exactly once, so it runs once per partial index k with partial k
standing in as the region's writer (partial S-1 for nodes split fewer ways):
its reads are checked against their producers and its consumers must start
after it.  Then every partial must
have ended before its region's finishing partial started."""
import numpy as np

import oracle


def check(w, tiles5, split, start, end):
    tiles5 = np.asarray(tiles5, np.int32)
    split = np.asarray(split, np.int32)
    start = np.asarray(start, np.uint32)
    end = np.asarray(end, np.uint32)
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

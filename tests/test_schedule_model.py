"""Host-side model of the GPU work decomposition (no GPU).

The CUDA tree kernel maps Listing 4's row tree onto warps: the tree is cut
at depth dw into work items, each item is evaluated in groups of 2^G slots
with a binary-counter stack, and the levels above the cut are combined by
ticket-holding second arrivers.  This model replays exactly that schedule
in Python -- item rows from the brev formula, the root-to-node walk, the
group occupancy rule, the stack, the ticket/slot indices, arbitrary arrival
orders -- and checks that

* every row is read exactly once and every element index is inside [0, n),
* every ticket index lies in [0, 2^dw - 1) and every slot index in
  [0, 2 (2^dw - 1)) of the vector's block,
* the value equals the oracle's Listing 4 recursion bit for bit (the
  combine is the oracle's v1_hypot, applied lane-wise).

It checks the index arithmetic the kernel relies on before the kernel
ever runs, and pins that the decomposition is the paper's tree.
"""
import random

import numpy as np
import pytest

import oracle
from paper_2509_06220_gb300 import inputs

_k1v = np.vectorize(lambda a, b: oracle.k1(a, b), otypes=[np.float64])


def brev(j, d):
    r = 0
    for _ in range(d):
        r = (r << 1) | (j & 1)
        j >>= 1
    return r


def clog2(m):
    d = 0
    while (1 << d) < m:
        d += 1
    return d


def node_rows(m, j, d):
    b = brev(j, d)
    if b >= m:
        return 0
    return ((m - b) + (1 << d) - 1) >> d


def node_start(m, j, d):
    start, size = 0, m
    for l in range(d - 1, -1, -1):
        left = (size + 1) >> 1
        if (j >> l) & 1:
            start += left
            size -= left
        else:
            size = left
    return start


def plan_single(n, P, sms, wpb, item_log2, G, maxl=10, dwmax=20):
    m = (n + P - 1) // P
    D = clog2(m)
    min_items = sms * wpb * 2
    dw = max(D - item_log2, clog2(min_items))
    dw = min(dw, D - G)
    dw = max(dw, 0)
    dw = min(dw, dwmax)
    k = D - dw
    assert k <= G + maxl
    return m, D, k, dw


class Model:
    def __init__(self, x, P, G):
        self.x, self.n, self.P, self.G = x, x.size, P, G
        self.reads = {}

    def load_row(self, row):
        P, n = self.P, self.n
        e0 = row * P
        assert 0 <= e0 < n, "row start outside the vector"
        self.reads[row] = self.reads.get(row, 0) + 1
        v = np.zeros(P)
        hi = min(n, e0 + P)
        v[:hi - e0] = self.x[e0:hi]
        return v

    def group(self, row0, tg):
        U = 1 << self.G
        assert 1 <= tg <= U
        buf, occ, r = [None] * U, [False] * U, row0
        for s in range(U):
            occ[s] = brev(s, self.G) < tg
            if occ[s]:
                buf[s] = self.load_row(r)
                r += 1
        w = U
        while w > 1:
            for s in range(w // 2):
                a, b = occ[2 * s], occ[2 * s + 1]
                if a and b:
                    buf[s] = _k1v(buf[2 * s], buf[2 * s + 1])
                elif a:
                    buf[s] = buf[2 * s]
                elif b:
                    buf[s] = buf[2 * s + 1]
                occ[s] = a or b
            w //= 2
        return buf[0]

    def item(self, start, t, k):
        G = self.G
        if k <= G:
            return self.group(start, t)
        L = k - G
        st, stf, row, r = [None] * L, 0, start, None
        for g in range(1 << L):
            tg = node_rows(t, g, L)
            fr = tg > 0
            if fr:
                r = self.group(row, tg)
                row += tg
            else:
                r = np.zeros(self.P)
            for l in range(L):
                if ((g >> l) & 1) == 0:
                    st[l] = r
                    stf = (stf | (1 << l)) if fr else (stf & ~(1 << l))
                    break
                fl = (stf >> l) & 1
                if fl:
                    r = _k1v(st[l], r) if fr else st[l]
                fr = fr or bool(fl)
        assert row == start + t, "item rows not consumed exactly"
        return r


def run_model(x, P, G, dw, seed=0):
    n = x.size
    m = (n + P - 1) // P
    D = clog2(m)
    k = D - dw
    mod = Model(x, P, G)
    items = 1 << dw
    nodes = items - 1
    tickets = [0] * max(nodes, 1)
    slots = {}
    order = list(range(items))
    random.Random(seed).shuffle(order)
    result = None
    vals = {}
    for i in order:  # arrival order of the warps finishing their items
        t = node_rows(m, i, dw)
        assert t >= 1
        vals[i] = mod.item(node_start(m, i, dw), t, k)
    # second arrivers climb; replay arrivals in the shuffled order
    for i in order:
        r = vals[i]
        h = (1 << dw) + i
        root = True
        while h > 1:
            si = h - 2
            assert 0 <= si < 2 * nodes
            slots[si] = r
            ti = (h >> 1) - 1
            assert 0 <= ti < nodes
            tickets[ti] += 1
            if tickets[ti] == 1:
                root = False
                break
            assert tickets[ti] == 2
            tickets[ti] = 0
            sib = slots[(h ^ 1) - 2]
            r = _k1v(sib, r) if (h & 1) else _k1v(r, sib)
            h >>= 1
        if root:
            assert result is None
            result = r
    assert all(t == 0 for t in tickets), "tickets must be back to zero"
    assert sorted(mod.reads) == list(range(m)) and set(mod.reads.values()) == {1}
    # lane reduction: R with contiguous pairing
    v = list(result)
    while len(v) > 1:
        v = [oracle.k1(v[2 * j], v[2 * j + 1]) for j in range(len(v) // 2)]
    return np.float64(v[0])


@pytest.mark.parametrize("P", [4, 8])
@pytest.mark.parametrize("G", [2, 3])
def test_model_equals_listing4(P, G):
    r = random.Random(P * 10 + G)
    ns = list(range(1, 12 * P)) + [r.randint(1, 300 * P) for _ in range(12)]
    base = inputs.vector(max(ns), seed=5, vec=1)
    for n in ns:
        x = base[:n]
        m = (n + P - 1) // P
        D = clog2(m)
        for dw in sorted({0, max(0, D - G), D // 2, max(0, D - G - 2)}):
            if D - dw > G + 10:
                continue
            got = run_model(x, P, G, dw, seed=n + dw)
            assert got.tobytes() == oracle.nrm(x, P=P).tobytes(), (n, dw)


def test_plan_single_limits():
    """The single-vector plan keeps dw <= 20 and k <= G + 10 up to 2^33 rows,
    and gives enough items to fill 152 SMs for the benchmark sizes."""
    for P in (64, 128):
        for lg in range(0, 34):
            n = (1 << lg) * P
            m, D, k, dw = plan_single(n, P, 152, 8, 7, 3)
            assert 0 <= dw <= 20 and k <= 13 and k == D - dw
        m, D, k, dw = plan_single(1 << 28, P, 152, 8, 7, 3)
        assert (1 << dw) >= 152 * 8


def slot_rank(s, tg, G):
    """The kernels' row of slot s in a group of tg occupied slots: the number
    of occupied slots before it, clamped to tg - 1 for an empty slot."""
    r = sum(1 for q in range(s) if brev(q, G) < tg)
    return min(r, tg - 1)


@pytest.mark.parametrize("G", [2, 3])
def test_ring_and_slot_rank_indices(G):
    """The index arithmetic of the ring path for partial work items: group g
    of an item of t rows (2^(k-G) <= t <= 2^k) has node_rows(t, g, k - G)
    rows, copied from a running row offset; slot_rank maps each occupied
    slot to the row the slot form assigns it (rows in slot order) and every
    slot to a row of the group; the tail group starts where the ring's
    groups end; and the slot form over those rows is the ceil-split tree of
    the group's rows."""
    U = 1 << G
    for tg in range(1, U + 1):
        seq, r = {}, 0
        for s in range(U):
            if brev(s, G) < tg:
                seq[s] = r
                r += 1
        assert r == tg
        for s in range(U):
            assert 0 <= slot_rank(s, tg, G) < tg
            if s in seq:
                assert slot_rank(s, tg, G) == seq[s]
        # the slot form (pairs of occupied slots combine, a lone one passes
        # up) builds the ceil-split tree of the tg rows
        def ceil_tree(lo, cnt):
            if cnt == 1:
                return lo
            left = (cnt + 1) // 2
            return (ceil_tree(lo, left), ceil_tree(lo + left, cnt - left))
        buf = [seq.get(s) for s in range(U)]
        occ = [s in seq for s in range(U)]
        w = U
        while w > 1:
            for s in range(w // 2):
                a, c = occ[2 * s], occ[2 * s + 1]
                if a and c:
                    buf[s] = (buf[2 * s], buf[2 * s + 1])
                elif c:
                    buf[s] = buf[2 * s + 1]
                elif a:
                    buf[s] = buf[2 * s]
                occ[s] = a or c
            w //= 2
        assert buf[0] == ceil_tree(0, tg)
    for k in range(G + 1, G + 7):
        L = k - G
        for t in range(1 << L, (1 << k) + 1):
            pref, rows = 0, []
            for g in range(1 << L):
                tq = node_rows(t, g, L)
                assert 1 <= tq <= U
                rows.append((pref, tq))
                pref += tq
            assert pref == t
            # the tail group (the last) starts at t - tg
            last0, lastn = rows[-1]
            assert last0 == t - lastn
            # groups are the item's subtrees at depth L: their row starts are
            # the root-to-node walk
            for g, (r0, tq) in enumerate(rows):
                assert r0 == node_start(t, g, L) and tq == node_rows(t, g, L)


@pytest.mark.parametrize("P", [64, 128])
def test_batch_stack_depth_bound(P):
    """The batch path sizes each warp's counter stack from a bound on the
    work-item depth k of every vector: with offsets (vectors never overlap)
    the ticket bound 2 (x_len / P + B + 1) / 2^item_log2 + 2 holds for the
    planner's first depth, so items never deepen, and each vector's k =
    min(D, item_log2), raised to D - DW_MAX when the cut would be deeper than
    DW_MAX, is at most max(min(dmax, item_log2), dmax - DW_MAX) for
    dmax = ceil(log2(ceil(x_len / P))).  The planner's rule replayed on
    random ragged batches, including very long vectors."""
    DW_MAX = 20
    rng = random.Random(P)
    for trial in range(300):
        item_log2 = rng.randint(4, 12)
        B = rng.randint(1, 64)
        kind = trial % 3
        if kind == 0:
            lens = [rng.randint(0, 1 << rng.randint(0, 20)) for _ in range(B)]
        elif kind == 1:
            lens = [1 << rng.randint(0, 36) for _ in range(B)]
        else:
            lens = [rng.randint(0, 1 << 40) for _ in range(B)]
        x_len = sum(lens)
        dmax = clog2(max(1, (x_len + P - 1) // P))
        kmax = max(min(dmax, item_log2), dmax - DW_MAX)
        nodes = 0
        for n in lens:
            if n == 0:
                continue
            m = (n + P - 1) // P
            D = clog2(m)
            k = min(D, item_log2)
            if D - k > DW_MAX:
                k = D - DW_MAX
            assert k <= kmax, (n, k, kmax)
            nodes += (1 << (D - k)) - 1
        node_cap = (2 * (x_len // P + B + 1) >> item_log2) + 2
        assert nodes <= node_cap, (nodes, node_cap)


"""Race check of the band-to-tridiagonal sweep schedule (CPU, no GPU).

The band stage of the two-stage reduction runs one sweep per CTA at a time;
sweep i waits only on two counts that sweep i - 1 publishes.  This test models
every phase of every task of every sweep with the matrix entries it reads from
and writes to global memory, builds the happens-before relation from program
order and the waits, and checks that any two accesses to one entry from
different sweeps, at least one a write, are ordered like the sequential
algorithm (sweep i - 1 first).  The phases and waits follow the kernel:

* R_0: the reflected column i, rows i+1 .. i+b (read and written) once
  crit[i-1] >= 2;
* task t with a successor, window [p, q), block below [q, qb):
  A (t >= 1): write-back of the deferred part of task t - 1 (its diagonal
  block's columns >= 1, rows >= column) and of the left block (rows [p, q),
  columns [p - b + 1, p)); then pre[i] = t;
  E: once pre[i-1] >= t + 1, the window's lower triangle and the block below
  are read but for their last column;
  C: once crit[i-1] >= t + 3, the last column (b + 1 entries) is read and
  column p of the window and of the block below written; then crit[i] = t + 2;
* the last task: A, then once crit[i-1] >= t + 3 everything read and written,
  then both counts at their end value.

A count that a sweep never reaches (it ends earlier) is reached at its end.
Planted mistakes (a wait one task too early) must produce races.
"""
import itertools

import pytest

DONE = 1 << 30


class Schedule:
    def __init__(self, n, b, e_need=1, c_need=3, r0_need=2):
        self.n, self.b = n, b
        self.nodes = []          # (sweep, label, reads, writes)
        self.anc = []            # ancestor bitsets
        self.races = []
        sweeps = []              # per sweep: {'pre': [(value, node)], 'crit': [(value, node)], 'end': node}
        for i in range(n - 2):
            prev = sweeps[-1] if sweeps else None
            info = {"pre": [], "crit": [], "end": None}
            last = None

            def node(label, reads, writes, waits=()):
                nonlocal last
                k = len(self.nodes)
                a = 0
                if last is not None:
                    a |= self.anc[last] | (1 << last)
                for w in waits:
                    if w is not None:
                        a |= self.anc[w] | (1 << w)
                self.nodes.append((i, label, frozenset(reads), frozenset(writes)))
                self.anc.append(a)
                last = k
                return k

            def released(kind, need):
                """the node after which count `kind` of sweep i - 1 is >= need"""
                if prev is None:
                    return None
                for v, nd in prev[kind]:
                    if v >= need:
                        return nd
                raise AssertionError("count never reached")

            p = i + 1
            col = {(r, i) for r in range(p, min(p + b, n))}
            k = node("R0", col, col, [released("crit", r0_need)])
            info["crit"].append((1, k))
            t = 0
            while True:
                p = i + 1 + b * t
                q = min(p + b, n)
                ln = q - p
                qb = min(q + b, n)
                lnb = qb - q
                nxt = q <= n - 2
                if t > 0:
                    pp = p - b
                    w = {(pp + r, pp + c) for c in range(1, b) for r in range(c, b)}
                    w |= {(p + r, p - b + c) for r in range(ln) for c in range(1, b)}
                    k = node("A%d" % t, (), w)
                    info["pre"].append((t, k))
                win = {(p + r, p + c) for c in range(ln) for r in range(c, ln)}
                below = {(q + r, p + c) for r in range(lnb) for c in range(ln)}
                if not nxt:
                    k = node("L%d" % t, win | below, win | below, [released("crit", t + c_need)])
                    info["pre"].append((DONE, k))
                    info["crit"].append((DONE, k))
                    info["end"] = k
                    break
                lastc = p + b - 1
                early = {e for e in win | below if e[1] != lastc}
                node("E%d" % t, early, (), [released("pre", t + e_need)])
                late = {e for e in win | below if e[1] == lastc}
                wr = {(p + r, p) for r in range(ln)} | {(q + r, p) for r in range(lnb)}
                k = node("C%d" % t, late, wr, [released("crit", t + c_need)])
                info["crit"].append((t + 2, k))
                t += 1
            sweeps.append(info)
        self.check()

    def check(self):
        acc = {}
        for k, (sw, _, rd, wr) in enumerate(self.nodes):
            for e in rd:
                acc.setdefault(e, []).append((k, False))
            for e in wr:
                acc.setdefault(e, []).append((k, True))
        self.pairs = 0
        for e, lst in acc.items():
            for (u, wu), (v, wv) in itertools.combinations(lst, 2):
                su, sv = self.nodes[u][0], self.nodes[v][0]
                if su == sv or not (wu or wv):
                    continue
                if su > sv:
                    u, v = v, u
                self.pairs += 1
                if not (self.anc[v] >> u) & 1:
                    self.races.append((e, self.nodes[u][:2], self.nodes[v][:2]))


@pytest.mark.parametrize("n,b", [(12, 4), (37, 4), (41, 8), (70, 32), (99, 32)])
def test_schedule_has_no_race(n, b):
    s = Schedule(n, b)
    assert s.pairs > 1000   # the check looked at many conflicting pairs
    assert not s.races, s.races[:5]


@pytest.mark.parametrize("mistake", [{"e_need": 0}, {"c_need": 2}, {"r0_need": 1}])
def test_planted_early_wait_is_a_race(mistake):
    # E reading the window before sweep i - 1 wrote its deferred part, C reading the last
    # column before sweep i - 1 formed it, R_0 reading its column too early
    assert Schedule(41, 8, **mistake).races

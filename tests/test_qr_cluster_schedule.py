"""Race check of the cluster panel QR's shared-memory protocol (CPU, no GPU).

Per reflector l every CTA of the cluster writes its parts into its own buffer
of parity l, arrives at the cluster barrier, waits on it, then reads every
CTA's buffer of parity l through distributed shared memory; one barrier per
reflector.  The model builds the happens-before relation of these phases
(program order; a wait completes after every CTA's arrive of the same
barrier) and checks that each read of a buffer sees the write of its own
reflector and that no later write to the buffer can overtake a read of it.
With one buffer instead of two the check must find a race.
"""
import pytest


def races(ncta, nref, buffers=2):
    nodes = []        # (cta, phase, l)
    anc = []
    idx = {}

    def add(key, preds):
        a = 0
        for p in preds:
            a |= anc[p] | (1 << p)
        idx[key] = len(nodes)
        nodes.append(key)
        anc.append(a)

    for l in range(nref):
        for x in range(ncta):
            prev = [idx[(x, "S", l - 1)]] if l > 0 else []
            add((x, "P", l), prev)                    # parts into own buffer l % buffers
        for x in range(ncta):
            add((x, "A", l), [idx[(x, "P", l)]])      # barrier.cluster.arrive.release
        for x in range(ncta):
            add((x, "W", l), [idx[(y, "A", l)] for y in range(ncta)])   # wait.acquire
        for x in range(ncta):
            add((x, "S", l), [idx[(x, "W", l)]])      # remote reads of every CTA's buffer
    add(("all", "end", nref), [idx[(x, "S", nref - 1)] for x in range(ncta)])   # final barrier

    def hb(u, v):
        return (anc[idx[v]] >> idx[u]) & 1

    found = []
    for y in range(ncta):              # the buffers of CTA y
        for l in range(nref):
            w = (y, "P", l)
            for x in range(ncta):
                r = (x, "S", l)
                if not hb(w, r):       # the read of reflector l must see its write
                    found.append((w, r))
                for l2 in range(l + 1, nref):   # a later write to the same buffer
                    if l2 % buffers == l % buffers and not hb(r, (y, "P", l2)):
                        found.append((r, (y, "P", l2)))
                        break
    return found


@pytest.mark.parametrize("ncta,nref", [(8, 32), (16, 32), (16, 5)])
def test_double_buffered_parts_have_no_race(ncta, nref):
    assert not races(ncta, nref)


def test_single_buffer_is_a_race():
    assert races(16, 32, buffers=1)

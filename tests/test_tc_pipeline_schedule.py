"""Race check of the warp-specialised tensor-core panel update's pipeline
(CPU, no GPU).

The kernel's three roles synchronise only through mbarriers waited on by
phase parity: the producer copies the Y digits of a column tile (mb_y, once
the MMAs of the previous tile are done: mb_acc) and streams the 8 X digits of
each tile through 3 slots (item j in slot j % 3: its copy is the (j/3)-th
completion of mb_full[slot], which the producer may issue once the MMAs of
item j - 3 have completed, the (j/3 - 1)-th completion of mb_empty[slot]); the
MMA issuer waits for mb_y on a new column tile, for mb_free (the epilogue has
read the previous tile's accumulators), for mb_full of each item, commits each
item's MMAs to mb_empty[slot] and each tile's to mb_acc; the epilogue waits
for mb_acc, reads the accumulators and arrives on mb_free.  This model runs
the three roles under random interleavings, with copies and MMAs completing
asynchronously at random later times, and checks at every step that no buffer
is overwritten while a reader still needs it, that no operand or accumulator
is read before it is complete, and that no wait is two phases behind its
barrier (a parity wait would then never return).
"""
import random

import pytest

SLOTS, DIG = 3, 8


class Barrier:
    def __init__(self, count):
        self.count, self.arrived, self.done = count, 0, 0   # done: completed phases

    def arrive(self):
        self.arrived += 1
        if self.arrived == self.count:
            self.arrived = 0
            self.done += 1


class Model:
    def __init__(self, tiles, rng):
        self.rng = rng
        self.tiles = tiles                       # list of column-tile indices, one per tile
        self.mb = {"y": Barrier(1), "acc": Barrier(1), "free": Barrier(4), "fin": Barrier(1)}
        for s in range(SLOTS):
            self.mb["full%d" % s] = Barrier(1)
            self.mb["empty%d" % s] = Barrier(1)
        self.pending = []                        # asynchronous operations: (kind, payload)
        self.slot_item = [None] * SLOTS          # item whose digits a slot holds (complete copy)
        self.slot_readers = [set() for _ in range(SLOTS)]   # items whose MMAs are still in flight
        self.y_tile = None                       # column tile of the Y buffer (complete copy)
        self.y_readers = 0                       # MMAs in flight reading Y
        self.acc_tile = None                     # tile whose accumulators are complete in TMEM
        self.acc_writers = 0                     # MMAs in flight writing the accumulators
        self.epi_reading = None
        self.errors = []
        self.roles = [self.producer(), self.mma(), self.epilogue()]

    # -- waits: a role yields ("wait", barrier, k) to wait for the k-th completion (0-based)
    def ready(self, name, k):
        done = self.mb[name].done
        if done > k + 1:
            self.errors.append("wait on %s for phase %d with %d completed: parity never returns" % (name, k, done))
        return done >= k + 1

    def producer(self):
        cur = None
        for tl, ct in enumerate(self.tiles):
            if ct != cur:
                if tl > 0:
                    yield ("wait", "acc", tl - 1)
                if self.y_readers:
                    self.errors.append("Y overwritten while MMAs read it")
                self.pending.append(("ycopy", ct))
                cur = ct
            for k in range(DIG):
                j = tl * DIG + k
                s = j % SLOTS
                if j >= SLOTS:
                    yield ("wait", "empty%d" % s, (j - SLOTS) // SLOTS)
                if self.slot_readers[s]:
                    self.errors.append("slot %d overwritten while item(s) %s are read" % (s, self.slot_readers[s]))
                self.slot_item[s] = None
                self.pending.append(("xcopy", (s, j)))
                yield ("step",)

    def mma(self):
        cur, yw = None, 0
        for tl, ct in enumerate(self.tiles):
            if ct != cur:
                yield ("wait", "y", yw)
                yw += 1
                cur = ct
                if self.y_tile != ct:
                    self.errors.append("MMAs of tile %d read Y before its copy landed" % tl)
            if tl > 0:
                yield ("wait", "free", tl - 1)
            if self.epi_reading is not None:
                self.errors.append("accumulators overwritten while the epilogue reads them")
            self.acc_tile = None
            for k in range(DIG):
                j = tl * DIG + k
                s = j % SLOTS
                yield ("wait", "full%d" % s, j // SLOTS)
                if self.slot_item[s] != j:
                    self.errors.append("MMA of item %d read slot %d holding %s" % (j, s, self.slot_item[s]))
                self.slot_readers[s].add(j)
                self.y_readers += 1
                self.acc_writers += 1
                self.pending.append(("mma", (s, j)))
                self.pending.append(("commit", "empty%d" % s))
                yield ("step",)
            self.pending.append(("commit_acc", tl))

    def epilogue(self):
        for tl in range(len(self.tiles)):
            yield ("wait", "acc", tl)
            if self.acc_tile != tl or self.acc_writers:
                self.errors.append("epilogue of tile %d read accumulators before the MMAs completed" % tl)
            self.epi_reading = tl
            yield ("step",)
            self.epi_reading = None
            for _ in range(4):                     # four epilogue warps arrive
                self.mb["free"].arrive()
            yield ("step",)

    # -- asynchronous completions, in issue order per kind (copies of a thread land in any order,
    # a commit completes only after every earlier MMA of the issuing thread)
    def complete_one(self):
        cands = []
        for i, (kind, _) in enumerate(self.pending):
            if kind in ("commit", "commit_acc"):
                if any(k == "mma" for k, _ in self.pending[:i]):
                    continue
            cands.append(i)
        if not cands:
            return False
        i = self.rng.choice(cands)
        kind, x = self.pending.pop(i)
        if kind == "ycopy":
            self.y_tile = x
            self.mb["y"].arrive()
        elif kind == "xcopy":
            s, j = x
            self.slot_item[s] = j
            self.mb["full%d" % s].arrive()
        elif kind == "mma":
            s, j = x
            self.slot_readers[s].discard(j)
            self.y_readers -= 1
            self.acc_writers -= 1
        elif kind == "commit":
            self.mb[x].arrive()
        elif kind == "commit_acc":
            self.acc_tile = x
            self.mb["acc"].arrive()
        return True

    def run(self):
        state = [None] * 3                         # the pending wait of each role
        alive = [True] * 3
        while any(alive) or self.pending:
            moves = []
            for r in range(3):
                if alive[r] and (state[r] is None or self.ready(state[r][1], state[r][2])):
                    moves.append(r)
            if self.pending:
                moves.append(-1)
            if not moves:
                self.errors.append("deadlock")
                break
            r = self.rng.choice(moves)
            if r < 0:
                self.complete_one()
                continue
            state[r] = None
            try:
                act = next(self.roles[r])
                if act[0] == "wait":
                    state[r] = act
            except StopIteration:
                alive[r] = False
        return self.errors


@pytest.mark.parametrize("seed", range(40))
def test_pipeline_has_no_race(seed):
    rng = random.Random(seed)
    ntile = rng.randint(1, 7)
    tiles, ct = [], 0
    for _ in range(ntile):                          # column tiles change every few tiles
        if rng.random() < 0.4:
            ct += 1
        tiles.append(ct)
    errors = Model(tiles, rng).run()
    assert not errors, errors[:3]


def test_planted_missing_empty_wait_is_caught():
    # the producer not waiting for the MMAs of item j - 3 before reusing its slot
    class Broken(Model):
        def producer(self):
            cur = None
            for tl, ct in enumerate(self.tiles):
                if ct != cur:
                    if tl > 0:
                        yield ("wait", "acc", tl - 1)
                    self.pending.append(("ycopy", ct))
                    cur = ct
                for k in range(DIG):
                    j = tl * DIG + k
                    s = j % SLOTS
                    if self.slot_readers[s]:
                        self.errors.append("slot %d overwritten while read" % s)
                    self.slot_item[s] = None
                    self.pending.append(("xcopy", (s, j)))
                    yield ("step",)

    caught = any(Broken([0, 0, 1], random.Random(s)).run() for s in range(40))
    assert caught

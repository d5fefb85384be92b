"""A model of the hand-off between warp 0 and warps 1-7 in the decision loop of
the slice kernel (spin channel, periodic: the pipelined path of
paper_2609_14668_b300/csrc/update.cuh), checked on the CPU.

The kernel's two parties use named barriers that have no time limit, so the
protocol must be right by construction.  The model replays each party's
sequence of barrier operations exactly as the kernel issues them:

* warp 0 publishes move a (site or -1) and arrives on TF(a & 1) (ids 2, 3),
  waits on DONE((a-1) & 1) (ids 4, 5) before it reads the block G^(a), and
  waits once more on the last DONE before it leaves;
* warps 1-7 wait on TF(a & 1), stop on site -1, else read G^(a), write
  G^(a+1) into the other buffer and arrive on DONE(a & 1).

Under random interleavings of the two parties (and random accept patterns,
with and without the n_delay stop) no barrier phase may receive more than its
256 threads, no party may wait forever, every phase must be complete at the
end, and warp 0 must never read the buffer warps 1-7 are writing."""
import random

import pytest


class _Barrier:
    def __init__(self):
        self.count = 0
        self.phase = 0


def _run(accepts, nd_stop, seed):
    rnd = random.Random(seed)
    bars = {i: _Barrier() for i in (2, 3, 4, 5)}
    slots = [None, None]
    writing = set()

    def warp0():
        tf = accepts[0] if accepts else -1
        slots[0] = tf
        yield ("arrive", 2)
        na, idx = 0, 0
        while tf >= 0:
            idx += 1
            if nd_stop is not None and idx == nd_stop:
                tn = -1
            else:
                tn = accepts[idx] if idx < len(accepts) else -1
            if na >= 1:
                yield ("sync", 5 if (na - 1) & 1 else 4)
            if tn >= 0:
                yield ("read", na & 1)
            ns = (na + 1) & 1
            slots[ns] = tn
            yield ("arrive", 3 if ns else 2)
            tf, na = tn, na + 1
        if na >= 1:
            yield ("sync", 5 if (na - 1) & 1 else 4)

    def trailing():
        na = 0
        while True:
            sl = na & 1
            yield ("sync", 3 if sl else 2)
            if slots[sl] < 0:
                return
            yield ("write", (na + 1) & 1)
            yield ("arrive", 5 if sl else 4)
            na += 1

    procs = {"w0": [warp0(), 32, False], "tr": [trailing(), 224, False]}
    waiting = {}
    for _ in range(100000):
        runnable = []
        for name, (gen, nthreads, done) in procs.items():
            if done:
                continue
            if name in waiting:
                b, ph = waiting[name]
                if bars[b].phase <= ph:
                    continue
                del waiting[name]
            runnable.append(name)
        if not runnable:
            if all(p[2] for p in procs.values()):
                break
            return "deadlock"
        name = rnd.choice(runnable)
        proc = procs[name]
        try:
            kind, arg = next(proc[0])
        except StopIteration:
            proc[2] = True
            continue
        if kind in ("arrive", "sync"):
            b = bars[arg]
            b.count += proc[1]
            if b.count > 256:
                return f"barrier {arg} over-subscribed"
            if b.count == 256:
                b.count, b.phase = 0, b.phase + 1
            elif kind == "sync":
                waiting[name] = (arg, b.phase)
            if name == "tr" and kind == "arrive":
                writing.clear()
        elif kind == "read" and arg in writing:
            return "warp 0 read a buffer being written"
        elif kind == "write":
            writing.clear()
            writing.add(arg)
    else:
        return "no progress"
    if any(b.count for b in bars.values()):
        return "unbalanced"
    return "ok"


@pytest.mark.parametrize("block", range(4))
def test_handoff_protocol(block):
    for trial in range(block * 500, (block + 1) * 500):
        r = random.Random(trial)
        n = r.randint(0, 16)
        accepts = sorted(r.sample(range(32), n))
        nd_stop = r.choice([None, r.randint(1, n)]) if n else None
        for s in range(4):
            assert _run(accepts, nd_stop, trial * 7 + s) == "ok", (accepts, nd_stop)


def test_model_detects_a_broken_protocol():
    """The same check fails when warp 0 publishes the next move before reading
    G^(a) (a planted mistake in the model, not in the kernel)."""
    bad = 0
    for trial in range(200):
        r = random.Random(trial)
        accepts = sorted(r.sample(range(32), 8))
        bad += _broken_run(accepts, trial) != "ok"
    assert bad > 0


def _broken_run(accepts, seed):
    """Warp 0 publishes move a+1 before it reads G^(a) and never waits on DONE."""
    rnd = random.Random(seed)
    slots = [None, None]
    writing = set()
    bars = {i: _Barrier() for i in (2, 3)}

    def warp0():
        tf = accepts[0]
        slots[0] = tf
        yield ("arrive", 2)
        na, idx = 0, 0
        while tf >= 0:
            idx += 1
            tn = accepts[idx] if idx < len(accepts) else -1
            ns = (na + 1) & 1
            slots[ns] = tn
            yield ("arrive", 3 if ns else 2)
            if tn >= 0:
                yield ("read", na & 1)
            tf, na = tn, na + 1

    def trailing():
        na = 0
        while True:
            sl = na & 1
            yield ("sync", 3 if sl else 2)
            if slots[sl] < 0:
                return
            yield ("write", (na + 1) & 1)
            yield ("end", None)
            na += 1

    procs = {"w0": [warp0(), 32, False], "tr": [trailing(), 224, False]}
    waiting = {}
    for _ in range(10000):
        runnable = [n for n, p in procs.items() if not p[2] and
                    (n not in waiting or bars[waiting[n][0]].phase > waiting[n][1])]
        for n in runnable:
            waiting.pop(n, None)
        if not runnable:
            return "ok" if all(p[2] for p in procs.values()) else "deadlock"
        name = rnd.choice(runnable)
        proc = procs[name]
        try:
            kind, arg = next(proc[0])
        except StopIteration:
            proc[2] = True
            continue
        if kind in ("arrive", "sync"):
            b = bars[arg]
            b.count += proc[1]
            if b.count > 256:
                return "over-subscribed"
            if b.count == 256:
                b.count, b.phase = 0, b.phase + 1
            elif kind == "sync":
                waiting[name] = (arg, b.phase)
        elif kind == "read" and arg in writing:
            return "race"
        elif kind == "write":
            writing.add(arg)
        elif kind == "end":
            writing.clear()
    return "no progress"

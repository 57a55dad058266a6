"""A model check, on the CPU, of the exchange protocol between the two CTAs of a column-split pair
(umma::cluster_exchange and its callers in the mixed and FP64 kernels).

Each CTA runs the same sequence of exchanges (both take the same RHST decisions): per step one
Varah exchange whose payload goes to a small buffer chosen by step parity; per RHST, and once at
the end, the mixed kernel makes four exchanges through one large buffer (Q's half, "read", P's
half, "read") and the FP64 kernel two (its columns into the other CTA's planes, "read"; at the
end only the first). An
exchange is: write the payload into the other CTA's buffer, one arrival on the other CTA's
mbarrier bars[k % 2] (count 1), a wait on this CTA's bars[k % 2] for the phase of parity
(k // 2) % 2, then read the received payload. The simulation interleaves the two CTAs' actions
at random and checks that (1) every wait is released by the arrival of the same exchange (the
other CTA never completes a phase twice before it is waited for, which would alias the parity),
(2) no payload overwrites one its receiver has not read yet, (3) neither CTA deadlocks.
"""
import random

import pytest


def _program(n_steps, rhst_steps, kernel="mixed"):
    """Exchange list of one CTA: (buffer written in the other CTA, or None for a bare signal)."""
    rhst = ([("big", 0), (None, None), ("big", 0), (None, None)] if kernel == "mixed"
            else [("big", 0), (None, None)])
    final = rhst if kernel == "mixed" else [("big", 0)]
    prog = []
    for i in range(n_steps):
        prog.append(("small", i & 1))
        if i in rhst_steps:
            prog += rhst
    return prog + final


class _Barrier:
    def __init__(self):
        self.completed = 0          # completed phases (count 1: one arrival completes a phase)

    def arrive(self):
        self.completed += 1

    def passed(self, parity):       # try_wait.parity: the phase of this parity has completed
        return self.completed % 2 != parity


def _simulate(prog, rng):
    n = len(prog)
    bars = [[_Barrier(), _Barrier()] for _ in range(2)]
    # buffers[cta][(kind, idx)] = (writer's exchange index, read by the owner?)
    buffers = [dict(), dict()]
    pc = [0, 0]                     # next exchange per CTA
    stage = [0, 0]                  # 0 write + arrive, 1 wait, 2 read
    while pc[0] < n or pc[1] < n:
        ready = [c for c in (0, 1) if pc[c] < n and
                 (stage[c] != 1 or bars[c][pc[c] % 2].passed((pc[c] // 2) % 2))]
        assert ready, f"deadlock at {pc}, stages {stage}"
        c = rng.choice(ready)
        k, peer = pc[c], 1 - c
        kind, idx = prog[k]
        if stage[c] == 0:
            if kind is not None:
                prev = buffers[peer].get((kind, idx))
                assert prev is None or prev[1], \
                    f"CTA {c} overwrites {kind}[{idx}] (exchange {prev[0]}) before it was read"
                buffers[peer][(kind, idx)] = (k, False)
            bars[peer][k % 2].arrive()
            stage[c] = 1
        elif stage[c] == 1:
            # released by the other CTA's arrival for this very exchange, not a later one
            assert bars[c][k % 2].completed == k // 2 + 1, (c, k, bars[c][k % 2].completed)
            stage[c] = 2
        else:
            if kind is not None:
                w, _ = buffers[c][(kind, idx)]
                assert w == k, f"CTA {c} reads the payload of exchange {w} at exchange {k}"
                buffers[c][(kind, idx)] = (w, True)
            pc[c] += 1
            stage[c] = 0


@pytest.mark.parametrize("kernel", ["mixed", "fp64"])
@pytest.mark.parametrize("seed", range(40))
def test_exchange_protocol_random_interleavings(seed, kernel):
    rng = random.Random(seed)
    n_steps = rng.randint(1, 12)
    rhst = {i for i in range(n_steps) if rng.random() < 0.4}
    _simulate(_program(n_steps, rhst, kernel), rng)


def test_a_single_barrier_would_alias():
    """The check has teeth: with one mbarrier for every exchange the other CTA can complete two
    phases before a wait and the parity test releases the wrong exchange (or none)."""
    prog = _program(3, {1})
    failures = 0
    for seed in range(200):
        rng = random.Random(seed)
        n = len(prog)
        bar = [_Barrier(), _Barrier()]
        pc, stage = [0, 0], [0, 0]
        try:
            while pc[0] < n or pc[1] < n:
                ready = [c for c in (0, 1) if pc[c] < n and
                         (stage[c] != 1 or bar[c].passed(pc[c] % 2))]
                assert ready
                c = rng.choice(ready)
                if stage[c] == 0:
                    bar[1 - c].arrive()
                    stage[c] = 1
                elif stage[c] == 1:
                    assert bar[c].completed == pc[c] + 1
                    stage[c] = 2
                else:
                    pc[c] += 1
                    stage[c] = 0
        except AssertionError:
            failures += 1
    assert failures > 0

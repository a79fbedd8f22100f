"""Model check of the tensor-core M2L kernel's mbarrier protocol (CPU).

The slab kernel (csrc/fmm_m2l_tc.cu) runs one producer thread and NISS
MMA-issuing threads.  Slabs go through 2 buffers (full/empty barriers, the
empty one counting NISS arrivals); offset matrices go through NBST stages
(full/empty barriers, one arrival each), offset t in stage t % NBST and
issuer t % NISS.  Every wait is a parity wait on the phase a thread needs,
which returns true as soon as the barrier's current phase has the other
parity: it cannot tell phase k from phase k - 2.  The host therefore picks
NISS = NBST in {2, 4}, so that a stage always has one waiting issuer, which
waits on its phases in order.

This test simulates random interleavings of the producer, the issuers and
the asynchronous completions (copies landing, MMAs finishing) and checks
that no parity wait ever returns before its phase has completed, and that
every run finishes.  It also checks that the rejected configuration (four
issuers on two stages) does break, so the model is sharp enough to matter.
"""
import random

import pytest


class _Barrier:
    def __init__(self, count):
        self.count, self.pending, self.phase = count, count, 0   # phase: index of the incomplete phase

    def arrive(self):
        self.pending -= 1
        if self.pending == 0:
            self.phase += 1
            self.pending = self.count

    def parity_wait(self, k):
        """Wait for the completion of phase k with a parity wait; raise if it
        would return before phase k completed."""
        ok = (self.phase & 1) != (k & 1)
        if ok and self.phase <= k:
            raise AssertionError("parity wait for phase %d returned in phase %d" % (k, self.phase))
        return ok


def _simulate(niss, nbst, seed, nslab=24):
    rnd = random.Random(seed)
    per_slab = [rnd.randint(5, 9) for _ in range(nslab)]   # offsets per slab (5..9, as in the kernel)
    sfull, sempty = [_Barrier(1), _Barrier(1)], [_Barrier(niss), _Barrier(niss)]
    bfull = [_Barrier(1) for _ in range(nbst)]
    bempty = [_Barrier(1) for _ in range(nbst)]
    # producer program: a slab, then the matrices of its offsets
    prod, t = [], 0
    for sl, n in enumerate(per_slab):
        prod.append(("slab", sl))
        for _ in range(n):
            prod.append(("mat", t))
            t += 1
    # issuer programs: wait for the slab, for each own offset wait for its
    # stage and commit its MMAs, then commit the slab
    iss = []
    for w in range(niss):
        prog, t = [], 0
        for sl, n in enumerate(per_slab):
            prog.append(("wslab", sl))
            for _ in range(n):
                if t % niss == w:
                    prog.append(("wmat", t))
                t += 1
            prog.append(("cslab", sl))
        iss.append(prog)
    pc = [0] * (niss + 1)
    pending = []   # asynchronous completions: barriers to arrive on
    for _ in range(10 ** 6):
        actors = [a for a in range(niss + 1) if pc[a] < len(prod if a == 0 else iss[a - 1])]
        if not actors and not pending:
            return
        choice = rnd.randrange(len(actors) + (1 if pending else 0))
        if choice == len(actors):
            pending.pop(rnd.randrange(len(pending))).arrive()
            continue
        a = actors[choice]
        if a == 0:
            kind, i = prod[pc[0]]
            if kind == "slab":
                if i < 2 or sempty[i & 1].parity_wait((i >> 1) - 1):
                    pending.append(sfull[i & 1]); pc[0] += 1
            else:
                if i < nbst or bempty[i % nbst].parity_wait(i // nbst - 1):
                    pending.append(bfull[i % nbst]); pc[0] += 1
        else:
            kind, i = iss[a - 1][pc[a]]
            if kind == "wslab":
                if sfull[i & 1].parity_wait(i >> 1):
                    pc[a] += 1
            elif kind == "wmat":
                if bfull[i % nbst].parity_wait(i // nbst):
                    pending.append(bempty[i % nbst]); pc[a] += 1   # commit: arrives when the MMAs finish
            else:
                pending.append(sempty[i & 1]); pc[a] += 1
    raise AssertionError("no progress: deadlock")


@pytest.mark.parametrize("niss,nbst", [(2, 2), (2, 4), (4, 4)])
def test_issuer_stage_configurations_are_safe(niss, nbst):
    for seed in range(200):
        _simulate(niss, nbst, seed)


def test_four_issuers_on_two_stages_break_the_parity_waits():
    broken = 0
    for seed in range(50):
        try:
            _simulate(4, 2, seed)
        except AssertionError:
            broken += 1
    assert broken > 0


# ---------------------------------------------------------------------------
# The kernel that builds the offset matrices on chip (csrc/fmm_m2l_tcgen.cu):
# a producer (slabs into 2 buffers, D vectors into ND stages), NISS issuers
# and G generator warps.  Generator warps wait for an offset's D vector
# (dfull, one arrival), release it (dempty, G arrivals), wait for their
# matrix stage to be free (bempty, one arrival: the issuer's commit) and
# mark it written (bfull, G arrivals); issuer t % NISS waits for bfull and
# commits to bempty; slabs as above.
# ---------------------------------------------------------------------------
def _simulate_gen(niss, nb, nd, ngen, seed, nslab=24):
    rnd = random.Random(seed)
    per_slab = [rnd.randint(5, 9) for _ in range(nslab)]
    tot = sum(per_slab)
    sfull, sempty = [_Barrier(1), _Barrier(1)], [_Barrier(niss), _Barrier(niss)]
    dfull = [_Barrier(1) for _ in range(nd)]
    dempty = [_Barrier(ngen) for _ in range(nd)]
    bfull = [_Barrier(ngen) for _ in range(nb)]
    bempty = [_Barrier(1) for _ in range(nb)]
    done = _Barrier(niss)
    prod, t = [], 0
    for sl, n in enumerate(per_slab):
        prod.append(("slab", sl))
        for _ in range(n):
            prod.append(("dvec", t))
            t += 1
    iss = []
    for w in range(niss):
        prog, t = [], 0
        for sl, n in enumerate(per_slab):
            prog.append(("wslab", sl))
            for _ in range(n):
                if t % niss == w:
                    prog.append(("wmat", t))
                t += 1
            prog.append(("cslab", sl))
        prog.append(("done", 0))
        iss.append(prog)
    gen = [[(step, k) for k in range(tot) for step in ("wd", "wb")] for _ in range(ngen)]
    progs = [prod] + iss + gen
    pc = [0] * len(progs)
    pending = []
    for _ in range(10 ** 7):
        actors = [a for a in range(len(progs)) if pc[a] < len(progs[a])]
        if not actors and not pending:
            assert done.phase == 1
            return
        choice = rnd.randrange(len(actors) + (1 if pending else 0))
        if choice == len(actors):
            pending.pop(rnd.randrange(len(pending))).arrive()
            continue
        a = actors[choice]
        kind, i = progs[a][pc[a]]
        if a == 0:
            if kind == "slab":
                if sempty[i & 1].parity_wait((i >> 1) - 1):
                    pending.append(sfull[i & 1]); pc[a] += 1
            elif dempty[i % nd].parity_wait(i // nd - 1):
                pending.append(dfull[i % nd]); pc[a] += 1
        elif a <= niss:
            if kind == "wslab":
                if sfull[i & 1].parity_wait(i >> 1):
                    pc[a] += 1
            elif kind == "wmat":
                if bfull[i % nb].parity_wait(i // nb):
                    pending.append(bempty[i % nb]); pc[a] += 1
            elif kind == "cslab":
                pending.append(sempty[i & 1]); pc[a] += 1
            else:
                pending.append(done); pc[a] += 1
        else:
            if kind == "wd":
                if dfull[i % nd].parity_wait(i // nd):
                    dempty[i % nd].arrive(); pc[a] += 1
            elif bempty[i % nb].parity_wait(i // nb - 1):
                bfull[i % nb].arrive(); pc[a] += 1
    raise AssertionError("no progress: deadlock")


@pytest.mark.parametrize("niss,nb", [(1, 2), (1, 3), (1, 4), (2, 2), (2, 4)])
def test_onchip_matrix_protocol_is_safe(niss, nb):
    for seed in range(60):
        _simulate_gen(niss, nb, 8, 4, seed, nslab=10)

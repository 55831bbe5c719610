"""The ordering contract of intent marking (Sec. 3.1.2), checked on the host.

The host-only simulator drives the same dependency tracker as the CUDA
contexts and logs each wait it inserts ("w<-c@s": context w waits for launch s
of context c) or elides ("w..c@s").  The rule under test: for accesses A then
B to one object on different contexts, B waits for A unless both are reads;
accesses on one context keep program order without waits.
"""

import pytest

from paper_2306_17801_gb300 import apcg

R, W, RW = apcg.READ, apcg.WRITE, apcg.READ_WRITE


@pytest.fixture(scope="module", autouse=True)
def lib():
    import __graft_entry__

    __graft_entry__.build()
    return apcg.load()


def waits(log):
    return [l for l in log if "<-" in l]


@pytest.mark.parametrize("m1,m2,ordered", [(W, W, True), (W, R, True), (R, W, True), (R, R, False), (RW, R, True), (R, RW, True)])
def test_pairwise_rule(m1, m2, ordered):
    s = apcg.Sim(2)
    s.op(0, [(7, m1)])
    s.op(1, [(7, m2)])
    assert waits(s.log()) == (["1<-0@1"] if ordered else [])


def test_same_context_needs_no_wait():
    s = apcg.Sim(1)
    for m in (W, R, W, RW, R):
        s.op(0, [(3, m)])
    assert s.log() == []


def test_write_waits_for_every_reader_since_last_write():
    s = apcg.Sim(4)
    s.op(0, [(1, W)])  # 0@1
    s.op(1, [(1, R)])  # waits 0@1
    s.op(2, [(1, R)])  # waits 0@1
    s.op(3, [(1, W)])  # waits readers 1@1, 2@1 and the writer 0@1
    w = waits(s.log())
    assert w[:2] == ["1<-0@1", "2<-0@1"]
    assert sorted(w[2:]) == sorted(["3<-0@1", "3<-1@1", "3<-2@1"])


def test_waits_are_elided_when_known_or_complete():
    s = apcg.Sim(3)
    s.op(0, [(1, W), (2, W)])  # one launch writes two objects: 0@1
    s.op(1, [(1, R)])  # 1<-0@1
    s.op(1, [(2, R)])  # already ordered after 0@1: elided
    s.op(0, [(3, W)])  # 0@2
    s.complete(0, 2)
    s.op(2, [(3, R)])  # finished: elided
    log = s.log()
    assert log == ["1<-0@1", "1..0@1", "2..0@2"]


def test_later_write_supersedes_earlier():
    s = apcg.Sim(3)
    s.op(0, [(5, W)])  # 0@1
    s.op(1, [(5, W)])  # 1<-0@1 ; now the writer is 1@1 and readers are cleared
    s.op(2, [(5, R)])  # waits only for 1@1
    assert waits(s.log()) == ["1<-0@1", "2<-1@1"]


def test_mixed_api_cg_listing_dependencies():
    """Accesses of one iteration of the mixed sync/async CG main loop (Sec. 3.3).

    Contexts: a=0, b=1, c=2 and 3 for the synchronous calls (global
    blocking, so each is complete before the next call starts).
    """
    P, Z, Wv, X, Rv, A, a, b, beta, betaold, dp = range(1, 12)
    s = apcg.Sim(4)
    s.op(0, [(beta, R), (betaold, R), (b, W)])  # b = beta / betaold      (a@1)
    s.op(3, [(Z, R), (P, RW)])  # VecAYPX(P, b.front(), Z) [sync]       (3@1)
    s.complete(3, 1)
    s.op(3, [(A, R), (P, R), (Wv, W)])  # MatMult(A, P, W)  [sync]      (3@2)
    s.complete(3, 2)
    n0 = len(s.log())
    s.op(1, [(P, R), (Wv, R), (a, W)])  # VecDotAsync(P, W, &a, b)      (b@1)
    assert waits(s.log()[n0:]) == []  # producers already finished
    n0 = len(s.log())
    s.op(2, [(beta, R), (a, RW)])  # a = beta / a on c: waits for the dot
    assert waits(s.log()[n0:]) == ["2<-1@1"]
    n0 = len(s.log())
    s.op(0, [(beta, R), (betaold, RW)])  # betaold = beta on a: concurrent with the above
    assert waits(s.log()[n0:]) == []
    n0 = len(s.log())
    s.op(1, [(a, R), (P, R), (X, RW)])  # VecAXPYAsync(X, a, P, b): waits for a on c
    assert waits(s.log()[n0:]) == ["1<-2@1"]
    n0 = len(s.log())
    s.op(2, [(a, R), (Wv, R), (Rv, RW)])  # VecAXPYAsync(R, -a, W, c): same context as a
    assert waits(s.log()[n0:]) == []
    n0 = len(s.log())
    s.op(3, [(Rv, R), (Z, W)])  # ApplyPreconditioner(R, Z) [sync]: only the second AXPY
    assert waits(s.log()[n0:]) == ["3<-2@2"]
    s.complete(3, 3)
    s.complete(2, 2)
    n0 = len(s.log())
    s.op(0, [(Z, R), (dp, W)])  # VecNormAsync(Z, &dp, a)
    assert waits(s.log()[n0:]) == []
    n0 = len(s.log())
    s.op(1, [(Z, R), (Rv, R), (beta, W)])  # VecDotAsync(Z, R, &beta, b): after the readers of beta
    assert waits(s.log()[n0:]) == ["1<-0@2"]

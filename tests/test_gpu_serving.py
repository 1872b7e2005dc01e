"""The serving loop: sessions admitted within a device-memory budget, evicted
to the host and re-admitted, requests batched over two CUDA streams as they
arrive.  Every session must end exactly where its requests applied one by one
(bdu_update, no batching, no eviction) leave it -- bit for bit in both forms
-- and in FP64 that is the oracle's result."""
import collections

import numpy as np
import pytest

import oracle as O
from paper_2509_02840_gb300 import bdu, inputs as I, serve as S

pytestmark = pytest.mark.gpu


def _replay(specs, reqs, precision, check_every):
    by_sid = collections.defaultdict(list)
    for q in sorted(reqs, key=lambda q: q.t_arrival):
        by_sid[q.sid].append(q)
    out = {}
    for sid, (m, n) in enumerate(specs):
        Q, d, e, P = I.factorization(m, n, config=4, which=sid)
        with bdu.Factorization(Q, d, e, P, precision=precision, check_every=check_every, reorth_every=1) as F:
            for q in by_sid[sid]:
                F.update(q.B, q.C)
            out[sid] = F.read()
    return out, by_sid


@pytest.mark.parametrize("precision", [bdu.FP64, bdu.MIXED])
def test_serving_equals_sequential_replay(precision):
    specs = I.serving_mix(12, lo=16, hi=200)
    check_every = 0 if precision == bdu.MIXED else None
    per = [S.reserve_bytes(m, n, precision) for m, n in specs]
    budget = max(per) + sorted(per)[len(per) // 2]  # room for about two sessions: forces evictions
    # one re-orthogonalization step after every column: a cadence that does not
    # depend on how long a session has been resident
    srv = S.Server(specs, precision, budget, max_batch=5, check_every=check_every, reorth_every=1)
    counter = collections.Counter()
    burst = S.poisson_arrivals(specs, 0.0, 24, seed=3, first_update=counter)
    res1 = srv.run(burst)
    trickle = S.poisson_arrivals(specs, 400.0, 40, seed=4, first_update=counter)
    res2 = srv.run(trickle)
    assert res1["requests"] == 24 and res2["requests"] == 40
    assert res1["evictions"] + res2["evictions"] > 0
    assert srv.peak_resident <= budget
    assert res2["latency_ms"]["p99"] >= res2["latency_ms"]["p50"] > 0
    final = {s.sid: s.read() for s in srv.sessions}
    srv.close()
    want, by_sid = _replay(specs, burst + trickle, precision, check_every)
    for sid, (m, n) in enumerate(specs):
        if not by_sid[sid]:
            continue  # never admitted: still the unrounded initial state
        for a, b in zip(final[sid], want[sid]):
            assert np.array_equal(a, b), (sid, m, n, len(by_sid[sid]))
    if precision == bdu.FP64:
        # two sessions checked against the oracle through all their updates
        for sid in sorted(by_sid, key=lambda k: -len(by_sid[k]))[:2]:
            m, n = specs[sid]
            Q, d, e, P = I.factorization(m, n, config=4, which=sid)
            for q in by_sid[sid]:
                Q, d, e, P, _ = O.update(Q, d, e, P, q.B, q.C)
            Qg, dg, eg, Pg = final[sid]
            assert np.array_equal(dg, d) and np.array_equal(eg, e)
            assert np.array_equal(Qg, Q) and np.array_equal(Pg, P)


def test_budget_below_one_session_is_rejected():
    specs = [(64, 32), (40, 40)]
    with pytest.raises(ValueError):
        S.Server(specs, bdu.FP64, budget_bytes=1000)


def test_automatic_check_acts_after_a_batch():
    """In the mixed form the check that falls due in a batch is enqueued
    without waiting and acted on by the next synchronizing call: a factor
    pushed off orthogonality is repaired by the time it is read."""
    import torch
    m = n = 192
    Q, d, e, P = I.factorization(m, n, config=0, which=21)
    g = np.random.default_rng(5)
    Qp = Q + 2e-5 * g.standard_normal((m, m)) / np.sqrt(m)
    before = np.linalg.norm(Qp.T @ Qp - np.eye(m), 2)
    B, C = I.dense_update(m, n, 0, config=0)
    tb = torch.from_numpy(B.reshape(-1, order="F").copy()).cuda()
    tc = torch.from_numpy(C.reshape(-1, order="F").copy()).cuda()
    torch.cuda.synchronize()
    with bdu.Factorization(Qp, d, e, P, precision=bdu.MIXED, reorth_tol=1e-7, check_every=1, reorth_every=0) as F:
        bdu.update_batch([F], [tb.data_ptr()], [tc.data_ptr()], [1])
        Qg, _, _, _ = F.read()
        st = F.stats()
    assert st["reorth_q"] == 1
    after = np.linalg.norm(Qg.T @ Qg - np.eye(m), 2)
    assert after < 0.2 * before and after < 5e-6


@pytest.mark.parametrize("precision", [bdu.FP64, bdu.MIXED])
def test_serving_large_sessions_equal_sequential_replay(precision):
    """The serving mix's full size range (m, n up to 2048): sessions of order
    >= 512 get a thread-block cluster each inside a batch, the smaller ones one
    block each on the second stream; every served session still ends bit for
    bit where its requests applied one by one leave it."""
    specs = [(2048, 2048), (1900, 1100), (1800, 600), (900, 700), (520, 512), (300, 200), (128, 64), (96, 90)]
    check_every = 0 if precision == bdu.MIXED else None
    per = [S.reserve_bytes(m, n, precision) for m, n in specs]
    budget = max(per) + sorted(per)[len(per) // 2]  # forces evictions
    srv = S.Server(specs, precision, budget, max_batch=4, check_every=check_every, reorth_every=1)
    counter = collections.Counter()
    burst = S.poisson_arrivals(specs, 0.0, 14, seed=13, first_update=counter)
    res1 = srv.run(burst)
    trickle = S.poisson_arrivals(specs, 50.0, 10, seed=14, first_update=counter)
    res2 = srv.run(trickle)
    assert res1["requests"] == 14 and res2["requests"] == 10
    assert res1["evictions"] + res2["evictions"] > 0
    assert srv.peak_resident <= budget
    final = {s.sid: s.read() for s in srv.sessions}
    srv.close()
    want, by_sid = _replay(specs, burst + trickle, precision, check_every)
    assert any(specs[sid][1] >= 512 for sid in by_sid)  # a cluster-engine session was served
    for sid, (m, n) in enumerate(specs):
        if not by_sid[sid]:
            continue
        for a, b in zip(final[sid], want[sid]):
            assert np.array_equal(a, b), (sid, m, n, len(by_sid[sid]))

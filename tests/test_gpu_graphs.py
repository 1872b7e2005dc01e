"""CUDA-graph replay of plain updates: the launch sequence of an update is
captured the first time a rank and pair of input buffers are seen and replayed
afterwards.  Replays must give exactly the results of separate launches (same
kernels, same order), in both forms, while ranks change, inputs come from host
or device buffers, and timing is switched on and off."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2509_02840_gb300 import bdu, inputs as I

pytestmark = pytest.mark.gpu

RANKS = [1, 1, 1, 2, 2, 1, 3, 1, 1]


def _run(precision, graphs, m, n, dev_inputs=False, timing_at=None):
    Q, d, e, P = I.factorization(m, n, config=0, which=41)
    # a fixed apply variant: the autotuner would drop the first update's graph
    nb = 8 if precision == bdu.FP64 else 1
    # (no re-orthogonalization cadence: its counters take part in the replay key)
    with bdu.Factorization(Q, d, e, P, precision=precision, graphs=graphs, nb=nb, reorth_every=0,
                           check_every=0 if precision == bdu.MIXED else None) as F:
        keep = []
        for h, r in enumerate(RANKS):
            if timing_at is not None:
                F.set_timing(h == timing_at)
            B, C = I.dense_update(m, n, h, config=0, r=r)
            if dev_inputs:
                tb = torch.from_numpy(B.reshape(-1, order="F").copy()).cuda()
                tc = torch.from_numpy(C.reshape(-1, order="F").copy()).cuda()
                keep.append((tb, tc))
                torch.cuda.synchronize()
                F.update_dev(tb.data_ptr(), tc.data_ptr(), r)
            else:
                F.update(B, C)
        out = F.read()
        st = F.stats()
    return out, st


@pytest.mark.parametrize("precision", [bdu.FP64, bdu.MIXED])
@pytest.mark.parametrize("m,n", [(96, 64), (300, 300), (700, 600)])
def test_replay_equals_separate_launches(precision, m, n):
    (a, sa), (b, sb) = _run(precision, True, m, n), _run(precision, False, m, n)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    # captures at ranks 1, 2, 1, 3, 1: the other four updates are replays
    assert sa["graph_replays"] == 4 and sb["graph_replays"] == 0
    assert sa["launches"] == sb["launches"] and sa["updates"] == sb["updates"] == sum(RANKS)
    assert sa["rot_left"] == sb["rot_left"] and sa["chase_steps"] == sb["chase_steps"]


def test_device_inputs_and_timing():
    m, n = 200, 150
    ref, _ = _run(bdu.FP64, False, m, n)
    # new device buffers on every call: every update is captured, none replayed
    got, st = _run(bdu.FP64, True, m, n, dev_inputs=True)
    assert st["graph_replays"] == 0
    for x, y in zip(got, ref):
        assert np.array_equal(x, y)
    # timing switched on for one update: that one launches separately
    got, st = _run(bdu.FP64, True, m, n, timing_at=2)
    for x, y in zip(got, ref):
        assert np.array_equal(x, y)
    assert st["graph_replays"] == 3 and st["timed_updates"] == 1


@pytest.mark.parametrize("precision", [bdu.FP64, bdu.MIXED])
def test_rank_r_pipeline_equals_column_by_column(precision):
    """A rank-r call runs column k's chase beside column k-1's application
    (with and without graph replay); the batched path applies the columns one
    after another.  All three must agree bit for bit, and the FP64 form with
    the oracle."""
    m, n = 300, 260
    Q, d, e, P = I.factorization(m, n, config=0, which=77)
    ranks = [3, 2, 2, 4, 4, 1, 2]
    ups = [I.dense_update(m, n, h, config=0, r=r) for h, r in enumerate(ranks)]
    kw = dict(precision=precision, nb=8 if precision == bdu.FP64 else 1, reorth_every=0,
              check_every=0 if precision == bdu.MIXED else None)
    outs = []
    for graphs in (True, False):
        with bdu.Factorization(Q, d, e, P, graphs=graphs, **kw) as F:
            for B, C in ups:
                F.update(B, C)
            st = F.stats()
            outs.append(F.read())
        if graphs:
            assert st["graph_replays"] == 2  # the second rank-2 and the second rank-4 call
    with bdu.Factorization(Q, d, e, P, **kw) as F:
        for B, C in ups:
            tb = torch.from_numpy(B.reshape(-1, order="F").copy()).cuda()
            tc = torch.from_numpy(C.reshape(-1, order="F").copy()).cuda()
            torch.cuda.synchronize()
            bdu.update_batch([F], [tb.data_ptr()], [tc.data_ptr()], [B.shape[1]])
        outs.append(F.read())
    for other in outs[1:]:
        for a, b in zip(outs[0], other):
            assert np.array_equal(a, b)
    if precision == bdu.FP64:
        for B, C in ups:
            Q, d, e, P, _ = O.update(Q, d, e, P, B, C)
        for a, b in zip(outs[0], (Q, d, e, P)):
            assert np.array_equal(a, b)



@pytest.mark.parametrize("every", [-1, 1, 3])
def test_replay_with_reorthogonalization_cadence(every):
    """The mixed form's re-orthogonalization cadence is host state that a
    replay must follow: graphs are replayed only when the cadence is where it
    was at capture, and the results equal separate launches bit for bit."""
    m, n = 300, 256
    Q, d, e, P = I.factorization(m, n, config=0, which=43)
    outs, stats = [], []
    for graphs in (True, False):
        with bdu.Factorization(Q, d, e, P, precision=bdu.MIXED, graphs=graphs, nb=1, reorth_every=every,
                               check_every=0) as F:
            for h, r in enumerate([1, 1, 1, 2, 2, 2, 1, 3, 1, 1]):
                F.update(*I.dense_update(m, n, h, config=0, r=r))
            outs.append(F.read())
            stats.append(F.stats())
    for a, b in zip(*outs):
        assert np.array_equal(a, b)
    assert stats[0]["reorth_q"] == stats[1]["reorth_q"] and stats[0]["reorth_p"] == stats[1]["reorth_p"]
    if every == 1:
        assert stats[0]["graph_replays"] >= 3

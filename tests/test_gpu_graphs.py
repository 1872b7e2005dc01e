"""CUDA-graph replay of plain updates: the launch sequence of an update is
captured the first time a rank and pair of input buffers are seen and replayed
afterwards.  Replays must give exactly the results of separate launches (same
kernels, same order), in both forms, while ranks change, inputs come from host
or device buffers, and timing is switched on and off."""
import numpy as np
import pytest
import torch

from paper_2509_02840_gb300 import bdu, inputs as I

pytestmark = pytest.mark.gpu

RANKS = [1, 1, 1, 2, 2, 1, 3, 1, 1]


def _run(precision, graphs, m, n, dev_inputs=False, timing_at=None):
    Q, d, e, P = I.factorization(m, n, config=0, which=41)
    # a fixed apply variant: the autotuner would drop the first update's graph
    nb = 8 if precision == bdu.FP64 else 1
    with bdu.Factorization(Q, d, e, P, precision=precision, graphs=graphs, nb=nb,
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

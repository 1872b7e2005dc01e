"""The serving loop's host-side policy, without a GPU: admission within the
device-memory budget, least-recently-used eviction of idle sessions only
(never a busy one, never one already picked for the batch being formed),
refusal when nothing can make room, the byte accounting, the reservation of
an m < n session (held as its transpose), and reproducible arrivals."""
import pytest

from paper_2509_02840_gb300 import bdu, serve


class FakeSession:
    def __init__(self, sid, nbytes):
        self.sid, self.bytes = sid, nbytes
        self.handle = None
        self.busy = False
        self.last_used = 0.0
        self.evictions = 0
        self.admits = 0

    def admit(self):
        self.handle = object()
        self.admits += 1

    def evict(self):
        self.handle = None
        self.evictions += 1


def _server(sessions, budget):
    srv = serve.Server.__new__(serve.Server)  # no CUDA streams: policy only
    srv.sessions = sessions
    srv.budget = budget
    srv.resident_bytes = 0
    srv.peak_resident = 0
    srv.max_batch = 64
    return srv


def test_admission_within_budget_and_lru_eviction():
    ss = [FakeSession(i, 40) for i in range(4)]
    srv = _server(ss, 100)
    assert srv._admit(ss[0], 1.0, {0}) and srv._admit(ss[1], 2.0, {1})
    assert srv.resident_bytes == 80 and srv.peak_resident == 80
    # full: the least recently used idle session (0) makes room
    assert srv._admit(ss[2], 3.0, {2})
    assert ss[0].handle is None and ss[0].evictions == 1 and ss[1].handle is not None
    assert srv.resident_bytes == 80 and srv.peak_resident == 80
    # an already resident session is admitted without any eviction
    assert srv._admit(ss[1], 4.0, {1}) and ss[1].admits == 1


def test_busy_and_protected_sessions_are_never_evicted():
    ss = [FakeSession(i, 40) for i in range(4)]
    srv = _server(ss, 100)
    srv._admit(ss[0], 1.0, {0})
    srv._admit(ss[1], 2.0, {1})
    ss[0].busy = True                      # in a batch in flight
    # session 1 is protected (already picked for the batch being formed):
    # nothing can be evicted, so session 2 waits
    assert not srv._admit(ss[2], 3.0, {1, 2})
    assert ss[2].handle is None and ss[0].handle is not None and ss[1].handle is not None
    assert srv.resident_bytes == 80
    # once session 0 is idle again it is the one evicted
    ss[0].busy = False
    assert srv._admit(ss[2], 4.0, {1, 2})
    assert ss[0].handle is None and ss[1].handle is not None


def test_reservation_of_a_wide_session_is_that_of_its_transpose():
    for prec in (bdu.FP64, bdu.MIXED):
        assert serve.reserve_bytes(300, 700, prec) == serve.reserve_bytes(700, 300, prec)
        assert serve.reserve_bytes(700, 300, prec) > serve.reserve_bytes(300, 300, prec)


def test_arrivals_are_reproducible_and_ordered():
    specs = [(96, 64), (128, 128), (300, 200)]
    a = serve.poisson_arrivals(specs, rate=50.0, count=40, seed=3)
    b = serve.poisson_arrivals(specs, rate=50.0, count=40, seed=3)
    assert [(q.sid, q.t_arrival, q.r) for q in a] == [(q.sid, q.t_arrival, q.r) for q in b]
    assert all(x.t_arrival <= y.t_arrival for x, y in zip(a, a[1:]))
    assert all(1 <= q.r <= 4 and q.B.shape == (specs[q.sid][0], q.r) for q in a)
    # a session's updates are numbered in arrival order: no two requests of a
    # session carry the same update
    seen = {}
    for q in a:
        key = (q.sid, q.B.tobytes())
        assert key not in seen
        seen[key] = True


def test_budget_smaller_than_one_session_is_refused():
    ss = [FakeSession(0, 150)]
    srv = _server(ss, 100)
    assert not srv._admit(ss[0], 1.0, {0}) and ss[0].handle is None

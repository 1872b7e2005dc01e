"""Serving loop: many resident factorizations updated by a stream of requests.

Each session holds one factorization A = Q Bd P^T; a request is one rank-r
update A <- A + B C^T of one session (Sec. 3.4 applied r times).  The loop

  * keeps sessions resident on the GPU within a device-memory budget: a
    session is admitted on demand, and when the budget is full the idle
    resident sessions are evicted least recently used first.  Eviction reads
    the state back to the host (bdu_read) and re-admission re-creates it from
    there (bdu_create), an exact round trip in both forms;
  * batches the oldest pending request of up to max_batch free sessions of any
    (m, n, r) into one bdu_update_batch call, and keeps up to two batches in
    flight on two CUDA streams (continuous batching: a request arriving while
    batches run joins the next one as soon as its session is free);
  * applies each session's requests in arrival order, so that every session
    ends where the same updates applied one by one leave it (in the mixed form
    exactly so when re-orthogonalization runs after every column,
    reorth_every=1: the default cadence counts columns per resident handle,
    and a re-admitted session starts counting afresh).

It reports rank-1 updates per second and the p50/p99 request latency (arrival
to the completion of its batch, seen by polling an event): first saturated
(every request present at the start), then under Poisson arrivals at a
fraction of that rate.

    python -m paper_2509_02840_gb300.serve [--sessions 256] [--seconds 20] [--fp64]
"""
import argparse
import collections
import json
import time

import numpy as np

from . import bdu, inputs


class Request:
    __slots__ = ("sid", "t_arrival", "B", "C", "r", "t_done")

    def __init__(self, sid, t_arrival, B, C):
        self.sid, self.t_arrival, self.B, self.C = sid, t_arrival, B, C
        self.r = B.shape[1]
        self.t_done = None


def reserve_bytes(m, n, precision, max_rank=4):
    """Device bytes to reserve for one session: the allocations of bdu_create,
    the workspace of a rank-max_rank update and, in the mixed form, the
    re-orthogonalization workspace that the first re-orthogonalization adds."""
    es = 8 if precision == bdu.FP64 else 4
    if m < n:
        m, n = n, m  # held as the transposed problem
    N = n + 1 if m > n else n
    T = (N - 1) + max(n - 2, 0) + 2 * (n if N == n + 1 else n - 1)
    tc = T * (n // 2 + 4)
    b = es * (m * m + n * n)                              # Q, P
    b += 8 * (6 * (N + 2) + 2 * (n + 2) + (m + 2))       # band, row 1, u, v
    if precision == bdu.MIXED:
        b += tc * (2 * 8 + 2 * 4)                         # FP32 (c, s) and int32 pair records
    else:
        b += tc * (4 * 8 + 2 * 4)                         # FP64 (c, s) and int32 pair records
    b += 8 * (T + 1) + 20 * (m + 1) + 8 * (3 * m + 8) + 256
    b += max_rank * (16 * (m + n) + 4 * (m + n)) + 8      # B, C, U, V and their nonzero lists
    if precision == bdu.MIXED:
        b += 8 * m * m + 8 * (m + 1) + 32 * (T + 1)       # FP64 scratch, spike copies, chase descriptors
        b += 16 * m * m                                   # re-orthogonalization workspace
        if m >= BLOCKED_FROM:
            # the blocked apply's workspace: a chunk of 16 bands of blocks (the
            # largest over the block orders), band ranges, progress words
            blobs = max(((m + nb) // (nb // 2) + 2) * part for nb, part in ((64, 23552), (96, 48128), (128, 81920)))
            b += 16 * blobs + 8 * (T // 32 + 2) + 16 * ((m + 128) // 128) * 8 * 4 + 1024
    return b


# factor orders from which the library's mixed form keeps the blocked
# tensor-core apply's workspace (and applies with it)
BLOCKED_FROM = 1024


class Session:
    def __init__(self, sid, m, n, precision, check_every=None, config=4, reorth_every=None):
        self.sid, self.m, self.n = sid, m, n
        self.precision = precision
        self.check_every = check_every
        self.reorth_every = reorth_every
        self.state = inputs.factorization(m, n, config=config, which=sid)  # host copy while evicted
        self.handle = None
        self.pending = collections.deque()
        self.busy = False
        self.last_used = 0.0
        self.bytes = reserve_bytes(m, n, precision)
        self.evictions = 0
        self.updates = 0

    def admit(self):
        Q, d, e, P = self.state
        # each session gets its own CUDA stream; batches order themselves after it
        self.handle = bdu.Factorization(Q, d, e, P, precision=self.precision, check_every=self.check_every,
                                        reorth_every=self.reorth_every)
        self.state = None
        self.bytes = max(self.bytes, self.handle.stats()["device_bytes"])

    def evict(self):
        self.state = self.handle.read()
        self.handle.close()
        self.handle = None
        self.evictions += 1

    def read(self):
        return self.handle.read() if self.handle is not None else self.state


class Server:
    def __init__(self, specs, precision=bdu.MIXED, budget_bytes=None, max_batch=64, check_every=None,
                 reorth_every=None):
        import torch
        self.torch = torch
        self.sessions = [Session(i, m, n, precision, check_every, reorth_every=reorth_every)
                         for i, (m, n) in enumerate(specs)]
        self.cuda = [torch.cuda.Stream(), torch.cuda.Stream()]
        self.budget = budget_bytes if budget_bytes is not None else sum(s.bytes for s in self.sessions)
        if max(s.bytes for s in self.sessions) > self.budget:
            raise ValueError("the budget is smaller than one session")
        self.resident_bytes = 0
        self.peak_resident = 0
        self.max_batch = max_batch
        self.in_flight = []  # (event, stream index, requests, device tensor, sessions)
        self.done = []
        self.batches = 0

    def _admit(self, s, now, protected):
        if s.handle is not None:
            return True
        if self.resident_bytes + s.bytes > self.budget:
            idle = [v for v in self.sessions
                    if v.handle is not None and not v.busy and v.sid not in protected]
            idle.sort(key=lambda v: v.last_used)
            for v in idle:
                if self.resident_bytes + s.bytes <= self.budget:
                    break
                v.evict()
                self.resident_bytes -= v.bytes
            if self.resident_bytes + s.bytes > self.budget:
                return False
        s.admit()
        if s.bytes > self.budget:
            raise RuntimeError(f"session {s.sid} ({s.m} x {s.n}) holds {s.bytes} device bytes, more than the "
                               f"budget of {self.budget}")
        self.resident_bytes += s.bytes
        self.peak_resident = max(self.peak_resident, self.resident_bytes)
        s.last_used = now
        return True

    def _retire(self):
        still = []
        for item in self.in_flight:
            ev, _, reqs, _, batch = item
            if ev.query():
                t = time.perf_counter()
                for q in reqs:
                    q.t_done = t
                for s in batch:
                    s.busy = False
                self.done.extend(reqs)
            else:
                still.append(item)
        self.in_flight = still

    def _launch(self, now):
        torch = self.torch
        used = {k for _, k, _, _, _ in self.in_flight}
        k = 0 if 0 not in used else 1
        cs = self.cuda[k]
        cands = sorted((s for s in self.sessions if s.pending and not s.busy),
                       key=lambda s: s.pending[0].t_arrival)
        batch, protected = [], set()
        for s in cands:
            if len(batch) == self.max_batch:
                break
            protected.add(s.sid)
            if self._admit(s, now, protected):
                batch.append(s)
        if not batch:
            return False
        reqs = [s.pending.popleft() for s in batch]
        # one pinned staging buffer and one host-to-device copy per batch
        sizes = [q.B.size + q.C.size for q in reqs]
        host = torch.empty(sum(sizes), dtype=torch.float64, pin_memory=True)
        hv = host.numpy()
        offs, o = [], 0
        for q in reqs:
            hv[o:o + q.B.size] = q.B.ravel(order="F")
            hv[o + q.B.size:o + q.B.size + q.C.size] = q.C.ravel(order="F")
            offs.append(o)
            o += q.B.size + q.C.size
        with torch.cuda.stream(cs):
            dev = host.to("cuda", non_blocking=True)
        base = dev.data_ptr()
        bdu.update_batch([s.handle for s in batch], [base + 8 * o for o in offs],
                         [base + 8 * (o + q.B.size) for o, q in zip(offs, reqs)], [q.r for q in reqs],
                         stream=cs.cuda_stream)
        ev = torch.cuda.Event()
        ev.record(cs)
        for s, q in zip(batch, reqs):
            s.busy = True
            s.last_used = now
            s.updates += q.r
        self.in_flight.append((ev, k, reqs, (host, dev), batch))
        self.batches += 1
        return True

    def run(self, arrivals, time_limit=None):
        """Serves the requests (t_arrival in seconds from the start) until all
        are done, or until time_limit seconds have passed (then the requests
        still waiting are dropped and do not count)."""
        arrivals = sorted(arrivals, key=lambda q: q.t_arrival)
        self.done = []
        batches0 = self.batches
        evictions0 = sum(s.evictions for s in self.sessions)
        t0 = time.perf_counter()
        for q in arrivals:
            q.t_arrival += t0
        nxt = 0
        while nxt < len(arrivals) or self.in_flight or any(s.pending for s in self.sessions):
            now = time.perf_counter()
            if time_limit is not None and now - t0 > time_limit:
                break
            while nxt < len(arrivals) and arrivals[nxt].t_arrival <= now:
                q = arrivals[nxt]
                self.sessions[q.sid].pending.append(q)
                nxt += 1
            self._retire()
            if not (len(self.in_flight) < 2 and self._launch(now)):
                time.sleep(0.0002)
        self.torch.cuda.synchronize()
        self._retire()
        for s in self.sessions:
            s.pending.clear()
        wall = time.perf_counter() - t0
        lat = np.array([1e3 * (q.t_done - q.t_arrival) for q in self.done])
        ups = sum(q.r for q in self.done)
        return {"requests": len(self.done), "updates": ups, "wall_s": wall, "updates_per_s": ups / wall,
                "latency_ms": {"p50": float(np.percentile(lat, 50)) if lat.size else None,
                               "p99": float(np.percentile(lat, 99)) if lat.size else None,
                               "samples": int(lat.size)},
                "batches": self.batches - batches0,
                "evictions": sum(s.evictions for s in self.sessions) - evictions0,
                "peak_resident_bytes": self.peak_resident, "budget_bytes": self.budget}

    def close(self):
        for s in self.sessions:
            if s.handle is not None:
                s.handle.close()
                s.handle = None


def poisson_arrivals(specs, rate, count, seed=0, config=4, first_update=None):
    """count requests of a Poisson process of the given rate (requests/s); each
    picks a session uniformly and is a rank r ~ U{1..4} update with N(0,1)
    entries.  first_update[sid] numbers the session's updates (advanced here)."""
    g = np.random.default_rng([inputs.SEED_BASE + config, 77, seed])
    h = first_update if first_update is not None else collections.Counter()
    t, out = 0.0, []
    for _ in range(count):
        t += g.exponential(1.0 / rate) if rate else 0.0
        sid = int(g.integers(len(specs)))
        m, n = specs[sid]
        B, C = inputs.serving_update(m, n, sid, h[sid], config=config)
        h[sid] += 1
        out.append(Request(sid, t, B, C))
    return out


def serve(num_sessions=256, seconds=20.0, precision=bdu.MIXED, budget_fraction=1 / 3, load=0.8,
          max_batch=64, seed=0, sat_per_session=4):
    """Saturation first (sat_per_session requests per session, all present
    at the start), then Poisson arrivals at `load` times the saturated request
    rate for about `seconds`; both on the same sessions, which carry their
    state over."""
    specs = inputs.serving_mix(num_sessions)
    total = sum(reserve_bytes(m, n, precision) for m, n in specs)
    srv = Server(specs, precision, int(total * budget_fraction), max_batch)
    counter = collections.Counter()
    sat = srv.run(poisson_arrivals(specs, 0.0, sat_per_session * num_sessions, seed, first_update=counter))
    rate = load * sat["requests"] / sat["wall_s"]
    arr = poisson_arrivals(specs, rate, max(1, int(rate * seconds)), seed + 1, first_update=counter)
    res = srv.run(arr, time_limit=3 * seconds)
    srv.close()
    return {"form": "fp64" if precision == bdu.FP64 else "mixed", "sessions": num_sessions,
            "budget_fraction": budget_fraction, "saturated": sat, "offered_requests_per_s": rate,
            "poisson": res}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--sessions", type=int, default=256)
    ap.add_argument("--seconds", type=float, default=20.0)
    ap.add_argument("--fp64", action="store_true")
    ap.add_argument("--budget-fraction", type=float, default=1 / 3)
    ap.add_argument("--max-batch", type=int, default=64)
    a = ap.parse_args()
    print(json.dumps(serve(a.sessions, a.seconds, bdu.FP64 if a.fp64 else bdu.MIXED, a.budget_fraction,
                           max_batch=a.max_batch)))


if __name__ == "__main__":
    main()

"""Continuous-batching request loop for REXI steps (the served form of the REXI time step).

Requests (one REXI linear step each, with their own truncation T, time step dt and pole count
N) arrive over time.  The engine keeps every admitted state resident in a device arena, and
each tick launches ONE ragged REXI step (rexi_ragged_*) over all admitted requests: requests
that arrive while a tick runs on the GPU are admitted -- their states copied into free arena
slots on a separate copy stream, overlapping the running tick -- and join the next tick.

Admission is by device memory: a request needs 2 x 3 x nlm complex128 of arena (input and
output slot) and its padded pole set in the pole arena; it waits while slots or memory are
short and is rejected with an error status (the others unaffected) when it can never fit or
its parameters are invalid.  Latency = completion time - arrival time; p50/p99 and steps/s
are reported.  All compute runs in librexi (argument marshalling only here).
"""
import bisect
import math
import time

import numpy as np

from . import rexi

OK, REJECTED = "ok", "rejected"


_CONTOURS = {}  # (N, quantised X) -> (p0, Xc) from the library's contour search


def contour(T, dt, omega, radius, phibar, N=None):
    """Default contour for a request: the covered half-width X of dt L, then (p0, Xc) with
    p0 <= Xc.  Below X = 20: Xc = 1.6 X, p0 = min(6, 1.6 X).  From X = 20 on, a fixed p0 fails:
    with p0 = 14 and 2048 poles the scalar REXI error is 2e5 at X = 182, so the contour comes from
    rexi_contour_select for the request's pole count, evaluated at X rounded up to a 5 % grid
    (X_q >= X covers the request's spectrum) and memoised, so that a stream of requests with
    continuous time steps costs a few hundred searches at most."""
    X = rexi.spectrum_bound(T, dt, omega, radius, phibar)
    if X < 20 or N is None:
        return (min(6.0, 1.6 * X), 1.6 * X) if X < 20 else (14.0, 1.4 * X)
    q = math.ceil(math.log(X / 20.0) / math.log(1.05))
    key = (int(N), q)
    if key not in _CONTOURS:
        _CONTOURS[key] = rexi.contour_select(20.0 * 1.05 ** q, int(N))
    return _CONTOURS[key]


def prepare_contours(pole_counts, Xmax):
    """Fills the contour table for every pole count served and every grid point of X up to Xmax
    (the planning work of a service, done once before requests arrive); returns the seconds
    it took."""
    t0 = time.perf_counter()
    qmax = math.ceil(math.log(max(Xmax, 20.0) / 20.0) / math.log(1.05))
    for N in pole_counts:
        for q in range(qmax + 1):
            key = (int(N), q)
            if key not in _CONTOURS:
                _CONTOURS[key] = rexi.contour_select(20.0 * 1.05 ** q, int(N))
    return time.perf_counter() - t0


class Request:
    __slots__ = ("rid", "arrival", "T", "dt", "N", "p0", "Xc", "state", "status", "error",
                 "result", "t_admit", "t_done", "slot")

    def __init__(self, rid, arrival, T, dt, N, state, p0=None, Xc=None):
        self.rid, self.arrival, self.T, self.dt, self.N = rid, arrival, int(T), float(dt), int(N)
        self.state = state
        self.p0, self.Xc = p0, Xc
        self.status = None
        self.error = None
        self.result = None
        self.t_admit = self.t_done = None
        self.slot = None

    @property
    def nlm(self):
        return (self.T + 1) * (self.T + 2) // 2

    @property
    def latency(self):
        return None if self.t_done is None else self.t_done - self.arrival


class _Arena:
    """First-fit allocator of complex128 elements in a fixed device buffer."""

    def __init__(self, cap):
        self.cap = cap
        self.free = [(0, cap)]  # sorted (start, length)

    def alloc(self, n):
        for i, (s, l) in enumerate(self.free):
            if l >= n:
                if l == n:
                    self.free.pop(i)
                else:
                    self.free[i] = (s + n, l - n)
                return s
        return None

    def release(self, s, n):
        i = bisect.bisect(self.free, (s, n))
        self.free.insert(i, (s, n))
        merged = []
        for a, b in self.free:
            if merged and merged[-1][0] + merged[-1][1] == a:
                merged[-1] = (merged[-1][0], merged[-1][1] + b)
            else:
                merged.append((a, b))
        self.free = merged


class ServingEngine:
    """Continuous-batching REXI server on one GPU.

    Tmax:       largest truncation served
    max_slots:  largest number of requests in one tick
    hbm_bytes:  device memory budget of the state arena (input + output slots)
    max_poles:  capacity of the pole arena (padded poles of the pole sets in flight)
    precision:  "mixed" (served form) or "fp64"
    """

    def __init__(self, Tmax=511, max_slots=64, hbm_bytes=2 << 30, max_poles=1 << 17,
                 precision="mixed", omega=None, radius=None, phibar=None):
        import torch
        from . import synthetic as syn
        self.torch = torch
        self.omega = syn.OMEGA if omega is None else omega
        self.radius = syn.RADIUS if radius is None else radius
        self.phibar = syn.PHIBAR if phibar is None else phibar
        self.Tmax, self.max_slots, self.max_poles = Tmax, max_slots, max_poles
        cap = int(hbm_bytes // (2 * 16))  # complex elements per arena (input and output)
        self.cap = cap
        self.stream = torch.cuda.Stream()
        self.copy_stream = torch.cuda.Stream()
        self.U0 = torch.zeros(cap, dtype=torch.complex128, device="cuda")
        self.U1 = torch.zeros(cap, dtype=torch.complex128, device="cuda")
        self.arena = _Arena(cap)
        self.plan = rexi.RaggedPlan(Tmax, max_slots, max_poles, cap // 3 + 1, self.omega, self.radius,
                                    self.phibar, precision=precision, stream=self.stream)
        self.queue = []       # arrived, not admitted
        self.active = []      # admitted, waiting for a tick
        self.done = []
        self.ticks = 0
        self.out_host = None  # pinned host buffer the results of a tick are copied into
        self.prepared = None  # (batch, upload event) whose launch is built for the next tick

    # ---- admission ---------------------------------------------------------------------
    def _validate(self, r):
        if not (1 <= r.T <= self.Tmax):
            return "truncation T=%d outside [1, %d]" % (r.T, self.Tmax)
        if not (1 <= r.N <= 8192) or not (r.dt > 0):
            return "bad N or dt"
        if 3 * r.nlm > self.cap:
            return "state of %d coefficients exceeds the device memory budget" % (3 * r.nlm)
        if (r.N + 31) // 32 * 32 > self.max_poles:
            return "pole set exceeds the pole arena"
        if r.state is None or r.state.shape != (3, r.nlm):
            return "state shape mismatch"
        return None

    def submit(self, r):
        err = self._validate(r)
        if err:
            r.status, r.error, r.t_done = REJECTED, err, time.perf_counter()
            self.done.append(r)
            return r
        if r.p0 is None:
            r.p0, r.Xc = contour(r.T, r.dt, self.omega, self.radius, self.phibar, r.N)
        self.queue.append(r)
        return r

    def _admit(self):
        """Moves queued requests into free arena slots (copies on the copy stream)."""
        torch = self.torch
        admitted = []
        npoles = sum((r.N + 31) // 32 * 32 for r in self.active)
        keep = []
        for r in self.queue:
            need_p = (r.N + 31) // 32 * 32
            if len(self.active) + len(admitted) >= self.max_slots or npoles + need_p > self.max_poles:
                keep.append(r)
                continue
            s = self.arena.alloc(3 * r.nlm)
            if s is None:
                keep.append(r)
                continue
            r.slot = s
            r.t_admit = time.perf_counter()
            with torch.cuda.stream(self.copy_stream):
                src = torch.from_numpy(np.ascontiguousarray(r.state.reshape(-1))).pin_memory()
                self.U0[s: s + 3 * r.nlm].copy_(src, non_blocking=True)
            npoles += need_p
            admitted.append(r)
        self.queue = keep
        return admitted

    # ---- one tick ------------------------------------------------------------------------
    def _prepare(self):
        """Admits what fits and builds its ragged launch (plan.set: host tile lists, uploads
        queued in stream order behind the work in flight).  Returns the batch, or None."""
        self.active.extend(self._admit())
        if not self.active:
            return None
        batch = self.active
        self.active = []
        ev = self.torch.cuda.Event()
        ev.record(self.copy_stream)   # the batch's state uploads
        self.plan.set([(r.T, r.N, r.dt, r.p0, r.Xc, r.slot) for r in batch])
        return batch, ev

    def tick(self, on_launch=None):
        """Launches one ragged REXI step over a batch of admitted requests and completes it.
        While it runs, late arrivals are admitted (on_launch callback) and the next batch's
        launch is built, so that the host work between two steps is only the copy-out."""
        torch = self.torch
        prep = self.prepared if self.prepared is not None else self._prepare()
        self.prepared = None
        if prep is None:
            return 0
        batch, ev = prep
        self.stream.wait_event(ev)
        self.plan.step(self.U0, self.U1)
        # the results back to the host in the same stream order: one asynchronous copy per
        # request into one pinned buffer, then one wait for the tick
        total = sum(3 * r.nlm for r in batch)
        if self.out_host is None or self.out_host.numel() < total:
            self.out_host = torch.empty(max(total, 3 * (self.Tmax + 1) * (self.Tmax + 2) // 2),
                                        dtype=torch.complex128, pin_memory=True)
        offs = []
        o = 0
        with torch.cuda.stream(self.stream):
            for r in batch:
                n = 3 * r.nlm
                self.out_host[o: o + n].copy_(self.U1[r.slot: r.slot + n], non_blocking=True)
                offs.append(o)
                o += n
        done_ev = torch.cuda.Event()
        done_ev.record(self.stream)
        if on_launch is not None:
            on_launch()                      # arrivals during the tick
        self.prepared = self._prepare()      # the next launch, built while this one runs
        done_ev.synchronize()
        now = time.perf_counter()
        host = self.out_host.numpy()
        for r, o in zip(batch, offs):
            r.result = host[o: o + 3 * r.nlm].reshape(3, r.nlm).copy()
            r.status = OK
            r.t_done = now
            self.arena.release(r.slot, 3 * r.nlm)
            self.done.append(r)
        self.ticks += 1
        return len(batch)

    def run(self, requests, clock=time.perf_counter):
        """Serves a list of requests with arrival times (seconds from start)."""
        pending = sorted(requests, key=lambda r: r.arrival)
        t0 = clock()
        for r in pending:
            r.arrival += t0
        i = 0

        def arrivals():
            nonlocal i
            now = clock()
            while i < len(pending) and pending[i].arrival <= now:
                self.submit(pending[i])
                i += 1

        while i < len(pending) or self.queue or self.active or self.prepared is not None:
            arrivals()
            if not self.queue and not self.active and self.prepared is None:
                if i < len(pending):
                    time.sleep(max(0.0, min(0.01, pending[i].arrival - clock())))
                continue
            self.tick(on_launch=arrivals)
        wall = clock() - t0
        return summarize(self.done, wall)

    def close(self):
        self.plan.close()


def summarize(done, wall):
    ok = [r for r in done if r.status == OK]
    lat = np.array([r.latency for r in ok]) if ok else np.zeros(1)
    return {"completed": len(ok), "rejected": len(done) - len(ok), "wall_s": wall,
            "steps_per_s": len(ok) / wall if wall > 0 else float("nan"),
            "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3)}


def one_at_a_time(requests, precision="fp64", Tmax=511, clock=time.perf_counter):
    """Reference service: requests processed one at a time (one instance per launch)."""
    import torch
    from . import synthetic as syn
    stream = torch.cuda.Stream()
    maxe = max(3 * r.nlm for r in requests)
    plan = rexi.RaggedPlan(Tmax, 1, max((r.N + 31) // 32 * 32 for r in requests) * 2, maxe // 3 + 1,
                           syn.OMEGA, syn.RADIUS, syn.PHIBAR, precision=precision, stream=stream)
    U0 = torch.zeros(maxe, dtype=torch.complex128, device="cuda")
    U1 = torch.zeros_like(U0)
    pending = sorted(requests, key=lambda r: r.arrival)
    t0 = clock()
    done = []
    for r in pending:
        arrival = t0 + r.arrival
        while clock() < arrival:
            time.sleep(max(0.0, min(0.01, arrival - clock())))
        if r.p0 is None:
            r.p0, r.Xc = contour(r.T, r.dt, syn.OMEGA, syn.RADIUS, syn.PHIBAR, r.N)
        n = 3 * r.nlm
        U0[:n].copy_(torch.from_numpy(r.state.reshape(-1)))
        plan.set([(r.T, r.N, r.dt, r.p0, r.Xc, 0)])
        with torch.cuda.stream(stream):
            plan.step(U0, U1)
        stream.synchronize()
        r.result = U1[:n].cpu().numpy().reshape(3, r.nlm)
        r.status = OK
        r.t_done = clock()
        r.arrival = arrival
        done.append(r)
    wall = clock() - t0
    plan.close()
    return summarize(done, wall)


def make_requests(count, seed=5, rate=1.0, Tmax=511, state_seed=1000):
    """Requests of the serving workload: Poisson arrivals at `rate` per second,
    T = round(exp(U[ln 63, ln 511])), dt = exp(U[ln 600, ln 14400]) s,
    N = 256 * 2^round(3 ln(dt/600)/ln 24); n^-1.5 Gaussian states."""
    from . import synthetic as syn
    out = []
    for k, q in enumerate(syn.request_stream(count, seed=seed, rate=rate)):
        T = min(q["T"], Tmax)
        out.append(Request(k, q["arrival"], T, q["dt"], q["N"], syn.gaussian_state(T, state_seed + k)))
    return out

"""Continuous-batching request server for randomized SVDs.

Requests (m x n matrix already on the device, k, p, q, sigma tolerance) arrive
over time.  The server keeps a set of *lanes*; each lane is one CUDA stream
with one batch plan (rsvd_batch_plan_create) for a class of requests:

* precision: a request's tolerance is relative on every sigma_i, i <= k.
  Requests with tol >= 1e-4 start on FP32 lanes, the rest on FP64 lanes
  (the matrix is promoted to FP64 on the device).  FP32 rounding moves each
  computed sigma by about u_32 sigma_1 (u_32 = 2^-24), i.e. by u_32
  sigma_1 / sigma_i relative, so whether FP32 meets a tolerance depends on
  the spectrum, which is known only once solved: an FP32 result is accepted
  when FP32_ERR_COEF u_32 sigma_1 / sigma_k <= tol (computed sigmas), and
  otherwise the request is promoted and solved again on an FP64 lane (its
  latency covers both solves);
* size: "small" lanes (k + p <= 80) and "big" lanes (k + p up to 288), so a
  few large problems never hold back the latency of the many small ones.

Whenever a lane is idle, it takes the oldest waiting requests of its class
that fit its slot count and the global HBM admission budget, and launches
them as one grouped solve; lanes run concurrently, so requests that arrive
while others are on the GPU are admitted as soon as a lane and memory free
up, and their work overlaps with the batches still in flight.  Every result
is the same as the request solved alone (the grouped kernels share no work
between problems).

The scheduling logic (``Server``) is independent of the GPU: it drives a
backend with ``launch(lane, requests)`` / ``poll(handle)``; ``TorchBackend``
is the CUDA one, and the tests use a simulated one.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Dict, List, Optional

FP32_TOL_LIMIT = 1e-4     # tolerances below this go to FP64 lanes
FP32_UNIT = 2.0 ** -24
FP32_ERR_COEF = 256.0     # FP32 sigma error bound: FP32_ERR_COEF * u_32 * sigma_1
SMALL_L_MAX = 80
BIG_L_MAX = 288


@dataclass
class Request:
    rid: int
    m: int
    n: int
    k: int
    p: int
    q: int
    tol: float
    seed: int
    arrival: float
    A: object = None              # device tensor (n, lda), column-major, FP32 or FP64
    # filled by the server
    lane: Optional[str] = None
    start: Optional[float] = None
    done: Optional[float] = None
    status: Optional[int] = None
    result: object = None
    precision: Optional[str] = None   # "f32" / "f64" once routed (promotion sets "f64")
    promoted: bool = False

    @property
    def l(self) -> int:
        return self.k + self.p

    @property
    def latency(self) -> Optional[float]:
        return None if self.done is None else self.done - self.arrival


def request_class(r: Request) -> str:
    prec = r.precision or ("f32" if r.tol >= FP32_TOL_LIMIT else "f64")
    size = "small" if r.l <= SMALL_L_MAX else "big"
    return f"{prec}-{size}"


def fp32_meets(sigma, tol: float) -> bool:
    """Whether an FP32 result's singular values (descending, length k) meet
    the relative tolerance on every sigma_i: the FP32 error bound
    FP32_ERR_COEF u_32 sigma_1, relative to the smallest sigma_k, must not
    exceed tol.  Non-finite or non-positive sigma_k fails."""
    s = [float(x) for x in sigma]
    if not s or not all(math.isfinite(x) for x in s) or s[-1] <= 0.0:
        return False
    return FP32_ERR_COEF * FP32_UNIT * s[0] / s[-1] <= tol


def footprint_bytes(r: Request) -> int:
    """Device bytes a request holds while admitted: its matrix in the lane's
    precision, the outputs, and its share of the lane workspace (the n x l,
    m x l and (m+n) x l buffers of the grouped solve)."""
    e = 4 if request_class(r).startswith("f32") else 8
    a = r.m * r.n * e
    out = (r.m * r.k + r.k * r.n) * e + r.k * 8
    ws = (3 * r.n + 2 * r.m + (r.m + r.n)) * r.l * e
    return a + out + ws


@dataclass
class LaneSpec:
    name: str               # request class served, e.g. "f32-small"
    max_count: int          # problems per batch
    rows_total: int         # sum of m over a batch
    cols_total: int         # sum of n over a batch
    l_max: int
    # "grouped": one grouped solve per batch (rsvd_solve_batched); "tensor":
    # one request at a time on an FP64 plan whose passes over A run on the
    # tensor cores (max_count 1; rows_total, cols_total bound m and n)
    engine: str = "grouped"
    lanes: int = 0          # lanes of this class (0: the server's default)


@dataclass
class Lane:
    spec: LaneSpec
    index: int
    busy: bool = False
    batch: List[Request] = field(default_factory=list)
    handle: object = None
    batches: int = 0

    @property
    def key(self) -> str:
        return f"{self.spec.name}#{self.index}"


class Server:
    """Continuous batching over lanes with HBM-footprint admission."""

    def __init__(self, lane_specs: List[LaneSpec], backend, hbm_budget_bytes: int,
                 lanes_per_class: int = 2, clock=None):
        self.backend = backend
        self.budget = hbm_budget_bytes
        self.in_use = 0
        self.lanes: List[Lane] = []
        for spec in lane_specs:
            if spec.engine == "tensor" and (spec.max_count != 1 or spec.name.startswith("f32")):
                raise ValueError("tensor lanes serve FP64 requests one at a time")
            for i in range(spec.lanes or lanes_per_class):
                lane = Lane(spec, i)
                backend.create_lane(lane)
                self.lanes.append(lane)
        self.queues: Dict[str, List[Request]] = {s.name: [] for s in lane_specs}
        self.finished: List[Request] = []
        self.clock = clock
        self.admission_stalls = 0
        self.promotions = 0

    def submit(self, r: Request, now: float = 0.0):
        r.precision = r.precision or ("f32" if r.tol >= FP32_TOL_LIMIT else "f64")
        cls = request_class(r)
        if cls not in self.queues:
            raise ValueError(f"no lane serves request class {cls}")
        spec = next(l.spec for l in self.lanes if l.spec.name == cls)
        if (footprint_bytes(r) > self.budget or r.l > spec.l_max or r.m > spec.rows_total or
                r.n > spec.cols_total):
            # can never be admitted: refuse now instead of blocking the class
            r.status, r.start, r.done = 4, now, now
            self.finished.append(r)
            return
        self.queues[cls].append(r)

    def _promote(self, r: Request, now: float):
        """FP32 did not meet r's tolerance: queue it again on the FP64 class,
        ahead of requests that arrived after it (FIFO by arrival)."""
        r.precision = "f64"
        r.promoted = True
        r.result = None
        self.promotions += 1
        cls = request_class(r)
        spec = next((l.spec for l in self.lanes if l.spec.name == cls), None)
        if (spec is None or footprint_bytes(r) > self.budget or r.l > spec.l_max or
                r.m > spec.rows_total or r.n > spec.cols_total):
            r.status, r.done = 4, now
            self.finished.append(r)
            return
        q = self.queues[cls]
        i = 0
        while i < len(q) and q[i].arrival <= r.arrival:
            i += 1
        q.insert(i, r)

    def _fill(self, lane: Lane, now: float) -> List[Request]:
        q = self.queues[lane.spec.name]
        take, rows, cols = [], 0, 0
        for r in q:
            if len(take) == lane.spec.max_count:
                break
            fp = footprint_bytes(r)
            if (rows + r.m > lane.spec.rows_total or cols + r.n > lane.spec.cols_total or
                    self.in_use + fp > self.budget):
                if not take:
                    self.admission_stalls += 1
                break                 # FIFO within a class: never overtake
            take.append(r)
            rows += r.m
            cols += r.n
            self.in_use += fp
        del q[:len(take)]
        for r in take:
            r.lane = lane.key
            r.start = now
        return take

    def step(self, now: float) -> int:
        """Completes finished batches and launches new ones; returns the number
        of requests completed."""
        completed = 0
        for lane in self.lanes:
            if lane.busy and self.backend.poll(lane):
                t = now if self.clock is None else self.clock()
                f32 = lane.spec.name.startswith("f32")
                sig = self.backend.sigmas(lane) if f32 else [None] * len(lane.batch)
                for r, st, s in zip(lane.batch, self.backend.statuses(lane), sig):
                    self.in_use -= footprint_bytes(r)
                    if f32 and st == 0 and not fp32_meets(s, r.tol):
                        self._promote(r, t)
                        continue
                    r.done = t
                    r.status = st
                    self.finished.append(r)
                    completed += 1
                lane.busy = False
                lane.batch = []
        for lane in self.lanes:
            if not lane.busy:
                batch = self._fill(lane, now)
                if batch:
                    self.backend.launch(lane, batch)
                    lane.busy = True
                    lane.batch = batch
                    lane.batches += 1
        return completed

    def pending(self) -> int:
        return sum(len(q) for q in self.queues.values()) + sum(len(l.batch) for l in self.lanes)


def percentile(xs: List[float], pct: float) -> float:
    if not xs:
        return float("nan")
    s = sorted(xs)
    i = min(len(s) - 1, max(0, int(math.ceil(pct / 100.0 * len(s))) - 1))
    return s[i]


def run(server: Server, requests: List[Request], now_fn, max_wall: float = 600.0,
        drain_s: Optional[float] = None) -> dict:
    """Feeds requests at their arrival times (now_fn: seconds since start)
    until every request has completed.  With drain_s, stops waiting drain_s
    after the last arrival: requests not finished by then are counted as
    unserved (their work still completes on the device, the results are
    dropped), and latencies cover the served requests only."""
    order = sorted(requests, key=lambda r: r.arrival)
    i = 0
    t0 = now_fn()
    last = order[-1].arrival if order else 0.0
    while True:
        now = now_fn() - t0
        while i < len(order) and order[i].arrival <= now:
            server.submit(order[i], now)
            i += 1
        server.step(now)
        if i == len(order) and server.pending() == 0:
            break
        if drain_s is not None and i == len(order) and now > last + drain_s:
            break
        if now > max_wall:
            raise RuntimeError("serving run exceeded its wall-clock limit")
    wall = now_fn() - t0
    lat = [r.latency for r in server.finished]
    unserved = len(order) - len(server.finished)
    return {"completed": len(server.finished), "unserved": unserved, "wall_s": wall,
            "throughput_rps": len(server.finished) / wall if wall > 0 else float("nan"),
            "p50_ms": percentile(lat, 50) * 1e3, "p99_ms": percentile(lat, 99) * 1e3,
            "max_ms": max(lat) * 1e3 if lat else float("nan"),
            "batches": sum(l.batches for l in server.lanes),
            "admission_stalls": server.admission_stalls,
            "promotions": server.promotions,
            "failed": sum(1 for r in server.finished if r.status != 0)}


class TorchBackend:
    """Runs lanes as CUDA streams with one rsvd batch plan each."""

    def __init__(self):
        import torch

        from . import rsvd as R
        self.torch = torch
        self.R = R
        self.state = {}

    def create_lane(self, lane: Lane):
        torch, R = self.torch, self.R
        # small problems on high-priority streams: their blocks are scheduled
        # ahead of a big batch's pending blocks as SMs free up
        stream = torch.cuda.Stream(priority=-1 if lane.spec.name.endswith("small") else 0)
        dt = R.F32 if lane.spec.name.startswith("f32") else R.F64
        if lane.spec.engine == "tensor":
            plan = R.Plan(lane.spec.rows_total, lane.spec.cols_total, lane.spec.l_max,
                          mode=R.F64_TENSOR, stream=stream)
        else:
            plan = R.BatchPlan(lane.spec.max_count, lane.spec.rows_total, lane.spec.cols_total,
                               lane.spec.l_max, dt, stream=stream)
        self.state[lane.key] = {"stream": stream, "plan": plan, "event": None, "dt": dt,
                                "tensor": lane.spec.engine == "tensor"}

    def launch(self, lane: Lane, batch: List[Request]):
        torch, R = self.torch, self.R
        st = self.state[lane.key]
        dtype = torch.float32 if st["dt"] == R.F32 else torch.float64
        with torch.cuda.stream(st["stream"]):
            items = []
            for r in batch:
                A = r.A if r.A.dtype == dtype else r.A.to(dtype)
                items.append((A, r.m, r.n, r.k, r.p, r.q, r.seed))
            if st["tensor"]:
                res = [st["plan"].solve(A, m, n, k, p, q, seed)
                       for (A, m, n, k, p, q, seed) in items]
            else:
                res = st["plan"].solve(items)
            ev = torch.cuda.Event()
            ev.record(st["stream"])
        for r, out in zip(batch, res):
            r.result = out
        st["event"] = ev
        st["items"] = items

    def poll(self, lane: Lane) -> bool:
        return self.state[lane.key]["event"].query()

    def statuses(self, lane: Lane) -> List[int]:
        st = self.state[lane.key]
        if st["tensor"]:
            return [st["plan"].status()] * len(lane.batch)
        return st["plan"].status()

    def sigmas(self, lane: Lane):
        """Host copies of each finished request's singular values (the lane's
        event has completed, so the copies do not wait on work in flight)."""
        return [r.result[1].cpu().tolist() for r in lane.batch]

"""Serving loop: Poisson request streams over several cached media, continuous batching.

Each medium has one set-up Context (its cached factorisation) and one dds_server; the library
admits by device memory: the context's budget (dds_set_memory_budget) caps what it holds, and the
server's slot count (its admission limit) is what fits in the rest.  A request carries 1..32
point sources (right-hand sides); each right-hand side becomes one server submission, and the
request completes when all of them have.  One worker thread per medium steps its server (the
C calls release the GIL), so the media's batched iterations overlap on the GPU; inside a
medium, sources that arrive while others are in flight join at the next FGMRES iteration.

This module only schedules: every arithmetic step runs inside libdds.
"""

from __future__ import annotations

import dataclasses
import threading
import time

import numpy as np

from . import dds, synth


@dataclasses.dataclass
class Medium:
    name: str
    n: tuple
    parts: tuple
    omega: float
    c: np.ndarray
    pml_cells: int = 12


def serving_media(seed: int = 5):
    """The three cached media of the serving workload: 256^2 constant (4x4 of 64, kappa = 32 pi),
    512^2 two-layer (8x8 of 64, omega = 64 pi), 1024^2 smooth random c in [1, 2] (16x16 of 64,
    omega = 128 pi, Gaussian covariance length 0.1); 12-cell PML."""
    return [
        Medium("const256", (256, 256), (4, 4), 32 * np.pi, synth.medium_constant((256, 256))),
        Medium("layer512", (512, 512), (8, 8), 64 * np.pi,
               synth.medium_two_layer((512, 512), 1.0 / 512)),
        Medium("random1024", (1024, 1024), (16, 16), 128 * np.pi,
               synth.medium_random((1024, 1024), 1.0 / 1024, seed)),
    ]


@dataclasses.dataclass
class Request:
    rid: int
    medium: int
    arrival: float
    centres: np.ndarray
    done_rhs: int = 0
    completion: float = 0.0
    iters: list = dataclasses.field(default_factory=list)
    relres: list = dataclasses.field(default_factory=list)


def poisson_requests(rng, count: int, rate: float, n_media: int, max_sources: int = 32):
    """Arrival times (s), medium (uniform) and 1..max_sources seeded source centres each."""
    t = 0.0
    out = []
    for rid in range(count):
        t += rng.exponential(1.0 / rate)
        m = int(rng.integers(0, n_media))
        k = int(rng.integers(1, max_sources + 1))
        out.append(Request(rid, m, t, rng.uniform(0.1, 0.9, size=(k, 2))))
    return out


class MediumWorker(threading.Thread):
    def __init__(self, idx, medium: Medium, budget_bytes, tol, maxit, rounds, t0):
        super().__init__(daemon=True)
        self.idx = idx
        self.medium = medium
        self.ctx = dds.Context(medium.n, 1.0 / medium.n[0], medium.omega, medium.c, medium.parts,
                               medium.pml_cells, 30.0, precision="mixed")
        # launch shapes picked by measurement for a typical batch (set-up work, before the budget
        # applies: the tuner's scratch is its own)
        self.tuned = self.ctx.autotune(32, rounds)
        # admission by device memory inside the library: the context's budget caps everything
        # it holds, and the server takes the slots that fit in what is left (at most 64)
        self.ctx.set_memory_budget(int(budget_bytes))
        self.server = dds.Server(self.ctx, 64, tol, maxit, rounds)
        self.slots = self.server.slots
        self.inbox = []
        self.lock = threading.Lock()
        self.pending = {}
        self.t0 = t0
        self.stop = False
        self.steps = 0
        self.rhs_done = 0
        self.error = None

    def close(self):
        """Destroy the server, then its context (after the worker has stopped)."""
        if self.server is not None:
            self.server.close()
            self.server = None
        if self.ctx is not None:
            self.ctx.close()
            self.ctx = None

    def put(self, req: Request):
        with self.lock:
            self.inbox.append(req)

    def run(self):
        h = 1.0 / self.medium.n[0]
        out = np.empty(self.ctx.G[::-1], dtype=np.complex128)
        # one extended source field, reused: each source is written on its compact support (the
        # Gaussian's cutoff box), submitted, and cleared again
        src = np.zeros(self.ctx.G[::-1], dtype=np.complex128)
        E = (self.ctx.G[0] - self.medium.n[0]) // 2
        try:
            while True:
                with self.lock:
                    new, self.inbox = self.inbox, []
                for req in new:
                    for k, centre in enumerate(req.centres):
                        sl, vals = synth.gaussian_source_patch(self.medium.n, h, centre, 2 * h)
                        box = tuple(slice(q.start + E, q.stop + E) for q in sl)
                        src[box] = vals
                        self.server.submit(src, req.rid * 64 + k)
                        src[box] = 0.0
                    self.pending[req.rid] = req
                active, queued = self.server.step()
                self.steps += 1
                while True:
                    res = self.server.poll(out)
                    if res is None:
                        break
                    tag, _, it, rel = res
                    req = self.pending[tag // 64]
                    req.done_rhs += 1
                    req.iters.append(it)
                    req.relres.append(rel)
                    self.rhs_done += 1
                    if req.done_rhs == len(req.centres):
                        req.completion = time.perf_counter() - self.t0
                        del self.pending[req.rid]
                if active == 0 and queued == 0 and not new:
                    # stop only once nothing is in flight and nothing waits in the inbox (the
                    # driver may add a request between this iteration's read and the stop flag)
                    with self.lock:
                        idle = not self.inbox
                    if self.stop and not self.pending and idle:
                        return
                    time.sleep(0.0005)
        except Exception as e:  # surfaced by the driver
            self.error = e


def run(requests, media=None, budget_bytes=40e9, tol=1e-6, maxit=30, rounds=3):
    """Serve `requests` (arrival times in seconds from the start) in real time.  Returns per-
    request latencies (s), wall time, RHS count and worker statistics."""
    media = serving_media() if media is None else media
    t0 = time.perf_counter()
    workers = [MediumWorker(i, m, budget_bytes / len(media), tol, maxit, rounds, t0)
               for i, m in enumerate(media)]
    setup = time.perf_counter() - t0
    t0 = time.perf_counter()
    for w in workers:
        w.t0 = t0
        w.start()
    for req in sorted(requests, key=lambda r: r.arrival):
        delay = req.arrival - (time.perf_counter() - t0)
        if delay > 0:
            time.sleep(delay)
        workers[req.medium].put(req)
    for w in workers:
        w.stop = True
    # every worker leaves the library before an error surfaces (a worker whose peer failed
    # still finishes its own requests), and the servers go before their contexts
    for w in workers:
        w.join()
    errors = [w.error for w in workers if w.error is not None]
    for w in workers:
        w.close()
    if errors:
        raise errors[0]
    wall = time.perf_counter() - t0
    lat = np.array([r.completion - r.arrival for r in requests])
    return {"latency_s": lat, "wall_s": wall, "setup_s": setup,
            "rhs": int(sum(len(r.centres) for r in requests)),
            "slots": [w.slots for w in workers], "steps": [w.steps for w in workers],
            "launch_shapes": [{k: w.tuned[k] for k in ("panel_width", "panels_per_cta",
                                                        "trace_ctas_per_sm")} for w in workers],
            "max_relres": float(max(max(r.relres) for r in requests)),
            "max_iters": [max([max(r.iters) for r in requests if r.medium == i and r.iters] or [0])
                          for i in range(len(media))],
            "p99_s": [float(np.percentile([r.completion - r.arrival for r in requests
                                            if r.medium == i] or [0.0], 99))
                      for i in range(len(media))]}

"""Continuous-batching server for world-stepping requests.

A request asks for one world (its seeded state and genome table) to be stepped a given number
of times. Requests arrive over time; the server admits them in arrival order as soon as the
memory they need fits in the budget and a batch slot is free, keeps every admitted world
resident on the device, and
steps all resident worlds together: one batched launch per pass over every world (the
library's coral_batch_*), so a request that arrives while others run joins the next step and
its work overlaps theirs on the device. A world that has done its steps is read back and freed,
which may admit waiting requests. Because the batched kernels run the same per-cell arithmetic
as single-world stepping, each result is identical to stepping the world alone.

The device side is behind a small backend interface (``CoralBackend``) so that the scheduling
logic can be exercised on the CPU with a fake backend.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np

# Device bytes per cell of a resident world: two state buffers (2 x 29 B), the pass-1 record
# and direction (17 B); plus per genome slot the FP32 and BF16 nets and genes (~8.6 KB at
# H = 32) and a fixed part (stats ring, partial sums, radiation scratch).
BYTES_PER_CELL = 2 * 29 + 17
BYTES_PER_SLOT = {0: 2400 + 2200, 16: 4200 + 2600, 32: 6600 + 4200, 48: 8900 + 6300, 64: 17300 + 10400}
FIXED_BYTES = 2 << 20


def world_bytes(n_cells: int, capacity: int, hidden: int) -> int:
    return n_cells * BYTES_PER_CELL + capacity * BYTES_PER_SLOT.get(hidden, 20000) + FIXED_BYTES


@dataclass(order=True)
class Request:
    arrival: float                      # seconds after the start of the run
    rid: int
    world: object = field(compare=False)
    steps: int = field(compare=False, default=1)


@dataclass
class Completed:
    rid: int
    arrival: float
    admitted: float
    finished: float
    steps: int
    cells: int
    result: dict                        # the world's channels after its last step


class CoralBackend:
    """Real device backend: substrates and batches of the CUDA library. Worlds given lazily
    (with a ``materialize`` method) are built on a host thread pool as soon as they are queued,
    so that building them overlaps the device's steps."""

    def __init__(self, path=None, build_threads: int = 4):
        from concurrent.futures import ThreadPoolExecutor
        from . import coral
        self.coral = coral
        self.path = coral.BF16_GROUPED if path is None else path
        self.pool = ThreadPoolExecutor(max_workers=build_threads)
        self.stepper = ThreadPoolExecutor(max_workers=1)
        self.futures = {}

    def prepare(self, world):
        if hasattr(world, "materialize") and id(world) not in self.futures:
            self.futures[id(world)] = self.pool.submit(world.materialize)

    def create(self, world):
        if hasattr(world, "materialize"):
            self.prepare(world)
            world = self.futures.pop(id(world)).result()
        return self.coral.substrate_for_world(world, self.path)

    def batch(self, handles):
        return self.coral.Batch(handles)

    def step(self, batch, n):
        return batch.step_timed(n)       # per-step device time (ms)

    def step_async(self, batch, n):
        """The same steps on a host thread (the call waits for the device without holding the
        interpreter), so that the server creates the next worlds meanwhile."""
        return self.stepper.submit(batch.step_timed, n)

    def read(self, handle):
        return handle.read_channels()

    def free(self, handle):
        handle.close()

    def free_batch(self, batch):
        batch.close()


class WorldServer:
    """Admits requests by memory budget and steps the resident worlds as one batch."""

    def __init__(self, backend, budget_bytes: int, chunk_steps: int = 4, clock=time.perf_counter,
                 sleep=time.sleep, max_worlds: int = 0, prefetch: int = 8):
        self.backend = backend
        self.budget = int(budget_bytes)
        self.chunk = max(1, int(chunk_steps))
        self.max_worlds = int(max_worlds)      # batch slots (0 = bounded by the budget only)
        self.prefetch = int(prefetch)          # queued requests whose worlds are built ahead
        self.clock = clock
        self.sleep = sleep

    def run(self, requests):
        """Serve `requests` (arrival times in seconds from now). Returns (completed, report).

        With a backend that steps asynchronously (``step_async``), the host work overlaps the
        device's chunk of steps: the next requests' worlds are admitted and created (until the
        chunk ends; they join the batch at the next rebuild), and the worlds that finished with
        the last chunk are read back (their memory is released at the next chunk end)."""
        pending = sorted(requests)
        waiting = []                     # arrived, not admitted (FIFO by arrival)
        active = {}                      # rid -> [request, handle, remaining, admitted_at, bytes]: in the batch
        joining = {}                     # admitted and created, joining at the next rebuild
        finished = []                    # left the batch, results not read yet
        to_free = []                     # read, released when the device is idle
        used = 0
        batch = None
        dirty = False
        step_lat = []                    # (batch step ms, resident worlds) per batched step
        req_step_ms = []                 # one entry per request-step: the device time of its step
        req_step_wall = []               # one entry per request-step: wall time between chunk ends / steps
        completed = []
        work = 0
        t0 = self.clock()
        peak_used = 0
        inflight = None                  # (future or result, steps, resident worlds)
        last_end = None                  # wall clock at the end of the last chunk
        asynchronous = hasattr(self.backend, "step_async")
        host = {"create_s": 0.0, "batch_s": 0.0, "read_s": 0.0, "free_s": 0.0, "wait_s": 0.0}

        def chunk_running():
            return asynchronous and inflight is not None and not inflight[0].done()

        def admit(during_chunk=False):
            nonlocal used, peak_used
            now = self.clock() - t0
            while pending and pending[0].arrival <= now:
                waiting.append(pending.pop(0))
            if hasattr(self.backend, "prepare"):
                for r in waiting[:self.prefetch]:
                    self.backend.prepare(r.world)
            # arrival order, while the budget and the slots allow (a request that can never fit
            # on its own is rejected rather than blocking the queue); during a chunk only until
            # it ends, so that the device does not wait for a burst of admissions
            while waiting and not (during_chunk and not chunk_running()):
                r = waiting[0]
                need = world_bytes(r.world.n_cells, r.world.capacity, r.world.hidden)
                if need > self.budget:
                    waiting.pop(0)
                    completed.append(Completed(r.rid, r.arrival, -1.0, -1.0, 0, r.world.n_cells, {}))
                    continue
                resident = len(active) + len(joining)
                if used + need > self.budget or (self.max_worlds and resident >= self.max_worlds):
                    break
                waiting.pop(0)
                c0 = self.clock()
                joining[r.rid] = [r, self.backend.create(r.world), r.steps, self.clock() - t0, need]
                host["create_s"] += self.clock() - c0
                used += need
                peak_used = max(peak_used, used)

        def read_finished():
            c0 = self.clock()
            for rid, (r, h, _, adm, need) in finished:
                res = self.backend.read(h)
                completed.append(Completed(rid, r.arrival, adm, self.clock() - t0, r.steps, r.world.n_cells, res))
                to_free.append((h, need))
            finished.clear()
            host["read_s"] += self.clock() - c0

        def release():
            nonlocal used
            c0 = self.clock()
            for h, need in to_free:
                self.backend.free(h)
                used -= need
            to_free.clear()
            host["free_s"] += self.clock() - c0

        while pending or waiting or active or joining or inflight or finished or to_free:
            if inflight is not None:
                read_finished()                               # overlaps the chunk
                admit(during_chunk=True)
                fut, n, resident = inflight
                c0 = self.clock()
                ms = fut.result() if asynchronous else fut
                host["wait_s"] += self.clock() - c0
                inflight = None
                for m in ms:
                    step_lat.append((float(m), resident))
                    req_step_ms.extend([float(m)] * resident)
                work += n * sum(v[0].world.n_cells for v in active.values())
                done = [rid for rid, v in active.items() if v[2] - n <= 0]
                for v in active.values():
                    v[2] -= n
                for rid in done:
                    finished.append((rid, active.pop(rid)))
                if done:
                    dirty = True
                end = self.clock()
                req_step_wall.extend([1e3 * (end - last_end) / n] * (resident * n))
                last_end = end
            release()                                         # the device is idle here
            if not asynchronous:
                read_finished()
                release()
            admit()
            if joining:
                active.update(joining)
                joining.clear()
                dirty = True
            if not active:
                read_finished()
                release()
                if batch is not None:
                    self.backend.free_batch(batch)
                    batch = None
                last_end = None
                if pending and not waiting:                   # idle until the next arrival
                    self.sleep(max(0.0, pending[0].arrival - (self.clock() - t0)))
                continue
            if dirty or batch is None:
                c0 = self.clock()
                if batch is not None:
                    self.backend.free_batch(batch)
                batch = self.backend.batch([v[1] for v in active.values()])
                dirty = False
                host["batch_s"] += self.clock() - c0
            if last_end is None:
                last_end = self.clock()
            n = min(self.chunk, min(v[2] for v in active.values()))
            if asynchronous:
                inflight = (self.backend.step_async(batch, n), n, len(active))
            else:
                inflight = (self.backend.step(batch, n), n, len(active))
        if batch is not None:
            self.backend.free_batch(batch)
        makespan = self.clock() - t0
        lat = np.array(req_step_ms) if req_step_ms else np.zeros(1)
        wall = np.array(req_step_wall) if req_step_wall else np.zeros(1)
        served = [c for c in completed if c.admitted >= 0]
        # per request: wall time from admission to its result, per step
        per_req = [1e3 * (c.finished - c.admitted) / c.steps for c in served if c.steps > 0] or [0.0]
        report = {
            "requests": len(completed), "served": len(served),
            "rejected": len(completed) - len(served),
            "makespan_s": makespan, "cell_updates": work,
            "cell_updates_per_s": work / makespan if makespan > 0 else 0.0,
            # device time of the batched step each request-step ran in
            "p50_step_device_ms": float(np.percentile(lat, 50)), "p99_step_device_ms": float(np.percentile(lat, 99)),
            # wall time per step between the ends of consecutive chunks, as each request-step saw
            # it: batch rebuilds on admission and completion, the steps and the read-back of
            # finished worlds included
            "p50_step_wall_ms": float(np.percentile(wall, 50)), "p99_step_wall_ms": float(np.percentile(wall, 99)),
            "p50_request_ms_per_step": float(np.percentile(per_req, 50)),
            "p99_request_ms_per_step": float(np.percentile(per_req, 99)),
            "batched_steps": len(step_lat),
            "mean_resident_worlds": float(np.mean([k for _, k in step_lat])) if step_lat else 0.0,
            "p50_queue_s": float(np.percentile([c.admitted - c.arrival for c in served], 50)) if served else 0.0,
            "p99_queue_s": float(np.percentile([c.admitted - c.arrival for c in served], 99)) if served else 0.0,
            "peak_resident_bytes": peak_used, "budget_bytes": self.budget, "max_worlds": self.max_worlds,
            "host_s": host,
        }
        return completed, report


def poisson_requests(n: int, rate: float, make_world, steps_range=(10, 1000), seed: int = 0):
    """n requests with exponential inter-arrival times (rate per second); make_world(rng, k)
    builds request k's world; steps uniform in steps_range."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, n, 5]))
    t = 0.0
    out = []
    for k in range(n):
        t += float(rng.exponential(1.0 / rate))
        steps = int(rng.integers(steps_range[0], steps_range[1] + 1))
        out.append(Request(t, k, make_world(rng, k), steps))
    return out

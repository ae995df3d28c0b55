"""Scheduling logic of the continuous-batching world server, on the CPU with a fake device
backend and a simulated clock: admission by memory budget in arrival order, worlds joining
and leaving the running batch, every request stepped exactly as often as it asked."""
import numpy as np

from paper_2406_09654_gb300 import serving, worlds


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t

    def sleep(self, dt):
        self.t += max(dt, 1e-6)


class FakeBackend:
    """Records batches; every step takes 1 ms per resident world of simulated time."""

    def __init__(self, clock):
        self.clock = clock
        self.steps = {}
        self.batches = []
        self.live = 0

    def create(self, world):
        self.live += 1
        self.steps[world.name] = 0
        return world

    def batch(self, handles):
        self.batches.append(sorted(h.name for h in handles))
        return list(handles)

    def step(self, batch, n):
        for h in batch:
            self.steps[h.name] += n
        self.clock.t += 1e-3 * n * len(batch)
        return np.full(n, 1.0 * len(batch), np.float32)

    def read(self, h):
        return {"steps": self.steps[h.name]}

    def free(self, h):
        self.live -= 1

    def free_batch(self, b):
        pass


def small(k, side=8):
    return worlds.make_square_world(side, 2, 32, seed=k, name=f"w{k}")


def test_every_request_is_served_with_its_step_count_and_overlaps():
    clock = FakeClock()
    be = FakeBackend(clock)
    reqs = [serving.Request(0.001 * k, k, small(k), steps=5 + 3 * k) for k in range(6)]
    srv = serving.WorldServer(be, budget_bytes=10**12, chunk_steps=2, clock=clock, sleep=clock.sleep)
    done, rep = srv.run(reqs)
    assert rep["served"] == 6 and be.live == 0
    for c in done:
        assert c.result["steps"] == reqs[c.rid].steps
    # a later request joined a batch while earlier ones were still running
    assert any(len(b) >= 3 for b in be.batches)
    assert rep["cell_updates"] == sum(r.steps * r.world.n_cells for r in reqs)


def test_budget_admission_in_arrival_order():
    clock = FakeClock()
    be = FakeBackend(clock)
    one = serving.world_bytes(small(0).n_cells, 2, 32)
    reqs = [serving.Request(0.0, k, small(k), steps=4) for k in range(4)]
    srv = serving.WorldServer(be, budget_bytes=2 * one, chunk_steps=4, clock=clock, sleep=clock.sleep)
    done, rep = srv.run(reqs)
    assert rep["served"] == 4 and rep["peak_resident_bytes"] <= 2 * one
    assert all(len(b) <= 2 for b in be.batches)
    order = sorted(done, key=lambda c: c.admitted)
    assert [c.rid for c in order] == [0, 1, 2, 3]
    assert order[2].admitted >= order[0].finished - 1e-12


def test_request_larger_than_budget_is_rejected_not_blocking():
    clock = FakeClock()
    be = FakeBackend(clock)
    big = worlds.make_square_world(64, 2, 32, seed=9, name="big")
    reqs = [serving.Request(0.0, 0, big, 3), serving.Request(0.0, 1, small(1), 3)]
    srv = serving.WorldServer(be, budget_bytes=serving.world_bytes(small(1).n_cells, 2, 32) + 10,
                              clock=clock, sleep=clock.sleep)
    done, rep = srv.run(reqs)
    assert rep["rejected"] == 1 and rep["served"] == 1
    assert {c.rid: c.admitted < 0 for c in done} == {0: True, 1: False}


def test_poisson_requests_are_sorted_and_seeded():
    f = worlds.request_world_factory((16, 64), (2, 10))
    a = serving.poisson_requests(12, 200.0, f, (10, 20), seed=1)
    b = serving.poisson_requests(12, 200.0, f, (10, 20), seed=1)
    assert [r.arrival for r in a] == [r.arrival for r in b]
    assert all(x.arrival < y.arrival for x, y in zip(a, b[1:]))
    assert all(16 <= r.world.width <= 64 and 10 <= r.steps <= 20 for r in a)


def test_batch_slots_bound_resident_worlds_and_queue_requests():
    clock = FakeClock()
    be = FakeBackend(clock)
    reqs = [serving.Request(0.001 * k, k, small(k), 5) for k in range(12)]
    srv = serving.WorldServer(be, budget_bytes=1 << 40, chunk_steps=2, clock=clock, sleep=clock.sleep, max_worlds=4)
    done, rep = srv.run(reqs)
    assert rep["served"] == 12 and all(len(b) <= 4 for b in be.batches)
    assert rep["p99_queue_s"] > 0 and rep["max_worlds"] == 4
    assert all(c.result["steps"] == 5 for c in done)
    assert rep["p50_step_wall_ms"] >= 0 and rep["p99_request_ms_per_step"] >= rep["p50_request_ms_per_step"]


def test_lazy_request_worlds_match_eager_ones():
    f_lazy = worlds.request_world_factory((16, 64), (2, 9), lazy=True)
    f_eager = worlds.request_world_factory((16, 64), (2, 9))
    a = serving.poisson_requests(5, 100.0, f_lazy, (3, 9), seed=2)
    b = serving.poisson_requests(5, 100.0, f_eager, (3, 9), seed=2)
    for ra, rb in zip(a, b):
        assert ra.world.n_cells == rb.world.n_cells and ra.world.capacity == rb.world.capacity
        w = ra.world.materialize()
        for k in ("E", "I", "C", "G", "R"):
            assert np.array_equal(getattr(w, k), getattr(rb.world, k))


def test_tree_voronoi_equals_plain_voronoi():
    for W, H, n, seed in [(37, 29, 5, 1), (64, 64, 60, 2), (300, 200, 256, 3), (7, 5, 35, 4), (10, 10, 1, 5)]:
        a = worlds._torus_voronoi(W, H, n, np.random.default_rng(seed))
        b = worlds._torus_voronoi_tree(W, H, n, np.random.default_rng(seed))
        assert np.array_equal(a, b)


class AsyncFakeBackend(FakeBackend):
    """step_async on a real worker thread; the step's world set is captured at submission, and
    worlds created while it runs must not be stepped by it."""

    def __init__(self, clock):
        super().__init__(clock)
        from concurrent.futures import ThreadPoolExecutor
        self.pool = ThreadPoolExecutor(max_workers=1)
        self.created_during = 0
        self.running = False

    def create(self, world):
        if self.running:
            self.created_during += 1
        return super().create(world)

    def step_async(self, batch, n):
        self.running = True
        members = list(batch)

        def run():
            for h in members:
                self.steps[h.name] += n
            return np.full(n, 1.0 * len(members), np.float32)

        fut = self.pool.submit(run)
        self.clock.t += 1e-3 * n * len(members)

        class Done:
            def done(inner):                 # a long chunk: still running until waited for
                return False

            def result(inner):
                out = fut.result()
                self.running = False
                return out
        return Done()


def test_overlapped_stepping_creates_next_worlds_during_a_chunk():
    clock = FakeClock()
    be = AsyncFakeBackend(clock)
    reqs = [serving.Request(0.0005 * k, k, small(k), steps=6 + 5 * k) for k in range(8)]
    srv = serving.WorldServer(be, budget_bytes=10**12, chunk_steps=3, clock=clock, sleep=clock.sleep)
    done, rep = srv.run(reqs)
    assert rep["served"] == 8 and be.live == 0
    for c in done:
        assert c.result["steps"] == reqs[c.rid].steps, (c.rid, c.result)
    assert be.created_during > 0
    assert rep["cell_updates"] == sum(r.steps * r.world.n_cells for r in reqs)
    assert set(rep["host_s"]) == {"create_s", "batch_s", "read_s", "free_s", "wait_s"}

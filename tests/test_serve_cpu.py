"""Scheduling logic of the served form on the CPU (no GPU, no library).

serve.Server's device calls go to a fake layer: contexts and batches that
record what they were asked to do, tensors backed by numpy, events that
complete at once.  What is checked is the host policy: admission under the
memory budget, least-recently-used eviction of idle walkers only, at most one
request of a walker per batched step, per-walker order, the deposit schedule,
and that every request completes."""
import time
import types

import numpy as np
import pytest

torch = pytest.importorskip("torch")


class FakeTensor:
    def __init__(self, shape, dtype=np.float32):
        self.a = np.zeros(shape, dtype=dtype)

    def pin_memory(self):
        return self

    def copy_(self, other, non_blocking=False):
        self.a[...] = other.a if isinstance(other, FakeTensor) else other
        return self

    def numpy(self):
        return self.a


class FakeEvent:
    def __init__(self, enable_timing=True):
        self.t = None

    def record(self, stream=None):
        self.t = time.perf_counter()

    def query(self):
        return True

    def synchronize(self):
        pass

    def elapsed_time(self, other):
        return (other.t - self.t) * 1e3


class _Ctx:
    def __enter__(self):
        return self

    def __exit__(self, *a):
        return False


def fake_torch():
    cuda = types.SimpleNamespace(Event=FakeEvent, stream=lambda s: _Ctx(), synchronize=lambda dev=None: None)
    return types.SimpleNamespace(
        cuda=cuda, float32=np.float32, float64=np.float64,
        empty=lambda shape, dtype=np.float32, device=None: FakeTensor(shape, dtype),
        zeros=lambda shape, dtype=np.float32, device=None: FakeTensor(shape, dtype),
        Tensor=FakeTensor)


class Log:
    def __init__(self):
        self.created, self.destroyed, self.steps = [], [], []


def fake_metad(log):
    class Metad:
        def __init__(self, params):
            self.params = params
            self.hills = None
            self.ctx = object()
            log.created.append(params.n_atoms)

        def load_hills(self, c, h):
            self.hills = (np.array(c), np.array(h))

        def get_hills(self):
            return self.hills

        def close(self):
            log.destroyed.append(self.params.n_atoms)

    class Batch:
        def __init__(self, ctxs):
            self.n = len(ctxs)
            self.launch_count = 0

        def set_tile(self, t):
            pass

        def step(self, pos, forces, accumulate=False, deposit=None, active=None):
            act = np.asarray(active)
            log.steps.append((act.copy(), np.asarray(deposit).copy()))
            self.launch_count += 15

        def collect(self, out):
            out[:, 0] = np.arange(out.shape[0])

        def close(self):
            pass

    return types.SimpleNamespace(Metad=Metad, Batch=Batch,
                                 metad_estimate_bytes=lambda p: 1000 * p.n_atoms)


@pytest.fixture
def serve_fake(monkeypatch):
    import paper_2510_06873_gb300.serve as serve
    log = Log()
    monkeypatch.setattr(serve, "torch", fake_torch())
    monkeypatch.setattr(serve, "_m", fake_metad(log))
    return serve, log


def walkers(serve, sizes):
    out = []
    for n in sizes:
        p = types.SimpleNamespace(n_atoms=n)
        out.append(serve.Walker(params=p, centres=np.zeros((3, 2)), heights=np.ones(3),
                                frames=[FakeTensor((n, 4)) for _ in range(2)]))
    return out


def trace(n_walkers, n_req, seed):
    g = np.random.default_rng(seed)
    arrivals = np.cumsum(g.exponential(2e-5, n_req))  # a burst: many requests queue up
    return arrivals, g.integers(0, n_walkers, n_req)


def test_every_request_completes_in_walker_order(serve_fake):
    serve, log = serve_fake
    ws = walkers(serve, [100, 200, 300, 400])
    srv = serve.Server(ws, stream=types.SimpleNamespace(device="cpu"), budget_bytes=10**12, deposit_every=3)
    arr, who = trace(4, 60, 1)
    out = srv.run(arr, who)
    srv.close()
    assert len(out.requests) == 60 and all(r.done >= 0 for r in out.requests)
    for w in range(4):
        rs = [r for r in out.requests if r.walker == w]
        assert [r.index for r in rs] == list(range(len(rs)))
        assert all(a.done <= b.done for a, b in zip(rs, rs[1:]))
        # deposits on every third request of the walker
        assert [r.deposit for r in rs] == [(k + 1) % 3 == 0 for k in range(len(rs))]
    # a batched step never carries two requests of one walker (active is a 0/1 mask)
    assert all(set(np.unique(a)) <= {0, 1} for a, _ in log.steps)
    assert sum(int(a.sum()) for a, _ in log.steps) == 60
    assert out.evictions == 0 and out.mean_batch > 1


def test_budget_admission_and_lru_eviction(serve_fake):
    serve, log = serve_fake
    sizes = [100, 200, 300, 400]
    ws = walkers(serve, sizes)
    per = [serve.walker_bytes(types.SimpleNamespace(n_atoms=n)) for n in sizes]
    budget = per[3] + per[2]  # the two largest fit together, never all four
    srv = serve.Server(ws, stream=types.SimpleNamespace(device="cpu"), budget_bytes=budget)
    arr, who = trace(4, 80, 2)
    out = srv.run(arr, who)
    # every walker's hill history survives eviction and re-admission
    for w in ws:
        hills = w.ctx.get_hills() if w.ctx is not None else w.saved
        assert hills is not None and np.array_equal(hills[1], np.ones(3))
    srv.close()
    assert out.peak_bytes <= budget
    assert out.evictions > 0
    assert len(log.created) == len(log.destroyed)  # every context created was closed
    assert all(r.done >= 0 for r in out.requests)


def test_preload_fills_the_budget_in_order(serve_fake):
    serve, log = serve_fake
    ws = walkers(serve, [100, 100, 100])
    one = serve.walker_bytes(types.SimpleNamespace(n_atoms=100))
    srv = serve.Server(ws, stream=types.SimpleNamespace(device="cpu"), budget_bytes=2 * one)
    assert srv.preload() == 2
    assert [w.ctx is not None for w in ws] == [True, True, False]
    srv.close()


def test_walker_larger_than_budget_is_refused(serve_fake):
    serve, _ = serve_fake
    with pytest.raises(ValueError):
        serve.Server(walkers(serve, [10_000]), stream=types.SimpleNamespace(device="cpu"), budget_bytes=1000)

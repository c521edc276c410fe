"""Served form: continuous batching of walker requests (serve.Server).

Walkers follow the served workload (wurtzite/liquid systems with log-uniform
atom counts, pre-deposited well-tempered hills, Poisson arrivals, a deposit
every 20 requests of a walker).  Each request's result must be the same alone
and in the mix: with resident walkers bit for bit, and within the parity
tolerances when a small memory budget forces evictions (an evicted walker's
neighbour list is rebuilt, which reorders its sums).
"""
import numpy as np
import pytest

import oracle
import synth
from parity_util import check_forces, kbdt, setup_hills

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_06873_gb300 import build
    build.build()
    d = torch.device("cuda:0")
    torch.cuda.set_stream(torch.cuda.Stream(d))
    return d


@pytest.fixture(scope="module")
def trace(dev):
    mp = synth.method_params(5)
    n_w, arrivals, walker_of = synth.served_trace(5, n_walkers=6, n_requests=150, rate_hz=20000.0, n_hi=3e4)
    systems = [synth.wurtzite_system(int(n_w[w]), cfg=5, sys=w) for w in range(len(n_w))]
    hills = []
    for s in systems:
        c = setup_hills(s, mp, 300, cfg=5)[0]
        hills.append((c, oracle.deposit_sequence(c, mp.sigma, mp.w0, kbdt(mp))))
    frames = [[torch.from_numpy(synth.perturbed_frame(s, f)).pin_memory() for f in range(3)] for s in systems]
    return mp, systems, hills, frames, arrivals, walker_of


def walkers(trace, stream):
    from paper_2510_06873_gb300 import metad, serve
    mp, systems, hills, frames, _, _ = trace
    out = []
    for s, (c, w), fr in zip(systems, hills, frames):
        p = metad.params_for(s.n, s.box, n_cv=2, sigma=mp.sigma, stream=stream.cuda_stream, hill_capacity=4096)
        out.append(serve.Walker(params=p, centres=c, heights=w, frames=fr))
    return out


def alone(trace, stream, dev):
    """Each walker's requests in its own order, one context per walker."""
    from paper_2510_06873_gb300 import metad
    mp, systems, hills, frames, arrivals, walker_of = trace
    res = {}
    with torch.cuda.stream(stream):
        for w, s in enumerate(systems):
            p = metad.params_for(s.n, s.box, n_cv=2, sigma=mp.sigma, stream=stream.cuda_stream, hill_capacity=4096)
            ctx = metad.Metad(p)
            ctx.load_hills(*hills[w])
            pos = torch.empty((s.n, 4), dtype=torch.float32, device=dev)
            F = torch.empty((s.n, 3), dtype=torch.float32, device=dev)
            count = int(np.sum(walker_of == w))
            for k in range(count):
                pos.copy_(frames[w][k % 3])
                ctx.step(pos, F, deposit=((k + 1) % 20 == 0))
                cv, V, _ = ctx.read_results()
                res[(w, k)] = (np.array(cv), V, F.cpu().numpy())
            ctx.close()
    return res


def test_served_results_equal_alone(dev, trace):
    from paper_2510_06873_gb300 import serve
    stream = torch.cuda.current_stream(dev)
    _, systems, _, _, arrivals, walker_of = trace
    srv = serve.Server(walkers(trace, stream), stream, budget_bytes=10**12, keep_forces=True)
    out = srv.run(arrivals, walker_of)
    srv.close()
    ref = alone(trace, stream, dev)
    assert len(out.requests) == len(arrivals)
    assert out.mean_batch > 1.0, "requests were never batched"
    for r in out.requests:
        cv, V, F = ref[(r.walker, r.index)]
        assert r.err == 0
        assert np.array_equal(r.cv, cv) and r.V == V, (r.walker, r.index)
        assert np.array_equal(r.forces, F), (r.walker, r.index)
    s = out.summary()
    assert 0 < s["p50_ms"] <= s["p99_ms"]
    assert out.evictions == 0


def test_plain_baseline_gives_the_same_results(dev, trace):
    from paper_2510_06873_gb300 import serve
    stream = torch.cuda.current_stream(dev)
    _, _, _, _, arrivals, walker_of = trace
    ws = walkers(trace, stream)
    out = serve.run_plain(ws, stream, arrivals, walker_of, keep_forces=True)
    for wk in ws:
        wk.ctx.close()
    ref = alone(trace, stream, dev)
    for r in out.requests:
        cv, V, F = ref[(r.walker, r.index)]
        assert np.array_equal(r.cv, cv) and r.V == V and np.array_equal(r.forces, F)


def test_small_budget_admission_and_eviction(dev, trace):
    from paper_2510_06873_gb300 import serve
    stream = torch.cuda.current_stream(dev)
    _, systems, _, _, arrivals, walker_of = trace
    ws = walkers(trace, stream)
    sizes = sorted(serve.walker_bytes(w.params) for w in ws)
    budget = sizes[-1] + sizes[-2] + sizes[0]  # never all six walkers at once
    srv = serve.Server(ws, stream, budget_bytes=budget, keep_forces=True)
    out = srv.run(arrivals, walker_of)
    srv.close()
    assert out.peak_bytes <= budget
    assert out.evictions > 0
    assert len(out.requests) == len(arrivals) and all(r.done > 0 for r in out.requests)
    by_walker = {}
    for r in out.requests:
        by_walker.setdefault(r.walker, []).append(r)
    for rs in by_walker.values():
        rs.sort(key=lambda r: r.index)
        assert all(a.done <= b.done for a, b in zip(rs, rs[1:])), "a walker's requests finished out of order"
    ref = alone(trace, stream, dev)
    for r in out.requests:
        cv, V, F = ref[(r.walker, r.index)]
        assert np.all(np.abs(r.cv - cv) <= 1e-6 * np.abs(cv))
        check_forces(r.forces.astype(np.float64), F.astype(np.float64))


def test_walker_larger_than_budget_is_refused(dev, trace):
    from paper_2510_06873_gb300 import serve
    stream = torch.cuda.current_stream(dev)
    ws = walkers(trace, stream)
    with pytest.raises(ValueError):
        serve.Server(ws, stream, budget_bytes=1024)


def test_served_requests_match_the_oracle(dev):
    """Served requests against the FP64 oracle at the parity tolerances.

    Three walkers of the served workload's construction: the largest and the
    smallest walker of the 32-walker trace (2k-500k atoms, log-uniform) and a
    mid-sized one, with the trace's arrival process (Poisson) restricted to
    them.  A hill is deposited every 5 requests of a walker (at that
    request's CVs), so sampled requests of the largest walker come both
    before and after deposits; the oracle carries the same hill history,
    each deposit's centre the CUDA path's CVs and its well-tempered height
    the oracle's own."""
    from paper_2510_06873_gb300 import metad, serve
    from parity_util import check_cv
    stream = torch.cuda.current_stream(dev)
    mp = synth.method_params(5)
    cfgp = synth.CONFIG_PARAMS[5]
    n_all, _, _ = synth.served_trace(5, n_walkers=cfgp["walkers"], n_requests=cfgp["requests"],
                                     rate_hz=cfgp["rate_hz"])
    order = np.argsort(n_all)
    pick = [int(order[-1]), int(order[len(order) // 2]), int(order[0])]
    assert n_all[pick[0]] >= 200_000
    systems = [synth.wurtzite_system(int(n_all[w]), cfg=5, sys=w) for w in pick]
    g = np.random.default_rng(55)
    n_req = 36
    walker_of = np.array([0] * 16 + [1] * 12 + [2] * 8)
    g.shuffle(walker_of)
    arrivals = np.cumsum(g.exponential(1.0 / cfgp["rate_hz"], n_req))
    every = 5
    hills, frames = [], []
    for s in systems:
        c = setup_hills(s, mp, 400, cfg=5)[0]
        hills.append((c, oracle.deposit_sequence(c, mp.sigma, mp.w0, kbdt(mp))))
        frames.append([torch.from_numpy(synth.perturbed_frame(s, f)).pin_memory() for f in range(3)])
    ws = []
    for s, (c, w), fr in zip(systems, hills, frames):
        p = metad.params_for(s.n, s.box, n_cv=2, sigma=mp.sigma, stream=stream.cuda_stream, hill_capacity=4096)
        ws.append(serve.Walker(params=p, centres=c, heights=w, frames=fr))
    srv = serve.Server(ws, stream, budget_bytes=10**12, deposit_every=every, keep_forces=True)
    out = srv.run(arrivals, walker_of)
    srv.close()
    by = {}
    for r in out.requests:
        by.setdefault(r.walker, []).append(r)
    for w, rs in by.items():
        rs.sort(key=lambda r: r.index)
        s = systems[w]
        p = oracle.params_from(mp, s.box)
        live_c, live_w = hills[w][0].copy(), hills[w][1].copy()
        sample = {0, 1, every - 1, every, every + 1, 2 * every + 1, len(rs) - 1} if w == 0 else {0, len(rs) - 1}
        for r in rs:
            if r.index in sample:
                frame = synth.perturbed_frame(s, r.index % 3)
                ref = oracle.step(frame, p, live_c, live_w, mp.sigma)
                check_cv(r.cv, ref["s"])
                assert abs(r.V - ref["V"]) <= 1e-5 * max(abs(ref["V"]), mp.w0), (w, r.index, r.V, ref["V"])
                check_forces(r.forces.astype(np.float64), ref["F"])
            if (r.index + 1) % every == 0:
                # the oracle's own chain: its hill at its own CVs of that frame
                frame = synth.perturbed_frame(s, r.index % 3)
                s_ref = oracle.cv(frame, p)[0]
                h = oracle.deposit_sequence(np.vstack([live_c, s_ref[None, :]]), mp.sigma, mp.w0, kbdt(mp),
                                            heights_prefix=live_w)[-1]
                live_c = np.vstack([live_c, s_ref[None, :]])
                live_w = np.append(live_w, h)
    assert len(by[0]) == 16 and sum(1 for r in by[0] if (r.index + 1) % every == 0) == 3

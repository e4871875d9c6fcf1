"""Serving (continuous batching): every result equals the oracle's and the
same query run alone.

Queries arrive in bursts while others are on the device; a small memory
budget forces memory-gated admission.  The bar is bit-exact equality of every
served level[] and parent[] with the CPU oracle (the result definition of
Theorem 1: hop distance and least-index parent), and with abfs_run of the same
query on the same GPU."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")

import paper_1906_03113_gb300 as abfs  # noqa: E402
from paper_1906_03113_gb300 import binding  # noqa: E402


def test_default_cfg_and_argument_checks():
    abfs.build()
    c = abfs.serve_default_cfg()
    assert c.max_slots >= 1 and c.queue_capacity >= 1 and c.memory_budget > 0
    assert c.idle_exit_ms >= 1 and c.params.unit_entries >= 256
    lib = abfs.load()
    import ctypes
    out = ctypes.c_void_p()
    assert lib.abfs_serve_start(None, 0, None, ctypes.byref(out)) == binding.ERR_INVALID_ARG
    assert lib.abfs_serve_stop(None, None) == binding.ERR_INVALID_ARG


@pytest.fixture(scope="module")
def graphs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    abfs.build()
    abfs.load()
    torch.cuda.set_device(0)
    gs = [synth.er_2_16(), synth.rmat(14, 16.0, seed=3), synth.grid(100, 37),
          synth.rgg_knn(1 << 15, 4, seed=4), synth.rmat(16, 8.0, seed=9)]
    dev = [abfs.graph_create(g.colptr, g.rowidx, directed=g.directed) for g in gs]
    yield gs, dev
    for G in dev:
        G.destroy()


def _queries(gs, count, seed):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        gi = int(rng.integers(len(gs)))
        deg = gs[gi].degrees()
        cand = np.nonzero(deg > 0)[0]
        out.append((gi, int(cand[rng.integers(cand.size)])))
    return out


def _serve_and_check(gs, dev, queries, cfg, bursts):
    srv = abfs.Server(dev, cfg)
    outs = []
    tickets = []
    per = (len(queries) + bursts - 1) // bursts
    for b in range(bursts):
        for gi, s in queries[b * per:(b + 1) * per]:
            lev = torch.empty(gs[gi].n, dtype=torch.int32, device="cuda")
            par = torch.empty(gs[gi].n, dtype=torch.int32, device="cuda")
            t = srv.submit(gi, s, lev, par)
            assert t is not None
            tickets.append(t)
            outs.append((gi, s, lev, par))
        if b == 0:
            # later bursts arrive while the first ones are on the device
            srv.poll(tickets[0])
    for t in tickets:
        assert srv.wait(t, 60000) == 0
    rep = srv.stop()
    assert rep["completed"] == len(queries) == rep["submitted"] and rep["failed"] == 0
    assert rep["launches"] >= 1 and 0 < rep["p50_ms"] <= rep["p99_ms"] <= rep["max_ms"]
    torch.cuda.synchronize()
    expect = {}
    for gi, s, lev, par in outs:
        if (gi, s) not in expect:
            expect[(gi, s)] = oracle.bfs(gs[gi], s)
        lo, po = expect[(gi, s)]
        lev_h, par_h = lev.cpu().numpy(), par.cpu().numpy()
        bad = np.nonzero(lev_h != lo)[0]
        assert bad.size == 0, f"served level != oracle: graph {gi} src {s} at {bad[:8]}"
        bad = np.nonzero(par_h != po)[0]
        assert bad.size == 0, f"served parent != oracle: graph {gi} src {s} at {bad[:8]}"
        la, pa = abfs.run(dev[gi], s)
        assert torch.equal(la, lev) and torch.equal(pa, par), (gi, s)
    return rep


@pytest.mark.gpu
def test_serve_mix_equals_alone(graphs):
    gs, dev = graphs
    cfg = abfs.serve_default_cfg(max_slots=32, memory_budget=2 << 30, idle_exit_ms=20)
    _serve_and_check(gs, dev, _queries(gs, 300, 1), cfg, bursts=6)


@pytest.mark.gpu
def test_serve_on_relabelled_graphs(graphs):
    """Served queries on graphs that carry a relabelled copy run on the input
    numbering; abfs_run of the same query runs on the copy; both equal the
    oracle."""
    gs, _ = graphs
    sub = [gs[1], gs[3], gs[4]]
    dev = [abfs.graph_create(g.colptr, g.rowidx, directed=g.directed) for g in sub]
    for G in dev:
        abfs.graph_relabel(G)
    cfg = abfs.serve_default_cfg(max_slots=16, memory_budget=2 << 30, idle_exit_ms=20)
    _serve_and_check(sub, dev, _queries(sub, 60, 5), cfg, bursts=3)
    for G in dev:
        G.destroy()


@pytest.mark.gpu
def test_serve_memory_gated_admission(graphs):
    gs, dev = graphs
    # a budget that holds only one or two queries of the largest graph at a time
    big = max(G.footprint() for G in dev)
    cfg = abfs.serve_default_cfg(max_slots=64, memory_budget=int(big * 2.2), idle_exit_ms=5)
    _serve_and_check(gs, dev, _queries(gs, 80, 2), cfg, bursts=3)


@pytest.mark.gpu
def test_serve_queue_full_is_busy(graphs):
    gs, dev = graphs
    cfg = abfs.serve_default_cfg(max_slots=1, queue_capacity=2, memory_budget=1 << 30)
    srv = abfs.Server(dev, cfg)
    bufs = [(torch.empty(gs[0].n, dtype=torch.int32, device="cuda"),
             torch.empty(gs[0].n, dtype=torch.int32, device="cuda")) for _ in range(64)]
    results = [srv.submit(0, 0, lv, pr) for lv, pr in bufs]
    assert any(r is None for r in results)          # some were refused: queue full
    for t in results:
        if t is not None:
            assert srv.wait(t, 60000) == 0
    rep = srv.stop()
    assert rep["completed"] == sum(r is not None for r in results)
    torch.cuda.synchronize()
    lo, po = oracle.bfs(gs[0], 0)
    for t, (lv, pr) in zip(results, bufs):
        if t is not None:
            assert np.array_equal(lv.cpu().numpy(), lo) and np.array_equal(pr.cpu().numpy(), po)


@pytest.mark.gpu
def test_serve_slot_reuse_under_churn():
    """Many short searches through few slots: each slot is reused hundreds of
    times while other CTAs still look at it, and every result still equals the
    oracle's and the query run alone."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    abfs.build()
    gs = [synth.er(3000, 4.0, seed=21), synth.grid(40, 25), synth.rgg_knn(4096, 4, seed=22),
          synth.rmat(12, 8.0, seed=23)]
    dev = [abfs.graph_create(g.colptr, g.rowidx, directed=g.directed) for g in gs]
    try:
        for trial in range(3):
            cfg = abfs.serve_default_cfg(max_slots=4 + 4 * trial, memory_budget=1 << 30,
                                         idle_exit_ms=20)
            _serve_and_check(gs, dev, _queries(gs, 1500, 30 + trial), cfg, bursts=5)
    finally:
        for G in dev:
            G.destroy()

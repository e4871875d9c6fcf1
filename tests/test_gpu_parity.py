"""Parity of the CUDA path (through the C-ABI) with the CPU oracle.

Levels and min-index parents are integers: the bar is bit-exact equality,
element by element, for every mode, parameter set and batch mix.
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1906_03113_gb300 as abfs  # noqa: E402

SUB = abfs.MODE_SUBMATRIX
PLAIN = abfs.MODE_PLAIN


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    abfs.build()
    abfs.load()
    torch.cuda.set_device(0)


def _check(g, src, level, parent, ctx=""):
    lev_o, par_o = oracle.bfs(g, src)
    lev = level.cpu().numpy() if hasattr(level, "cpu") else level
    par = parent.cpu().numpy() if hasattr(parent, "cpu") else parent
    bad = np.nonzero(lev != lev_o)[0]
    assert bad.size == 0, f"{ctx}: level mismatch at {bad[:8]} ({lev[bad[:8]]} vs {lev_o[bad[:8]]})"
    bad = np.nonzero(par != par_o)[0]
    assert bad.size == 0, f"{ctx}: parent mismatch at {bad[:8]} ({par[bad[:8]]} vs {par_o[bad[:8]]})"
    return lev_o


def _e_adj(g, lev):
    cols = np.repeat(np.arange(g.n), g.degrees())
    lj = lev[cols]
    li = lev[g.rowidx.astype(np.int64)]
    return int(((lj >= 0) & (li == lj + 1)).sum())


def _params(mode=SUB, **kw):
    return abfs.default_params(mode=mode, **kw)


MODES = [
    ("sub", dict(mode=SUB)),
    ("plain", dict(mode=PLAIN)),
    ("sub_shrink", dict(mode=SUB, shrink_theta=0.3, shrink_max=3)),
    ("sub_small_units", dict(mode=SUB, tile=32, narrow_max=0, narrow_edges=0, unit_entries=256)),
    ("plain_small_units", dict(mode=PLAIN, tile=64, narrow_max=32, narrow_edges=256,
                               unit_entries=512)),
    ("sub_narrow_all", dict(mode=SUB, tile=1024, narrow_max=1 << 30, narrow_edges=1 << 30)),
    ("sub_wide_all", dict(mode=SUB, tile=256, narrow_max=0, narrow_edges=0, ctas_per_sm=1)),
    ("sub_shrink_every", dict(mode=SUB, tile=128, narrow_max=0, narrow_edges=0, shrink_theta=0.05,
                              shrink_max=20, unit_entries=1024)),
    # narrow levels through the block bookkeeping instead of resident runs
    ("sub_narrow_blocks", dict(mode=SUB, narrow_resident=0)),
    ("plain_narrow_blocks", dict(mode=PLAIN, narrow_resident=0)),
    # resident runs over whole searches: small chunks, several slot windows
    ("sub_resident_all", dict(mode=SUB, tile=64, narrow_max=1 << 30, narrow_edges=1 << 30)),
    ("plain_resident_all", dict(mode=PLAIN, tile=96, narrow_max=1 << 30, narrow_edges=1 << 30)),
    # resident runs interrupted by shrinks (matrix switches inside and between runs)
    ("sub_resident_shrink", dict(mode=SUB, tile=64, narrow_max=1 << 30, narrow_edges=1 << 30,
                                 shrink_theta=0.05, shrink_max=20)),
    # every wide level claims by reductions and a bitmap scan
    ("sub_scan_all", dict(mode=SUB, tile=256, narrow_max=0, narrow_edges=0, claim_scan=1,
                          unit_entries=512)),
    ("sub_scan_shrink", dict(mode=SUB, narrow_max=64, narrow_edges=1024, claim_scan=1,
                             shrink_theta=0.1, shrink_max=8)),
    ("sub_no_scan", dict(mode=SUB, claim_scan=0)),
    # frequent narrow <-> wide transitions
    ("sub_resident_mixed", dict(mode=SUB, tile=128, narrow_max=300, narrow_edges=3000,
                                unit_entries=512)),
    # hybrid: bottom-up levels by the usual thresholds, on every level after the
    # first, and alternating with top-down ones (every kind of hand-over)
    ("sub_hybrid", dict(mode=SUB, bottom_up_alpha=14, bottom_up_beta=24)),
    ("sub_hybrid_always", dict(mode=SUB, bottom_up_alpha=0xFFFFFFFF, bottom_up_beta=0xFFFFFFFF)),
    ("sub_hybrid_alternate", dict(mode=SUB, bottom_up_alpha=0xFFFFFFFF, bottom_up_beta=0,
                                  narrow_max=0, narrow_edges=0, unit_entries=256)),
    ("sub_hybrid_scan", dict(mode=SUB, bottom_up_alpha=0xFFFFFFFF, bottom_up_beta=0, claim_scan=1,
                             narrow_max=0, narrow_edges=0)),
]

# cluster runs: none (single-CTA narrow runs), other cluster sizes, whole
# searches in cluster runs, frequent run <-> wide transitions, the comparator's
# two steps per level, shrinks ending runs, several chunks per member
MODES += [
    ("sub_no_cluster", dict(mode=SUB, cluster_ctas=1)),
    ("plain_no_cluster", dict(mode=PLAIN, cluster_ctas=1)),
    ("sub_cluster2", dict(mode=SUB, cluster_ctas=2)),
    ("sub_cluster4_all", dict(mode=SUB, cluster_ctas=4, cluster_min=0, cluster_max=1 << 30,
                              cluster_edges=1 << 30)),
    ("sub_cluster8_all", dict(mode=SUB, cluster_ctas=8, cluster_min=0, cluster_max=1 << 30,
                              cluster_edges=1 << 30)),
    ("sub_cluster16_all", dict(mode=SUB, cluster_ctas=16, cluster_min=0, cluster_max=1 << 30,
                               cluster_edges=1 << 30)),
    ("sub_cluster16_one_per_sm", dict(mode=SUB, cluster_ctas=16, ctas_per_sm=1)),
    ("plain_cluster_all", dict(mode=PLAIN, cluster_min=0, cluster_max=1 << 30,
                               cluster_edges=1 << 30)),
    ("sub_cluster_mixed", dict(mode=SUB, cluster_min=64, cluster_max=300, cluster_edges=3000,
                               narrow_max=40, narrow_edges=400, unit_entries=512)),
    ("plain_cluster_mixed", dict(mode=PLAIN, cluster_min=64, cluster_max=300, cluster_edges=3000,
                                 narrow_max=40, narrow_edges=400)),
    ("sub_cluster_shrink", dict(mode=SUB, tile=64, cluster_min=0, cluster_max=1 << 30,
                                cluster_edges=1 << 30, shrink_theta=0.05, shrink_max=20)),
    ("sub_cluster_small_tile", dict(mode=SUB, tile=32, cluster_min=0, cluster_max=1 << 30,
                                    cluster_edges=1 << 30)),
]

HYBRID = ("sub_hybrid", "sub_hybrid_always", "sub_hybrid_alternate", "sub_hybrid_scan")


def _small_graphs():
    star_leaves = 20000
    return {
        "fig1_path": synth.from_arcs(5, [0, 1, 2, 2], [3, 4, 3, 4], directed=False),
        "er_2000": synth.er(2000, 3.0, seed=2),
        "er_2_16": synth.er_2_16(),
        "rmat_14": synth.rmat(14, 16.0, seed=3),
        "grid_100x37": synth.grid(100, 37),
        "grid_1x1000": synth.grid(1, 1000),
        "rgg_2_15": synth.rgg_knn(1 << 15, 4, seed=4),
        "star": synth.from_arcs(star_leaves + 1, [0] * star_leaves, list(range(1, star_leaves + 1)),
                                directed=False),
        "path_3000": synth.from_arcs(3000, list(range(2999)), list(range(1, 3000)), directed=False),
        "complete_200": synth.from_arcs(200, [i for i in range(200) for j in range(i + 1, 200)],
                                        [j for i in range(200) for j in range(i + 1, 200)], directed=False),
        "dicycle_777": synth.from_arcs(777, list(range(777)), [(i + 1) % 777 for i in range(777)],
                                       directed=True),
        "two_components": synth.from_arcs(100, list(range(49)) + list(range(50, 99)),
                                          list(range(1, 50)) + list(range(51, 100)), directed=False),
        "no_edges": synth.from_arcs(77, [], [], directed=False),
        # one vertex; a path ending just past a bitmap word (ragged last word)
        "one_vertex": synth.from_arcs(1, [], [], directed=False),
        "path_33": synth.from_arcs(33, list(range(32)), list(range(1, 33)), directed=False),
    }


@pytest.fixture(scope="module")
def small():
    gs = _small_graphs()
    dev = {k: abfs.graph_create(g.colptr, g.rowidx, directed=g.directed, validate=True)
           for k, g in gs.items()}
    yield gs, dev
    for G in dev.values():
        G.destroy()


def _sources(g):
    deg = g.degrees()
    cand = [0, g.n - 1, int(np.argmax(deg)), g.n // 2]
    nz = np.nonzero(deg > 0)[0]
    if nz.size:
        cand.append(int(nz[len(nz) // 3]))
    return sorted(set(int(c) for c in cand))


@pytest.mark.parametrize("mode_name,kw", MODES, ids=[m[0] for m in MODES])
def test_small_graphs_all_modes(small, mode_name, kw):
    gs, dev = small
    p = _params(**kw)
    for name, g in gs.items():
        for s in _sources(g):
            level, parent, st = abfs.run(dev[name], s, params=p, stats=True)
            torch.cuda.synchronize()
            assert st["status"] == 0, (name, s, st)
            lev_o = _check(g, s, level, parent, f"{mode_name}/{name}/src{s}")
            reached = lev_o >= 0
            assert st["reached"] == int(reached.sum()), (name, s, st)
            assert st["levels"] == int(lev_o.max()) + 1, (name, s, st)
            nnz_c = int(g.degrees()[reached].sum())
            assert st["nnz_reached"] == nnz_c, (name, s, st)
            if mode_name in HYBRID:
                # bottom-up levels read rows until the first frontier entry:
                # the entry counters of Claim 1 and E_adj do not apply
                continue
            if kw.get("mode") == PLAIN:
                assert st["entries_read"] == nnz_c and st["entries_unmasked"] == nnz_c
            else:
                # rows that pass the mask are exactly the entries j -> i with
                # level(i) = level(j) + 1 (E_adj): the multiplies of Theorem 1
                assert st["entries_unmasked"] == _e_adj(g, lev_o), (name, s, st)
            if kw.get("mode") == PLAIN:
                pass
            elif not kw.get("shrink_theta"):
                # each reached column is read exactly once (Claim 1)
                assert st["entries_read"] == nnz_c, (name, s, st)
                assert st["entries_unmasked"] <= nnz_c
            else:
                assert st["entries_read"] <= nnz_c


def test_fig1_frontiers_through_gpu(small):
    gs, dev = small
    level, parent = abfs.run(dev["fig1_path"], 1)
    assert level.cpu().tolist() == [4, 0, 2, 3, 1]
    assert parent.cpu().tolist() == [3, 1, 4, 2, 1]


def test_invalid_source_rejected(small):
    gs, dev = small
    with pytest.raises(abfs.AbfsError) as ei:
        abfs.run(dev["er_2000"], 2000)
    assert ei.value.status == 1


def test_run_host_matches(small):
    gs, dev = small
    g = gs["rmat_14"]
    s = _sources(g)[-1]
    lev_h, par_h = abfs.run_host(dev["rmat_14"], s)
    _check(g, s, lev_h, par_h, "run_host")


RELABEL = ["rmat_14", "er_2000", "grid_100x37", "rgg_2_15", "star", "path_3000", "no_edges"]


@pytest.mark.parametrize("name", RELABEL)
def test_relabelled_graph_all_modes(small, name):
    """A graph relabelled by column-length class (abfs_graph_relabel): every
    mode equals the oracle in the input's labels -- the submatrix searches run
    on the copy (wide, reduction, resident, cluster and shrink paths), the
    comparator, the hybrid, path counts and batches keep the input numbering."""
    gs, _ = small
    g = gs[name]
    G = abfs.graph_create(g.colptr, g.rowidx, directed=g.directed)
    abfs.graph_relabel(G)
    abfs.graph_relabel(G)  # a second call changes nothing
    for mode_name, kw in MODES:
        p = _params(**kw)
        for s in _sources(g):
            level, parent, st = abfs.run(G, s, params=p, stats=True)
            assert st["status"] == 0, (name, mode_name, s)
            _check(g, s, level, parent, f"relabelled {name} {mode_name} src{s}")
    s = _sources(g)[-1]
    lev_h, par_h = abfs.run_host(G, s)
    _check(g, s, lev_h, par_h, f"relabelled {name} run_host")
    lev, par, st = abfs.run_host_many(G, _sources(g))
    assert st == [0] * len(_sources(g))
    for i, s in enumerate(_sources(g)):
        _check(g, s, lev[i], par[i], f"relabelled {name} run_host_many #{i}")
    level, parent, sigma = abfs.run_counts(G, s)
    _check(g, s, level, parent, f"relabelled {name} counts")
    assert np.array_equal(sigma.cpu().numpy().view(np.uint64), oracle.path_counts(g, s))
    level, parent, tr = abfs.run_trace(G, s)
    _check(g, s, level, parent, f"relabelled {name} trace")
    best, _ = abfs.tune(G, _sources(g)[:2])
    level, parent = abfs.run(G, s)
    _check(g, s, level, parent, f"relabelled {name} tuned")
    srcs = _sources(g)
    levels, parents, st = abfs.run_batch([G] * len(srcs), srcs)
    torch.cuda.synchronize()
    assert all(x == 0 for x in st), st
    for i, s in enumerate(srcs):
        _check(g, s, levels[i], parents[i], f"relabelled {name} batch #{i}")
    G.destroy()


def test_run_host_many_matches(small):
    """Many searches into host memory: two device buffers alternate and each
    search's outputs are copied out while the next one runs, so the third and
    fourth searches reuse buffers whose copies had to finish first."""
    gs, dev = small
    for name in ("rmat_14", "rgg_2_15"):
        g = gs[name]
        base = _sources(g)
        srcs = [base[0], base[-1], base[1 % len(base)], base[0], base[-1]]
        for count in (1, 2, len(srcs)):
            lev = torch.full((count, g.n), 7, dtype=torch.int32).pin_memory()
            par = torch.full((count, g.n), 7, dtype=torch.int32).pin_memory()
            _, _, st = abfs.run_host_many(dev[name], srcs[:count], lev, par)
            assert st == [0] * count, st
            for i, s in enumerate(srcs[:count]):
                _check(g, s, lev[i], par[i], f"run_host_many {name} {count} #{i}")
    # pageable host arrays work too (the copies then do not overlap)
    g = gs["rmat_14"]
    base = _sources(g)
    lev, par, st = abfs.run_host_many(dev["rmat_14"], base[:3])
    assert st == [0, 0, 0]
    for i, s in enumerate(base[:3]):
        _check(g, s, lev[i], par[i], "run_host_many pageable")
    with pytest.raises(abfs.AbfsError) as ei:
        abfs.run_host_many(dev["rmat_14"], [0, g.n])
    assert ei.value.status == 1


def test_repeated_runs_identical(small):
    gs, dev = small
    g = gs["rmat_14"]
    s = int(np.argmax(g.degrees()))
    ref = None
    for _ in range(5):
        level, parent = abfs.run(dev["rmat_14"], s)
        cur = (level.cpu().numpy().copy(), parent.cpu().numpy().copy())
        _check(g, s, cur[0], cur[1], "repeated run")
        if ref is not None:
            assert np.array_equal(ref[0], cur[0]) and np.array_equal(ref[1], cur[1])
        ref = cur


def test_exhaustive_tiny_graphs_in_one_batch():
    """Every directed graph on 4 vertices and every undirected graph on 5,
    from every source, as instances of persistent batch launches."""
    jobs = []
    for n, directed in ((4, True), (5, False)):
        pairs = ([(i, j) for i in range(n) for j in range(n) if i != j] if directed
                 else [(i, j) for i in range(n) for j in range(i + 1, n)])
        for mask in range(1 << len(pairs)):
            arcs = [pairs[b] for b in range(len(pairs)) if mask >> b & 1]
            g = synth.from_arcs(n, [a for a, _ in arcs], [b for _, b in arcs], directed=directed)
            jobs.append(g)
    for mode in (SUB, PLAIN):
        dev = [abfs.graph_create(g.colptr, g.rowidx, directed=g.directed) for g in jobs]
        graphs, srcs, hosts = [], [], []
        for G, g in zip(dev, jobs):
            for s in range(g.n):
                graphs.append(G)
                srcs.append(s)
                hosts.append(g)
        levels, parents, st = abfs.run_batch(graphs, srcs, params=_params(mode=mode, tile=32,
                                                                           unit_entries=256))
        torch.cuda.synchronize()
        assert all(x == 0 for x in st)
        for g, s, L, P in zip(hosts, srcs, levels, parents):
            _check(g, s, L, P, f"tiny mode{mode}")
        for G in dev:
            G.destroy()


def test_batch_alone_equals_mix(small):
    gs, dev = small
    names = ["er_2_16", "rmat_14", "grid_100x37", "rgg_2_15", "star", "path_3000", "no_edges"]
    graphs, srcs, hosts = [], [], []
    for nm in names:
        for s in _sources(gs[nm])[:3]:
            graphs.append(dev[nm])
            srcs.append(s)
            hosts.append(gs[nm])
    for kw in (dict(mode=SUB), dict(mode=PLAIN), dict(mode=SUB, shrink_theta=0.4, shrink_max=2),
               dict(mode=SUB, bottom_up_alpha=5, bottom_up_beta=24),
               dict(mode=SUB, bottom_up_alpha=0xFFFFFFFF, bottom_up_beta=0)):
        p = _params(**kw)
        levels, parents, st = abfs.run_batch(graphs, srcs, params=p)
        torch.cuda.synchronize()
        assert all(x == 0 for x in st), st
        for G, g, s, L, P in zip(graphs, hosts, srcs, levels, parents):
            la, pa = abfs.run(G, s, params=p)
            assert torch.equal(la, L) and torch.equal(pa, P), (g.name, s, kw)
            _check(g, s, L, P, f"batch {kw}")


def test_batch_plan_replays(small):
    gs, dev = small
    graphs = [dev["rmat_14"], dev["er_2_16"], dev["grid_100x37"]]
    hosts = [gs["rmat_14"], gs["er_2_16"], gs["grid_100x37"]]
    srcs = [int(np.argmax(h.degrees())) for h in hosts]
    plan = abfs.BatchPlan(graphs, srcs)
    for rep in range(3):
        for L in plan.levels:
            L.fill_(7)
        plan.launch()
        assert plan.status() == [0, 0, 0]
        for g, s, L, P in zip(hosts, srcs, plan.levels, plan.parents):
            _check(g, s, L, P, f"plan replay {rep}")
    plan.destroy()


def test_tune_keeps_results(small, tmp_path):
    gs, dev = small
    g = gs["rmat_14"]
    srcs = _sources(g)[:2]
    cache = str(tmp_path / "tune.json")
    best, ms = abfs.tune(dev["rmat_14"], srcs, SUB, cache)
    assert ms > 0 and best.tile >= 32
    best2, ms2 = abfs.tune(dev["rmat_14"], srcs, SUB, cache)   # from the cache
    assert best2.as_dict() == best.as_dict()
    level, parent = abfs.run(dev["rmat_14"], srcs[0])          # uses the tuned params
    _check(g, srcs[0], level, parent, "tuned")
    # tuning the comparator leaves the graph's default (submatrix) set alone:
    # without params a search still masks before it multiplies
    abfs.tune(dev["rmat_14"], srcs, PLAIN)
    level, parent, st = abfs.run(dev["rmat_14"], srcs[0], stats=True)
    _check(g, srcs[0], level, parent, "tuned after a comparator tune")
    assert st["entries_unmasked"] < st["entries_read"], st


def test_batch_tune_picks_a_valid_set(small, tmp_path):
    gs, dev = small
    names = ["er_2000", "rmat_14", "grid_100x37", "rgg_2_15"]
    graphs = [dev[n] for n in names]
    srcs = [_sources(gs[n])[0] for n in names]
    cache = str(tmp_path / "batch_tune.json")
    best, ms = abfs.batch_tune(graphs, srcs, SUB, cache)
    assert ms > 0 and best.unit_entries in (512, 1024, 4096)
    best2, _ = abfs.batch_tune(graphs, srcs, SUB, cache)   # from the cache
    assert best2.as_dict() == best.as_dict()
    plan = abfs.BatchPlan(graphs, srcs, params=best)
    plan.launch()
    assert plan.status() == [0] * len(names)
    for n, s, L, P in zip(names, srcs, plan.levels, plan.parents):
        _check(gs[n], s, L, P, f"tuned batch {n}")
    plan.destroy()


def _kinds(trace):
    return {r["kind"] for r in trace}


def test_hybrid_runs_bottom_up_only_where_allowed():
    """Bottom-up levels appear on an undirected graph with ascending columns and
    not on the same graph with shuffled columns, nor on a directed graph, nor
    when path counts are requested; every result equals the oracle's."""
    p = _params(bottom_up_alpha=0xFFFFFFFF, bottom_up_beta=0xFFFFFFFF)
    g = synth.rmat(14, 16.0, seed=3)
    s = int(np.argmax(g.degrees()))
    G = abfs.graph_create(g.colptr, g.rowidx, directed=False)
    level, parent, trace = abfs.run_trace(G, s, params=p)
    assert "bottom_up" in _kinds(trace)
    _check(g, s, level, parent, "sorted hybrid")
    level, parent, sigma = abfs.run_counts(G, s, params=p)
    _check(g, s, level, parent, "hybrid with counts")
    assert np.array_equal(sigma.cpu().numpy().view(np.uint64), oracle.path_counts(g, s))
    # relabelled, the graph still offers the hybrid its bottom-up levels: such
    # searches keep the input numbering, whose columns ascend
    abfs.graph_relabel(G)
    level, parent, trace = abfs.run_trace(G, s, params=p)
    assert "bottom_up" in _kinds(trace)
    _check(g, s, level, parent, "relabelled hybrid")
    G.destroy()
    # the same graph with each column's rows in a seeded random order
    rng = np.random.default_rng(7)
    rows = g.rowidx.copy()
    for v in range(g.n):
        a, b = int(g.colptr[v]), int(g.colptr[v + 1])
        rows[a:b] = rng.permutation(rows[a:b])
    H = abfs.graph_create(g.colptr, rows, directed=False)
    level, parent, trace = abfs.run_trace(H, s, params=p)
    assert "bottom_up" not in _kinds(trace) and "bu_prep" not in _kinds(trace)
    _check(g, s, level, parent, "shuffled columns")
    H.destroy()
    d = synth.rgg_knn(1 << 14, 4, seed=4)
    D = abfs.graph_create(d.colptr, d.rowidx, directed=True)
    level, parent, trace = abfs.run_trace(D, 0, params=p)
    assert "bottom_up" not in _kinds(trace)
    _check(d, 0, level, parent, "directed hybrid")
    D.destroy()


def test_cluster_runs_take_the_thin_levels():
    """A thin search (a 300 x 200 grid from a corner) runs its levels in
    cluster runs when the launch has clusters (trace entries marked 3, with the
    run's CTA count), and in single-CTA narrow runs without; both exact."""
    g = synth.grid(300, 200)
    G = abfs.graph_create(g.colptr, g.rowidx, directed=False)
    level, parent, trace = abfs.run_trace(G, 0, params=_params(cluster_min=256), cap=1 << 14)
    runs = [r for r in trace if r.get("alone") == 3]
    assert len(runs) > 100 and all(2 <= r["items"] <= 16 for r in runs)
    _check(g, 0, level, parent, "cluster runs")
    level, parent, trace = abfs.run_trace(G, 0, params=_params(cluster_ctas=1, cluster_min=256),
                                          cap=1 << 14)
    assert not [r for r in trace if r.get("alone") == 3]
    _check(g, 0, level, parent, "no clusters")
    G.destroy()


def test_cluster_parameter_rules():
    G = abfs.graph_create(*(lambda g: (g.colptr, g.rowidx))(synth.er(100, 3.0, seed=1)))
    for bad in (dict(cluster_ctas=0), dict(cluster_ctas=17)):
        with pytest.raises(abfs.AbfsError) as ei:
            abfs.run(G, 0, params=_params(**bad))
        assert ei.value.status == 1
    G.destroy()


def test_hybrid_parameter_rules():
    G = abfs.graph_create(*(lambda g: (g.colptr, g.rowidx))(synth.er(100, 3.0, seed=1)))
    for bad in (dict(mode=PLAIN, bottom_up_alpha=14),
                dict(bottom_up_alpha=14, shrink_theta=0.5, shrink_max=1)):
        with pytest.raises(abfs.AbfsError) as ei:
            abfs.run(G, 0, params=_params(**bad))
        assert ei.value.status == 1
    G.destroy()


def test_calibrate_reports_rates():
    c = abfs.calibrate(16)
    assert c["words"] == 1 << 16 and c["ops"] > 0
    assert c["red_gops"] > 1.0 and c["load_gops"] > 1.0
    with pytest.raises(abfs.AbfsError):
        abfs.calibrate(40)


def test_device_inputs_and_validation():
    g = synth.rmat(12, 8.0, seed=5)
    cp = torch.from_numpy(g.colptr.view(np.int32)).cuda()
    ri = torch.from_numpy(g.rowidx.view(np.int32)).cuda()
    G = abfs.graph_create(cp, ri, directed=False, validate=True)
    s = int(np.argmax(g.degrees()))
    level, parent = abfs.run(G, s)
    _check(g, s, level, parent, "device input")
    G.destroy()


# ---------------------------------------------------------------------------
# full-size workloads
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def rmat22():
    g = synth.rmat_22()
    G = abfs.graph_create(g.colptr, g.rowidx, directed=False)
    yield g, G
    G.destroy()


def test_rmat22_16_sources(rmat22):
    g, G = rmat22
    srcs = synth.sources_with_degree(g, 16, seed=1)
    for kw in (dict(mode=SUB), dict(mode=PLAIN), dict(mode=SUB, shrink_theta=0.6, shrink_max=1),
               dict(mode=SUB, bottom_up_alpha=14, bottom_up_beta=24)):
        p = _params(**kw)
        for s in srcs[: (16 if kw == dict(mode=SUB) else 4)]:
            level, parent, st = abfs.run(G, int(s), params=p, stats=True)
            assert st["status"] == 0
            _check(g, int(s), level, parent, f"rmat22 {kw} src{s}")


def test_rmat22_relabelled(rmat22):
    """The same graph relabelled by column-length class: the levels and the
    least-index parents, in the input's labels, are the oracle's."""
    g, _ = rmat22
    G = abfs.graph_create(g.colptr, g.rowidx, directed=False)
    abfs.graph_relabel(G)
    srcs = synth.sources_with_degree(g, 16, seed=1)
    for kw in (dict(mode=SUB), dict(mode=SUB, shrink_theta=0.6, shrink_max=1),
               dict(mode=SUB, cluster_ctas=16), dict(mode=PLAIN)):
        for s in srcs[:3]:
            level, parent, st = abfs.run(G, int(s), params=_params(**kw), stats=True)
            assert st["status"] == 0
            _check(g, int(s), level, parent, f"rmat22 relabelled {kw} src{s}")
    G.destroy()


def test_rmat22_batch_64_sources(rmat22):
    g, G = rmat22
    srcs = synth.sources_with_degree(g, 64, seed=2)
    levels, parents, st = abfs.run_batch([G] * 64, srcs)
    torch.cuda.synchronize()
    assert all(x == 0 for x in st)
    for i in range(64):
        _check(g, int(srcs[i]), levels[i], parents[i], f"rmat22 batch {i}")


def test_batch_512_graphs_as_benchmarked():
    """The benchmark's 512-graph batch (seeded ER/R-MAT, n in [2^10, 2^18]) in one
    persistent launch with the batch autotuner's parameters: every status is OK
    and every one of the 512 searches equals the oracle bit for bit."""
    specs = synth.batch_specs(512, seed=1)
    hosts = [synth.make_batch_graph(sp) for sp in specs]
    graphs = [abfs.graph_create(h.colptr, h.rowidx, directed=False) for h in hosts]
    srcs = [int(synth.sources_with_degree(h, 1, seed=1 + i)[0]) if (h.degrees() > 0).any() else 0
            for i, h in enumerate(hosts)]
    for p in (abfs.batch_tune(graphs, srcs)[0], _params(bottom_up_alpha=5, bottom_up_beta=24)):
        plan = abfs.BatchPlan(graphs, srcs, params=p)
        plan.launch()
        assert plan.status() == [0] * len(graphs)
        for i in range(len(graphs)):
            _check(hosts[i], srcs[i], plan.levels[i], plan.parents[i], f"batch512 graph {i}")
        plan.destroy()
    for G in graphs:
        G.destroy()


def test_grid_4096():
    g = synth.grid_4096()
    G = abfs.graph_create(g.colptr, g.rowidx, directed=False)
    # the last set is the autotuner's choice for this graph: 16-CTA clusters, one CTA per SM
    for kw in (dict(mode=SUB), dict(mode=PLAIN), dict(mode=SUB, cluster_ctas=1),
               dict(mode=SUB, cluster_ctas=16), dict(mode=SUB, cluster_ctas=16, ctas_per_sm=1)):
        level, parent, st = abfs.run(G, 0, params=_params(**kw), stats=True)
        assert st["status"] == 0 and st["levels"] == 8191
        lev = level.cpu().numpy()
        par = parent.cpu().numpy()
        v = np.arange(g.n)
        r, c = v // 4096, v % 4096
        assert np.array_equal(lev, r + c)                     # Manhattan distance
        exp = np.where(r > 0, v - 4096, v - 1)
        exp[0] = 0
        assert np.array_equal(par, exp)
    G.destroy()


def test_rgg_2_22():
    g = synth.rgg_2_22()
    G = abfs.graph_create(g.colptr, g.rowidx, directed=True)
    for kw in (dict(mode=SUB), dict(mode=PLAIN), dict(mode=SUB, cluster_ctas=1),
               dict(mode=SUB, cluster_ctas=16, ctas_per_sm=1)):
        level, parent = abfs.run(G, 0, params=_params(**kw))
        _check(g, 0, level, parent, f"rgg22 {kw}")
    G.destroy()

"""Parity of abfs_run_counts (shortest-path counts, the all-nonzero variant over
the arithmetic semiring) with the CPU oracle, through the C-ABI.

Counts are integers mod 2^64: the bar is bit-exact equality of sigma, level and
parent, element by element, for every submatrix-mode parameter set.
"""
import math

import numpy as np
import pytest

import oracle
import synth
from test_gpu_parity import MODES, SUB, PLAIN, _check, _params, _small_graphs, _sources

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1906_03113_gb300 as abfs  # noqa: E402

MOD = 1 << 64


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    abfs.build()
    abfs.load()
    torch.cuda.set_device(0)


def _u64(t):
    return t.cpu().numpy().view(np.uint64)


def _check_counts(g, s, level, parent, sigma, ctx):
    _check(g, s, level, parent, ctx)
    want = oracle.path_counts(g, s)
    got = _u64(sigma)
    bad = np.nonzero(got != want)[0]
    assert bad.size == 0, f"{ctx}: sigma mismatch at {bad[:8]} ({got[bad[:8]]} vs {want[bad[:8]]})"


@pytest.fixture(scope="module")
def small():
    gs = _small_graphs()
    dev = {k: abfs.graph_create(g.colptr, g.rowidx, directed=g.directed, validate=True)
           for k, g in gs.items()}
    yield gs, dev
    for G in dev.values():
        G.destroy()


SUB_MODES = [m for m in MODES if m[1].get("mode") == SUB]


@pytest.mark.parametrize("mode_name,kw", SUB_MODES, ids=[m[0] for m in SUB_MODES])
def test_small_graphs_counts(small, mode_name, kw):
    gs, dev = small
    p = _params(**kw)
    for name, g in gs.items():
        for s in _sources(g):
            level, parent, sigma, st = abfs.run_counts(dev[name], s, params=p, stats=True)
            torch.cuda.synchronize()
            assert st["status"] == 0, (name, s, st)
            _check_counts(g, s, level, parent, sigma, f"{mode_name}/{name}/src{s}")
            # the counts leave the search itself unchanged
            la, pa = abfs.run(dev[name], s, params=p)
            assert torch.equal(la, level) and torch.equal(pa, parent)


def test_duplicates_and_self_loops_count_as_integer_entries():
    # 0 -> 1 twice, 0 -> 2, 1 -> 3, 2 -> 3 three times, 3 -> 3, 3 -> 4 twice
    colptr = np.array([0, 3, 4, 7, 10, 10], dtype=np.uint32)
    rowidx = np.array([1, 1, 2, 3, 3, 3, 3, 3, 4, 4], dtype=np.uint32)
    g = synth.Graph(colptr, rowidx, True)
    G = abfs.graph_create(colptr, rowidx, directed=True)
    for kw in (dict(), dict(narrow_max=0, narrow_edges=0, claim_scan=1, unit_entries=256)):
        level, parent, sigma = abfs.run_counts(G, 0, params=_params(**kw))
        assert _u64(sigma).tolist() == [1, 2, 1, 5, 10]
        _check_counts(g, 0, level, parent, sigma, f"duplicates {kw}")
    G.destroy()


def test_comparator_mode_and_null_counts_rejected(small):
    gs, dev = small
    with pytest.raises(abfs.AbfsError) as ei:
        abfs.run_counts(dev["er_2000"], 0, params=_params(mode=PLAIN))
    assert ei.value.status == 8  # ABFS_ERR_UNSUPPORTED
    lev = torch.empty(2000, dtype=torch.int32, device="cuda")
    rc = abfs.load().abfs_run_counts(dev["er_2000"].handle, 0, lev.data_ptr(), lev.data_ptr(),
                                     None, None, None, None)
    assert rc == 1  # ABFS_ERR_INVALID_ARG


@pytest.mark.parametrize("d", [10, 16])
def test_hypercube_factorials(d):
    """Q_d from 0: sigma(v) = popcount(v)!, every level wide and dense in paths."""
    n = 1 << d
    v = np.arange(n, dtype=np.int64)
    src = np.concatenate([v[(v >> b) & 1 == 0] for b in range(d)])
    dst = np.concatenate([v[(v >> b) & 1 == 0] | (1 << b) for b in range(d)])
    g = synth.from_arcs(n, src, dst, directed=False)
    G = abfs.graph_create(g.colptr, g.rowidx, directed=False)
    fact = np.array([math.factorial(k) for k in range(d + 1)], dtype=np.uint64)
    pop = np.array([bin(x).count("1") for x in range(n)])
    for kw in (dict(), dict(claim_scan=1, narrow_max=0, narrow_edges=0)):
        level, parent, sigma = abfs.run_counts(G, 0, params=_params(**kw))
        assert np.array_equal(_u64(sigma), fact[pop]), kw
        assert np.array_equal(level.cpu().numpy(), pop)
    G.destroy()


def test_batch_plan_with_counts(small):
    """A mixed batch with path counts in one launch (replayed twice, hybrid
    parameters given: searches with counts stay top-down) equals the oracle."""
    gs, dev = small
    names = ["er_2_16", "rmat_14", "grid_100x37", "rgg_2_15", "star", "path_3000", "no_edges",
             "dicycle_777", "one_vertex"]
    graphs, srcs, hosts = [], [], []
    for nm in names:
        for s in _sources(gs[nm])[:2]:
            graphs.append(dev[nm])
            srcs.append(s)
            hosts.append(gs[nm])
    for p in (_params(), _params(bottom_up_alpha=5, bottom_up_beta=24)):
        plan = abfs.BatchPlan(graphs, srcs, params=p, counts=True)
        for rep in range(2):
            for t in plan.sigmas:
                t.fill_(7)
            plan.launch()
            assert plan.status() == [0] * len(graphs)
            for g, s, L, P, S in zip(hosts, srcs, plan.levels, plan.parents, plan.sigmas):
                _check_counts(g, s, L, P, S, f"batch counts {g.name} src{s} rep{rep}")
        plan.destroy()
    with pytest.raises(abfs.AbfsError) as ei:
        abfs.BatchPlan(graphs[:1], srcs[:1], params=_params(mode=PLAIN), counts=True)
    assert ei.value.status == 8  # ABFS_ERR_UNSUPPORTED


# ---------------------------------------------------------------------------
# full-size workloads
# ---------------------------------------------------------------------------

def test_grid_4096_binomials():
    """sigma(r, c) = C(r + c, r) mod 2^64 on the 4096^2 grid, checked on a seeded
    sample of vertices plus the corners and the first row and column."""
    W = 4096
    g = synth.grid_4096()
    G = abfs.graph_create(g.colptr, g.rowidx, directed=False)
    level, parent, sigma, st = abfs.run_counts(G, 0, params=_params(), stats=True)
    assert st["status"] == 0 and st["levels"] == 8191
    sig = _u64(sigma)
    rng = np.random.default_rng(1)
    verts = np.concatenate([rng.integers(0, W * W, 2000), [0, W - 1, W * (W - 1), W * W - 1],
                            np.arange(W), np.arange(W) * W])
    for v in verts.tolist():
        r, c = divmod(v, W)
        assert int(sig[v]) == math.comb(r + c, r) % MOD, (r, c)
    lev = level.cpu().numpy()
    vv = np.arange(g.n)
    assert np.array_equal(lev, vv // W + vv % W)
    G.destroy()


def test_rmat22_counts():
    g = synth.rmat_22()
    G = abfs.graph_create(g.colptr, g.rowidx, directed=False)
    s = int(synth.sources_with_degree(g, 16, seed=1)[0])
    level, parent, sigma, st = abfs.run_counts(G, s, stats=True)
    assert st["status"] == 0
    _check_counts(g, s, level, parent, sigma, "rmat22")
    G.destroy()


def test_rgg_2_22_counts():
    g = synth.rgg_2_22()
    G = abfs.graph_create(g.colptr, g.rowidx, directed=True)
    level, parent, sigma = abfs.run_counts(G, 0)
    _check_counts(g, 0, level, parent, sigma, "rgg22")
    G.destroy()

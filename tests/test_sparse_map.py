"""The sparse niv map (only the finite entries, nnz(N) of Sec. 2.4): chosen for
large k, e.g. the paper's Erdos-Renyi DAGs (Sec. 5) whose path covers have
k ~ 0.3 n chains. Host structures on CPU; transforms on GPU (marked gpu)."""
import numpy as np
import pytest

import oracle
import posetgen as pg
import paper_2211_13706_gb300 as mz


def _exports(plan):
    return {w: plan.export(w) for w in (mz.MZ_EXPORT_NIV, mz.MZ_EXPORT_LEVEL, mz.MZ_EXPORT_ULEVEL,
                                        mz.MZ_EXPORT_CHAIN_ID)}


@pytest.mark.parametrize("maker", [
    lambda: (pg.paper_example(), np.array([1, 0, 1, 0, 2, 3, 1, 3, 0, 2, 3, 0], np.int32)),
    lambda: (lambda p: (p, p.chain_id))(pg.planted_chain_poset(500, 7, 2, cross_p=5 / 500)),
    lambda: (pg.er_dag(400, 4, 3), None),
    lambda: (pg.er_dag(300, 6, 4), None),
])
def test_sparse_equals_dense_and_oracle(maker):
    p, cid = maker()
    dense = mz.Plan(p.n, p.src, p.dst, cid, host_only=True, niv_format=1, build_transpose=True)
    sparse = mz.Plan(p.n, p.src, p.dst, cid, host_only=True, niv_format=2, build_transpose=True)
    assert sparse.info["sparse"] == 1 and dense.info["sparse"] == 0
    for key in ("n", "k", "nnz", "levels", "ulevels", "levels_T", "ulevels_T", "edges"):
        assert dense.info[key] == sparse.info[key], key
    de, se = _exports(dense), _exports(sparse)
    for w in de:
        assert (de[w] == se[w]).all()
    Z = oracle.closure(p.n, p.src, p.dst)
    chains = sparse.export(mz.MZ_EXPORT_CHAIN_ID)
    assert (se[mz.MZ_EXPORT_NIV] == oracle.niv(Z, chains)).all()
    assert (sparse.export(mz.MZ_EXPORT_NIV, dual=True) == oracle.niv(np.ascontiguousarray(Z.T), chains)).all()


def test_auto_format_and_er_structure():
    p = pg.er_dag(3000, 4, 5)
    plan = mz.Plan(p.n, p.src, p.dst, None, host_only=True)
    info = plan.info
    assert info["k"] > 512 and info["sparse"] == 1          # a path cover of an ER DAG: k ~ 0.3 n
    assert info["nnz"] < 0.05 * info["n"] * info["k"]
    q = pg.planted_chain_poset(2000, 32, 1, cross_deg=2)
    assert mz.Plan(q.n, q.src, q.dst, q.chain_id, host_only=True).info["sparse"] == 0


def test_sparse_bad_chains():
    with pytest.raises(mz.MzError) as e:
        mz.mz_build(3, [0, 0], [1, 2], chain_id=[0, 1, 1], host_only=True, niv_format=2)
    assert e.value.status == mz.MZ_ERR_BAD_CHAINS


@pytest.mark.gpu
@pytest.mark.parametrize("batch", [1, 4])
def test_sparse_parity_gpu(batch):
    import torch
    from gpu_util import assert_close
    cases = [(pg.er_dag(2000, 4, 6), None, 2), (pg.er_dag(1500, 6, 7), None, 2),
             (lambda q: (q, q.chain_id, 2))(pg.planted_chain_poset(1200, 9, 8, cross_p=4 / 1200))]
    for p, cid, fmt in cases:
        plan = mz.Plan(p.n, p.src, p.dst, cid, build_transpose=True, niv_format=fmt)
        assert plan.info["sparse"] == 1
        Z = oracle.closure(p.n, p.src, p.dst)
        mu = oracle.mobius_function(Z)
        f = pg.function_values(p.n, batch, "i64:1000", 9)
        x = torch.from_numpy(f if batch > 1 else f[:, 0].copy()).cuda()
        g, r, m_ = plan.zeta(x), plan.zeta_T(x), plan.mobius(x)
        back, backT = plan.mobius(g), plan.mobius_T(r)
        plan.check()
        shape = (p.n, batch)
        g, r, m_, back, backT = (t.cpu().numpy().reshape(shape) for t in (g, r, m_, back, backT))
        assert (g == Z.astype(np.int64) @ f).all(), p.name
        assert (r == Z.T.astype(np.int64) @ f).all(), p.name
        assert (m_ == mu.T @ f).all(), p.name
        assert (back == f).all() and (backT == f).all(), p.name
        ff = pg.function_values(p.n, 1, "f64u", 10)[:, 0]
        gf = plan.zeta(torch.from_numpy(ff).cuda()).cpu().numpy()
        assert_close(gf, oracle.zeta(Z, ff), oracle.zeta(Z, np.abs(ff)), mz.MZ_F64, p.name)


@pytest.mark.gpu
@pytest.mark.parametrize("degree", [4, 6])
def test_er_paper_scale_sampled(degree):
    """ER DAGs as in the paper's Sec. 5 (n = 2^20, average degree 4 and 6), sparse map:
    sampled zeta rows exact, Moebius(zeta(f)) = f exactly, Z f_out = g on sampled rows."""
    import torch
    p = pg.er_dag(1 << 20, degree, 11)
    plan = mz.Plan(p.n, p.src, p.dst, None)
    assert plan.info["sparse"] == 1
    f = pg.function_values(p.n, 1, "i64:1000", 12)[:, 0]
    x = torch.from_numpy(f).cuda()
    g = plan.zeta(x)
    back = plan.mobius(g)
    y = plan.mobius(x)
    plan.check()
    assert torch.equal(back, x)
    rows = np.random.default_rng(1).choice(p.n, 12, replace=False).tolist()
    gg = g.cpu().numpy()
    assert (gg[rows] == oracle.zeta_rows(p.n, p.src, p.dst, f, rows)).all()
    res, _ = oracle.mobius_residual_rows(p.n, p.src, p.dst, y.cpu().numpy(), f, rows)
    assert all(int(v) % (1 << 64) == 0 for v in res)


def test_sparse_host_build_threads_agree(monkeypatch):
    # levels of >= 4096 nodes run on several host threads; the plan must not depend on it
    p = pg.er_dag(150000, 6, 8)
    plans = {}
    for t in ("1", "4"):
        monkeypatch.setenv("MZ_HOST_THREADS", t)
        plans[t] = mz.Plan(p.n, p.src, p.dst, None, host_only=True, niv_format=2)
    a, b = plans["1"], plans["4"]
    for key in ("k", "nnz", "levels", "ulevels"):
        assert a.info[key] == b.info[key], key
    for w in (mz.MZ_EXPORT_ULEVEL, mz.MZ_EXPORT_LEVEL, mz.MZ_EXPORT_CHAIN_ID):
        assert np.array_equal(a.export(w), b.export(w))
    # a broken chain is reported at the same node either way
    cid = a.export(mz.MZ_EXPORT_CHAIN_ID).copy()
    lvl = a.export(mz.MZ_EXPORT_LEVEL)
    x = int(np.flatnonzero(lvl == 5)[0])
    cid[x] = cid[int(np.flatnonzero(lvl == 9)[0])]
    msgs = []
    for t in ("1", "4"):
        monkeypatch.setenv("MZ_HOST_THREADS", t)
        with pytest.raises(mz.MzError) as e:
            mz.Plan(p.n, p.src, p.dst, cid, host_only=True, niv_format=2)
        assert e.value.status == mz.MZ_ERR_BAD_CHAINS
        msgs.append(str(e.value))
    assert msgs[0] == msgs[1]

"""Plans of many posets (mz_build_batch): host structures on CPU (host-only plans)
and, marked gpu, parity of every transform against the oracle, poset by poset."""
import numpy as np
import pytest

import oracle
import posetgen as pg
import paper_2211_13706_gb300 as mz


def mixed_posets():
    ps = [pg.paper_example(), pg.planted_chain_poset(700, 5, 3, cross_p=4 / 700), pg.boolean_lattice(5),
          pg.antichain_poset(9), pg.chain_poset(300, seed=2), pg.planted_chain_poset(1200, 12, 4, cross_deg=2),
          pg.Poset(n=1, src=np.zeros(0, np.int32), dst=np.zeros(0, np.int32))]
    cids = [None, ps[1].chain_id, None, None, ps[4].chain_id, ps[5].chain_id, None]
    return ps, cids


def test_batch_host_structures():
    ps, cids = mixed_posets()
    plan = mz.Plan.batch([(p.n, p.src, p.dst, c) for p, c in zip(ps, cids)], host_only=True, build_transpose=True)
    info = plan.info
    singles = [mz.Plan(p.n, p.src, p.dst, c, host_only=True) for p, c in zip(ps, cids)]
    assert info["components"] == len(ps)
    assert info["n"] == sum(p.n for p in ps)
    assert info["k"] == sum(s.info["k"] for s in singles)
    assert info["nnz"] == sum(s.info["nnz"] for s in singles)
    assert info["levels"] == max(s.info["levels"] for s in singles)
    assert info["ulevels"] == max(s.info["ulevels"] for s in singles)
    off = np.cumsum([0] + [p.n for p in ps])
    lv = plan.export(mz.MZ_EXPORT_LEVEL)
    cid = plan.export(mz.MZ_EXPORT_CHAIN_ID)
    topo = plan.export(mz.MZ_EXPORT_TOPO)
    koff = np.cumsum([0] + [s.info["k"] for s in singles])
    for i, (p, s) in enumerate(zip(ps, singles)):
        assert (lv[off[i]:off[i + 1]] == oracle.heights(p.n, p.src, p.dst)).all()
        assert (cid[off[i]:off[i + 1]] == s.export(mz.MZ_EXPORT_CHAIN_ID) + koff[i]).all()
        t = topo[off[i]:off[i + 1]] - off[i]
        pos = np.empty(p.n, np.int64)
        pos[t] = np.arange(p.n)
        assert (pos[p.src] < pos[p.dst]).all()
    with pytest.raises(mz.MzError) as e:
        plan.export(mz.MZ_EXPORT_NIV)
    assert e.value.status == mz.MZ_ERR_UNSUPPORTED


def test_batch_errors_name_the_poset():
    ps, _ = mixed_posets()
    bad = [(p.n, p.src, p.dst, None) for p in ps[:3]] + [(3, [0, 1, 2], [1, 2, 0], None)]
    with pytest.raises(mz.MzError) as e:
        mz.Plan.batch(bad, host_only=True)
    assert e.value.status == mz.MZ_ERR_CYCLE and "poset 3" in str(e.value)


@pytest.mark.gpu
@pytest.mark.parametrize("sched", [mz.MZ_SCHED_ULEVEL, mz.MZ_SCHED_ANTICHAIN])
@pytest.mark.parametrize("batch", [1, 4, 3])
def test_batch_parity_int64(sched, batch):
    import torch
    ps, cids = mixed_posets()
    plan = mz.Plan.batch([(p.n, p.src, p.dst, c) for p, c in zip(ps, cids)], build_transpose=True,
                         mobius_schedule=sched)
    off = np.cumsum([0] + [p.n for p in ps])
    f = pg.function_values(int(off[-1]), batch, "i64:1000", 5)
    x = torch.from_numpy(f if batch > 1 else f[:, 0].copy()).cuda()
    g = plan.zeta(x)
    back = plan.mobius(g)
    r = plan.zeta_T(x)
    m = plan.mobius(x)
    plan.check()
    g, back, r, m = (t.cpu().numpy().reshape(-1, batch) for t in (g, back, r, m))
    assert (back == f).all()
    for i, p in enumerate(ps):
        Z = oracle.closure(p.n, p.src, p.dst)
        sl = slice(off[i], off[i + 1])
        assert (g[sl] == Z.astype(np.int64) @ f[sl]).all(), p.name
        assert (r[sl] == Z.T.astype(np.int64) @ f[sl]).all(), p.name
        mu = oracle.mobius_function(Z)
        assert (m[sl] == mu.T @ f[sl]).all(), p.name


@pytest.mark.gpu
@pytest.mark.parametrize("dtype", [mz.MZ_F64, mz.MZ_F32C])
def test_batch_parity_float(dtype):
    import torch
    from gpu_util import assert_close
    ps, cids = mixed_posets()
    plan = mz.Plan.batch([(p.n, p.src, p.dst, c) for p, c in zip(ps, cids)])
    off = np.cumsum([0] + [p.n for p in ps])
    f = pg.function_values(int(off[-1]), 4, "f64u" if dtype == mz.MZ_F64 else "f32u", 6)
    if dtype == mz.MZ_F64:
        x = torch.from_numpy(f).cuda()
    else:
        x = torch.from_numpy(np.stack([f, np.zeros_like(f)])).cuda()
    g = plan.zeta(x)
    plan.check()
    gv = g.cpu().numpy()
    gv = gv if dtype == mz.MZ_F64 else gv[0].astype(np.float64) + gv[1].astype(np.float64)
    for i, p in enumerate(ps):
        Z = oracle.closure(p.n, p.src, p.dst)
        sl = slice(off[i], off[i + 1])
        for b in range(4):
            fb = f[sl, b].astype(np.float64)
            assert_close(gv[sl, b], oracle.zeta(Z, fb), oracle.zeta(Z, np.abs(fb)), dtype, f"{p.name} col {b}")

"""The device build (mz_build_opts::device_build): the niv recurrence of Thm. 4
(Alg. 2), the U levels, the gather tiles and the Moebius rows computed by
kernels. The plan must be the host build's, entry for entry: the same exports,
the same plan info, and bit-identical transforms (same layouts, same order of
additions). Argument checks run on the CPU; everything else is marked gpu."""
import numpy as np
import pytest

import oracle
import posetgen as pg
import paper_2211_13706_gb300 as mz

EXPORTS = (mz.MZ_EXPORT_NIV, mz.MZ_EXPORT_LEVEL, mz.MZ_EXPORT_ULEVEL, mz.MZ_EXPORT_CHAIN_ID,
           mz.MZ_EXPORT_CHAIN_POS, mz.MZ_EXPORT_TOPO)
INFO_KEYS = ("n", "k", "nnz", "edges", "levels", "ulevels", "levels_T", "ulevels_T", "max_chain", "sparse",
             "device_bytes")


def test_device_build_argument_checks():
    with pytest.raises(mz.MzError) as e:
        mz.mz_build(3, [0, 1], [1, 2], device_build=True, host_only=True)
    assert e.value.status == mz.MZ_ERR_INVALID_ARG
    for bad in (3, -1):
        with pytest.raises(mz.MzError) as e:
            mz.mz_build(3, [0, 1], [1, 2], device_build=bad)
        assert e.value.status == mz.MZ_ERR_INVALID_ARG
    p = pg.paper_example()
    # several posets on the device: dense maps only (a 600-chain antichain keeps a sparse map)
    q600 = pg.antichain_poset(600)
    with pytest.raises(mz.MzError) as e:
        mz.mz_build_batch([(p.n, p.src, p.dst, None), (q600.n, q600.src, q600.dst, None)], device_build=True)
    assert e.value.status == mz.MZ_ERR_UNSUPPORTED
    # a dense map on the device holds at most 512 chains: refused before any device work
    q = pg.antichain_poset(600)
    with pytest.raises(mz.MzError) as e:
        mz.mz_build(q.n, q.src, q.dst, device_build=True, niv_format=1)
    assert e.value.status == mz.MZ_ERR_UNSUPPORTED and "512" in str(e.value)


def _cases():
    ex = pg.paper_example()
    bl = pg.boolean_lattice(8)
    dl, _ = pg.divisor_lattice(720)
    pl = pg.planted_chain_poset(4096, 16, 1, cross_p=4 / 4096)
    pl33 = pg.planted_chain_poset(3000, 33, 2, cross_deg=3)
    pl300 = pg.planted_chain_poset(6000, 300, 3, cross_deg=2)
    return [
        ("paper_example", ex, None),
        ("boolean_lattice_8", bl, None),
        ("divisor_lattice_720", dl, None),
        ("chain_500", pg.chain_poset(500, 1), None),
        ("antichain_100", pg.antichain_poset(100), None),
        ("planted_4096_k16", pl, pl.chain_id),
        ("planted_3000_k33", pl33, pl33.chain_id),
        ("planted_6000_k300", pl300, pl300.chain_id),
        ("planted_4096_matching", pl, None),
        ("er_400_deg3", pg.er_dag(400, 3, 9), None),
        ("tiny_dag", pg.random_dag_tiny(40, 0.2, 5), None),
    ]


CASES = _cases()


def _pair(p, cid, **kw):
    host = mz.Plan(p.n, p.src, p.dst, cid, **kw)
    dev = mz.Plan(p.n, p.src, p.dst, cid, device_build=True, **kw)
    return host, dev


@pytest.mark.gpu
@pytest.mark.parametrize("name,p,cid", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("schedule", [mz.MZ_SCHED_ULEVEL, mz.MZ_SCHED_ANTICHAIN])
def test_device_build_equals_host_build(name, p, cid, schedule):
    host, dev = _pair(p, cid, build_transpose=True, mobius_schedule=schedule)
    for key in INFO_KEYS:
        assert host.info[key] == dev.info[key], key
    for dual in (False, True):
        for w in EXPORTS:
            assert np.array_equal(host.export(w, dual=dual), dev.export(w, dual=dual)), (w, dual)
    # the map itself against the oracle's niv (independent of both builds)
    Z = oracle.closure(p.n, p.src, p.dst)
    chains = dev.export(mz.MZ_EXPORT_CHAIN_ID)
    assert np.array_equal(dev.export(mz.MZ_EXPORT_NIV), oracle.niv(Z, chains))
    assert np.array_equal(dev.export(mz.MZ_EXPORT_NIV, dual=True), oracle.niv(np.ascontiguousarray(Z.T), chains))


@pytest.mark.gpu
@pytest.mark.parametrize("name,p,cid", CASES[:6] + CASES[7:8], ids=[c[0] for c in CASES[:6] + CASES[7:8]])
def test_device_built_transforms_bit_identical(name, p, cid):
    import torch
    host, dev = _pair(p, cid, build_transpose=True)
    xi = torch.from_numpy(pg.function_values(p.n, 3, "i64:1000", 4)).cuda()
    xf = torch.from_numpy(pg.function_values(p.n, 3, "f64u", 5)).cuda()
    for op in ("zeta", "mobius", "zeta_T", "mobius_T"):
        for x in (xi, xf):
            a = getattr(host, op)(x)
            b = getattr(dev, op)(x)
            host.check()
            dev.check()
            assert torch.equal(a, b), op
    # int64 against the oracle's exact zeta
    want = oracle.zeta(oracle.closure(p.n, p.src, p.dst), xi.cpu().numpy())
    assert np.array_equal(dev.zeta(xi).cpu().numpy(), want)


@pytest.mark.gpu
def test_device_build_bad_chains_same_error():
    p = pg.planted_chain_poset(2000, 8, 4, cross_deg=2)
    bad = p.chain_id.copy()
    # move one element to another chain: that chain is no longer totally ordered
    bad[np.flatnonzero(bad == 0)[len(bad) // 40]] = 1
    errs = []
    for device_build in (False, True):
        with pytest.raises(mz.MzError) as e:
            mz.mz_build(p.n, p.src, p.dst, bad, device_build=device_build)
        errs.append((e.value.status, str(e.value).split(":", 1)[-1]))
    assert errs[0][0] == errs[1][0] == mz.MZ_ERR_BAD_CHAINS
    assert errs[0][1] == errs[1][1]


@pytest.mark.gpu
def test_device_build_full_size_planted():
    """n = 2^20, k = 64 chains of 16384: the maps, levels and nnz equal the host build's."""
    p = pg.planted_chain_poset(1 << 20, 64, 1)
    host, dev = _pair(p, p.chain_id)
    for key in INFO_KEYS:
        assert host.info[key] == dev.info[key], key
    for w in (mz.MZ_EXPORT_NIV, mz.MZ_EXPORT_ULEVEL):
        assert np.array_equal(host.export(w), dev.export(w)), w


def _sparse_cases():
    pl7 = pg.planted_chain_poset(500, 7, 2, cross_p=5 / 500)
    return [
        ("paper_example", pg.paper_example(), None, 2),
        ("planted_500_k7", pl7, pl7.chain_id, 2),
        ("boolean_lattice_7", pg.boolean_lattice(7), None, 2),
        ("antichain_600", pg.antichain_poset(600), None, 0),
        ("er_3000_deg4", pg.er_dag(3000, 4, 11), None, 0),
        ("er_2000_deg6", pg.er_dag(2000, 6, 12), None, 0),
    ]


SPARSE_CASES = _sparse_cases()


@pytest.mark.gpu
@pytest.mark.parametrize("name,p,cid,fmt", SPARSE_CASES, ids=[c[0] for c in SPARSE_CASES])
@pytest.mark.parametrize("schedule", [mz.MZ_SCHED_ULEVEL, mz.MZ_SCHED_ANTICHAIN])
def test_sparse_device_build_equals_host_build(name, p, cid, fmt, schedule):
    host, dev = _pair(p, cid, build_transpose=True, mobius_schedule=schedule, niv_format=fmt)
    assert dev.info["sparse"] == 1
    for key in INFO_KEYS:
        assert host.info[key] == dev.info[key], key
    for dual in (False, True):
        for w in EXPORTS:
            assert np.array_equal(host.export(w, dual=dual), dev.export(w, dual=dual)), (w, dual)
    Z = oracle.closure(p.n, p.src, p.dst)
    chains = dev.export(mz.MZ_EXPORT_CHAIN_ID)
    assert np.array_equal(dev.export(mz.MZ_EXPORT_NIV), oracle.niv(Z, chains))


@pytest.mark.gpu
@pytest.mark.parametrize("name,p,cid,fmt", SPARSE_CASES[3:], ids=[c[0] for c in SPARSE_CASES[3:]])
def test_sparse_device_built_transforms_bit_identical(name, p, cid, fmt):
    import torch
    host, dev = _pair(p, cid, build_transpose=True, niv_format=fmt)
    xi = torch.from_numpy(pg.function_values(p.n, 2, "i64:1000", 6)).cuda()
    xf = torch.from_numpy(pg.function_values(p.n, 2, "f64u", 7)).cuda()
    for op in ("zeta", "mobius", "zeta_T", "mobius_T"):
        for x in (xi, xf):
            a = getattr(host, op)(x)
            b = getattr(dev, op)(x)
            host.check()
            dev.check()
            assert torch.equal(a, b), op


@pytest.mark.gpu
def test_sparse_device_build_bad_chains_same_error():
    p = pg.planted_chain_poset(2000, 8, 4, cross_deg=2)
    bad = p.chain_id.copy()
    bad[np.flatnonzero(bad == 0)[len(bad) // 40]] = 1
    errs = []
    for device_build in (False, True):
        with pytest.raises(mz.MzError) as e:
            mz.mz_build(p.n, p.src, p.dst, bad, device_build=device_build, niv_format=2)
        errs.append((e.value.status, str(e.value).split(":", 1)[-1]))
    assert errs[0][0] == errs[1][0] == mz.MZ_ERR_BAD_CHAINS
    assert errs[0][1] == errs[1][1]


@pytest.mark.gpu
def test_sparse_device_build_er_paper_scale():
    """The paper's ER DAG at n = 2^20, average degree 4 (path cover, k ~ 0.27 n): plan info, U
    levels and the fp64 transforms equal the host-built plan's bit for bit."""
    import torch
    p = pg.er_dag(1 << 20, 4, 1)
    host, dev = _pair(p, None)
    for key in INFO_KEYS:
        assert host.info[key] == dev.info[key], key
    assert np.array_equal(host.export(mz.MZ_EXPORT_ULEVEL), dev.export(mz.MZ_EXPORT_ULEVEL))
    x = torch.from_numpy(pg.function_values(p.n, 1, "f64u", 8)[:, 0]).cuda()
    for op in ("zeta", "mobius"):
        a, b = getattr(host, op)(x), getattr(dev, op)(x)
        host.check()
        dev.check()
        assert torch.equal(a, b), op


# ----------------------------------------------------------------------------- plans of several posets

def _batch_posets():
    ps = [pg.planted_chain_poset(2048, 256, 31, cross_deg=2), pg.paper_example(),
          pg.planted_chain_poset(1500, 100, 32, cross_deg=2), pg.boolean_lattice(6),
          pg.planted_chain_poset(3000, 7, 33, cross_deg=2), pg.chain_poset(700, seed=34),
          pg.antichain_poset(40), pg.planted_chain_poset(1024, 4, 35, cross_p=4 / 1024),
          pg.er_dag(500, 3, 36), pg.Poset(n=1, src=np.zeros(0, np.int32), dst=np.zeros(0, np.int32))]
    cids = [p.chain_id if p.name.startswith(("planted", "chain")) else None for p in ps]
    return [(p.n, p.src, p.dst, c) for p, c in zip(ps, cids)]


BATCH_INFO = INFO_KEYS + ("components", "wave_rows", "wave_entries")


@pytest.mark.gpu
@pytest.mark.parametrize("schedule", [mz.MZ_SCHED_ULEVEL, mz.MZ_SCHED_ANTICHAIN])
def test_batch_device_build_equals_host_build(schedule):
    """Ten posets of uneven n and k (1 to 256 chains) in one plan: the device build's plan
    has the host build's info and exports, and every int64 transform is bit-identical."""
    import torch
    posets = _batch_posets()
    host = mz.Plan.batch(posets, build_transpose=True, mobius_schedule=schedule)
    dev = mz.Plan.batch(posets, build_transpose=True, mobius_schedule=schedule, device_build=True)
    for key in BATCH_INFO:
        assert host.info[key] == dev.info[key], key
    for dual in (False, True):
        for w in EXPORTS:
            if w != mz.MZ_EXPORT_NIV:
                assert np.array_equal(host.export(w, dual=dual), dev.export(w, dual=dual)), (w, dual)
    n = host.info["n"]
    for batch in (1, 32):
        f = pg.function_values(n, batch, "i64:1000", 40 + batch)
        x = torch.from_numpy(f if batch > 1 else f[:, 0].copy()).cuda()
        for name in ("zeta", "mobius", "zeta_T", "mobius_T"):
            a, b = getattr(host, name)(x), getattr(dev, name)(x)
            host.check()
            dev.check()
            assert torch.equal(a, b), (name, batch)
        assert torch.equal(dev.mobius(dev.zeta(x)), x)
        dev.check()


@pytest.mark.gpu
def test_batch_device_build_names_the_poset_of_a_bad_chain():
    posets = _batch_posets()
    n, src, dst, _ = posets[4]
    bad = np.arange(n, dtype=np.int32) % 2            # two "chains" that are not totally ordered
    posets[4] = (n, src, dst, bad)
    with pytest.raises(mz.MzError) as e:
        mz.Plan.batch(posets, device_build=True)
    assert e.value.status == mz.MZ_ERR_BAD_CHAINS and "poset 4" in str(e.value)


# ----------------------------------------------------------------------------- Alg. 1 on the device

def _matching_cases():
    pl = pg.planted_chain_poset(4096, 16, 1, cross_p=4 / 4096)
    return [("paper_example", pg.paper_example()), ("boolean_lattice_8", pg.boolean_lattice(8)),
            ("divisor_lattice_720", pg.divisor_lattice(720)[0]), ("chain_500", pg.chain_poset(500, 1)),
            ("antichain_100", pg.antichain_poset(100)), ("planted_4096_k16", pl),
            ("er_400_deg3", pg.er_dag(400, 3, 9)), ("tiny_dag", pg.random_dag_tiny(40, 0.2, 5)),
            ("er_20000_deg6", pg.er_dag(20000, 6, 3)), ("er_20000_deg2", pg.er_dag(20000, 2, 4))]


MATCHING_CASES = _matching_cases()


def _assert_path_cover(p, plan):
    """Every chain of the plan is a path of edges: consecutive members joined by an edge
    from the upper one to the lower one (u -> v means v <= u)."""
    cid = plan.export(mz.MZ_EXPORT_CHAIN_ID)
    pos = plan.export(mz.MZ_EXPORT_CHAIN_POS)
    edges = set(zip(np.asarray(p.src).tolist(), np.asarray(p.dst).tolist()))
    order = np.lexsort((pos, cid))
    c, q = cid[order], pos[order]
    assert (q[np.r_[True, c[1:] != c[:-1]]] == 0).all()            # each chain starts at position 0
    for a, b in zip(order[:-1], order[1:]):
        if cid[a] == cid[b]:
            assert pos[b] == pos[a] + 1 and (int(b), int(a)) in edges, (int(a), int(b))


@pytest.mark.gpu
@pytest.mark.parametrize("name,p", MATCHING_CASES, ids=[c[0] for c in MATCHING_CASES])
def test_device_matching_gives_a_minimum_path_cover(name, p):
    """device_build = 2: Alg. 1's matching on the device. The chains are a path cover with as
    many chains as the host's maximum matching gives (both are maximum), and the int64
    transforms of the plan equal those of the host-chained plan (and the oracle's)."""
    import torch
    host = mz.Plan(p.n, p.src, p.dst, None, build_transpose=True)
    dev = mz.Plan(p.n, p.src, p.dst, None, build_transpose=True, device_build=2)
    assert dev.info["k"] == host.info["k"], (dev.info["k"], host.info["k"])
    _assert_path_cover(p, dev)
    f = pg.function_values(p.n, 1, "i64:1000", 5)[:, 0]
    x = torch.from_numpy(f).cuda()
    for op in ("zeta", "mobius", "zeta_T", "mobius_T"):
        a, b = getattr(host, op)(x), getattr(dev, op)(x)
        host.check()
        dev.check()
        assert torch.equal(a, b), op
    if p.n <= 4096:
        Z = oracle.closure(p.n, p.src, p.dst)
        assert np.array_equal(dev.zeta(x).cpu().numpy(), oracle.zeta(Z, f))


@pytest.mark.gpu
def test_device_matching_er_paper_scale():
    """The paper's ER DAG at n = 2^20, average degree 4, chains by the device's matching:
    the host's number of chains, a path cover, and int64 transforms equal to the host plan's."""
    import torch
    p = pg.er_dag(1 << 20, 4, 1)
    host = mz.Plan(p.n, p.src, p.dst, None, device_build=True)
    dev = mz.Plan(p.n, p.src, p.dst, None, device_build=2)
    assert dev.info["k"] == host.info["k"]
    cid = dev.export(mz.MZ_EXPORT_CHAIN_ID)
    pos = dev.export(mz.MZ_EXPORT_CHAIN_POS)
    order = np.lexsort((pos, cid))
    same = cid[order][1:] == cid[order][:-1]
    lo, hi = order[:-1][same], order[1:][same]                      # consecutive members: hi directly above lo
    key = lambda a, b: a.astype(np.int64) * p.n + b
    assert np.isin(key(hi, lo), key(np.asarray(p.src), np.asarray(p.dst))).all()
    x = torch.from_numpy(pg.function_values(p.n, 1, "i64:1000", 6)[:, 0]).cuda()
    for op in ("zeta", "mobius"):
        a, b = getattr(host, op)(x), getattr(dev, op)(x)
        host.check()
        dev.check()
        assert torch.equal(a, b), op

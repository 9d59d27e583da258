"""int64 transforms are exact modulo 2^64 for every input, INT64_MIN included.

The Moebius forward substitution marks an unfinished prefix word with INT64_MIN;
a prefix that really equals INT64_MIN is published through an escape flag. These
tests make prefixes hit that value on purpose (chosen on the host from the plan's
exported chains and the oracle's mu) and compare the GPU with the exact result
reduced modulo 2^64, under both schedules and at several batch sizes (one lane per
row, G lanes per row, and the generic kernel for a batch that is not a power of 2).
"""
import numpy as np
import pytest
import torch

import oracle
import posetgen as pg
import paper_2211_13706_gb300 as mz

pytestmark = pytest.mark.gpu

INT64_MIN = np.int64(-(1 << 63))


def _mod64_matvec(W, v):
    """W @ v modulo 2^64 (W small integers, v int64), as int64."""
    return (W.astype(np.int64).astype(np.uint64) @ v.astype(np.int64).view(np.uint64)).view(np.int64)


@pytest.fixture(scope="module")
def inst():
    p = pg.planted_chain_poset(2000, 8, 12, cross_deg=2)
    Z = oracle.closure(p.n, p.src, p.dst)
    mu = oracle.mobius_function(Z)
    return p, Z, mu


def _referenced(plan):
    """Elements some row of another chain reads: niv_j(x) = y with j = chain(y) != chain(x)."""
    N = plan.export(mz.MZ_EXPORT_NIV)
    cid = plan.export(mz.MZ_EXPORT_CHAIN_ID)
    ref = np.zeros(N.shape[0], bool)
    for x in range(N.shape[0]):
        for j in range(N.shape[1]):
            if j != cid[x] and N[x, j] >= 0:
                ref[N[x, j]] = True
    return ref


def _prefixes(plan, f):
    """y' = V f: on every chain, the sum of f over the chain's elements up to x (mod 2^64)."""
    cid = plan.export(mz.MZ_EXPORT_CHAIN_ID)
    pos = plan.export(mz.MZ_EXPORT_CHAIN_POS)
    y = np.zeros(len(f), np.uint64)
    fu = f.astype(np.int64).view(np.uint64)
    for c in np.unique(cid):
        idx = np.flatnonzero(cid == c)
        idx = idx[np.argsort(pos[idx])]
        y[idx] = np.cumsum(fu[idx], dtype=np.uint64)
    return y.view(np.int64)


def _sentinel_input(plan, p, Z, mu):
    """g with two prefixes y' equal to INT64_MIN: a minimal element some other chain reads
    (y' = g there), and a read element with dependencies, its g shifted so that its
    prefix lands exactly on INT64_MIN."""
    ref = _referenced(plan)
    lv = plan.export(mz.MZ_EXPORT_LEVEL)
    ul = plan.export(mz.MZ_EXPORT_ULEVEL)
    g = pg.function_values(p.n, 1, "i64:1000", 9)[:, 0]
    y0 = int(np.flatnonzero(ref & (lv == 1))[0])
    g[y0] = INT64_MIN
    cand = np.flatnonzero(ref & (ul >= 2))
    x1 = int(cand[len(cand) // 2])
    y = _prefixes(plan, _mod64_matvec(mu.T, g))
    # y'(x1) = g(x1) - (prefixes of x1's dependencies, which do not involve g(x1))
    g_u = g.view(np.uint64).copy()
    with np.errstate(over="ignore"):                     # unsigned arithmetic modulo 2^64
        g_u[x1] = g_u[x1] + (INT64_MIN.view(np.uint64) - y.view(np.uint64)[x1])
    g = g_u.view(np.int64)
    yy = _prefixes(plan, _mod64_matvec(mu.T, g))
    assert yy[y0] == INT64_MIN and yy[x1] == INT64_MIN
    return g


@pytest.mark.parametrize("sched", [mz.MZ_SCHED_ULEVEL, mz.MZ_SCHED_ANTICHAIN])
@pytest.mark.parametrize("batch", [1, 3, 4, 32])
def test_prefix_equal_to_int64_min(inst, sched, batch):
    p, Z, mu = inst
    plan = mz.Plan(p.n, p.src, p.dst, p.chain_id, mobius_schedule=sched)
    g = _sentinel_input(plan, p, Z, mu)
    # column b: g plus b at the elements no other chain reads (their prefixes are not
    # published), so every column still meets INT64_MIN at the same two prefixes
    ref = _referenced(plan)
    G = np.stack([g + np.where(ref, 0, b).astype(np.int64) for b in range(batch)], axis=1)
    x = torch.from_numpy(G if batch > 1 else G[:, 0].copy()).cuda()
    got = plan.mobius(x)
    plan.check()
    got = got.cpu().numpy().reshape(p.n, batch)
    for b in range(batch):
        want = _mod64_matvec(mu.T, G[:, b])
        assert np.array_equal(got[:, b], want), (sched, batch, b, np.flatnonzero(got[:, b] != want)[:5])
        # and back: zeta of the result is g again, modulo 2^64
        assert np.array_equal(_mod64_matvec(Z, want), G[:, b])
    back = plan.zeta(plan.mobius(x))
    plan.check()
    assert torch.equal(back, x)


def test_zeta_wraps_modulo_2_64(inst):
    p, Z, _ = inst
    plan = mz.Plan(p.n, p.src, p.dst, p.chain_id)
    f = pg.function_values(p.n, 1, "i64:1000", 10)[:, 0]
    f[::7] = INT64_MIN
    f[3::11] = np.int64((1 << 63) - 1)
    got = plan.zeta(torch.from_numpy(f).cuda())
    plan.check()
    assert np.array_equal(got.cpu().numpy(), _mod64_matvec(Z, f))

"""The forward substitution with a look-ahead of one level against the one without.

With the U-level schedule and a warp per row, a row may compute up to seven of its
dependencies one level below it from their own rows, so that it waits only for words
published two levels down. Every row's value is formed in one fixed order wherever it is
computed, so the look-ahead must return the bits of the kernel without it, for int64,
fp64 and F32C alike, and int64 must equal the oracle's M g exactly. The posets cover
every segment width (rows of up to 32, 64, 128 and 256 entries), a plan whose rows are
too long for the look-ahead tables, a plan of several posets, launch shapes without
pacing and with several blocks per SM, the full-size planted posets (n = 2^20, k = 64
and n = 2^22, k = 128), and the withheld-row test hook.
"""
import numpy as np
import pytest
import torch

import oracle
import posetgen as pg
import paper_2211_13706_gb300 as mz
from gpu_util import to_device

pytestmark = pytest.mark.gpu

KINDS = {mz.MZ_I64: "i64:1000", mz.MZ_F64: "f64u", mz.MZ_F32C: "f32u"}


def _bits(t):
    return t.contiguous().view(torch.uint8)


def _mobius(plan, x, lookahead, **shape):
    mz.mz_plan_tune(plan.handle, mobius_lanes=32, mobius_lookahead=lookahead, **shape)
    y = plan.mobius(x)
    plan.check()
    return y


def _same_bits(plan, x, **shape):
    """Moebius of x with and without the look-ahead; returns the look-ahead's result
    after checking that both have the same bits."""
    a = _mobius(plan, x, 1, **shape)
    b = _mobius(plan, x, 2, **shape)
    assert torch.equal(_bits(a), _bits(b)), shape
    return a


@pytest.mark.parametrize("k,width", [(20, 2), (60, 4), (120, 8), (250, 16)])
def test_every_width_same_bits_and_exact(k, width):
    p = pg.planted_chain_poset(3000, k, 40 + k, cross_deg=3)
    plan = mz.Plan(p.n, p.src, p.dst, p.chain_id)
    info = plan.info
    assert info["lookahead_width"] == width
    assert info["lookahead_max_local"] == min(32 // width, 8) - 1
    assert 0 < info["wave_critical_rows"] <= info["wave_rows"]
    Z = oracle.closure(p.n, p.src, p.dst)
    mu = oracle.mobius_function(Z)
    for dtype in (mz.MZ_I64, mz.MZ_F64, mz.MZ_F32C):
        g = pg.function_values(p.n, 1, KINDS[dtype], 7)[:, 0]
        x = to_device(g, dtype)
        for shape in ({}, dict(mobius_pace_ns=-1), dict(mobius_blocks_per_sm=4, mobius_pace_ns=300)):
            y = _same_bits(plan, x, **shape)
            if dtype == mz.MZ_I64:
                assert np.array_equal(y.cpu().numpy(), mu.T @ g), (k, shape)
        mz.mz_plan_tune(plan.handle, mobius_pace_ns=600, mobius_blocks_per_sm=2)


def test_rows_too_long_keep_no_tables():
    p = pg.planted_chain_poset(2000, 300, 9, cross_deg=3)
    plan = mz.Plan(p.n, p.src, p.dst, p.chain_id)
    assert plan.info["lookahead_width"] == 0
    g = pg.function_values(p.n, 1, "i64:1000", 8)[:, 0]
    Z = oracle.closure(p.n, p.src, p.dst)
    y = _same_bits(plan, to_device(g, mz.MZ_I64))
    assert np.array_equal(y.cpu().numpy(), oracle.mobius_function(Z).T @ g)


def test_antichain_schedule_keeps_no_tables():
    p = pg.planted_chain_poset(2000, 30, 10, cross_deg=3)
    plan = mz.Plan(p.n, p.src, p.dst, p.chain_id, mobius_schedule=mz.MZ_SCHED_ANTICHAIN)
    assert plan.info["lookahead_width"] == 0


def test_several_posets_same_bits():
    ps = [pg.planted_chain_poset(2048, 100, 31, cross_deg=2), pg.paper_example(),
          pg.planted_chain_poset(1500, 40, 32, cross_deg=3), pg.boolean_lattice(6),
          pg.chain_poset(700, seed=34), pg.planted_chain_poset(1024, 4, 35, cross_p=4 / 1024)]
    cids = [p.chain_id if p.name.startswith(("planted", "chain")) else None for p in ps]
    plan = mz.Plan.batch([(p.n, p.src, p.dst, c) for p, c in zip(ps, cids)])
    assert plan.info["lookahead_width"] == 8
    off = np.cumsum([0] + [p.n for p in ps])
    n = int(off[-1])
    g = pg.function_values(n, 1, "i64:1000", 11)[:, 0]
    y = _same_bits(plan, to_device(g, mz.MZ_I64)).cpu().numpy()
    for i, p in enumerate(ps):
        Z = oracle.closure(p.n, p.src, p.dst)
        sl = slice(off[i], off[i + 1])
        assert np.array_equal(y[sl], oracle.mobius_function(Z).T @ g[sl]), p.name
    for dtype in (mz.MZ_F64, mz.MZ_F32C):
        _same_bits(plan, to_device(pg.function_values(n, 1, KINDS[dtype], 12)[:, 0], dtype))


@pytest.mark.parametrize("n,k", [(1 << 20, 64), (1 << 22, 128)])
def test_full_size_same_bits_and_round_trip(n, k):
    p = pg.planted_chain_poset(n, k, 1, cross_deg=3 if k == 64 else 2)
    plan = mz.Plan(p.n, p.src, p.dst, p.chain_id, device_build=True)
    assert plan.info["lookahead_width"] == k // 16
    f = pg.function_values(p.n, 1, "i64:1048576", 13)[:, 0]
    x = to_device(f, mz.MZ_I64)
    g = plan.zeta(x)
    assert torch.equal(_same_bits(plan, g), x)
    for dtype in (mz.MZ_F64, mz.MZ_F32C):
        _same_bits(plan, to_device(pg.function_values(p.n, 1, KINDS[dtype], 14)[:, 0], dtype))


@pytest.mark.parametrize("withhold", [3, 200, 900])
def test_withheld_row_still_times_out(withhold):
    """The test hook's withheld row is never published and never computed by a reader
    either: some wait runs out and mz_check reports it."""
    p = pg.planted_chain_poset(20000, 24, 3, cross_deg=3)
    bad = mz.Plan(p.n, p.src, p.dst, p.chain_id, spin_limit=20000, debug_withhold=withhold)
    assert bad.info["lookahead_width"] == 2
    mz.mz_plan_tune(bad.handle, mobius_lanes=32, mobius_lookahead=1)
    bad.mobius(to_device(pg.function_values(p.n, 1, "i64:1000", 15)[:, 0], mz.MZ_I64))
    with pytest.raises(mz.MzError) as e:
        bad.check()
    assert e.value.status == mz.MZ_ERR_TIMEOUT

"""GPU parity of the batched float transforms against the oracle.

The batched forms (B functions per poset, many posets per plan) are what the
4096-poset workload times: F32C and fp64 at B = 32, one plan of posets of uneven
n and k, replayed from a captured CUDA graph, under launch shapes an autotuner
picks. Each case is compared element by element with the oracle on sampled
columns (the last column b = B - 1 included), with the componentwise metrics of
gpu_util: zeta against Z|f|, Moebius by its residual against Z|f_out| + |g| and
by its forward error against |M| Z |f|.
"""
import numpy as np
import pytest
import torch

import oracle
import posetgen as pg
import paper_2211_13706_gb300 as mz
from paper_2211_13706_gb300 import autotune
from gpu_util import assert_close, from_device, to_device

pytestmark = pytest.mark.gpu

SCHEDS = [mz.MZ_SCHED_ULEVEL, mz.MZ_SCHED_ANTICHAIN]
FLOATS = [mz.MZ_F64, mz.MZ_F32C]


def _kind(dtype):
    return "f64u" if dtype == mz.MZ_F64 else "f32u"


def _exact(col, dtype):
    """The input column as the oracle sees it (fp32 data upcast exactly)."""
    return np.asarray(col, np.float64)


def _check_zeta_cols(got, f, Z, dtype, cols, what):
    for b in cols:
        ex = _exact(f[:, b], dtype)
        assert_close(got[:, b], oracle.zeta(Z, ex), oracle.zeta(Z, np.abs(ex)), dtype, f"{what} zeta col {b}")


def _check_mobius_cols(out, g, Z, mu, dtype, cols, what):
    for b in cols:
        ex = _exact(g[:, b], dtype)
        ref = oracle.mobius(Z, ex, "mu", mu=mu)
        res = oracle.zeta(Z, out[:, b]) - ex
        assert_close(res, np.zeros_like(res), oracle.zeta(Z, np.abs(out[:, b])) + np.abs(ex), dtype,
                     f"{what} mobius residual col {b}")
        fwd = np.abs(mu.T).astype(np.float64) @ (Z.astype(np.float64) @ np.abs(ref))
        assert_close(out[:, b], ref, fwd, dtype, f"{what} mobius forward col {b}")


# ----------------------------------------------------------------------------- one poset, B up to 32

@pytest.fixture(scope="module")
def c1():
    p = pg.planted_chain_poset(4096, 16, 1, cross_p=4 / 4096)
    Z = oracle.closure(p.n, p.src, p.dst)
    return p, Z, oracle.mobius_function(Z)


@pytest.mark.parametrize("sched", SCHEDS)
@pytest.mark.parametrize("dtype", FLOATS)
def test_c1_float_mobius_batched(c1, dtype, sched):
    """Moebius at B = 4, 16, 32 (every lane-group width of the batched wavefront, B = 32 the
    one the batched workload runs) on n = 4096, k = 16."""
    p, Z, mu = c1
    plan = mz.Plan(p.n, p.src, p.dst, p.chain_id, mobius_schedule=sched)
    for batch in (4, 16, 32):
        g = pg.function_values(p.n, batch, _kind(dtype), 40 + batch)
        out = from_device(plan.mobius(to_device(g, dtype)), dtype)
        plan.check()
        _check_mobius_cols(out, g, Z, mu, dtype, sorted({0, batch // 2 - 1, batch - 1}), f"B={batch}")


# ----------------------------------------------------------------------------- many posets, B = 32

def _uneven_posets():
    """Posets of uneven n and k (k from 1 to 256), as one batched plan holds them."""
    ps = [pg.planted_chain_poset(2048, 256, 31, cross_deg=2),
          pg.paper_example(),
          pg.planted_chain_poset(1500, 100, 32, cross_deg=2),
          pg.boolean_lattice(6),
          pg.planted_chain_poset(3000, 7, 33, cross_deg=2),
          pg.chain_poset(700, seed=34),
          pg.antichain_poset(40),
          pg.planted_chain_poset(1024, 4, 35, cross_p=4 / 1024)]
    cids = [p.chain_id if p.name.startswith(("planted", "chain")) else None for p in ps]
    return ps, cids


@pytest.fixture(scope="module")
def multi():
    ps, cids = _uneven_posets()
    Zs = [oracle.closure(p.n, p.src, p.dst) for p in ps]
    mus = [oracle.mobius_function(Z) for Z in Zs]
    off = np.cumsum([0] + [p.n for p in ps])
    return ps, cids, Zs, mus, off


def _cols(batch):
    return (0, 13, batch - 1)


def _check_multi(multi, f, g_out, m_in, m_out, dtype, what):
    ps, _, Zs, mus, off = multi
    for i, p in enumerate(ps):
        sl = slice(off[i], off[i + 1])
        _check_zeta_cols(g_out[sl], f[sl], Zs[i], dtype, _cols(f.shape[1]), f"{what} {p.name}")
        _check_mobius_cols(m_out[sl], m_in[sl], Zs[i], mus[i], dtype, _cols(f.shape[1]), f"{what} {p.name}")


@pytest.mark.parametrize("sched", SCHEDS)
@pytest.mark.parametrize("dtype", FLOATS)
def test_multi_poset_float_b32(multi, dtype, sched):
    """One plan of 8 posets (k = 1 ... 256), B = 32: zeta and Moebius of every poset
    against the oracle, columns 0, 13 and 31."""
    ps, cids, _, _, off = multi
    plan = mz.Plan.batch([(p.n, p.src, p.dst, c) for p, c in zip(ps, cids)], mobius_schedule=sched)
    n = int(off[-1])
    f = pg.function_values(n, 32, _kind(dtype), 50)
    gm = pg.function_values(n, 32, _kind(dtype), 51)
    g_out = from_device(plan.zeta(to_device(f, dtype)), dtype)
    m_out = from_device(plan.mobius(to_device(gm, dtype)), dtype)
    plan.check()
    _check_multi(multi, f, g_out, gm, m_out, dtype, "multi")


@pytest.mark.parametrize("dtype", FLOATS + [mz.MZ_I64])
def test_multi_poset_cuda_graph_replay(multi, dtype):
    """zeta then Moebius captured once in a CUDA graph and replayed on two different
    inputs copied into the captured buffer: each replay matches the oracle (int64 bit for
    bit, floats within tolerance), so replay re-runs the whole path rather than reusing
    results."""
    ps, cids, Zs, mus, off = multi
    plan = mz.Plan.batch([(p.n, p.src, p.dst, c) for p, c in zip(ps, cids)])
    n = int(off[-1])
    kind = "i64:1000" if dtype == mz.MZ_I64 else _kind(dtype)
    inputs = [pg.function_values(n, 32, kind, s) for s in (60, 61)]
    x = to_device(inputs[0], dtype)
    g = torch.empty_like(x)
    y = torch.empty_like(x)
    m_in = torch.empty_like(x)
    m_out = torch.empty_like(x)

    def step():
        plan.zeta(x, out=g)
        plan.mobius(m_in, out=m_out)

    m_in.copy_(x)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        step()                                  # workspaces exist before the capture
    torch.cuda.current_stream().wait_stream(side)
    cg = torch.cuda.CUDAGraph()
    with torch.cuda.graph(cg):
        step()
    for f in inputs:
        x.copy_(to_device(f, dtype))
        m_in.copy_(x)
        g.fill_(0)
        m_out.fill_(0)
        cg.replay()
        torch.cuda.synchronize()
        plan.check()
        gv, mv = from_device(g, dtype), from_device(m_out, dtype)
        if dtype == mz.MZ_I64:
            for i, p in enumerate(ps):
                sl = slice(off[i], off[i + 1])
                assert (gv[sl] == Zs[i].astype(np.int64) @ f[sl]).all(), p.name
                assert (mv[sl] == mus[i].T @ f[sl]).all(), p.name
        else:
            _check_multi(multi, f, gv, f, mv, dtype, "graph replay")
    del y


def test_every_autotune_shape(multi):
    """Every launch shape the autotuner may pick: int64 zeta and Moebius bit-exact, and F32C
    within tolerance, under each; then the shape autotune.tune itself picks."""
    ps, cids, Zs, mus, off = multi
    plan = mz.Plan.batch([(p.n, p.src, p.dst, c) for p, c in zip(ps, cids)])
    n = int(off[-1])
    fi = pg.function_values(n, 32, "i64:1000", 70)
    ff = pg.function_values(n, 32, "f32u", 71)
    xi, xf = to_device(fi, mz.MZ_I64), to_device(ff, mz.MZ_F32C)
    want_z = [Zs[i].astype(np.int64) @ fi[off[i]:off[i + 1]] for i in range(len(ps))]
    want_m = [mus[i].T @ fi[off[i]:off[i + 1]] for i in range(len(ps))]
    shapes = [dict(gather_blocks_per_sm=gb, mobius_blocks_per_sm=mb, mobius_pace_ns=pc)
              for gb in autotune.CANDIDATES["gather_blocks_per_sm"]
              for mb in autotune.CANDIDATES["mobius_blocks_per_sm"]
              for pc in autotune.CANDIDATES["mobius_pace_ns"]]
    # one function per row: every lane count with every blocks-per-SM choice
    xi1 = to_device(fi[:, :1].copy(), mz.MZ_I64)
    for lanes in autotune.CANDIDATES["mobius_lanes"]:
        for mb in autotune.CANDIDATES["mobius_blocks_per_sm"]:
            mz.mz_plan_tune(plan.handle, mobius_lanes=lanes, mobius_blocks_per_sm=mb)
            gm1 = plan.mobius(xi1).cpu().numpy()
            plan.check()
            for i in range(len(ps)):
                sl = slice(off[i], off[i + 1])
                assert (gm1[sl, 0] == want_m[i][:, 0]).all(), (lanes, mb, ps[i].name)
    for sh in shapes:
        mz.mz_plan_tune(plan.handle, **sh)
        gz = plan.zeta(xi).cpu().numpy()
        gm = plan.mobius(xi).cpu().numpy()
        plan.check()
        for i in range(len(ps)):
            sl = slice(off[i], off[i + 1])
            assert (gz[sl] == want_z[i]).all(), (sh, ps[i].name)
            assert (gm[sl] == want_m[i]).all(), (sh, ps[i].name)
    for sh in shapes[::7] + [autotune.tune(plan, xf)]:
        mz.mz_plan_tune(plan.handle, **sh)
        gv = from_device(plan.zeta(xf), mz.MZ_F32C)
        mv = from_device(plan.mobius(xf), mz.MZ_F32C)
        plan.check()
        for i, p in enumerate(ps[:4]):
            sl = slice(off[i], off[i + 1])
            _check_zeta_cols(gv[sl], ff[sl], Zs[i], mz.MZ_F32C, (31,), f"{sh} {p.name}")
            _check_mobius_cols(mv[sl], ff[sl], Zs[i], mus[i], mz.MZ_F32C, (31,), f"{sh} {p.name}")


@pytest.mark.parametrize("batch", [32, 64, 128])
def test_f32c_pair_gathers(multi, batch):
    """B a power of two >= 32 takes the packed-pair F32C gathers (zeta, and the Moebius leaf
    gather) over prefixes and double-word copies stored in column pairs, one to four
    column pairs per lane. Zeta and Moebius of every poset against the oracle on sampled
    columns; and the Moebius, whose every stage works column by column in a fixed order
    (no tile shape enters it, unlike the chain scan's), must give each column the bits the
    same column gets at B = 16, where each word is one (hi, lo) pair and no pair layout is
    used."""
    ps, cids, Zs, mus, off = multi
    plan = mz.Plan.batch([(p.n, p.src, p.dst, c) for p, c in zip(ps, cids)])
    n = int(off[-1])
    f = pg.function_values(n, batch, "f32u", 80 + batch)
    lo = (pg.function_values(n, batch, "f32u", 90 + batch) * np.float32(2.0 ** -30)).astype(np.float32)
    x = to_device((f, lo), mz.MZ_F32C)
    g = from_device(plan.zeta(x), mz.MZ_F32C)
    m = plan.mobius(x)
    plan.check()
    exact = f.astype(np.float64) + lo.astype(np.float64)
    mv = from_device(m, mz.MZ_F32C)
    cols = (0, 17, batch - 1)
    for i, p in enumerate(ps):
        sl = slice(off[i], off[i + 1])
        for b in cols:
            ex = exact[sl, b]
            assert_close(g[sl, b], oracle.zeta(Zs[i], ex), oracle.zeta(Zs[i], np.abs(ex)), mz.MZ_F32C,
                         f"B={batch} {p.name} zeta col {b}")
            res = oracle.zeta(Zs[i], mv[sl, b]) - ex
            assert_close(res, np.zeros_like(res), oracle.zeta(Zs[i], np.abs(mv[sl, b])) + np.abs(ex), mz.MZ_F32C,
                         f"B={batch} {p.name} mobius residual col {b}")
    for s in range(0, batch, 16):
        ms = plan.mobius(to_device((f[:, s:s + 16].copy(), lo[:, s:s + 16].copy()), mz.MZ_F32C))
        plan.check()
        assert torch.equal(m[:, :, s:s + 16].contiguous().view(torch.int32), ms.view(torch.int32)), s

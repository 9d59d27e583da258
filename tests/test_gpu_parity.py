"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Small and medium instances are compared element by element with the dense
oracle (exact arithmetic, correctly rounded floats); the full-size planted
posets (n = 2^20, k = 64 and n = 2^22, k = 128) are checked on sampled rows
that the oracle computes one by one, and through the identities
M (Z f) = f and Z (M g) = g on every element."""
import numpy as np
import pytest
import torch

import oracle
import posetgen as pg
import paper_2211_13706_gb300 as mz
from gpu_util import TOL, assert_close, exact_input, from_device, run, to_device

pytestmark = pytest.mark.gpu

DTYPES = [mz.MZ_I64, mz.MZ_F64, mz.MZ_F32C]
SCHEDS = [mz.MZ_SCHED_ULEVEL, mz.MZ_SCHED_ANTICHAIN]


def values(n, batch, dtype, seed, kind=None):
    if dtype == mz.MZ_I64:
        return pg.function_values(n, batch, kind or "i64:1000", seed)
    if dtype == mz.MZ_F64:
        return pg.function_values(n, batch, kind or "f64u", seed)
    return pg.function_values(n, batch, kind or "f32u", seed)


def squeeze(x, batch):
    return x[:, 0] if batch == 1 else x


def check_zeta(plan, Z, f, dtype, what):
    got = run(plan, "zeta", f, dtype)
    ex = exact_input(f, dtype)
    ref = oracle.zeta(Z, ex)
    mag = oracle.zeta(Z, np.abs(from_abs(ex)))
    assert_close(got, ref, mag, dtype, what)
    return got


def check_mobius(plan, Z, g, dtype, what, mu=None):
    """int64: bit-exact against the oracle's M g. Floats: the backward error (the
    residual Z f_out - g, exact) within TOL of Z|f_out| + |g|, and the forward error
    within TOL of |M| Z |f| (the componentwise condition of the triangular solve)."""
    got = run(plan, "mobius", g, dtype)
    ex = exact_input(g, dtype)
    if mu is None:
        mu = oracle.mobius_function(Z)
    ref = oracle.mobius(Z, ex, "mu", mu=mu)
    if dtype == mz.MZ_I64:
        assert_close(got, ref, None, dtype, what)
        return got
    gval = from_abs(ex) if not isinstance(ex, tuple) else ex[0].astype(np.float64) + ex[1].astype(np.float64)
    res = oracle.zeta(Z, got) - gval
    assert_close(res, np.zeros_like(res), oracle.zeta(Z, np.abs(got)) + np.abs(gval), dtype, what + " residual")
    fwd_mag = np.abs(mu.T).astype(np.float64) @ (Z.astype(np.float64) @ np.abs(ref))
    assert_close(got, ref, fwd_mag, dtype, what + " forward")
    return got


def from_abs(ex):
    if isinstance(ex, tuple):
        return np.abs(ex[0].astype(np.float64)) + np.abs(ex[1].astype(np.float64))
    return ex


# ----------------------------------------------------------------------------- the paper's example

@pytest.mark.parametrize("sched", SCHEDS)
@pytest.mark.parametrize("dtype", DTYPES)
def test_paper_example(dtype, sched):
    p = pg.paper_example()
    cid = np.array([1, 0, 1, 0, 2, 3, 1, 3, 0, 2, 3, 0], dtype=np.int32)
    plan = mz.Plan(p.n, p.src, p.dst, cid, build_transpose=True, mobius_schedule=sched)
    Z = oracle.closure(p.n, p.src, p.dst)
    for batch in (1, 3):
        f = squeeze(values(12, batch, dtype, 1), batch)
        g = check_zeta(plan, Z, f, dtype, "example zeta")
        if dtype == mz.MZ_I64:
            Zp = np.loadtxt("tests/golden/paper_example_Z.txt", dtype=np.int64)
            Mp = np.loadtxt("tests/golden/paper_example_M.txt", dtype=np.int64)
            assert (g == Zp @ f).all()
            assert (run(plan, "mobius", g, dtype) == f).all()
            assert (run(plan, "mobius", f, dtype) == Mp @ f).all()
            assert (run(plan, "zeta_T", f, dtype) == Zp.T @ f).all()
            assert (run(plan, "mobius_T", f, dtype) == Mp.T @ f).all()
        else:
            check_mobius(plan, Z, f, dtype, "example mobius")


# ----------------------------------------------------------------------------- C1-sized instance

@pytest.fixture(scope="module")
def c1():
    p = pg.planted_chain_poset(4096, 16, 1, cross_p=4 / 4096)
    Z = oracle.closure(p.n, p.src, p.dst)
    mu = oracle.mobius_function(Z)
    return p, Z, mu


@pytest.mark.parametrize("sched", SCHEDS)
def test_c1_int64_exact(c1, sched):
    """n = 4096, k = 16 chains of 256, f uniform integers in [-1000, 1000]: bit-exact."""
    p, Z, mu = c1
    plan = mz.Plan(p.n, p.src, p.dst, p.chain_id, build_transpose=True, mobius_schedule=sched)
    f = values(p.n, 1, mz.MZ_I64, 2)[:, 0]
    g = run(plan, "zeta", f, mz.MZ_I64)
    assert (g == oracle.zeta(Z, f)).all()
    back = run(plan, "mobius", g, mz.MZ_I64)
    assert (back == f).all()
    assert (run(plan, "mobius", f, mz.MZ_I64) == oracle.mobius(Z, f, "mu", mu=mu)).all()
    assert (run(plan, "zeta_T", f, mz.MZ_I64) == oracle.zeta_T(Z, f)).all()
    assert (run(plan, "mobius_T", f, mz.MZ_I64) == oracle.mobius_T(Z, f, mu=mu)).all()


@pytest.mark.parametrize("batch", [2, 3, 4, 16, 32, 33, 64])
def test_c1_int64_batched(c1, batch):
    p, Z, mu = c1
    plan = mz.Plan(p.n, p.src, p.dst, p.chain_id)
    f = values(p.n, batch, mz.MZ_I64, 3)
    g = run(plan, "zeta", f, mz.MZ_I64)
    ref = np.stack([Z.astype(np.int64) @ f[:, b] for b in range(batch)], axis=1)
    assert (g == ref).all()
    assert (run(plan, "mobius", g, mz.MZ_I64) == f).all()


@pytest.mark.parametrize("sched", SCHEDS)
@pytest.mark.parametrize("dtype", [mz.MZ_F64, mz.MZ_F32C])
def test_c1_float(c1, dtype, sched):
    p, Z, mu = c1
    plan = mz.Plan(p.n, p.src, p.dst, p.chain_id, mobius_schedule=sched)
    for kind in ("u", "ln"):
        f = values(p.n, 1, dtype, 4, ("f64" if dtype == mz.MZ_F64 else "f32") + kind)[:, 0]
        check_zeta(plan, Z, f, dtype, f"c1 zeta {kind}")
        g = oracle.zeta(Z, exact_input(f, dtype))          # exact g, rounded to fp64
        gin = g if dtype == mz.MZ_F64 else _split(g)
        check_mobius(plan, Z, gin, dtype, f"c1 mobius {kind}", mu=mu)


@pytest.mark.parametrize("sched", SCHEDS)
@pytest.mark.parametrize("dtype", [mz.MZ_F64, mz.MZ_F32C])
def test_c1_float_batched(c1, dtype, sched):
    """Batched floats (B = 4, 16, 32): sampled columns within tolerance of the oracle."""
    p, Z, mu = c1
    plan = mz.Plan(p.n, p.src, p.dst, p.chain_id, mobius_schedule=sched)
    for batch in (4, 16, 32):
        f = values(p.n, batch, dtype, 21, ("f64" if dtype == mz.MZ_F64 else "f32") + "u")
        got = run(plan, "zeta", f, dtype)
        for b in range(0, batch, 5):
            ex = exact_input(f[:, b], dtype)
            assert_close(got[:, b], oracle.zeta(Z, ex), oracle.zeta(Z, np.abs(from_abs(ex))), dtype,
                         f"batched zeta B={batch} col {b}")
    g = values(p.n, 4, dtype, 22, ("f64" if dtype == mz.MZ_F64 else "f32") + "u")
    gin = g if dtype == mz.MZ_F64 else (g, np.zeros_like(g))
    out = run(plan, "mobius", gin, dtype)
    for b in (0, 3):
        ex = exact_input(g[:, b], dtype)
        ref = oracle.mobius(Z, ex, "mu", mu=mu)
        gval = from_abs(ex) if not isinstance(ex, tuple) else ex[0].astype(np.float64)
        res = oracle.zeta(Z, out[:, b]) - gval
        assert_close(res, np.zeros_like(res), oracle.zeta(Z, np.abs(out[:, b])) + np.abs(gval), dtype,
                     f"batched mobius residual col {b}")
        fwd = np.abs(mu.T).astype(np.float64) @ (Z.astype(np.float64) @ np.abs(ref))
        assert_close(out[:, b], ref, fwd, dtype, f"batched mobius forward col {b}")


@pytest.mark.parametrize("sched", SCHEDS)
@pytest.mark.parametrize("batch", [8, 32])
def test_c1_int64_batched_round_trip_both_schedules(c1, sched, batch):
    p, Z, mu = c1
    plan = mz.Plan(p.n, p.src, p.dst, p.chain_id, mobius_schedule=sched, build_transpose=True)
    f = values(p.n, batch, mz.MZ_I64, 23)
    g = run(plan, "zeta", f, mz.MZ_I64)
    assert (g == (Z.astype(np.int64) @ f)).all()
    assert (run(plan, "mobius", g, mz.MZ_I64) == f).all()
    h = run(plan, "zeta_T", f, mz.MZ_I64)
    assert (h == (Z.T.astype(np.int64) @ f)).all()
    assert (run(plan, "mobius_T", h, mz.MZ_I64) == f).all()


def _split(x):
    hi = x.astype(np.float32)
    lo = (x - hi.astype(np.float64)).astype(np.float32)
    return hi, lo


# ----------------------------------------------------------------------------- edge cases

@pytest.mark.parametrize("dtype", DTYPES)
def test_edge_cases(dtype):
    cases = [
        pg.Poset(n=1, src=np.zeros(0, np.int32), dst=np.zeros(0, np.int32), chain_id=np.zeros(1, np.int32)),
        pg.antichain_poset(77),
        pg.chain_poset(9001, seed=3),             # one chain over several scan tiles, ragged tail
        pg.planted_chain_poset(1000, 1, 5),        # k = 1 via the generator
        pg.planted_chain_poset(1537, 7, 6, cross_p=6 / 1537),   # chain lengths not multiples of 32
        pg.boolean_lattice(7),
    ]
    for p in cases:
        Z = oracle.closure(p.n, p.src, p.dst)
        plan = mz.Plan(p.n, p.src, p.dst, p.chain_id, build_transpose=True)
        f = values(p.n, 1, dtype, 7)[:, 0]
        g = check_zeta(plan, Z, f, dtype, p.name)
        if dtype == mz.MZ_I64:
            assert (run(plan, "mobius", g, dtype) == f).all(), p.name
            assert (run(plan, "zeta_T", f, dtype) == oracle.zeta_T(Z, f)).all(), p.name
        if p.n <= 2000:
            mu = oracle.mobius_function(Z)
            check_mobius(plan, Z, f if dtype != mz.MZ_F32C else _split(f.astype(np.float64)), dtype,
                         p.name + " mobius", mu=mu)


def test_long_chain_many_tiles_int64():
    """A total order of 100003 elements: the scan spans 25 tiles (decoupled look-back)."""
    p = pg.chain_poset(100003, seed=4)
    plan = mz.Plan(p.n, p.src, p.dst, p.chain_id)
    f = values(p.n, 1, mz.MZ_I64, 8)[:, 0]
    order = np.concatenate([p.src[:1], p.dst])[::-1]          # bottom first
    want = np.empty(p.n, np.int64)
    want[order] = np.cumsum(f[order])
    g = run(plan, "zeta", f, mz.MZ_I64)
    assert (g == want).all()
    assert (run(plan, "mobius", g, mz.MZ_I64) == f).all()


def test_path_cover_plan_matches_planted_plan():
    p = pg.planted_chain_poset(3000, 12, 9, cross_p=3 / 3000)
    a = mz.Plan(p.n, p.src, p.dst, p.chain_id)
    b = mz.Plan(p.n, p.src, p.dst, None)
    f = values(p.n, 2, mz.MZ_I64, 10)
    ga, gb = run(a, "zeta", f, mz.MZ_I64), run(b, "zeta", f, mz.MZ_I64)
    assert (ga == gb).all()
    assert (run(b, "mobius", ga, mz.MZ_I64) == f).all()


# ----------------------------------------------------------------------------- paper-scale instances

@pytest.fixture(scope="module")
def c2():
    p = pg.planted_chain_poset(1 << 20, 64, 1, cross_deg=3)
    plan = mz.Plan(p.n, p.src, p.dst, p.chain_id)
    return p, plan


def test_c2_int64_sampled_rows_and_identities(c2):
    """n = 2^20, k = 64, f uniform in [-2^20, 2^20]: sampled rows exact, M Z f = f exactly."""
    p, plan = c2
    f = values(p.n, 1, mz.MZ_I64, 11, "i64:1048576")[:, 0]
    g = run(plan, "zeta", f, mz.MZ_I64)
    rows = np.random.default_rng(0).choice(p.n, 24, replace=False).tolist()
    assert (g[rows] == oracle.zeta_rows(p.n, p.src, p.dst, f, rows)).all()
    back = run(plan, "mobius", g, mz.MZ_I64)
    assert (back == f).all()
    # Moebius of an arbitrary g: on these posets |M g| far exceeds 2^63 (it grows like
    # 10^(0.23 * U-levels)), so the int64 result is exact modulo 2^64: Z f_out = g mod 2^64
    f2 = run(plan, "mobius", f, mz.MZ_I64)
    res, _ = oracle.mobius_residual_rows(p.n, p.src, p.dst, f2, f, rows)
    assert all(int(r) % (1 << 64) == 0 for r in res)


def test_c2_fp64(c2):
    p, plan = c2
    f = values(p.n, 1, mz.MZ_F64, 12)[:, 0]
    g = run(plan, "zeta", f, mz.MZ_F64)
    rows = np.random.default_rng(1).choice(p.n, 16, replace=False).tolist()
    ref = oracle.zeta_rows(p.n, p.src, p.dst, f, rows)
    mag = oracle.zeta_rows(p.n, p.src, p.dst, np.abs(f), rows)
    assert_close(g[rows], ref, mag, mz.MZ_F64, "c2 fp64 zeta rows")
    # backward error of the Moebius transform of rounded data (its forward error is
    # governed by |M|, astronomically large here, for any algorithm)
    back = run(plan, "mobius", g, mz.MZ_F64)
    res, rmag = oracle.mobius_residual_rows(p.n, p.src, p.dst, back, g, rows)
    assert_close(res, np.zeros_like(res), rmag, mz.MZ_F64, "c2 fp64 mobius residual rows")
    # exactly representable data (integers times 2^-20): every operation is exact
    fe = values(p.n, 1, mz.MZ_I64, 13, "i64:1000")[:, 0].astype(np.float64) * 2.0 ** -20
    ge = run(plan, "zeta", fe, mz.MZ_F64)
    assert (ge[rows] == oracle.zeta_rows(p.n, p.src, p.dst, fe, rows)).all()
    assert (run(plan, "mobius", ge, mz.MZ_F64) == fe).all()


@pytest.fixture(scope="module")
def c3():
    p = pg.planted_chain_poset(1 << 22, 128, 1, cross_deg=2)
    plan = mz.Plan(p.n, p.src, p.dst, p.chain_id)
    return p, plan


@pytest.mark.parametrize("kind", ["u", "ln"])
def test_c3_f32c_vs_fp64_zeta(c3, kind):
    """n = 2^22, k = 128: F32C and fp64 zeta on sampled rows within tolerance of the
    exact oracle (uniform [-1, 1] and log-normal sigma = 3 with random signs)."""
    p, plan = c3
    f32 = values(p.n, 1, mz.MZ_F32C, 13, "f32" + kind)[:, 0]
    rows = np.random.default_rng(2).choice(p.n, 8, replace=False).tolist()
    ref = oracle.zeta_rows(p.n, p.src, p.dst, f32.astype(np.float64), rows)
    mag = oracle.zeta_rows(p.n, p.src, p.dst, np.abs(f32.astype(np.float64)), rows)
    gc = run(plan, "zeta", f32, mz.MZ_F32C)
    assert_close(gc[rows], ref, mag, mz.MZ_F32C, "c3 f32c zeta rows")
    g64 = run(plan, "zeta", f32.astype(np.float64), mz.MZ_F64)
    assert_close(g64[rows], ref, mag, mz.MZ_F64, "c3 fp64 zeta rows")


def test_c3_exact_round_trips(c3):
    """Integer-valued data: the F32C pairs hold every partial sum exactly (< 2^48) and
    the fp64 prefixes too, so Moebius(zeta(f)) = f bit for bit in both float forms."""
    p, plan = c3
    fi = values(p.n, 1, mz.MZ_I64, 14, "i64:1000")[:, 0]
    x = to_device(fi.astype(np.float32), mz.MZ_F32C)
    back = plan.mobius(plan.zeta(x))
    plan.check()
    assert torch.equal(back, x)
    x64 = to_device(fi.astype(np.float64), mz.MZ_F64)
    back64 = plan.mobius(plan.zeta(x64))
    plan.check()
    assert torch.equal(back64, x64)


# ----------------------------------------------------------------------------- failure detection

@pytest.mark.parametrize("dtype", [mz.MZ_I64, mz.MZ_F64])
def test_bounded_wait_reports_timeout_and_context_survives(dtype):
    """A withheld publication makes the waits run out: the kernels return, mz_check
    reports MZ_ERR_TIMEOUT once, and the context and other plans keep working."""
    p = pg.planted_chain_poset(20000, 8, 3, cross_deg=2)
    bad = mz.Plan(p.n, p.src, p.dst, p.chain_id, spin_limit=20000, debug_withhold=3)
    f = values(p.n, 1, dtype, 14)[:, 0]
    x = to_device(f, dtype)
    bad.zeta(x)
    with pytest.raises(mz.MzError) as e:
        bad.check()
    assert e.value.status == mz.MZ_ERR_TIMEOUT
    bad.mobius(x)
    with pytest.raises(mz.MzError) as e:
        bad.check()
    assert e.value.status == mz.MZ_ERR_TIMEOUT
    bad.check()                                     # cleared
    good = mz.Plan(p.n, p.src, p.dst, p.chain_id)
    if dtype == mz.MZ_I64:
        g = run(good, "zeta", f, dtype)
        assert (run(good, "mobius", g, dtype) == f).all()


def test_launch_counts():
    p = pg.planted_chain_poset(5000, 8, 2, cross_deg=2)
    plan = mz.Plan(p.n, p.src, p.dst, p.chain_id)
    x = to_device(values(p.n, 1, mz.MZ_I64, 1)[:, 0], mz.MZ_I64)
    plan.zeta(x)
    assert mz.mz_last_launch_count() == 2
    plan.mobius(x)
    assert mz.mz_last_launch_count() == 4            # init, forward substitution, leaf gather, V^-1
    plan.check()
    anti = mz.Plan(p.n, p.src, p.dst, p.chain_id, mobius_schedule=mz.MZ_SCHED_ANTICHAIN)
    anti.mobius(x)
    assert mz.mz_last_launch_count() == 2            # init, forward substitution writing f
    anti.check()


def test_argument_errors_on_device():
    p = pg.paper_example()
    plan = mz.Plan(p.n, p.src, p.dst, None)
    x = torch.zeros(12, dtype=torch.int64, device="cuda")
    with pytest.raises(mz.MzError) as e:
        plan.zeta(x, out=x)                          # overlapping input and output
    assert e.value.status == mz.MZ_ERR_INVALID_ARG
    with pytest.raises(mz.MzError) as e:
        plan.zeta_T(x)                               # built without the dual
    assert e.value.status == mz.MZ_ERR_UNSUPPORTED
    ws, wsb = plan.workspace(mz.MZ_I64, 1)
    y = torch.empty_like(x)
    with pytest.raises(mz.MzError) as e:
        mz.mz_zeta(plan.handle, mz.MZ_I64, x.data_ptr(), y.data_ptr(), 1, ws, 64, 0)
    assert e.value.status == mz.MZ_ERR_INVALID_ARG


# ----------------------------------------------------------------------------- autograd (transposes)

def test_autograd_backward_is_the_transpose():
    p = pg.planted_chain_poset(700, 5, 4, cross_p=4 / 700)
    Z = oracle.closure(p.n, p.src, p.dst)
    mu = oracle.mobius_function(Z)
    plan = mz.Plan(p.n, p.src, p.dst, p.chain_id, build_transpose=True)
    rng = np.random.default_rng(5)
    f = torch.tensor(rng.uniform(-1, 1, (p.n, 2)), dtype=torch.float64, device="cuda", requires_grad=True)
    w = torch.tensor(rng.uniform(-1, 1, (p.n, 2)), dtype=torch.float64, device="cuda")
    h = torch.tensor(rng.uniform(-1, 1, (p.n, 2)), dtype=torch.float64, device="cuda")
    loss = (w * mz.MobiusFn.apply(mz.ZetaFn.apply(f, plan) * h, plan)).sum()
    loss.backward()
    # d loss / d f = Z^T (h * M^T w)
    inner = oracle.mobius_T(Z, w.cpu().numpy(), mu=mu) * h.cpu().numpy()
    want = oracle.zeta_T(Z, inner)
    got = f.grad.cpu().numpy()
    assert np.abs(got - want).max() <= 1e-9 * np.abs(want).max()
    # central finite differences on a few coordinates (eps = 1e-3, fp64)
    with torch.no_grad():
        for (i, b) in [(0, 0), (123, 1), (p.n - 1, 0)]:
            e = torch.zeros_like(f)
            e[i, b] = 1e-3
            lp = (w * mz.MobiusFn.apply(mz.ZetaFn.apply(f + e, plan) * h, plan)).sum()
            lm = (w * mz.MobiusFn.apply(mz.ZetaFn.apply(f - e, plan) * h, plan)).sum()
            fd = (lp - lm).item() / 2e-3
            assert abs(fd - got[i, b]) <= 1e-6 * max(1.0, abs(got[i, b]))


# ----------------------------------------------------------------------------- lanes per row (one function)

@pytest.mark.parametrize("lanes", [1, 2, 4, 8, 32])
def test_c1_wavefront_lanes_per_row(c1, lanes):
    """One function with the U-level schedule: 1 to 32 lanes share a row of the forward
    substitution (chunks of 16 entries dealt to the lanes, sums met by shuffles): int64
    bit-exact and floats within tolerance under each."""
    p, Z, mu = c1
    plan = mz.Plan(p.n, p.src, p.dst, p.chain_id, build_transpose=True)
    assert mz.mz_plan_tune(plan.handle, mobius_lanes=lanes)["mobius_lanes"] == lanes
    f = values(p.n, 1, mz.MZ_I64, 31)[:, 0]
    assert (run(plan, "mobius", f, mz.MZ_I64) == oracle.mobius(Z, f, "mu", mu=mu)).all()
    assert (run(plan, "mobius_T", f, mz.MZ_I64) == oracle.mobius_T(Z, f, mu=mu)).all()
    assert (run(plan, "mobius", run(plan, "zeta", f, mz.MZ_I64), mz.MZ_I64) == f).all()
    for dtype in (mz.MZ_F64, mz.MZ_F32C):
        g = values(p.n, 1, dtype, 32)[:, 0]
        check_mobius(plan, Z, g if dtype == mz.MZ_F64 else _split(g.astype(np.float64)), dtype,
                     f"lanes {lanes} mobius", mu=mu)


@pytest.mark.parametrize("k", [10, 20, 60, 120, 250, 500])
def test_wavefront_tree_widths(k):
    """A warp per row meets the chunk sums in a butterfly only as wide as the plan's longest
    row (1 to 32 chunks of 16 entries here; the wider levels, which add only zeros, are
    one plus_zero): int64 exact against the oracle, fp64 within tolerance, and the same bits
    under every launch shape (results never depend on timing)."""
    p = pg.planted_chain_poset(2500, k, 60 + k, cross_deg=3)
    plan = mz.Plan(p.n, p.src, p.dst, p.chain_id)
    Z = oracle.closure(p.n, p.src, p.dst)
    mu = oracle.mobius_function(Z)
    f = values(p.n, 1, mz.MZ_I64, 61)[:, 0]
    g = values(p.n, 1, mz.MZ_F64, 62)[:, 0]
    xf = to_device(g, mz.MZ_F64)
    ref = None
    for shape in (dict(mobius_blocks_per_sm=2, mobius_pace_ns=600), dict(mobius_blocks_per_sm=1, mobius_pace_ns=-1),
                  dict(mobius_blocks_per_sm=4, mobius_pace_ns=300)):
        mz.mz_plan_tune(plan.handle, mobius_lanes=32, **shape)
        assert (run(plan, "mobius", f, mz.MZ_I64) == oracle.mobius(Z, f, "mu", mu=mu)).all(), shape
        y = plan.mobius(xf)
        plan.check()
        if ref is None:
            ref = y
            check_mobius(plan, Z, g, mz.MZ_F64, f"k={k} mobius", mu=mu)
        assert torch.equal(y.view(torch.int64), ref.view(torch.int64)), shape


@pytest.mark.parametrize("lanes", [1, 4, 16])
def test_c2_int64_round_trip_lanes_per_row(c2, lanes):
    p, plan = c2
    mz.mz_plan_tune(plan.handle, mobius_lanes=lanes)
    f = values(p.n, 1, mz.MZ_I64, 33, "i64:1048576")[:, 0]
    x = to_device(f, mz.MZ_I64)
    back = plan.mobius(plan.zeta(x))
    plan.check()
    mz.mz_plan_tune(plan.handle, mobius_lanes=4)
    assert torch.equal(back, x)

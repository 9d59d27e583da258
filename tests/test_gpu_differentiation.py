"""Differentiation: loss = sum(w * Moebius(zeta(f) * h)) with B = 16 functions on the
n = 2^20, k = 64 planted poset (cross out-degree 3); the backward pass runs the
transposed transforms, i.e. zeta and Moebius of the dual poset.

At this size the Moebius transform of generic data is astronomically large (it
grows like 10^(0.23 * U-levels)), so the full-size checks are exact ones: the
adjoint identities <Z u, v> = <u, Z^T v> and <M u, v> = <u, M^T v> in int64
(exact modulo 2^64), and central differences on the well-conditioned zeta part.
The full loss is checked on a 2048-node down-set of the same poset (a down-set
is convex, so it is a sub-poset): autograd against the oracle's Z^T and M^T and
against central differences (eps = 1e-3)."""
import numpy as np
import pytest
import torch

import oracle
import posetgen as pg
import paper_2211_13706_gb300 as mz
from gpu_util import assert_close

pytestmark = pytest.mark.gpu
B = 16


@pytest.fixture(scope="module")
def c5():
    p = pg.planted_chain_poset(1 << 20, 64, 5, cross_deg=3)
    plan = mz.Plan(p.n, p.src, p.dst, p.chain_id, build_transpose=True)
    return p, plan


def _wrap_dot(a, b):
    """<a, b> in int64 with wrap-around (exact modulo 2^64)."""
    return int((a * b).sum().item())


def test_adjoint_identities_exact(c5):
    p, plan = c5
    gen = torch.Generator(device="cuda").manual_seed(3)
    u = torch.randint(-1000, 1001, (p.n, B), generator=gen, device="cuda", dtype=torch.int64)
    v = torch.randint(-1000, 1001, (p.n, B), generator=gen, device="cuda", dtype=torch.int64)
    zu, ztv = plan.zeta(u), plan.zeta_T(v)
    mu, mtv = plan.mobius(u), plan.mobius_T(v)
    plan.check()
    assert _wrap_dot(zu, v) == _wrap_dot(u, ztv)
    assert _wrap_dot(mu, v) == _wrap_dot(u, mtv)
    assert torch.equal(plan.mobius(zu), u) and torch.equal(plan.mobius_T(ztv), v)


def test_zeta_gradient_by_central_differences(c5):
    p, plan = c5
    gen = torch.Generator(device="cuda").manual_seed(4)
    f = (torch.rand((p.n, B), generator=gen, device="cuda", dtype=torch.float64) * 2 - 1).requires_grad_()
    w = torch.rand((p.n, B), generator=gen, device="cuda", dtype=torch.float64) * 2 - 1
    loss = (w * mz.ZetaFn.apply(f, plan)).sum()
    loss.backward()
    eps = 1e-3
    with torch.no_grad():
        for i, b in [(0, 0), (12345, 7), (p.n - 1, 15), (777777, 3)]:
            e = torch.zeros_like(f)
            e[i, b] = eps
            lp = (w * mz.ZetaFn.apply(f + e, plan)).sum().item()
            lm = (w * mz.ZetaFn.apply(f - e, plan)).sum().item()
            fd = (lp - lm) / (2 * eps)
            assert abs(fd - f.grad[i, b].item()) <= 1e-6 * max(1.0, abs(fd))


@pytest.fixture(scope="module")
def sub(c5):
    p, _ = c5
    h = oracle.heights(p.n, p.src, p.dst)
    counts = np.cumsum(np.bincount(h))
    lvl = int(np.searchsorted(counts, 2048))
    q, _ = pg.sub_poset(p, h <= lvl)
    Z = oracle.closure(q.n, q.src, q.dst)
    mu = oracle.mobius_function(Z)
    plan = mz.Plan(q.n, q.src, q.dst, q.chain_id, build_transpose=True)
    return q, Z, mu, plan


def test_subinstance_is_a_down_set(c5, sub):
    q, Z, _, _ = sub
    assert 1500 <= q.n <= 4096
    # zeta rows of the sub-poset equal the full poset's zeta rows at the same nodes
    p, plan = c5
    h = oracle.heights(p.n, p.src, p.dst)
    keep = np.flatnonzero(h <= np.sort(h)[q.n - 1])[: q.n]
    f = pg.function_values(p.n, 1, "i64:1000", 9)[:, 0]
    g = plan.zeta(torch.from_numpy(f).cuda()).cpu().numpy()
    assert (oracle.zeta(Z, f[keep]) == g[keep]).all()


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_loss_gradient_on_subinstance(sub, dtype):
    q, Z, mu, plan = sub
    rng = np.random.default_rng(6)
    f0, w0, h0 = (rng.uniform(-1, 1, (q.n, B)) for _ in range(3))
    f = torch.tensor(f0, dtype=dtype, device="cuda", requires_grad=True)
    w = torch.tensor(w0, dtype=dtype, device="cuda")
    hh = torch.tensor(h0, dtype=dtype, device="cuda")
    loss = (w * mz.MobiusFn.apply(mz.ZetaFn.apply(f, plan) * hh, plan)).sum()
    loss.backward()
    got = f.grad.double().cpu().numpy()
    # dL/df = Z^T (h * M^T w), by the oracle in exact arithmetic (inputs as the GPU saw them)
    wv = w.double().cpu().numpy()
    hv = hh.double().cpu().numpy()
    mtw = oracle.mobius_T(Z, wv, mu=mu)
    want = oracle.zeta_T(Z, mtw * hv)
    # magnitude the error is measured against: the componentwise condition of M^T w
    # (|M^T| |Z^T| |M^T w|), carried through the product with h and through Z^T
    Zt = Z.T.astype(np.float64)
    cond = np.abs(mu).astype(np.float64) @ (Zt @ np.abs(mtw))
    mag = Zt @ (np.abs(hv) * cond)
    tol = 1e-12 if dtype == torch.float64 else 1e-5      # fp32 autograd rounds each transform to fp32
    err = np.abs(got - want) / np.maximum(mag, 1e-300)
    assert err.max() <= tol, err.max()
    # central differences, eps = 1e-3, in fp64
    with torch.no_grad():
        fd_f = torch.tensor(f0, dtype=torch.float64, device="cuda")
        wd, hd = w.double(), hh.double()
        for (i, b) in [(0, 0), (q.n // 2, 5), (q.n - 1, 15)]:
            e = torch.zeros_like(fd_f)
            e[i, b] = 1e-3
            lp = (wd * mz.MobiusFn.apply(mz.ZetaFn.apply(fd_f + e, plan) * hd, plan)).sum().item()
            lm = (wd * mz.MobiusFn.apply(mz.ZetaFn.apply(fd_f - e, plan) * hd, plan)).sum().item()
            fd = (lp - lm) / 2e-3
            assert abs(fd - got[i, b]) <= max(1e-6, tol * 10) * max(1.0, abs(fd), mag[i, b])


def test_f32c_transposes_on_subinstance(sub):
    """The compensated pair path of the transposes within 1e-10 of the exact oracle."""
    q, Z, mu, plan = sub
    h = pg.function_values(q.n, B, "f32u", 8)
    x = torch.from_numpy(np.stack([h, np.zeros_like(h)])).cuda()
    zt = plan.zeta_T(x)
    mt = plan.mobius_T(x)
    plan.check()
    zt = zt.double().cpu().numpy()
    mt = mt.double().cpu().numpy()
    for b in (0, 9):
        hb = h[:, b].astype(np.float64)
        assert_close(zt[0][:, b] + zt[1][:, b], oracle.zeta_T(Z, hb), oracle.zeta_T(Z, np.abs(hb)),
                     mz.MZ_F32C, f"zeta_T col {b}")
        ref = oracle.mobius_T(Z, hb, mu=mu)
        fwd = np.abs(mu).astype(np.float64) @ (Z.T.astype(np.float64) @ np.abs(ref))
        assert_close(mt[0][:, b] + mt[1][:, b], ref, fwd, mz.MZ_F32C, f"mobius_T col {b}")

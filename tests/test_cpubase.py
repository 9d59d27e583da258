"""The CPU timing baseline (the paper's fast transforms with OpenMP, cpubase/) against
the oracle: int64 exact, fp64 close; host only."""
import numpy as np
import pytest

import cpubase
import oracle
import posetgen as pg
import paper_2211_13706_gb300 as mz


def _cpu_plan(p, cid):
    plan = mz.Plan(p.n, p.src, p.dst, cid, host_only=True, niv_format=1)
    return cpubase.CpuPlan(plan, mz.MZ_EXPORT_NIV, mz.MZ_EXPORT_CHAIN_ID, mz.MZ_EXPORT_CHAIN_POS,
                           mz.MZ_EXPORT_LEVEL, mz.MZ_EXPORT_ULEVEL)


@pytest.mark.parametrize("maker", [
    lambda: (pg.paper_example(), None),
    lambda: (lambda q: (q, q.chain_id))(pg.planted_chain_poset(1500, 12, 3, cross_p=4 / 1500)),
    lambda: (pg.boolean_lattice(7), None),
    lambda: (pg.er_dag(600, 4, 2), None),
])
def test_cpu_baseline_matches_oracle(maker):
    p, cid = maker()
    cp = _cpu_plan(p, cid)
    Z = oracle.closure(p.n, p.src, p.dst)
    f = pg.function_values(p.n, 1, "i64:1000", 5)[:, 0]
    g = cp.zeta(f)
    assert np.array_equal(g, oracle.zeta(Z, f))
    assert np.array_equal(cp.mobius(g), f)
    assert np.array_equal(cp.mobius_u(g), f)          # U-level schedule, same exact result
    h = pg.function_values(p.n, 1, "i64:1000", 6)[:, 0]
    assert np.array_equal(cp.zeta(cp.mobius(h)), h)
    x = pg.function_values(p.n, 1, "f64u", 7)[:, 0]
    gx = cp.zeta(x)
    assert np.allclose(gx, oracle.zeta(Z, x), rtol=1e-12, atol=1e-12)
    assert np.allclose(cp.mobius(gx), x, rtol=1e-9, atol=1e-9)


def test_cpu_baseline_threads():
    assert cpubase.threads() >= 1

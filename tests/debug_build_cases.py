"""Transforms through the MZ_DEBUG build of the library, checked against the oracle.

Run as a script with MZ_LIBRARY=debug (tests/test_gpu_debug_build.py does): every
kernel then checks each index it takes from the niv map or a plan table, and the
library fills workspaces and outputs with a poison pattern before each transform.
Every case must leave the status word clear (no MZ_ERR_BOUNDS) and give the oracle's
result: int64 bit for bit, F32C within the tolerance of the other GPU tests, so a
word the kernels failed to write (still poison) or an index outside its array
fails it. Prints one line per case and exits non-zero on the first failure.
"""
import os
import sys

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))
sys.path.insert(0, HERE)

import oracle  # noqa: E402
import posetgen as pg  # noqa: E402
import paper_2211_13706_gb300 as mz  # noqa: E402
from gpu_util import assert_close, from_device, to_device  # noqa: E402


def exact_cases(name, plan, parts, batch):
    """int64 zeta, Moebius and (with the dual) their transposes of every poset in the plan."""
    n = plan.n
    f = pg.function_values(n, batch, "i64:1000", 3 + batch)
    f = f[:, 0].copy() if batch == 1 else f
    x = torch.from_numpy(f).cuda()
    outs = {"zeta": plan.zeta(x), "mobius": plan.mobius(x)}
    if plan.info["has_transpose"]:
        outs["zeta_T"] = plan.zeta_T(x)
        outs["mobius_T"] = plan.mobius_T(x)
    plan.check()
    off = 0
    for p, Z, mu in parts:
        sl = slice(off, off + p.n)
        fx = f[sl]
        want = {"zeta": Z.astype(np.int64) @ fx, "mobius": mu.T @ fx,
                "zeta_T": Z.T.astype(np.int64) @ fx, "mobius_T": mu @ fx}
        for k, v in outs.items():
            assert np.array_equal(v.cpu().numpy()[sl], want[k]), (name, p.name, k, batch)
        off += p.n


def f32c_cases(name, plan, parts, batch):
    n = plan.n
    f = pg.function_values(n, batch, "f32u", 7 + batch)
    f = f[:, 0].copy() if batch == 1 else f
    x = to_device(f, mz.MZ_F32C)
    g = from_device(plan.zeta(x), mz.MZ_F32C)
    m = from_device(plan.mobius(x), mz.MZ_F32C)
    plan.check()
    off = 0
    for p, Z, mu in parts:
        sl = slice(off, off + p.n)
        ex = f[sl].astype(np.float64)
        gg, mm = g[sl], m[sl]
        if batch > 1:
            ex, gg, mm = ex[:, -1], gg[:, -1], mm[:, -1]
        assert_close(gg, oracle.zeta(Z, ex), oracle.zeta(Z, np.abs(ex)), mz.MZ_F32C, f"{name} {p.name} zeta")
        res = oracle.zeta(Z, mm) - ex
        assert_close(res, np.zeros_like(res), oracle.zeta(Z, np.abs(mm)) + np.abs(ex), mz.MZ_F32C,
                     f"{name} {p.name} mobius residual")
        off += p.n


def parts_of(ps):
    out = []
    for p in ps:
        Z = oracle.closure(p.n, p.src, p.dst)
        out.append((p, Z, oracle.mobius_function(Z)))
    return out


def main():
    assert mz.LIBRARY_PATH.endswith("libmz_debug.so"), mz.LIBRARY_PATH
    torch.cuda.set_device(0)
    planted = pg.planted_chain_poset(3000, 24, 5, cross_deg=3)
    er = pg.er_dag(1500, 4, 6)
    singles = {
        "dense": (planted, dict(build_transpose=True)),
        "dense_antichain": (planted, dict(mobius_schedule=mz.MZ_SCHED_ANTICHAIN)),
        "sparse": (er, dict(niv_format=2, build_transpose=True)),
        "device_build": (planted, dict(device_build=True)),
    }
    for name, (p, opts) in singles.items():
        cid = p.chain_id if p.name.startswith(("planted", "chain")) else None
        plan = mz.Plan(p.n, p.src, p.dst, cid, **opts)
        parts = parts_of([p])
        for batch in (1, 3, 32):
            exact_cases(name, plan, parts, batch)
        for batch in (1, 32):
            f32c_cases(name, plan, parts, batch)
        print("ok", name, flush=True)
        plan.close()
    ps = [pg.planted_chain_poset(1024, 100, 11, cross_deg=2), pg.paper_example(), pg.boolean_lattice(5),
          pg.planted_chain_poset(700, 6, 12, cross_deg=2)]
    cids = [p.chain_id if p.name.startswith("planted") else None for p in ps]
    for name, opts in (("batch", {}), ("batch_device_build", dict(device_build=True))):
        plan = mz.Plan.batch([(p.n, p.src, p.dst, c) for p, c in zip(ps, cids)], **opts)
        parts = parts_of(ps)
        for batch in (1, 32):
            exact_cases(name, plan, parts, batch)
            f32c_cases(name, plan, parts, batch)
        print("ok", name, flush=True)
        plan.close()
    # both lane counts of the one-function wavefront under the checks
    plan = mz.Plan(planted.n, planted.src, planted.dst, planted.chain_id)
    parts = parts_of([planted])
    for lanes in (32, 1):
        mz.mz_plan_tune(plan.handle, mobius_lanes=lanes)
        exact_cases(f"lanes{lanes}", plan, parts, 1)
    print("ok wavefront shapes", flush=True)
    print("all debug cases ok")


if __name__ == "__main__":
    main()

"""CPU tests of the C ABI's host side: the library loads and exports every
declared symbol, and the host build (order, chains, niv map, levels, errors)
agrees with the oracle. Plans here are built host-only: no GPU is touched."""
import ctypes
import os
import re
from math import comb

import numpy as np
import pytest

import oracle
import posetgen as pg
import paper_2211_13706_gb300 as mz

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "mz.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mz_[a-z_A-Z0-9]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    names = declared_functions()
    assert len(names) >= 13
    for name in names:
        assert hasattr(mz.lib, name), name
    assert sorted(mz.EXPORTED) == names
    assert mz.LIBRARY_PATH.endswith("libmz.so")


def header_struct(name):
    """(field, C type) of the typedef struct `name` in mz.h, in order."""
    text = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "mz.h")).read(), flags=re.S)
    body = re.search(r"typedef struct \{([^}]*)\}\s*" + name + r"\s*;", text).group(1)
    fields = []
    for decl in body.split(";"):
        decl = " ".join(decl.split())
        if not decl:
            continue
        m = re.match(r"(.*?)\s*\(\s*\*\s*(\w+)\s*\)\s*\(.*\)$", decl)      # function pointer
        if m:
            fields.append((m.group(2), "ptr"))
            continue
        m = re.match(r"(.*?)(\**)\s*(\w+)$", decl)
        fields.append((m.group(3), "ptr" if m.group(2) else m.group(1).strip()))
    return fields


@pytest.mark.parametrize("cname,cls", [("mz_build_opts", "_Opts"), ("mz_plan_info_t", "PlanInfo"),
                                       ("mz_tuning", "Tuning")])
def test_binding_structs_mirror_the_header(cname, cls):
    """The binding's ctypes structures have the header's fields, in order, with the same
    types, so that the library and the binding agree on every offset."""
    ctype = {"int32_t": ctypes.c_int32, "int64_t": ctypes.c_int64, "ptr": ctypes.c_void_p}
    want = [(f, ctype[t]) for f, t in header_struct(cname)]
    got = list(getattr(mz, cls)._fields_)
    assert got == want


def test_status_strings():
    for code, name in enumerate(["MZ_OK", "MZ_ERR_INVALID_ARG", "MZ_ERR_CYCLE", "MZ_ERR_BAD_CHAINS", "MZ_ERR_OOM",
                                 "MZ_ERR_CUDA", "MZ_ERR_TIMEOUT", "MZ_ERR_UNSUPPORTED", "MZ_ERR_NO_DEVICE",
                                 "MZ_ERR_BOUNDS"]):
        assert mz.lib.mz_status_string(code).decode() == name


def build_host(p, chain_id="planted", **kw):
    cid = p.chain_id if isinstance(chain_id, str) else chain_id
    return mz.Plan(p.n, p.src, p.dst, cid, host_only=True, **kw)


def niv_nodes_from_oracle(p, chain_id):
    Z = oracle.closure(p.n, p.src, p.dst)
    return Z, oracle.niv(Z, chain_id)


def check_u_levels(ul, N, chain_id):
    """Levels of U's dependency graph: every dependency strictly lower, and every
    row above level 0 has a dependency exactly one level lower (longest path)."""
    n, k = N.shape
    for x in range(n):
        deps = [N[x, j] for j in range(k) if j != chain_id[x] and N[x, j] >= 0]
        if not deps:
            assert ul[x] == 0
        else:
            assert all(ul[d] < ul[x] for d in deps)
            assert max(ul[d] for d in deps) == ul[x] - 1


def test_paper_example_host_structures():
    p = pg.paper_example()
    cid = np.array([1, 0, 1, 0, 2, 3, 1, 3, 0, 2, 3, 0], dtype=np.int32)   # Z_1..Z_4 of the example
    plan = build_host(p, cid)
    info = plan.info
    assert info["n"] == 12 and info["k"] == 4 and info["nnz"] == 32 and info["levels"] == 5
    got = plan.export(mz.MZ_EXPORT_NIV)
    Z, want = niv_nodes_from_oracle(p, cid)
    assert (got == want).all()
    assert (plan.export(mz.MZ_EXPORT_LEVEL) == oracle.heights(p.n, p.src, p.dst)).all()
    check_u_levels(plan.export(mz.MZ_EXPORT_ULEVEL), want, cid)
    topo = plan.export(mz.MZ_EXPORT_TOPO)
    pos = np.empty(12, dtype=np.int64)
    pos[topo] = np.arange(12)
    assert (pos[p.src] < pos[p.dst]).all()
    cpos = plan.export(mz.MZ_EXPORT_CHAIN_POS)
    for j in range(4):                  # positions count from the bottom of each chain
        members = np.flatnonzero(cid == j)
        order = members[np.argsort(cpos[members])]
        assert all(Z[b, a] for a, b in zip(order, order[1:]))


@pytest.mark.parametrize("seed", [1, 2])
def test_planted_host_structures_match_oracle(seed):
    p = pg.planted_chain_poset(600, 6, seed, cross_p=4 / 600)
    plan = build_host(p, build_transpose=True)
    Z, want = niv_nodes_from_oracle(p, p.chain_id)
    assert (plan.export(mz.MZ_EXPORT_NIV) == want).all()
    assert plan.info["nnz"] == int((want >= 0).sum())
    assert (plan.export(mz.MZ_EXPORT_LEVEL) == oracle.heights(p.n, p.src, p.dst)).all()
    check_u_levels(plan.export(mz.MZ_EXPORT_ULEVEL), want, p.chain_id)
    assert plan.info["ulevels"] == plan.export(mz.MZ_EXPORT_ULEVEL).max() + 1
    # dual plan: the niv map of the poset with every edge flipped (closure = Z^T)
    Nd = oracle.niv(np.ascontiguousarray(Z.T), p.chain_id)
    assert (plan.export(mz.MZ_EXPORT_NIV, dual=True) == Nd).all()
    assert (plan.export(mz.MZ_EXPORT_LEVEL, dual=True) == oracle.heights(p.n, p.dst, p.src)).all()


def test_duplicate_and_transitive_edges_change_nothing():
    p = pg.planted_chain_poset(300, 4, 3, cross_p=5 / 300)
    Z = oracle.closure(p.n, p.src, p.dst)
    rng = np.random.default_rng(0)
    xs, ys = np.nonzero(Z & ~np.eye(p.n, dtype=bool))
    pick = rng.choice(xs.size, 200, replace=False)
    src = np.concatenate([p.src, p.src[:50], xs[pick]]).astype(np.int32)
    dst = np.concatenate([p.dst, p.dst[:50], ys[pick]]).astype(np.int32)
    a = build_host(p)
    b = mz.Plan(p.n, src, dst, p.chain_id, host_only=True)
    assert (a.export(mz.MZ_EXPORT_NIV) == b.export(mz.MZ_EXPORT_NIV)).all()
    assert b.info["edges"] == len(set(zip(src.tolist(), dst.tolist())))


@pytest.mark.parametrize("m", [4, 5, 6])
def test_path_cover_of_boolean_lattice_has_width_many_chains(m):
    """Alg. 1 on the cover graph of 2^[m]: a symmetric chain decomposition exists in the
    Hasse diagram, so a minimum path cover has C(m, m/2) paths = the width (Dilworth)."""
    p = pg.boolean_lattice(m)
    plan = mz.Plan(p.n, p.src, p.dst, None, host_only=True)
    assert plan.info["k"] == comb(m, m // 2)
    Z = oracle.closure(p.n, p.src, p.dst)
    cid = plan.export(mz.MZ_EXPORT_CHAIN_ID)
    assert (plan.export(mz.MZ_EXPORT_NIV) == oracle.niv(Z, cid)).all()


def test_path_cover_of_paper_example():
    p = pg.paper_example()
    plan = mz.Plan(p.n, p.src, p.dst, None, host_only=True)
    assert plan.info["k"] == 4          # width of the example (antichain {3,4,5,6}, Fig. 2)


def test_build_errors():
    with pytest.raises(mz.MzError) as e:
        mz.mz_build(3, [0, 1, 2], [1, 2, 0], host_only=True)
    assert e.value.status == mz.MZ_ERR_CYCLE
    with pytest.raises(mz.MzError) as e:
        mz.mz_build(3, [0, 1], [1, 1], host_only=True)
    assert e.value.status == mz.MZ_ERR_CYCLE          # self-loop
    with pytest.raises(mz.MzError) as e:
        mz.mz_build(3, [0], [3], host_only=True)
    assert e.value.status == mz.MZ_ERR_INVALID_ARG
    with pytest.raises(mz.MzError) as e:
        mz.mz_build(0, [], [], host_only=True)
    assert e.value.status == mz.MZ_ERR_INVALID_ARG
    # two incomparable elements put on one chain
    with pytest.raises(mz.MzError) as e:
        mz.mz_build(3, [0, 0], [1, 2], chain_id=[0, 1, 1], host_only=True)
    assert e.value.status == mz.MZ_ERR_BAD_CHAINS
    # a chain that skips an element in between is still a chain (comparable, transitively)
    h = mz.mz_build(3, [0, 1], [1, 2], chain_id=[5, 9, 5], host_only=True)
    assert mz.mz_plan_info(h)["k"] == 2
    mz.mz_destroy(h)


def test_host_only_plan_refuses_transforms():
    p = pg.paper_example()
    plan = build_host(p, None)
    with pytest.raises(mz.MzError) as e:
        mz.mz_zeta(plan.handle, mz.MZ_I64, 256, 4096, 1, 1 << 20, 1 << 20, 0)   # pointers never touched
    assert e.value.status == mz.MZ_ERR_NO_DEVICE
    with pytest.raises(mz.MzError) as e:
        mz.mz_zeta_T(plan.handle, mz.MZ_I64, 256, 4096, 1, 1 << 20, 1 << 20, 0)
    assert e.value.status in (mz.MZ_ERR_NO_DEVICE, mz.MZ_ERR_UNSUPPORTED)
    assert mz.mz_workspace_size(plan.handle, mz.MZ_F64, 3) >= (12 + 4) * 3 * 8


def test_singletons_and_antichain():
    plan = mz.Plan(1, [], [], None, host_only=True)
    assert plan.info["k"] == 1 and plan.info["levels"] == 1 and plan.info["nnz"] == 1
    q = pg.antichain_poset(50)
    plan = mz.Plan(q.n, q.src, q.dst, None, host_only=True)
    assert plan.info["k"] == 50 and plan.info["nnz"] == 50 and plan.info["ulevels"] == 1


def test_torch_allocator_option_on_host_only_plan():
    # host-only plans allocate no device memory: the callbacks are set but never called
    p = pg.paper_example()
    plan = mz.Plan(p.n, p.src, p.dst, None, host_only=True, torch_allocator=True, build_transpose=True)
    assert plan.info["device_bytes"] == 0
    assert plan.export(mz.MZ_EXPORT_LEVEL).max() == 5
    plan.close()

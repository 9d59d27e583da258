"""Plan files (mz_plan_save / mz_plan_load): the one-time precomputation written to a file
and read back.

On the CPU, host-only plans of every kind (caller's chains and Alg. 1's path cover, dense
and sparse maps, the dual, plans of several posets) round-trip: the plan info and every
export are equal, and saving the loaded plan gives the same bytes. Damaged or crafted
files are refused with MZ_ERR_INVALID_ARG naming what failed: a wrong magic, a bad
checksum, a truncated file, and a file whose checksum is right but whose niv map points
outside the slot array. On the GPU a loaded plan's transforms equal the built plan's bit
for bit, and a plan whose map was built on the device cannot be saved.
"""
import struct

import numpy as np
import pytest

import posetgen as pg
import paper_2211_13706_gb300 as mz

EXPORTS = (mz.MZ_EXPORT_CHAIN_ID, mz.MZ_EXPORT_CHAIN_POS, mz.MZ_EXPORT_LEVEL, mz.MZ_EXPORT_ULEVEL,
           mz.MZ_EXPORT_TOPO)


def _cases():
    pl = pg.planted_chain_poset(3000, 33, 2, cross_deg=3)
    ex = pg.paper_example()
    return {
        "paper_example_chains": ([(ex.n, ex.src, ex.dst, np.array([1, 0, 1, 0, 2, 3, 1, 3, 0, 2, 3, 0], np.int32))],
                                 dict(build_transpose=True)),
        "boolean_lattice_path_cover": ([(lambda p: (p.n, p.src, p.dst, None))(pg.boolean_lattice(6))], {}),
        "planted_dense_dual": ([(pl.n, pl.src, pl.dst, pl.chain_id)], dict(build_transpose=True)),
        "antichain_sparse": ([(lambda p: (p.n, p.src, p.dst, None))(pg.antichain_poset(600))], {}),
        "er_sparse_dual": ([(lambda p: (p.n, p.src, p.dst, None))(pg.er_dag(2000, 3, 4))],
                           dict(build_transpose=True, niv_format=2)),
        "several_posets": ([(pl.n, pl.src, pl.dst, pl.chain_id), (ex.n, ex.src, ex.dst, None),
                            (lambda p: (p.n, p.src, p.dst, None))(pg.chain_poset(100, 3))],
                           dict(build_transpose=True)),
    }


CASES = _cases()


def _build(posets, **opts):
    if len(posets) == 1:
        n, s, d, c = posets[0]
        return mz.Plan(n, s, d, c, **opts)
    return mz.Plan.batch(posets, **opts)


def _same_plans(a, b):
    assert a.info == b.info
    sides = (False, True) if a.info["has_transpose"] else (False,)
    for dual in sides:
        for what in EXPORTS:
            assert np.array_equal(a.export(what, dual), b.export(what, dual)), (what, dual)
        if a.info["components"] == 1:
            assert np.array_equal(a.export(mz.MZ_EXPORT_NIV, dual), b.export(mz.MZ_EXPORT_NIV, dual)), dual


@pytest.mark.parametrize("name", sorted(CASES))
def test_host_plan_round_trip(tmp_path, name):
    posets, opts = CASES[name]
    plan = _build(posets, host_only=True, **opts)
    f1, f2 = tmp_path / "a.mzplan", tmp_path / "b.mzplan"
    plan.save(str(f1))
    back = mz.Plan.load(str(f1), host_only=True)
    _same_plans(plan, back)
    back.save(str(f2))
    assert f1.read_bytes() == f2.read_bytes()


def _fnv1a(b: bytes) -> int:
    h = 1469598103934665603
    for x in b:
        h = ((h ^ x) * 1099511628211) & 0xFFFFFFFFFFFFFFFF
    return h


def _reseal(body: bytes) -> bytes:
    return body + struct.pack("<Q", _fnv1a(body))


def _refused(path, fragment):
    with pytest.raises(mz.MzError) as e:
        mz.Plan.load(str(path), host_only=True)
    assert e.value.status == mz.MZ_ERR_INVALID_ARG
    assert fragment in str(e.value), str(e.value)


def test_damaged_and_crafted_files_are_refused(tmp_path):
    p = pg.planted_chain_poset(500, 6, 3, cross_deg=2)
    plan = mz.Plan(p.n, p.src, p.dst, p.chain_id, host_only=True)
    good = tmp_path / "good.mzplan"
    plan.save(str(good))
    raw = good.read_bytes()
    bad = tmp_path / "bad.mzplan"
    _refused(tmp_path / "missing.mzplan", "cannot open")
    bad.write_bytes(b"")
    _refused(bad, "magic")
    bad.write_bytes(b"NOTAPLAN" + raw[8:])
    _refused(bad, "magic")
    flipped = bytearray(raw)
    flipped[len(raw) // 2] ^= 0x40
    bad.write_bytes(bytes(flipped))
    _refused(bad, "checksum")
    bad.write_bytes(_reseal(raw[:len(raw) // 2]))
    _refused(bad, "truncated")
    # a right checksum over a map entry outside the slot array: the first entry of the dense
    # map, after the header (24 bytes), the side's scalars (44) and seven arrays
    n, k = plan.info["n"], plan.info["k"]
    off = 24 + 44 + 5 * (8 + 4 * n) + (8 + 8 * (k + 1)) + (8 + 4 * (n + k)) + 8
    body = bytearray(raw[:-8])
    assert struct.unpack_from("<i", body, off)[0] in range(n + k)
    struct.pack_into("<i", body, off, n + k + 7)
    bad.write_bytes(_reseal(bytes(body)))
    _refused(bad, "dense map entries")
    # the untouched file still loads
    mz.Plan.load(str(good), host_only=True)


@pytest.mark.parametrize("kind", ["dense", "sparse"])
def test_mutated_files_never_load_out_of_range(tmp_path, kind):
    """Random 4-byte words of a valid file overwritten with random values (small, negative,
    huge), checksum recomputed: the loader either refuses the file with MZ_ERR_INVALID_ARG
    or gives a plan whose exports stay in range; it never crashes."""
    if kind == "dense":
        p = pg.planted_chain_poset(300, 5, 8, cross_deg=2)
        plan = mz.Plan(p.n, p.src, p.dst, p.chain_id, host_only=True, build_transpose=True)
    else:
        p = pg.er_dag(300, 3, 8)
        plan = mz.Plan(p.n, p.src, p.dst, None, host_only=True, niv_format=2)
    good = tmp_path / "good.mzplan"
    plan.save(str(good))
    body = good.read_bytes()[:-8]
    rng = np.random.default_rng(11)
    bad = tmp_path / "bad.mzplan"
    loaded = refused = 0
    for _ in range(300):
        m = bytearray(body)
        for _ in range(int(rng.integers(1, 4))):
            off = int(rng.integers(24, len(m) - 4)) & ~3
            val = int(rng.choice([rng.integers(-3, 3), rng.integers(0, 2 * p.n), rng.integers(-2**31, 2**31)]))
            struct.pack_into("<i", m, off, val)
        bad.write_bytes(_reseal(bytes(m)))
        try:
            q = mz.Plan.load(str(bad), host_only=True)
        except mz.MzError as e:
            assert e.status == mz.MZ_ERR_INVALID_ARG, str(e)
            refused += 1
            continue
        loaded += 1
        n, k = q.info["n"], q.info["k"]
        cid = q.export(mz.MZ_EXPORT_CHAIN_ID)
        assert ((cid >= 0) & (cid < k)).all()
        topo = q.export(mz.MZ_EXPORT_TOPO)
        assert np.array_equal(np.sort(topo), np.arange(n))
        niv = q.export(mz.MZ_EXPORT_NIV)
        assert ((niv >= -1) & (niv < n)).all()
        q.close()
    assert refused > 0


def test_save_and_load_arguments(tmp_path):
    p = pg.paper_example()
    plan = mz.Plan(p.n, p.src, p.dst, None, host_only=True)
    with pytest.raises(mz.MzError) as e:
        plan.save(str(tmp_path / "no_such_dir" / "x.mzplan"))
    assert e.value.status == mz.MZ_ERR_INVALID_ARG
    plan.save(str(tmp_path / "x.mzplan"))
    with pytest.raises(mz.MzError) as e:
        mz.Plan.load(str(tmp_path / "x.mzplan"), host_only=True, mobius_schedule=7)
    assert e.value.status == mz.MZ_ERR_INVALID_ARG


# ----------------------------------------------------------------------------- device plans

@pytest.mark.gpu
@pytest.mark.parametrize("name", ["planted_dense_dual", "er_sparse_dual", "several_posets"])
def test_loaded_plan_transforms_equal(tmp_path, name):
    """A plan loaded into the device runs the built plan's kernels on the same layouts:
    zeta, Moebius and the transposes equal bit for bit (int64 and fp64), under both
    schedules."""
    import torch
    posets, opts = CASES[name]
    n = sum(q[0] for q in posets)
    f = tmp_path / "p.mzplan"
    _build(posets, host_only=True, **opts).save(str(f))
    for sched in (mz.MZ_SCHED_ULEVEL, mz.MZ_SCHED_ANTICHAIN):
        built = _build(posets, mobius_schedule=sched, **opts)
        loaded = mz.Plan.load(str(f), mobius_schedule=sched)
        assert loaded.info == built.info
        for kind, dt in (("i64:1000", torch.int64), ("f64u", torch.float64)):
            x = torch.from_numpy(pg.function_values(n, 1, kind, 3)[:, 0]).cuda()
            for op in ("zeta", "mobius", "zeta_T", "mobius_T"):
                a, b = getattr(built, op)(x), getattr(loaded, op)(x)
                built.check()
                loaded.check()
                assert torch.equal(a.view(torch.int64), b.view(torch.int64)), (name, sched, kind, op)


@pytest.mark.gpu
def test_device_built_plan_is_not_saved(tmp_path):
    p = pg.planted_chain_poset(2000, 8, 5, cross_deg=2)
    plan = mz.Plan(p.n, p.src, p.dst, p.chain_id, device_build=True)
    with pytest.raises(mz.MzError) as e:
        plan.save(str(tmp_path / "d.mzplan"))
    assert e.value.status == mz.MZ_ERR_UNSUPPORTED

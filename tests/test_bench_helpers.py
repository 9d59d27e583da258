"""Host logic of bench.py: the algorithmic byte counts behind the roofline, the gate on
the committed ncu traffic figures, and the CPU baseline of the paper's method."""
import numpy as np

import bench
import posetgen as pg
import paper_2211_13706_gb300 as mz


def test_algorithmic_bytes_c2():
    n, k, B, nnz = 1 << 20, 64, 1, 67098120
    assert bench.algorithmic_bytes("niv_gather", n, k, B, nnz) == 4 * nnz + 4 * n + 8 * n
    assert round(bench.algorithmic_bytes("niv_gather", n, k, B, nnz) / 1e6, 1) == 281.0
    assert round(bench.algorithmic_bytes("mob_wave", n, k, B, nnz) / 1e6, 1) == 293.6   # every row
    # U-level schedule: the forward substitution reads only its rows' entries
    assert bench.algorithmic_bytes("mob_wave", n, k, B, nnz, (1000, 60000)) == 4 * 60000 + 12 * 1000 + 16 * 1000
    assert bench.algorithmic_bytes("mob_leaf", n, k, B, nnz, (1000, 60000)) == 4 * nnz + 8 * n + 16 * (n - 1000)
    assert round(bench.algorithmic_bytes("chain_scan", n, k, B, nnz) / 1e6, 1) == 21.0
    # every function column adds its own values, the map is read once
    assert bench.algorithmic_bytes("niv_gather", n, k, 32, nnz) - bench.algorithmic_bytes("niv_gather", n, k, 1, nnz) \
        == 8 * n * 31


def test_traffic_figures_follow_the_kernel_sources(tmp_path, monkeypatch):
    # the committed ncu figures count only while the kernel sources hash to their capture
    (tmp_path / "profiles").mkdir()
    csrc = tmp_path / "paper_2211_13706_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for f in ("mz_kernels.cu", "mz_arith.cuh"):
        (csrc / f).write_bytes(open(f"{bench.ROOT}/paper_2211_13706_gb300/csrc/{f}", "rb").read())
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h = bench.kernel_source_hash()
    (tmp_path / "profiles" / "ncu_traffic.txt").write_text(f"# c\nsource_hash: {h}\nmob_wave/c2/f64 = 123  # x\n")
    assert bench.load_traffic("mob_wave", "c2", "f64") == 123.0
    assert bench.load_traffic("mob_wave", "c3", "f64") is None
    (csrc / "mz_kernels.cu").write_bytes(b"changed")
    assert bench.load_traffic("mob_wave", "c2", "f64") is None


def test_cpu_paper_method_line():
    p = pg.planted_chain_poset(3000, 12, 4, cross_deg=2)
    plan = mz.Plan(p.n, p.src, p.dst, p.chain_id, host_only=True)
    f = pg.function_values(p.n, 1, "i64:1048576", 2)[:, 0]
    out = bench.cpu_paper_method(mz, plan, f, "i64")
    assert out["kind"] == "paper_method_cpu" and out["check"]["moebius_of_zeta_is_f"]
    assert out["one_core"]["threads"] == 1 and out["all_cores"]["value"] > 0
    x = pg.function_values(p.n, 1, "f64u", 3)[:, 0]
    z = bench.cpu_paper_method(mz, plan, x, "f64", gpu_g=np.zeros(p.n))
    assert "zeta_vs_gpu_max_rel" in z["check"]


def test_accuracy_leg_measures_errors():
    """The CPU-baseline leg's accuracy figures: exact results score 0, a perturbed zeta row
    and a perturbed Moebius value show up with about the size of the perturbation."""
    import oracle
    p = pg.planted_chain_poset(400, 5, 3, cross_p=4 / 400)
    Z = oracle.closure(p.n, p.src, p.dst)
    f = pg.function_values(p.n, 1, "f32u", 4)[:, 0].astype(np.float64)
    g = oracle.zeta(Z, f)
    m = oracle.mobius(Z, g)
    hi = f.astype(np.float32)
    pair = lambda x: (x.astype(np.float32), (x - x.astype(np.float32).astype(np.float64)).astype(np.float32))
    outs = {"f64": (f, g, m), "f32c": ((hi, np.zeros_like(hi)), pair(g), pair(m))}
    acc = bench.accuracy_leg([("small", p, outs, 30)], budget_s=60)
    assert acc["small"]["rows"] == 30
    assert acc["small"]["f64"]["zeta_max_rel"] < 1e-15 and acc["small"]["f64"]["mobius_residual_max_rel"] < 1e-15
    assert acc["small"]["f32c"]["zeta_max_rel"] < 1e-12
    bad_g = g.copy()
    rows = np.random.default_rng(7).choice(p.n, 30, replace=False)
    bad_g[rows[0]] *= 1 + 1e-6
    e = bench.oracle_row_errors(p, {"f64": (f, bad_g, m)}, [int(rows[0])])
    assert 1e-8 < e["f64"]["zeta_max_rel"] < 1e-5


def test_plan_file_leg(monkeypatch):
    """The plan-file variant: a host-only plan saved, loaded back (the loader is pointed at
    host-only loads, as there is no device here), sizes and times reported; a failure
    becomes an error entry instead of ending the bench line."""
    p = pg.planted_chain_poset(2000, 8, 4, cross_deg=2)
    plan = mz.Plan(p.n, p.src, p.dst, p.chain_id, host_only=True)
    real_load = mz.Plan.load
    monkeypatch.setattr(mz.Plan, "load", classmethod(lambda cls, path, **kw: real_load(path, host_only=True)))
    out = bench.time_plan_file(mz, plan, plan.info)
    assert out["same_plan_info"] and out["bytes"] > 4 * p.n * 8 and out["load_s"] >= 0
    monkeypatch.setattr(mz.Plan, "load", classmethod(lambda cls, path, **kw: (_ for _ in ()).throw(OSError("x"))))
    assert "error" in bench.time_plan_file(mz, plan, plan.info)

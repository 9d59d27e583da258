"""Pins for the CPU oracle: each check compares it with something it does not compute itself.

Sources of truth: the matrices and facts the paper prints for its 12-element
running example (tests/golden/, each file cites its passage), textbook closed
forms (Boolean lattice, divisor lattice, chains, antichains), a library
routine on independent data (numpy's matrix inverse, math.fsum), Yates'
subset-sum recursion, and brute force over every DAG on 6 labelled nodes.
"""
import math
import os

import numpy as np
import pytest

import oracle
import posetgen as pg

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def load_mat(name):
    return np.loadtxt(os.path.join(GOLD, f"paper_example_{name}.txt"), dtype=np.int64)


def load_facts():
    facts = {}
    for line in open(os.path.join(GOLD, "paper_example_facts.txt")):
        if line.startswith("#") or not line.strip():
            continue
        key, rest = line.split(":", 1)
        facts[key.strip()] = rest.split("--")[0].strip()
    return facts


def load_N():
    rows = []
    for line in open(os.path.join(GOLD, "paper_example_N.txt")):
        if line.startswith("#") or not line.strip():
            continue
        rows.append([-1 if t == "inf" else int(t) - 1 for t in line.split()])
    return np.array(rows, dtype=np.int64)


def example_chain_ids():
    facts = load_facts()
    cid = np.full(12, -1, dtype=np.int32)
    for j in range(4):
        for e in facts[f"chain_{j + 1}"].split():
            cid[int(e) - 1] = j
    assert (cid >= 0).all()
    return cid


# ----------------------------------------------------------------------------- the paper's example

@pytest.fixture(scope="module")
def example():
    A = load_mat("A")
    src, dst = np.nonzero(A)
    p = pg.paper_example()
    # the built-in copy of the edge list matches the fixture
    assert sorted(zip(p.src.tolist(), p.dst.tolist())) == sorted(zip(src.tolist(), dst.tolist()))
    Z = oracle.closure(12, src, dst)
    return src, dst, Z


def test_example_closure_is_printed_Z(example):
    _, _, Z = example
    assert (Z.astype(np.int64) == load_mat("Z")).all()


def test_example_mu_is_printed_M(example):
    _, _, Z = example
    mu = oracle.mobius_function(Z)
    M = mu.T                                   # M[x, y] = mu(y, x)
    assert (M == load_mat("M")).all()
    assert (M @ load_mat("Z") == np.eye(12, dtype=np.int64)).all()


def test_example_transforms_match_printed_matrices(example):
    _, _, Z = example
    rng = np.random.default_rng(0)
    f = rng.integers(-1000, 1001, size=12)
    g = oracle.zeta(Z, f)
    assert (g == load_mat("Z") @ f).all()
    assert (oracle.mobius(Z, g, "mu") == load_mat("M") @ g).all()
    assert (oracle.mobius(Z, g, "backsub") == f).all()
    # g(x_1) written out in Sec. 2.2: f(x1) + f(x3) + f(x4) + f(x6) + ... + f(x12)
    assert g[0] == f[0] + f[2] + f[3] + sum(f[5:12])


def test_example_niv_is_printed_N(example):
    _, _, Z = example
    N = oracle.niv(Z, example_chain_ids())
    assert (N == load_N()).all()
    facts = load_facts()
    assert int((N >= 0).sum()) == int(facts["nnz_N"])
    assert sorted((N[3] + 1).tolist()) == sorted(int(t) for t in facts["niv_4"].split())
    assert sorted((np.flatnonzero(Z[3]) + 1).tolist()) == [int(t) for t in facts["out_4"].split()]


def test_example_factorisation_U_V(example):
    _, _, Z = example
    cid = example_chain_ids()
    N = oracle.niv(Z, cid)
    U = np.zeros((12, 12), dtype=np.int64)
    for x in range(12):
        for z in N[x]:
            if z >= 0:
                U[x, z] = 1
    V = (Z & (cid[:, None] == cid[None, :])).astype(np.int64)   # closure of the chains
    assert (U == load_mat("U")).all()
    assert (V == load_mat("V")).all()
    assert (U @ V == load_mat("Z")).all()                    # Eq. (zfac)
    assert (V @ load_mat("Vinv") == np.eye(12, dtype=np.int64)).all()
    assert (load_mat("B") @ load_mat("Binv") == np.eye(12, dtype=np.int64)).all()
    # B = P V P^-1 with the printed cycles, B[i][j] = V[p(i)][p(j)]
    facts = load_facts()
    p = list(range(12))
    for cyc in facts["perm_cycles"].split("|"):
        c = [int(t) - 1 for t in cyc.split()]
        for a, b in zip(c, c[1:] + c[:1]):
            p[a] = b
    B = np.array([[V[p[i], p[j]] for j in range(12)] for i in range(12)])
    assert (B == load_mat("B")).all()
    # operation counts, Sec. 3 example: n - k scan additions, nnz(N) - n gather additions
    n, k, nnz = 12, 4, int((N >= 0).sum())
    assert n - k == int(facts["scan_adds"])
    assert nnz - n == int(facts["gather_adds"])
    assert nnz - k == int(facts["total_adds"])


def test_example_levels(example):
    src, dst, Z = example
    h = oracle.heights(12, src, dst)
    facts = load_facts()
    assert h.max() == int(facts["num_levels"])
    chain = [int(t) - 1 for t in facts["longest_chain"].split()]
    assert all(Z[a, b] for a, b in zip(chain, chain[1:]))     # it is a chain
    assert len(chain) == h.max()                              # Mirsky: #levels = longest chain
    for lv in range(1, h.max() + 1):
        nodes = np.flatnonzero(h == lv)
        sub = Z[np.ix_(nodes, nodes)]
        assert (sub == np.eye(nodes.size, dtype=bool)).all()  # each level is an antichain
    anti = [int(t) - 1 for t in facts["longest_antichain"].split()]
    assert (Z[np.ix_(anti, anti)] == np.eye(4, dtype=bool)).all()


# ----------------------------------------------------------------------------- closed forms

def yates_subset_sums(f, m):
    g = np.array(f, dtype=object)
    for b in range(m):
        for s in range(1 << m):
            if s >> b & 1:
                g[s] += g[s ^ (1 << b)]
    return g


@pytest.mark.parametrize("m", [4, 7])
def test_boolean_lattice(m):
    p = pg.boolean_lattice(m)
    Z = oracle.closure(p.n, p.src, p.dst)
    S = np.arange(p.n)
    assert (Z == ((S[:, None] & S[None, :]) == S[None, :])).all()      # T <= S iff T subset of S
    rng = np.random.default_rng(m)
    f = rng.integers(-10 ** 6, 10 ** 6, size=p.n)
    assert (oracle.zeta(Z, f) == yates_subset_sums(f, m).astype(np.int64)).all()
    mu = oracle.mobius_function(Z)
    pc = np.array([bin(int(v)).count("1") for v in S])
    sign = 1 - 2 * (np.abs(pc[None, :] - pc[:, None]) % 2)
    want = np.where(Z.T, sign, 0)                    # mu(T, S) = (-1)^|S \ T| for T subset of S
    assert (mu == want).all()
    h = oracle.heights(p.n, p.src, p.dst)
    assert (h == pc + 1).all() and h.max() == m + 1
    # up-set sums: superset sums by Yates on complemented masks
    r = oracle.zeta_T(Z, f)
    comp = (p.n - 1) ^ S
    assert (r == yates_subset_sums(f[comp], m)[comp].astype(np.int64)).all()


def test_boolean_lattice_float_rows_are_correctly_rounded():
    m = 6
    p = pg.boolean_lattice(m)
    Z = oracle.closure(p.n, p.src, p.dst)
    f = pg.function_values(p.n, 1, "f64ln", 3)[:, 0]
    g = oracle.zeta(Z, f)
    for s in range(p.n):
        sub = [f[t] for t in range(p.n) if t & s == t]
        assert g[s] == math.fsum(sub)


def mobius_nt(d):
    mu, q = 1, 2
    while q * q <= d:
        if d % q == 0:
            d //= q
            if d % q == 0:
                return 0
            mu = -mu
        q += 1
    return -mu if d > 1 else mu


def test_divisor_lattice():
    p, divs = pg.divisor_lattice(720720)
    assert p.n == 240
    Z = oracle.closure(p.n, p.src, p.dst)
    assert (Z == (divs[:, None] % divs[None, :] == 0)).all()
    rng = np.random.default_rng(5)
    f = rng.integers(-1000, 1001, size=p.n)
    g = oracle.zeta(Z, f)
    for i, d in enumerate(divs):
        assert g[i] == sum(int(f[j]) for j, e in enumerate(divs) if d % e == 0)
    mu = oracle.mobius_function(Z)
    for i, e in enumerate(divs):
        for j, d in enumerate(divs):
            assert mu[i, j] == (mobius_nt(int(d // e)) if d % e == 0 else 0)


def test_chain_and_antichain():
    p = pg.chain_poset(50, seed=1)
    Z = oracle.closure(p.n, p.src, p.dst)
    order = np.concatenate([p.src[:1], p.dst])             # top ... bottom
    f = np.random.default_rng(1).integers(-100, 101, size=p.n)
    g = oracle.zeta(Z, f)
    assert (g[order[::-1]] == np.cumsum(f[order[::-1]])).all()   # prefix sums from the bottom
    mu = oracle.mobius_function(Z)
    want = np.eye(p.n, dtype=np.int64)
    for a, b in zip(order[1:], order[:-1]):                 # b covers a
        want[a, b] = -1
    assert (mu == want).all()
    q = pg.antichain_poset(20)
    Zq = oracle.closure(q.n, q.src, q.dst)
    assert (Zq == np.eye(20, dtype=bool)).all()
    assert (oracle.mobius_function(Zq) == np.eye(20, dtype=np.int64)).all()


# ----------------------------------------------------------------------------- brute force

def test_all_dags_on_six_nodes():
    pairs = [(i, j) for i in range(6) for j in range(i + 1, 6)]
    rng = np.random.default_rng(6)
    for mask in range(1 << len(pairs)):
        e = [pairs[b] for b in range(len(pairs)) if mask >> b & 1]
        src = np.array([a for a, _ in e], dtype=np.int64)
        dst = np.array([b for _, b in e], dtype=np.int64)
        Z = oracle.closure(6, src, dst)
        # brute force reachability: powers of the adjacency matrix
        A = np.zeros((6, 6), dtype=np.int64)
        A[src, dst] = 1
        R = np.eye(6, dtype=np.int64)
        P = np.eye(6, dtype=np.int64)
        for _ in range(6):
            P = P @ A
            R = R + P
        assert (Z == (R > 0)).all()
        mu = oracle.mobius_function(Z)
        inv = np.rint(np.linalg.inv(Z.astype(np.float64))).astype(np.int64)
        assert (mu.T == inv).all()
        if mask % 97 == 0:
            f = rng.integers(-50, 51, size=6)
            assert (oracle.mobius(Z, oracle.zeta(Z, f)) == f).all()


# ----------------------------------------------------------------------------- planted posets

@pytest.fixture(scope="module")
def planted():
    p = pg.planted_chain_poset(768, 8, 11, cross_p=4 / 768)
    Z = oracle.closure(p.n, p.src, p.dst)
    return p, Z


def test_topological_order_is_a_linear_extension(planted):
    p, Z = planted
    order = oracle.topological_order(p.n, p.src, p.dst)
    pos = np.empty(p.n, dtype=np.int64)
    pos[order] = np.arange(p.n)
    assert (pos[p.src] < pos[p.dst]).all()
    with pytest.raises(oracle.CycleError):
        oracle.topological_order(3, [0, 1, 2], [1, 2, 0])


def test_niv_satisfies_reachability_theorem(planted):
    """Thm. 3: out(x) is the disjoint union over chains j of {z in Z_j : z <= niv_j(x)}."""
    p, Z = planted
    N = oracle.niv(Z, p.chain_id)
    for x in range(0, p.n, 7):
        rebuilt = np.zeros(p.n, dtype=bool)
        for j in range(N.shape[1]):
            if N[x, j] >= 0:
                rebuilt |= (p.chain_id == j) & Z[N[x, j]]
        assert (rebuilt == Z[x]).all()


def test_mobius_two_routes_agree_and_invert_zeta(planted):
    p, Z = planted
    f = pg.function_values(p.n, 2, "i64:1000", 4)
    g = oracle.zeta(Z, f)
    mu = oracle.mobius_function(Z)
    assert (oracle.mobius(Z, g, "mu", mu=mu) == f).all()
    assert (oracle.mobius(Z, g, "backsub") == f).all()
    assert ((mu.T.astype(object) @ Z.astype(object)) == np.eye(p.n, dtype=object)).all()
    h = pg.function_values(p.n, 1, "i64:1000", 5)[:, 0]
    assert (oracle.mobius_T(Z, oracle.zeta_T(Z, h), mu=mu) == h).all()
    # the transposes are the transforms of the dual poset (all edges flipped, Sec. 2.1)
    Zd = oracle.closure(p.n, p.dst, p.src)
    assert (Zd == Z.T).all()
    assert (oracle.zeta_T(Z, h) == oracle.zeta(Zd, h)).all()


def test_float_transforms_exact(planted):
    p, Z = planted
    f = pg.function_values(p.n, 1, "f64u", 7)[:, 0]
    g = oracle.zeta(Z, f)
    for x in range(0, p.n, 31):
        assert g[x] == math.fsum(f[Z[x]])
    # cancellation that plain fp64 summation gets wrong
    Zc = oracle.closure(3, [0, 1], [1, 2])
    assert oracle.zeta(Zc, np.array([1e16, 1.0, -1e16]))[0] == 1.0
    # Moebius of an exactly representable g: both routes, exact results
    fi = pg.function_values(p.n, 1, "i64:1000", 8)[:, 0].astype(np.float64) * 2.0 ** -20
    gi = oracle.zeta(Z, fi)
    assert (oracle.mobius(Z, gi, "mu") == fi).all()
    assert (oracle.mobius(Z, gi, "backsub") == fi).all()
    # an (hi, lo) fp32 pair input is the exact sum hi + lo
    hi = f.astype(np.float32)
    lo = (f - hi.astype(np.float64)).astype(np.float32)
    g2 = oracle.zeta(Z, (hi, lo))
    ref = oracle.zeta(Z, hi.astype(np.float64) + lo.astype(np.float64))
    assert (g2 == ref).all()


def test_sampled_rows_match_dense(planted):
    p, Z = planted
    f = pg.function_values(p.n, 1, "i64:1000", 9)[:, 0]
    g = oracle.zeta(Z, f)
    rows = list(range(0, p.n, 37))
    assert (oracle.zeta_rows(p.n, p.src, p.dst, f, rows) == g[rows]).all()
    res, mag = oracle.mobius_residual_rows(p.n, p.src, p.dst, f, g, rows)
    assert (res == 0).all() and (mag > 0).all()
    bad = f.copy()
    bad[int(np.flatnonzero(Z[rows[3]])[-1])] += 1
    res, _ = oracle.mobius_residual_rows(p.n, p.src, p.dst, bad, g, rows)
    assert res[3] == 1


def test_exact_values_roundtrip():
    from fractions import Fraction
    a = np.array([0.1, -3.5, 1e-300, 2.0 ** 60, 0.0, -np.finfo(np.float64).tiny])
    V, s = oracle.exact_values(a)
    assert all(Fraction(v, 1 << s) == Fraction(float(x)) for v, x in zip(V, a))
    hi = np.array([1.0, 2.5, -7.0], np.float32)
    lo = np.array([1e-9, -1e-12, 0.0], np.float32)
    V, s = oracle.exact_values((hi, lo))
    assert all(Fraction(v, 1 << s) == Fraction(float(h)) + Fraction(float(l)) for v, h, l in zip(V, hi, lo))

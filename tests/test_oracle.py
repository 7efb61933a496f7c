"""Pins of the CPU oracle against facts fixed by the paper and by mathematics
(closed forms, finite differences, textbook recursions, brute force), so that
a dropped term, a wrong index or a transposed operand in the oracle fails."""
import json
import os

import numpy as np
import pytest

import oracle
from oracle import con
from paper_2405_14060_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _spins(x):
    return 2 * np.asarray(x) - 1


def _unflatten(idx, cards):
    out = []
    for c in reversed(cards):
        out.append(idx % c)
        idx //= c
    return list(reversed(out))


# ------------------------------------------------------------ closed forms

def test_tree_ising_closed_form():
    """Tree Ising without fields: Z = 2^n prod_e cosh(J_e); p(s_i=+1)=1/2."""
    for n, seed in ((11, 1), (160, 2)):
        m = synth.tree_ising(n, seed)
        J = np.array([np.log(t[3]) for t in m.tables])   # table[1,1] = exp(J)
        expect = n * np.log(2.0) + np.sum(np.log(np.cosh(J)))
        assert abs(oracle.ve_pr(m) - expect) < 1e-10 * max(1, abs(expect))
        if n <= 20:
            assert abs(oracle.brute_pr(m) - expect) < 1e-10
        lz, marg = oracle.ve_mar(m)
        assert abs(lz - expect) < 1e-9
        for p in marg:
            np.testing.assert_allclose(p, [0.5, 0.5], atol=1e-12)


def test_tree_ising_edge_correlation_from_joint():
    """E[s_i s_j] = tanh(J_ij) on every tree edge (closed form)."""
    m = synth.tree_ising(9, 7)
    joint = oracle.brute_joint(m)
    cards = [2] * m.nvars
    X = np.array([_unflatten(i, cards) for i in range(len(joint))])
    S = _spins(X)
    for sc, t in zip(m.scopes, m.tables):
        i, j = sc
        J = np.log(t[3])
        corr = np.sum(joint * S[:, i] * S[:, j])
        assert abs(corr - np.tanh(J)) < 1e-12


def test_free_spins_with_fields():
    """J = 0: Z = prod_i 2 cosh(h_i), p(s_i=+1) = e^h / (2 cosh h)."""
    m = synth.grid_ising(4, 3)
    for k, sc in enumerate(m.scopes):
        if len(sc) == 2:
            m.tables[k] = np.ones(4)
    h = np.array([0.5 * np.log(t[1] / t[0]) for sc, t in zip(m.scopes, m.tables)
                  if len(sc) == 1])
    expect = np.sum(np.log(2 * np.cosh(h)))
    assert abs(oracle.brute_pr(m) - expect) < 1e-12
    assert abs(oracle.ve_pr(m) - expect) < 1e-12
    _, marg = oracle.ve_mar(m)
    for i, p in enumerate(marg):
        assert abs(p[1] - np.exp(h[i]) / (2 * np.cosh(h[i]))) < 1e-12


def test_bayes_net_normalisation():
    """A Bayesian network sums to one; evidence on parentless variables
    gives p(e) = prod of their prior CPT entries."""
    small = synth.bayes_net(12, 5)
    assert abs(oracle.brute_pr(small)) < 1e-12
    big = synth.bayes_net(300, synth.BASE_SEED + 3)
    assert abs(oracle.ve_pr(big)) < 1e-9
    roots = [(int(sc[0]), t) for sc, t in zip(big.scopes, big.tables) if len(sc) == 1]
    rng = np.random.default_rng(0)
    ev = np.full(big.nvars, -1, np.int32)
    expect = 0.0
    for v, t in roots[:25]:
        ev[v] = int(rng.integers(0, big.card[v]))
        expect += np.log(t[ev[v]])
    assert abs(oracle.ve_pr(big, ev) - expect) < 1e-9


# --------------------------------------------------- brute force vs VE

@pytest.mark.parametrize("seed", [0, 1, 2])
def test_elimination_matches_enumeration(seed):
    m = synth.random_markov(11, 14, 3, seed, cards=(2, 3))
    rng = np.random.default_rng(seed)
    ev = np.full(m.nvars, -1, np.int32)
    for v in rng.choice(m.nvars, 3, replace=False):
        ev[v] = int(rng.integers(0, m.card[v]))
    lzb, mb = oracle.brute_mar(m, ev)
    lzv, mv = oracle.ve_mar(m, ev)
    assert abs(lzb - lzv) < 1e-11
    assert abs(oracle.ve_pr(m, ev) - lzb) < 1e-11
    for a, b in zip(mb, mv):
        np.testing.assert_allclose(a, b, atol=1e-12)
    xb, lb = oracle.brute_map(m, ev)
    xv, lv = oracle.ve_map(m, ev)
    assert abs(lb - lv) < 1e-11
    np.testing.assert_array_equal(xb, xv)
    assert abs(oracle.log_weight(m, xv) - lv) < 1e-11


def test_order_independence():
    m = synth.grid_ising(6, 11)
    o1, _ = oracle.minfill_order(m)
    o2 = np.random.default_rng(3).permutation(m.nvars).astype(np.int32)
    assert abs(oracle.ve_pr(m, order=o1) - oracle.ve_pr(m, order=o2)) < 1e-12


# ------------------------------------------------------ MAR by derivatives

def test_marginals_are_log_z_derivatives():
    """d log Z / d h_i = E[s_i] = 2 p(s_i=+1) - 1 (central differences)."""
    m = synth.grid_ising(5, 17)
    _, marg = oracle.ve_mar(m)
    eps = 1e-5
    unary = [k for k, sc in enumerate(m.scopes) if len(sc) == 1]
    for k in unary[::4]:
        i = int(m.scopes[k][0])
        t0 = m.tables[k].copy()
        m.tables[k] = t0 * np.exp(eps * np.array([-1.0, 1.0]))
        lp = oracle.ve_pr(m)
        m.tables[k] = t0 * np.exp(-eps * np.array([-1.0, 1.0]))
        lm = oracle.ve_pr(m)
        m.tables[k] = t0
        fd = (lp - lm) / (2 * eps)
        assert abs(fd - (2 * marg[i][1] - 1)) < 1e-8


def test_clamped_marginal_matches_propagation():
    m = synth.grid_ising(6, 19)
    _, marg = oracle.ve_mar(m)
    for v in (0, 7, 20, 35):
        np.testing.assert_allclose(oracle.clamped_marginal(m, v), marg[v], atol=1e-12)


def test_bn_marginals_with_evidence():
    m = synth.bayes_net(14, 23)
    rng = np.random.default_rng(1)
    ev = synth.random_evidence(m, 0.2, rng)
    lzb, mb = oracle.brute_mar(m, ev)
    lzv, mv = oracle.ve_mar(m, ev)
    assert abs(lzb - lzv) < 1e-11
    for v, (a, b) in enumerate(zip(mb, mv)):
        np.testing.assert_allclose(a, b, atol=1e-12)
        assert abs(b.sum() - 1) < 1e-12
        if ev[v] >= 0:
            assert b[ev[v]] == 1.0


# --------------------------------------------------------------- MPE / MAP

def _viterbi(m):
    """Textbook max-product recursion on the chain of synth.chain_model."""
    n = m.nvars
    un = {int(sc[0]): np.log(t) for sc, t in zip(m.scopes, m.tables) if len(sc) == 1}
    pair = {int(sc[0]): np.log(t).reshape(m.card[sc[0]], m.card[sc[1]])
            for sc, t in zip(m.scopes, m.tables) if len(sc) == 2}
    delta = un[0].copy()
    back = []
    for i in range(1, n):
        s = delta[:, None] + pair[i - 1]
        back.append(np.argmax(s, axis=0))
        delta = s.max(axis=0) + un[i]
    x = [int(np.argmax(delta))]
    for b in reversed(back):
        x.append(int(b[x[-1]]))
    return np.array(x[::-1]), float(delta.max())


def test_map_chain_viterbi():
    for seed in range(3):
        m = synth.chain_model(40, [2, 3, 4] * 13 + [2], seed)
        xv, lv = _viterbi(m)
        xo, lo = oracle.ve_map(m)
        np.testing.assert_array_equal(xo, xv)
        assert abs(lo - lv) < 1e-10
    m = synth.chain_model(14, [2] * 14, 9)
    xb, lb = oracle.brute_map(m)
    xv, lv = _viterbi(m)
    np.testing.assert_array_equal(xb, xv)


def test_map_bn_local_optimality():
    w = synth.workload(3)
    m, ev = w.model, w.evid[0]
    x, lp = oracle.ve_map(m, ev)
    assert abs(oracle.log_weight(m, x) - lp) < 1e-9
    for v in range(m.nvars):
        if ev[v] >= 0:
            assert x[v] == ev[v]
            continue
        for y in range(m.card[v]):
            if y == x[v]:
                continue
            x2 = x.copy()
            x2[v] = y
            assert oracle.log_weight(m, x2) <= lp + 1e-12


# --------------------------------------------------------------------- MMAP

def test_mmap_small_matches_enumeration():
    for seed in range(3):
        m = synth.bayes_net(14, 40 + seed)
        rng = np.random.default_rng(seed)
        ev = synth.random_evidence(m, 0.2, rng)
        q = synth.mmap_query(m, ev, 0.4, rng)
        xb, lb = oracle.brute_mmap(m, q, ev)
        xv, lv = oracle.ve_mmap(m, q, ev)
        assert abs(lb - lv) < 1e-11
        np.testing.assert_array_equal(xb, xv)


def test_mmap_consistency_large():
    """The returned value equals log PR with Q clamped at q*, and no single
    flip of a query variable improves it."""
    w = synth.workload(3)
    m, ev, q = w.model, w.evid[0], w.query
    x, lp = oracle.ve_mmap(m, q, ev)
    e2 = ev.copy()
    e2[q] = x
    assert abs(oracle.ve_pr(m, e2) - lp) < 1e-9
    for i in range(0, len(q), 9):
        for y in range(m.card[q[i]]):
            if y == x[i]:
                continue
            e3 = e2.copy()
            e3[q[i]] = y
            assert oracle.ve_pr(m, e3) <= lp + 1e-12


# ------------------------------------------------------- joint marginals

def test_joint_marginal_tree_ising_closed_form():
    """Tree Ising without fields: an edge's pair marginal is
    exp(J s_i s_j) / (4 cosh J), and two spins joined through k have
    p(s_i, s_j) = (1 + s_i s_j tanh J_ik tanh J_kj) / 4 (closed forms)."""
    m = synth.tree_ising(12, 5)
    S = np.array([-1.0, 1.0])
    nbr = {}
    for sc, t in zip(m.scopes, m.tables):
        i, j = (int(x) for x in sc)
        J = np.log(t[3])
        nbr.setdefault(i, {})[j] = J
        nbr.setdefault(j, {})[i] = J
        expect = np.exp(J * np.outer(S, S)) / (4 * np.cosh(J))
        np.testing.assert_allclose(oracle.brute_joint_marginal(m, [i, j]), expect, atol=1e-12)
        np.testing.assert_allclose(oracle.clamped_joint_marginal(m, [j, i]), expect.T, atol=1e-12)
    k = next(v for v in nbr if len(nbr[v]) >= 2)
    i, j = list(nbr[k])[:2]
    t = np.tanh(nbr[k][i]) * np.tanh(nbr[k][j])
    expect = (1 + t * np.outer(S, S)) / 4
    np.testing.assert_allclose(oracle.brute_joint_marginal(m, [i, j]), expect, atol=1e-12)


def test_joint_marginal_enumeration_matches_clamped_elimination():
    """The enumeration route and the Bayes route (Z(e, Q = q) / Z(e) by
    elimination) agree; single-variable sets give the marginals; observed
    query variables put all mass on their value; every table sums to 1."""
    m = synth.random_markov(9, 12, 3, 8, cards=(2, 3, 4))
    ev = np.full(m.nvars, -1, np.int32)
    ev[4] = 1
    for query in ([2], [0, 5], [7, 1, 3], [3, 4], [8, 4, 6]):
        a = oracle.brute_joint_marginal(m, query, ev)
        b = oracle.clamped_joint_marginal(m, query, ev)
        assert a.shape == tuple(int(m.card[v]) for v in query)
        np.testing.assert_allclose(a, b, atol=1e-12)
        assert abs(a.sum() - 1) < 1e-12
        if 4 in query:
            ax = query.index(4)
            assert np.all(np.take(a, [x for x in range(int(m.card[4])) if x != 1], axis=ax) == 0)
    _, marg = oracle.brute_mar(m, ev)
    for v in (0, 2, 6):
        np.testing.assert_allclose(oracle.brute_joint_marginal(m, [v], ev), marg[v], atol=1e-12)


# ------------------------------------------------------------------ sampling

def test_sampling_matches_joint():
    m = synth.random_markov(7, 8, 3, 5, cards=(2, 3))
    ev = np.full(m.nvars, -1, np.int32)
    ev[2] = 1
    joint = oracle.brute_joint(m, ev)
    n = 60000
    free = [v for v in range(m.nvars) if ev[v] < 0]
    u = np.random.default_rng(0).random(n * len(free))
    s = oracle.ve_sample(m, n, u, ev)
    assert np.all(s[:, 2] == 1)
    cards = [int(m.card[v]) for v in free]
    idx = np.zeros(n, np.int64)
    for v, c in zip(free, cards):
        idx = idx * c + s[:, v]
    emp = np.bincount(idx, minlength=len(joint)) / n
    tv = 0.5 * np.abs(emp - joint).sum()
    assert tv < 0.02
    # chi-square over cells with expected count >= 5
    exp_cnt = joint * n
    keep = exp_cnt >= 5
    chi2 = np.sum((emp[keep] * n - exp_cnt[keep]) ** 2 / exp_cnt[keep])
    dof = keep.sum() - 1
    assert chi2 < dof + 6 * np.sqrt(2 * dof)


# -------------------------------------------------- contraction definition

def _golden():
    with open(os.path.join(GOLD, "paper_examples.json")) as f:
        return json.load(f)


def test_con_matrix_multiplication():
    """Eq. matrix-multiplication-contraction: con({i,j,k},{A_ij,B_jk},{i,k}) = AB."""
    g = _golden()["matmul"]
    rng = np.random.default_rng(0)
    A, B = rng.random((3, 4)), rng.random((4, 5))
    out = con.con_naive([tuple(g["A"]), tuple(g["B"])], [A, B], tuple(g["out"]))
    np.testing.assert_allclose(out, A @ B, rtol=1e-14)
    np.testing.assert_allclose(con.con_dense([tuple(g["A"]), tuple(g["B"])], [A, B],
                                             tuple(g["out"])), A @ B, rtol=1e-14)


def test_con_hyperedge_example():
    """Eq. more-complex-contraction (scope list of its second line; label l is
    a hyperedge shared by A, B and C)."""
    g = _golden()["five_tensor"]
    rng = np.random.default_rng(1)
    n = 3
    labels = [tuple(g["scopes"][k]) for k in "ABCDE"]
    ts = [rng.random([n] * len(l)) for l in labels]
    ref = np.einsum("il,l,kjl,kmn,jn->im", *ts)
    np.testing.assert_allclose(con.con_naive(labels, ts, tuple(g["out"])), ref, rtol=1e-13)
    np.testing.assert_allclose(con.con_dense(labels, ts, tuple(g["out"])), ref, rtol=1e-13)


def test_tcon_matches_maxplus_matmul():
    rng = np.random.default_rng(2)
    A, B = rng.normal(size=(4, 6)), rng.normal(size=(6, 3))
    s = A[:, :, None] + B[None, :, :]
    val, arg = con.tcon_dense([("i", "j"), ("j", "k")], [A, B], ("i", "k"))
    np.testing.assert_array_equal(val, s.max(axis=1))
    np.testing.assert_array_equal(arg, s.argmax(axis=1))
    v2, a2 = con.tcon_naive([("i", "j"), ("j", "k")], [A, B], ("i", "k"))
    np.testing.assert_array_equal(v2, val)
    for (i, k), (j,) in a2.items():
        assert j == arg[i, k]


def test_map_gap_is_the_enumerated_runner_up():
    """oracle.map_gap: the gap between the MAP assignment and the best other
    assignment equals the one read off the enumerated joint distribution
    (log of the top two probabilities), with and without evidence."""
    for seed in range(3):
        m = synth.random_markov(9, 12, 3, 50 + seed, cards=(2, 3))
        ev = np.full(m.nvars, -1, np.int32)
        if seed:
            ev[seed] = 1
        x, lp, gap = oracle.map_gap(m, ev)
        p = np.sort(oracle.brute_joint(m, ev))[::-1]
        assert abs(gap - (np.log(p[0]) - np.log(p[1]))) < 1e-9
        xb, lb = oracle.brute_map(m, ev)
        np.testing.assert_array_equal(x, xb)
        assert abs(lp - lb) < 1e-9

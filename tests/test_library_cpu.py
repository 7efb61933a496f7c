"""Host-side checks of libtn that need no GPU: the library loads and exports
every symbol include/tn.h declares, input validation, UAI I/O, tree
validation, and the planner's complexity accounting against an independent
recomputation of the keep rule."""
import os
import re
import tempfile

import numpy as np
import pytest

from paper_2405_14060_gb300 import build, synth, tn

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()


def _declared():
    with open(os.path.join(ROOT, "include", "tn.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(tn_[a-z_]+)\s*\(", text)))


def test_exports_every_declared_symbol():
    L = tn.lib()
    names = _declared()
    assert names, "no declarations found"
    for n in names:
        assert hasattr(L, n), n
    assert sorted(tn.EXPORTS) == names


def test_model_validation_errors():
    with pytest.raises(tn.TNError) as e:
        tn.Model.from_arrays([2, 0], [[0, 1]], [np.ones(0)])
    assert e.value.status == 1
    with pytest.raises(tn.TNError):
        tn.Model.from_arrays([2, 2], [[0, 2]], [np.ones(4)])
    with pytest.raises(tn.TNError):
        tn.Model.from_arrays([2, 2], [[0, 0]], [np.ones(4)])
    with pytest.raises(tn.TNError):
        tn.Model.from_arrays([2, 2], [[0, 1]], [np.array([1.0, -1.0, 1.0, 1.0])])
    with pytest.raises(tn.TNError):
        tn.Model.from_arrays([2, 2], [[0, 1]], [np.array([1.0, np.inf, 1.0, 1.0])])


def test_joint_marginal_argument_errors():
    """tn_joint_mar rejects a repeated or out-of-range query variable, an
    empty query, evidence out of range and a joint domain above 65536
    assignments before any device work (TN_E_ARG)."""
    m = synth.grid_ising(5, 1)
    M = tn.Model.from_synth(m)
    ev = np.full(m.nvars, -1, np.int32)
    for bad in ([3, 3], [m.nvars], [-1], [], list(range(17))):
        with pytest.raises(tn.TNError) as e:
            M.joint_mar(bad, ev)
        assert e.value.status == 1, bad
    ev[0] = 2
    with pytest.raises(tn.TNError) as e:
        M.joint_mar([1], ev)
    assert e.value.status == 1


def test_uai_roundtrip_and_parse_errors():
    m = synth.bayes_net(10, 3)
    with tempfile.TemporaryDirectory() as d:
        p = os.path.join(d, "m.uai")
        synth.write_uai(m, p)
        M = tn.Model.from_uai(p)
        assert M.nvars == m.nvars and M.nfactors == m.nfactors
        m2 = synth.read_uai(p)
        for a, b in zip(m.tables, m2.tables):
            np.testing.assert_array_equal(a, b)
        bad = os.path.join(d, "bad.uai")
        with open(bad, "w") as f:
            f.write("MARKOV\n2\n2 2\n1\n2 0 1\n3\n1 1 1\n")
        with pytest.raises(tn.TNError) as e:
            tn.Model.from_uai(bad)
        assert e.value.status == 2
        with open(bad, "w") as f:
            f.write("GRAPH\n")
        with pytest.raises(tn.TNError) as e:
            tn.Model.from_uai(bad)
        assert e.value.status == 2


def test_uai_evidence_and_query_files():
    """Evidence files in both UAI forms (one block, or a count of blocks) and
    MMAP query files read back to the arrays they were written from; malformed
    files and out-of-range entries are TN_E_PARSE."""
    m = synth.bayes_net(12, 4)
    ev = synth.evidence_batch(m, 3, 0.3, 9)
    q = [7, 2, 10]
    with tempfile.TemporaryDirectory() as d:
        pu = os.path.join(d, "m.uai")
        synth.write_uai(m, pu)
        M = tn.Model.from_uai(pu)
        pe = os.path.join(d, "m.uai.evid")
        synth.write_evidence(ev, pe)
        np.testing.assert_array_equal(M.read_evidence(pe), ev)
        # the single-block form
        obs = np.nonzero(ev[1] >= 0)[0]
        with open(pe, "w") as f:
            f.write(" ".join([str(len(obs))] + [f"{v} {ev[1][v]}" for v in obs]))
        np.testing.assert_array_equal(M.read_evidence(pe), ev[1:2])
        pq = os.path.join(d, "m.uai.query")
        synth.write_query(q, pq)
        np.testing.assert_array_equal(M.read_query(pq), q)
        for text in ("2 0 1", "1 1 12 0", "1 1 0 5", "1 2 0 1 0 0", "x"):
            with open(pe, "w") as f:
                f.write(text)
            with pytest.raises(tn.TNError) as e:
                M.read_evidence(pe)
            assert e.value.status == 2, text
        for text in ("3 1 2", "2 1 1", "1 40"):
            with open(pq, "w") as f:
                f.write(text)
            with pytest.raises(tn.TNError) as e:
                M.read_query(pq)
            assert e.value.status == 2, text
        with pytest.raises(tn.TNError) as e:
            M.read_evidence(os.path.join(d, "missing.evid"))
        assert e.value.status == 1


def test_tree_validation():
    m = synth.grid_ising(3, 1)
    M = tn.Model.from_synth(m)
    n = M.nleaves
    l, r = M.optimize_order(0)
    M.set_order(l, r)
    bad_l = l.copy()
    bad_l[-1] = bad_l[0]                    # a tensor contracted twice
    with pytest.raises(tn.TNError) as e:
        M.set_order(bad_l, r)
    assert e.value.status == 3
    bad_r = r.copy()
    bad_r[0] = n + 5                        # child not earlier than its parent
    with pytest.raises(tn.TNError):
        M.set_order(l, bad_r)
    with pytest.raises(tn.TNError):
        M.set_order(l[:-1], r[:-1])         # too few nodes


def _keep_rule_stats(m, left, right):
    """Independent recomputation: a label is kept at a node iff some leaf
    outside the node's subtree holds it (output labels are empty)."""
    leaves = [set(map(int, s)) for s in m.scopes] + [{v} for v in range(m.nvars)]
    n = len(leaves)
    sub = [{i} for i in range(n)]
    labels = [set(s) for s in leaves]
    muladds, sc = 0, 0
    for i, (a, b) in enumerate(zip(left, right)):
        me = n + i
        sub.append(sub[a] | sub[b])
        outside = set()
        for j in range(n):
            if j not in sub[me]:
                outside |= leaves[j]
        u = labels[a] | labels[b]
        labels.append({v for v in u if v in outside})
        muladds += int(np.prod([m.card[v] for v in u]))
        sc = max(sc, int(np.prod([m.card[v] for v in labels[me]])))
    return np.log2(muladds), np.log2(sc)


@pytest.mark.parametrize("method", [0, 1])
def test_tree_stats_match_keep_rule(method):
    m = synth.random_markov(9, 12, 3, 4, cards=(2, 3))
    M = tn.Model.from_synth(m)
    l, r = M.optimize_order(method, 4, 7)
    M.set_order(l, r)
    st = M.tree_stats(1, "fp64")
    tc, sc = _keep_rule_stats(m, l, r)
    assert abs(st["tc"] - tc) < 1e-9
    assert abs(st["sc"] - sc) < 1e-9
    assert st["nodes"] == M.nleaves - 1


def test_elimination_tree_is_valid_and_deterministic():
    m = synth.grid_ising(6, 2)
    M = tn.Model.from_synth(m)
    l1, r1 = M.tree_from_elimination(np.arange(m.nvars))
    l2, r2 = M.tree_from_elimination(np.arange(m.nvars))
    np.testing.assert_array_equal(l1, l2)
    M.set_order(l1, r1)
    assert M.tree_stats()["sc"] == 6.0      # a row sweep keeps one row (+1 label)  of 6
    g1 = M.optimize_order(0)
    g2 = M.optimize_order(0)
    np.testing.assert_array_equal(g1[0], g2[0])


def test_slicing_reduces_space_complexity():
    """Slicing removes the sliced labels from every tensor: the per-slice
    space complexity drops and the total time grows by at most the number of
    slices."""
    m = synth.grid_ising(8, 3)
    M = tn.Model.from_synth(m)
    l, r = M.tree_from_elimination(np.arange(m.nvars))
    M.set_order(l, r)
    full = M.tree_stats()
    # every boundary of a row sweep holds one spin of each column: slicing
    # column 0 removes one label from each of them
    M.set_order(l, r, slice_vars=list(range(0, m.nvars, 8)))
    sl = M.tree_stats()
    assert sl["sc"] == full["sc"] - 1
    assert sl["tc"] <= full["tc"] + 8 + 1e-9
    with pytest.raises(tn.TNError):
        M.set_order(l, r, slice_vars=[3, 3])
    with pytest.raises(tn.TNError):
        M.set_order(l, r, slice_vars=[m.nvars])


def _tree_logz(m, left, right):
    """log Z by contracting the model's tensors (plus unity vectors) along a
    given tree with numpy.einsum in float64, max-normalising every
    intermediate and keeping the log of the factor on the side."""
    from collections import Counter
    leaves = [list(map(int, s)) for s in m.scopes] + [[v] for v in range(m.nvars)]
    total = Counter()
    for L in leaves:
        total.update(L)
    ts = [np.asarray(t, float).reshape([int(m.card[v]) for v in s])
          for s, t in zip(m.scopes, m.tables)]
    ts += [np.ones(int(m.card[v])) for v in range(m.nvars)]
    labels = [list(L) for L in leaves]
    cnt = [Counter(L) for L in leaves]
    logs = 0.0
    for a, b in zip(left, right):
        c = cnt[a] + cnt[b]
        keep = [v for v in dict.fromkeys(labels[a] + labels[b]) if c[v] < total[v]]
        idx = {v: i for i, v in enumerate(dict.fromkeys(labels[a] + labels[b]))}
        out = np.einsum(ts[a], [idx[v] for v in labels[a]], ts[b], [idx[v] for v in labels[b]],
                        [idx[v] for v in keep])
        mx = float(np.max(out))
        logs += np.log(mx)
        ts.append(out / mx)
        labels.append(keep)
        cnt.append(Counter({v: c[v] for v in keep}))
    return logs + float(np.log(np.sum(ts[-1])))


def test_reassociate_keeps_the_contraction_and_cuts_read_write():
    """Re-associated chains (associativity of the contraction, Sec. Tensor
    networks): same log Z along both trees, fewer entries read and written,
    same number of pairwise contractions."""
    import oracle
    m = synth.grid_ising(14, 3)
    M = tn.Model.from_synth(m)
    l, r = M.optimize_order(0)
    M.set_order(l, r)
    s0 = M.tree_stats(1, "fp32")
    l2, r2 = M.reassociate(l, r)
    assert (l2 != l).any() or (r2 != r).any()
    M.set_order(l2, r2)                      # a valid tree
    s1 = M.tree_stats(1, "fp32")
    assert s1["nodes"] == s0["nodes"]
    assert s1["rw"] < s0["rw"] - 0.5
    assert s1["sc"] <= s0["sc"]
    z0, z1 = _tree_logz(m, l, r), _tree_logz(m, l2, r2)
    assert abs(z0 - z1) < 1e-10 * abs(z0)
    assert abs(z1 - oracle.ve_pr(m)) < 1e-10 * abs(z1)
    # nothing to do on small tensors: the tree comes back unchanged
    ms = synth.grid_ising(6, 1)
    Ms = tn.Model.from_synth(ms)
    ls, rs = Ms.optimize_order(0)
    l3, r3 = Ms.reassociate(ls, rs)
    np.testing.assert_array_equal(l3, ls)
    np.testing.assert_array_equal(r3, rs)
    with pytest.raises(tn.TNError) as e:
        bad = ls.copy()
        bad[-1] = bad[0]
        Ms.reassociate(bad, rs)
    assert e.value.status == 3


def test_choose_slices_reaches_target():
    """Greedy slice selection: the per-slice space complexity reaches the
    target and slicing never increases the total multiply-add count by more
    than the number of slices."""
    m = synth.grid_ising(10, 4)
    M = tn.Model.from_synth(m)
    l, r = M.optimize_order(0)
    M.set_order(l, r)
    full = M.tree_stats()
    sl = M.choose_slices(full["sc"] - 3, 8, l, r)
    assert 1 <= len(sl) <= 8 and len(set(sl)) == len(sl)
    M.set_order(l, r, slice_vars=sl)
    st = M.tree_stats()
    assert st["sc"] <= full["sc"] - 3
    assert st["tc"] <= full["tc"] + len(sl) + 1e-9
    # already at the target: nothing to slice
    assert M.choose_slices(full["sc"], 8, l, r) == []
    # the current tree is used when none is given
    M.set_order(l, r)
    assert M.choose_slices(full["sc"] - 3, 8) == sl


def test_incremental_annealing_order_search():
    """Method 4 (incrementally evaluated annealing from the better of the
    elimination and bisection trees): a valid tree, deterministic for a seed,
    the 12 x 12 grid within two labels of its width, and on workload 4's
    random 3-regular graph at least 8x fewer multiply-adds than method 2 with
    the same restarts at no larger space complexity."""
    m = synth.grid_ising(12, 5)
    M = tn.Model.from_synth(m)
    l1, r1 = M.optimize_order(4, 4, 9)
    l2, r2 = M.optimize_order(4, 4, 9)
    np.testing.assert_array_equal(l1, l2)
    np.testing.assert_array_equal(r1, r2)
    M.set_order(l1, r1)
    st = M.tree_stats()
    assert st["nodes"] == M.nleaves - 1
    assert st["sc"] <= 12 + 2
    m4 = synth.workload(4).model
    M4 = tn.Model.from_synth(m4)
    M4.set_order(*M4.optimize_order(2, 4, 1))
    s2 = M4.tree_stats()
    M4.set_order(*M4.optimize_order(4, 4, 1))
    s4 = M4.tree_stats()
    assert s4["sc"] <= s2["sc"]
    assert s4["tc"] <= s2["tc"] - 3


def test_order_search_on_tiny_models():
    """Every order-search method returns a valid tree for networks of two,
    three and five leaves (a single factor over one variable upwards)."""
    cases = (([2], [[0]], [np.array([1.0, 2.0])]),
             ([3, 2], [[0, 1]], [np.arange(1, 7, dtype=float)]),
             ([2, 2, 2], [[0, 1], [1, 2]], [np.ones(4), np.ones(4)]))
    for card, scopes, tables in cases:
        M = tn.Model.from_arrays(card, scopes, tables)
        for method in range(5):
            M.set_order(*M.optimize_order(method, 3, 0))
            assert M.tree_stats()["nodes"] == M.nleaves - 1


def test_partition_order_search():
    """Recursive bisection (method 3, kept only where it beats the
    elimination heuristics, then annealed): a valid tree, deterministic for a
    seed, within two labels of the 12 x 12 grid's width, and never worse than
    the elimination heuristics on a random 3-regular graph."""
    m = synth.grid_ising(12, 5)
    M = tn.Model.from_synth(m)
    l1, r1 = M.optimize_order(3, 4, 9)
    l2, r2 = M.optimize_order(3, 4, 9)
    np.testing.assert_array_equal(l1, l2)
    np.testing.assert_array_equal(r1, r2)
    M.set_order(l1, r1)
    st = M.tree_stats()
    assert st["nodes"] == M.nleaves - 1
    assert st["sc"] <= 12 + 2
    # on a random 3-regular graph it does not lose to the elimination heuristics
    m3 = synth.rrg3_ising(60, 7)
    M3 = tn.Model.from_synth(m3)
    M3.set_order(*M3.optimize_order(1, 8, 1))
    sc1 = M3.tree_stats()["sc"]
    M3.set_order(*M3.optimize_order(3, 4, 1))
    assert M3.tree_stats()["sc"] <= sc1

"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Tolerances: FP64 log Z within 1e-10 absolute and marginals within 1e-10;
FP32 / TF32 / BF16 log Z within 1e-4 relative (|dlogZ| / |logZ|) and
marginals within 1e-3 absolute; MPE / MMAP assignments bit-exact (continuous
random tables make ties vanish; the oracle's certificate below guards it).
"""
import numpy as np
import pytest

import oracle
from oracle import con
from paper_2405_14060_gb300 import synth, tn

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def _marg_close(M, marg_row, ref, atol):
    for v, (a, b) in enumerate(zip(M.split(marg_row), ref)):
        assert np.max(np.abs(a - b)) <= atol, (v, a, b)


SMALL = [
    ("grid4", lambda: synth.grid_ising(4, 3)),
    ("rand11", lambda: synth.random_markov(11, 14, 3, 5, cards=(2, 3))),
    ("bn14", lambda: synth.bayes_net(14, 9)),
    ("chain12", lambda: synth.chain_model(12, [2, 3, 4] * 4, 2)),
]


@pytest.mark.parametrize("name,mk", SMALL)
@pytest.mark.parametrize("method", [0, 1])
def test_pr_mar_small_fp64(name, mk, method):
    m = mk()
    M = tn.Model.from_synth(m)
    M.set_order(*M.optimize_order(method, 4, 3))
    rng = np.random.default_rng(1)
    ev = synth.random_evidence(m, 0.2, rng)
    lz_ref, marg_ref = oracle.brute_mar(m, ev)
    lz, marg = M.mar(ev, prec="fp64")
    assert abs(lz[0] - lz_ref) < 1e-10
    assert abs(M.pr(ev, prec="fp64")[0] - lz_ref) < 1e-10
    _marg_close(M, marg[0], marg_ref, 1e-10)


def _dense_model(layout, seed):
    """Three factors A(r, s), W(s, t), V(t, r): r = 12 binary variables (4096
    positions), s = cards (3, 2, 2, 2) (24 summed combinations), t = cards
    (5, 2, 2) (20 new ones).  With the tree ((A, W'), V'), where W' collects
    the unity vectors of s and t and V' those of r, the node (A, W') is a
    dense absorb (24 x 20 combinations, more than the register-blocked
    kernels take), its adjoint A-bar another (20 x 24) and W'-bar a dense
    reduce.  layout "sfast": A's summed labels fastest (four at a time);
    "mixed": A's labels interleaved (planned 16-byte chunks); "ternary":
    ternary position labels and 30 x 30 combinations (one entry at a
    time)."""
    rng = np.random.default_rng(seed)
    if layout == "ternary":
        # 8 ternary positions (no 16-byte quads, no repeating 128-position
        # tiles) and 30 x 30 combinations: the one-entry-per-copy and
        # one-entry-per-store modes
        r, s, t = list(range(8)), [8, 9, 10], [11, 12, 13]
        card = np.array([3] * 8 + [3, 5, 2] + [5, 3, 2], np.int32)
        sa = r + s
    else:
        r, s, t = list(range(12)), [12, 13, 14, 15], [16, 17, 18]
        card = np.array([2] * 12 + [3, 2, 2, 2] + [5, 2, 2], np.int32)
        sa = r + s if layout == "sfast" else [s[0]] + r[:6] + [s[1], s[2]] + r[6:] + [s[3]]
    scopes = [np.array(sa, np.int32), np.array(s + t, np.int32), np.array(t + r, np.int32)]
    tables = [rng.uniform(0.5, 1.5, size=int(np.prod(card[sc]))) for sc in scopes]
    m = synth.Model(card, scopes, tables, "MARKOV", "dense_" + layout)
    nleaves = 3 + m.nvars
    left, right, nid = [], [], nleaves
    w = 1
    for v in s + t:
        left.append(w), right.append(3 + v)
        w, nid = nid, nid + 1
    vv = 2
    for v in r:
        left.append(vv), right.append(3 + v)
        vv, nid = nid, nid + 1
    left.append(0), right.append(w)
    c, nid = nid, nid + 1
    left.append(c), right.append(vv)
    return m, left, right


@pytest.mark.parametrize("layout", ["sfast", "mixed", "ternary"])
def test_dense_absorb_and_reduce_nodes(layout):
    m, left, right = _dense_model(layout, 7)
    M = tn.Model.from_synth(m)
    M.set_order(left, right)
    rng = np.random.default_rng(3)
    ev = np.stack([np.full(m.nvars, -1, np.int32)] +
                  [synth.random_evidence(m, 0.15, rng) for _ in range(2)])
    refs = [oracle.ve_mar(m, e) for e in ev]
    lz, marg = M.mar(ev, prec="fp64")
    for b, (lz_ref, marg_ref) in enumerate(refs):
        assert abs(lz[b] - lz_ref) < 1e-10
        _marg_close(M, marg[b], marg_ref, 1e-10)
    for prec in ("fp32", "bf16"):
        lz, marg = M.mar(ev, prec=prec)
        for b, (lz_ref, marg_ref) in enumerate(refs):
            assert abs(lz[b] - lz_ref) <= 1e-4 * abs(lz_ref)
            _marg_close(M, marg[b], marg_ref, 1e-3)


@pytest.mark.parametrize("prec", ["fp32", "tf32", "bf16"])
def test_pr_mar_small_reduced(prec):
    m = synth.grid_ising(4, 5)
    M = tn.Model.from_synth(m)
    lz_ref, marg_ref = oracle.brute_mar(m)
    lz, marg = M.mar(prec=prec)
    assert abs(lz[0] - lz_ref) <= 1e-4 * abs(lz_ref)
    _marg_close(M, marg[0], marg_ref, 1e-3)


def test_batched_evidence_matches_per_item():
    m = synth.random_markov(10, 13, 3, 8, cards=(2, 3))
    M = tn.Model.from_synth(m)
    ev = synth.evidence_batch(m, 5, 0.3, 11)
    lz, marg = M.mar(ev, prec="fp64")
    for b in range(ev.shape[0]):
        lzr, mr = oracle.brute_mar(m, ev[b])
        assert abs(lz[b] - lzr) < 1e-10
        _marg_close(M, marg[b], mr, 1e-10)
    lz32 = M.pr(ev, prec="fp32")
    np.testing.assert_allclose(lz32, lz, rtol=1e-4)


def test_joint_marginals_match_oracle():
    """Joint marginals of variable sets (the query labels sliced into one
    batched PR) against the oracle's enumeration, with an observed query
    variable; an edge of a 160-spin tree Ising model against its closed form
    exp(J s_i s_j) / (4 cosh J); argument errors."""
    m = synth.random_markov(9, 12, 3, 8, cards=(2, 3, 4))
    M = tn.Model.from_synth(m)
    ev = np.full(m.nvars, -1, np.int32)
    ev[4] = 1
    lz_ref = oracle.brute_pr(m, ev)
    for query in ([2], [0, 5], [7, 1, 3], [8, 4, 6]):
        ref = oracle.brute_joint_marginal(m, query, ev)
        for prec, tol in (("fp64", 1e-10), ("fp32", 1e-4)):
            lz, P = M.joint_mar(query, ev, prec=prec)
            assert P.shape == ref.shape
            np.testing.assert_allclose(P, ref, rtol=0, atol=tol)
            assert abs(lz - lz_ref) <= (1e-10 if prec == "fp64" else 1e-4 * max(1.0, abs(lz_ref)))
    t = synth.tree_ising(160, 2)
    T = tn.Model.from_synth(t)
    i, j = (int(x) for x in t.scopes[17])
    J = np.log(t.tables[17][3])
    S = np.array([-1.0, 1.0])
    _, P = T.joint_mar([i, j], prec="fp64")
    np.testing.assert_allclose(P, np.exp(J * np.outer(S, S)) / (4 * np.cosh(J)), atol=1e-12)
    for bad in ([2, 2], [m.nvars], []):
        with pytest.raises(tn.TNError):
            M.joint_mar(bad)


def test_impossible_evidence():
    m = synth.chain_model(4, [2, 2, 2, 2], 1)
    m.tables[0] = np.array([0.0, 1.0])          # x0 = 0 has zero weight
    M = tn.Model.from_synth(m)
    ev = np.array([0, -1, -1, -1], np.int32)
    assert M.pr(ev)[0] == -np.inf
    with pytest.raises(tn.TNError):
        M.mar(ev)
    with pytest.raises(tn.TNError):
        M.map(ev)


def test_workload1_full():
    w = synth.workload(1)
    m = w.model
    M = tn.Model.from_synth(m)          # greedy order (the default)
    lz_ref, marg_ref = oracle.ve_mar(m)
    lz, marg = M.mar(prec="fp64")
    assert abs(lz[0] - lz_ref) < 1e-10
    _marg_close(M, marg[0], marg_ref, 1e-10)
    assert abs(M.pr(prec="fp64")[0] - lz_ref) < 1e-10
    for prec in ("fp32", "tf32", "bf16"):
        lz2, marg2 = M.mar(prec=prec)
        assert abs(lz2[0] - lz_ref) <= 1e-4 * abs(lz_ref), prec
        _marg_close(M, marg2[0], marg_ref, 1e-3)
        assert abs(M.pr(prec=prec)[0] - lz_ref) <= 1e-4 * abs(lz_ref), prec
    # a second tree (min-fill elimination) with different micro / streaming splits
    M.set_order(*M.optimize_order(1, 4, 11))
    for prec in ("fp64", "fp32"):
        tol = 1e-10 if prec == "fp64" else 1e-4 * abs(lz_ref)
        assert abs(M.pr(prec=prec)[0] - lz_ref) <= tol
        lz3, marg3 = M.mar(prec=prec)
        assert abs(lz3[0] - lz_ref) <= tol
        _marg_close(M, marg3[0], marg_ref, 1e-10 if prec == "fp64" else 1e-3)


def test_map_small_and_workload3():
    for name, mk in SMALL:
        m = mk()
        M = tn.Model.from_synth(m)
        ev = synth.random_evidence(m, 0.2, np.random.default_rng(4))
        xb, lb = oracle.brute_map(m, ev)
        for prec in ("fp64", "fp32"):
            x, lp = M.map(ev, prec=prec)
            np.testing.assert_array_equal(x, xb)
            assert abs(lp - lb) < (1e-9 if prec == "fp64" else 1e-3 * max(1, abs(lb)))
    w = synth.workload(3)
    m, ev = w.model, w.evid[0]
    xo, lo = oracle.ve_map(m, ev)
    M = tn.Model.from_synth(m)
    for prec in ("fp64", "fp32"):
        x, lp = M.map(ev, prec=prec)
        np.testing.assert_array_equal(x, xo)
        assert abs(oracle.log_weight(m, x) - lo) < 1e-9


# Worst-case FP32 rounding of a max-normalised tropical contraction over these
# trees: each root entry is a chain of at most ~1000 additions whose operands
# stay below 32 in magnitude after normalisation, 0.5 ulp(32) = 1.9e-6 each.
FP32_MAXPLUS_BOUND = 1000 * 2.0 ** -19


def _same_map_or_tie(m, x, ref, bound):
    """The GPU's MAP assignment is the oracle's, or (certificate) the oracle's
    runner-up gap is within the rounding bound and x scores within it."""
    if np.array_equal(x, np.asarray(ref["assign"])):
        return
    lw = oracle.log_weight(m, x)
    assert ref["gap"] <= bound and ref["logp"] - lw <= bound, (ref["gap"], ref["logp"] - lw)


def test_map_at_size_against_oracle():
    """MAP with tropical tensors of 2^21 entries: a 20 x 20 grid Ising model
    on the library's greedy tree, FP64 and FP32 max-plus, against the
    oracle's stored MAP (max-sum elimination along the row sweep); and the
    300-variable Bayesian network.  The oracle's stored gap to the runner-up
    assignment certifies FP32 exactness (it must exceed the FP32 bound of the
    max-normalised contraction, else a tie within rounding is accepted)."""
    g = _golden()
    ref = g["grid20_map"]
    m = synth.grid_ising(20, 20240620)
    M = tn.Model.from_synth(m)
    M.set_order(*M.optimize_order(0))
    assert M.tree_stats(1, "fp32")["sc"] >= 20
    x64, lp64 = M.map(prec="fp64")
    np.testing.assert_array_equal(x64, ref["assign"])
    assert abs(lp64 - ref["logp"]) < 1e-9
    x32, lp32 = M.map(prec="fp32")
    _same_map_or_tie(m, x32, ref, FP32_MAXPLUS_BOUND)
    assert abs(lp32 - ref["logp"]) <= FP32_MAXPLUS_BOUND
    rb = g["bn300_map"]
    w = synth.workload(3)
    B = tn.Model.from_synth(w.model)
    for prec, bound in (("fp64", 1e-9), ("fp32", FP32_MAXPLUS_BOUND)):
        x, lp = B.map(w.evid[0], prec=prec)
        _same_map_or_tie(w.model, x, rb, bound)
        assert abs(lp - rb["logp"]) <= bound


def test_mmap_small_and_workload3():
    for seed in range(3):
        m = synth.bayes_net(14, 40 + seed)
        rng = np.random.default_rng(seed)
        ev = synth.random_evidence(m, 0.2, rng)
        q = synth.mmap_query(m, ev, 0.4, rng)
        xb, lb = oracle.brute_mmap(m, q, ev)
        M = tn.Model.from_synth(m)
        for prec in ("fp64", "fp32"):
            x, lp = M.mmap(q, ev, prec=prec)
            np.testing.assert_array_equal(x, xb)
            assert abs(lp - lb) < (1e-9 if prec == "fp64" else 1e-3)
        # same query and observed variables, other values: the cached
        # programs replay with the new evidence
        ev2 = ev.copy()
        obs = np.nonzero(ev >= 0)[0]
        ev2[obs] = (ev[obs] + 1) % m.card[obs]
        xb2, lb2 = oracle.brute_mmap(m, q, ev2)
        x2, lp2 = M.mmap(q, ev2, prec="fp32")
        np.testing.assert_array_equal(x2, xb2)
        assert abs(lp2 - lb2) < 1e-3
    w = synth.workload(3)
    xo, lo = oracle.ve_mmap(w.model, w.query, w.evid[0])
    M = tn.Model.from_synth(w.model)
    for prec in ("fp64", "fp32"):
        x, lp = M.mmap(w.query, w.evid[0], prec=prec)
        np.testing.assert_array_equal(x, xo)
        assert abs(lp - lo) < (1e-8 if prec == "fp64" else 1e-3)


def test_sampling_small_chi_square():
    m = synth.random_markov(7, 8, 3, 5, cards=(2, 3))
    ev = np.full(m.nvars, -1, np.int32)
    ev[2] = 1
    joint = oracle.brute_joint(m, ev)
    M = tn.Model.from_synth(m)
    n = 200000
    s = M.sample(n, seed=7, evid=ev, prec="fp64")
    assert np.all(s[:, 2] == 1)
    free = [v for v in range(m.nvars) if ev[v] < 0]
    idx = np.zeros(n, np.int64)
    for v in free:
        idx = idx * int(m.card[v]) + s[:, v]
    emp = np.bincount(idx, minlength=len(joint))
    expc = joint * n
    keep = expc >= 5
    chi2 = np.sum((emp[keep] - expc[keep]) ** 2 / expc[keep])
    dof = int(keep.sum()) - 1
    assert chi2 < dof + 6 * np.sqrt(2 * dof), (chi2, dof)
    s2 = M.sample(1000, seed=7, evid=ev, prec="fp64")
    np.testing.assert_array_equal(s2, s[:1000])     # counter-based: reproducible


# ------------------------------------------------------ pairwise contraction

CASES = [
    # sizes, labels A, labels B, labels C
    ([3, 4, 5], [0, 1], [1, 2], [0, 2]),                 # matmul
    ([2, 3, 2, 3, 2, 2], [0, 3], [3], [0]),              # matvec
    ([2] * 12, [0, 1, 2, 3, 4, 5, 6, 7, 8, 9], [9, 10, 11], [10, 0, 1, 2, 3, 4, 5, 6, 7, 8, 11]),
    ([3, 2, 4, 5, 2], [0, 1, 2], [2, 3, 1], [3, 0, 1]),  # batch label 1
    ([2] * 16, list(range(16)), list(range(16)), []),   # full trace, split-K
    ([5, 7, 3, 2], [0, 1, 2], [3], [0, 3]),              # labels summed in one operand
    # batched strided GEMM (groups below the tensor-core tile sizes):
    # ragged M = 300, N = 70, K = 37; A summed-fastest, C column-fastest
    ([300, 37, 70], [0, 1], [1, 2], [0, 2]),
    # a shared kept label (group G) fastest in C, labels interleaved
    ([3, 50, 9, 20, 6], [1, 0, 3], [3, 2, 0, 4], [2, 1, 4, 0]),
    # long summed space, tiny output: split over blocks, partials reduced
    ([2] * 14 + [3], [14] + list(range(13)), list(range(14)), [14, 13]),
    # column side larger than the row side (operand roles swapped)
    ([4, 100, 30], [0, 1], [1, 2], [0, 2]),
    # at most 8 columns (the 128 x 8 tile): ragged rows, long summed space split
    ([130, 600, 7], [0, 1], [1, 2], [0, 2]),
    # 6 columns, a group label fastest in C, summed space split
    ([3, 9, 2000, 6], [0, 1, 2], [0, 2, 3], [3, 1, 0]),
    # at least 128 columns: ragged both ways
    ([200, 45, 300], [0, 1], [1, 2], [0, 2]),
    # the same with a group label and the rows fastest in C
    ([2, 150, 20, 130], [0, 1, 2], [0, 2, 3], [0, 3, 1]),
    # summed space of at most 8 (half K steps): K = 6, and K = 8 with a group
    ([150, 6, 90], [0, 1], [1, 2], [0, 2]),
    ([2, 130, 8, 20], [0, 1, 2], [0, 2, 3], [0, 1, 3]),
]


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("dtype", ["float64", "float32"])
def test_contract_dev_matches_definition(case, dtype):
    sizes, la, lb, lc = CASES[case]
    rng = np.random.default_rng(case)
    A = rng.random([sizes[v] for v in la])
    B = rng.random([sizes[v] for v in lb])
    ref = con.con_dense([tuple(la), tuple(lb)], [A, B], tuple(lc))
    dt = getattr(torch, dtype)
    tA = torch.tensor(A, dtype=dt, device="cuda").contiguous()
    tB = torch.tensor(B, dtype=dt, device="cuda").contiguous()
    tC = torch.zeros([sizes[v] for v in lc] or [1], dtype=dt, device="cuda")
    tn.contract_dev(sizes, la, tA, lb, tB, lc, tC)
    got = tC.cpu().numpy().reshape(np.shape(ref))
    tol = 1e-12 if dtype == "float64" else 2e-5
    np.testing.assert_allclose(got, ref, rtol=tol, atol=0)
    # tropical
    ref_v, ref_i = con.tcon_dense([tuple(la), tuple(lb)], [np.log(A), np.log(B)], tuple(lc))
    tA = torch.tensor(np.log(A), dtype=dt, device="cuda").contiguous()
    tB = torch.tensor(np.log(B), dtype=dt, device="cuda").contiguous()
    am = torch.zeros(tC.numel(), dtype=torch.int32, device="cuda")
    tn.contract_dev(sizes, la, tA, lb, tB, lc, tC, semiring=1, argmax=am)
    # argmax order: labels of A not in C (A's order), then B-only labels
    elim = [v for v in la if v not in lc] + [v for v in lb if v not in lc and v not in la]
    elim_ref = [v for v in dict.fromkeys(la + lb) if v not in lc]
    assert elim == elim_ref
    gv = tC.cpu().numpy().reshape(np.shape(ref_v))
    if dtype == "float64":
        np.testing.assert_allclose(gv, ref_v, rtol=0, atol=1e-12)
        np.testing.assert_array_equal(am.cpu().numpy().reshape(np.shape(ref_i)), ref_i)
    else:
        np.testing.assert_allclose(gv, ref_v, rtol=0, atol=1e-4 * max(1, np.abs(ref_v).max()))


# ----------------------------------------------------------- GEMM form
# sizes, labels A, labels B, labels C: every group >= 64 so the GEMM path runs
GEMM_CASES = [
    ([2] * 24, list(range(16)), list(range(8, 24)), list(range(8)) + list(range(16, 24))),
    # ragged groups (m = 65, n = 111, k = 77), a batch label of size 3
    ([5, 13, 3, 37, 7, 11, 3], [6, 0, 1, 4, 5], [6, 4, 5, 2, 3], [6, 0, 1, 2, 3]),
    # output in a non-canonical order (n before m): scatter through a workspace
    ([4, 4, 4, 4, 4, 4, 2], [0, 1, 2, 3], [2, 3, 4, 5, 6], [4, 5, 6, 0, 1]),
    # several tiles in every direction: m = 512, n = 768, k = 384
    ([8, 64, 3, 256, 128, 3], [0, 1, 4, 5], [4, 5, 2, 3], [0, 1, 2, 3]),
    # row operand stored K-slow (its preparation is a tiled transpose), output
    # [n][m] (scatter through a tiled transpose)
    ([2] * 20, list(range(6, 14)) + list(range(6)), list(range(14, 20)) + list(range(6, 14)),
     list(range(14, 20)) + list(range(6))),
    # interleaved non-binary labels on both operands and the output
    ([3, 25, 7, 36, 9, 30], [2, 0, 3, 1], [3, 5, 2, 4], [5, 0, 4, 1]),
]
GEMM_TOL = {"fp64": 1e-12, "fp32": 1e-5, "tf32": 2e-3, "bf16": 1.5e-2}


@pytest.mark.parametrize("case", range(len(GEMM_CASES)))
@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32", "bf16"])
def test_gemm_form_matches_definition(case, prec):
    sizes, la, lb, lc = GEMM_CASES[case]
    rng = np.random.default_rng(100 + case)
    A = rng.random([sizes[v] for v in la])
    B = rng.random([sizes[v] for v in lb])
    ref = np.einsum(A, la, B, lb, lc)
    dt = torch.float64 if prec == "fp64" else torch.float32
    tA = torch.tensor(A, dtype=dt, device="cuda").contiguous()
    tB = torch.tensor(B, dtype=dt, device="cuda").contiguous()
    tC = torch.zeros([sizes[v] for v in lc], dtype=dt, device="cuda")
    for _ in range(2):      # twice: workspaces and pipeline state are reused cleanly
        tC.zero_()
        tn.contract_dev(sizes, la, tA, lb, tB, lc, tC, prec=prec)
        got = tC.cpu().numpy()
        err = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
        assert err <= GEMM_TOL[prec], (prec, err)


# shapes of the batched strided GEMM (groups G, M, N, K in scattered layouts)
# for its tensor-core gather form: sizes, labels A, labels B, labels C
GATHER_CASES = [
    ([300, 37, 70], [0, 1], [1, 2], [0, 2]),                       # A summed-fastest
    ([3, 50, 9, 20, 6], [1, 0, 3], [3, 2, 0, 4], [2, 1, 4, 0]),    # G label fastest in C
    ([4, 100, 30], [0, 1], [1, 2], [0, 2]),                        # roles swapped
    ([2] * 18, list(range(13)) + [13, 14], [13, 14, 15, 16, 17],   # M = 2^13, K = 4, N = 8
     list(range(13)) + [15, 16, 17]),
    ([512, 40, 300, 2], [3, 0, 1], [3, 1, 2], [3, 2, 0]),          # N = 300: two 256-wide tiles
    ([2] * 20, list(range(20)), [5, 12], [5, 12]),                 # M = N = 2, K = 2^18
    ([1000, 64, 48], [1, 0], [2, 1], [0, 2]),                      # A rows strided by 64
    # M = 4096, K = 8, N = 128 with the output's fastest label on the N side
    ([2] * 22, list(range(15)), list(range(12, 22)), list(range(12)) + list(range(15, 22))),
]


@pytest.mark.parametrize("case", range(len(GATHER_CASES)))
def test_gather_gemm_tf32_matches_definition(case):
    """The batched strided GEMM with TF32 inputs (the tensor-core gather form
    where it applies, else the CUDA-core form) against the definition, twice
    in a row (shared-memory ring and TMEM reused cleanly)."""
    sizes, la, lb, lc = GATHER_CASES[case]
    rng = np.random.default_rng(300 + case)
    A = rng.random([sizes[v] for v in la])
    B = rng.random([sizes[v] for v in lb])
    ref = np.einsum(A, la, B, lb, lc)
    tA = torch.tensor(A, dtype=torch.float32, device="cuda")
    tB = torch.tensor(B, dtype=torch.float32, device="cuda")
    tC = torch.zeros([sizes[v] for v in lc], dtype=torch.float32, device="cuda")
    for _ in range(2):
        tC.fill_(float("nan"))
        tn.contract_dev(sizes, la, tA, lb, tB, lc, tC, prec="tf32")
        got = tC.cpu().numpy()
        err = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
        assert err <= 2e-3, (case, err)


def test_autograd_factor_marginals():
    """d log Z / d log T_f[x] is the factor marginal: a unary factor's equals
    the oracle's variable marginal, each sums to one, and finite differences
    of log Z agree."""
    from paper_2405_14060_gb300.autograd import log_partition
    m = synth.grid_ising(4, 21)
    M = tn.Model.from_synth(m)
    ev = np.full(m.nvars, -1, np.int32)
    ev[5] = 1
    lz_ref, marg_ref = oracle.brute_mar(m, ev)
    lt = torch.tensor(np.log(np.concatenate(m.tables)), dtype=torch.float64, device="cuda",
                      requires_grad=True)
    evt = torch.tensor(ev, device="cuda")
    lz, marg = log_partition(M, lt, evt)
    assert abs(lz.item() - lz_ref) < 1e-10
    lz.sum().backward()
    g = lt.grad.cpu().numpy()
    off = np.cumsum([0] + [len(t) for t in m.tables])
    for f, sc in enumerate(m.scopes):
        gf = g[off[f]:off[f + 1]]
        assert abs(gf.sum() - 1.0) < 1e-10
        if len(sc) == 1:
            np.testing.assert_allclose(gf, marg_ref[int(sc[0])], atol=1e-10)
    eps = 1e-6
    base = lt.detach().clone()
    for idx in (0, 7, off[-1] - 1):
        up, dn = base.clone(), base.clone()
        up[idx] += eps
        dn[idx] -= eps
        fd = (log_partition(M, up, evt)[0].item() - log_partition(M, dn, evt)[0].item()) / (2 * eps)
        assert abs(fd - g[idx]) < 1e-7


def _golden():
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "fullsize_oracle.json")) as f:
        return json.load(f)


def test_workload2_full_size():
    """24 x 24 grid (576 spins) at full size against the oracle's stored
    values (tests/golden/make_fullsize_oracle.py): log Z by FP64 bucket
    elimination and p(s_v) of six seeded spins by conditioning.  FP64 within
    1e-10 (log Z absolute, marginals absolute); TF32 / BF16 / FP32 within
    1e-4 relative (log Z) and 1e-3 (marginals); central differences of the
    GPU's FP64 log Z give the same magnetisation (d log Z / d h_i = 2 p_i - 1,
    a property at any size)."""
    g = _golden()["grid24"]
    w = synth.workload(2)
    m = w.model
    lz_ref = g["logz"]
    M = tn.Model.from_synth(m)

    def check(lz, marg, prec):
        tol = 1e-10 if prec == "fp64" else 1e-4 * abs(lz_ref)
        assert abs(lz[0] - lz_ref) <= tol, (prec, lz[0] - lz_ref)
        sp = M.split(marg[0])
        for v, p in zip(g["spins"], g["marg"]):
            err = np.max(np.abs(sp[v] - np.asarray(p)))
            assert err <= (1e-10 if prec == "fp64" else 1e-3), (prec, v, err)
        assert abs(M.pr(prec=prec)[0] - lz_ref) <= tol, prec
    for prec in ("fp64", "tf32", "bf16", "fp32"):
        check(*M.mar(prec=prec), prec)
    lz64, marg64 = M.mar(prec="fp64")
    unary = [k for k, sc in enumerate(m.scopes) if len(sc) == 1]
    eps = 1e-4
    sp = M.split(marg64[0])
    for k in unary[::290]:
        i = int(m.scopes[k][0])
        t0 = m.tables[k].copy()
        lzs = []
        for sgn in (1, -1):
            m.tables[k] = t0 * np.exp(sgn * eps * np.array([-1.0, 1.0]))
            lzs.append(tn.Model.from_synth(m).pr(prec="fp64")[0])
        m.tables[k] = t0
        fd = (lzs[0] - lzs[1]) / (2 * eps)
        assert abs(fd - (2 * sp[i][1] - 1)) < 1e-6
    # the 24 x 24 benchmark's tree: greedy with re-associated absorption chains
    M.set_order(*M.reassociate(*M.optimize_order(0)))
    for prec in ("fp64", "tf32", "bf16", "fp32"):
        check(*M.mar(prec=prec), prec)
    # the split reductions sum their chunk partials in a fixed order: repeated
    # solves agree bit for bit
    for prec in ("tf32", "fp64"):
        lza, ma = M.mar(prec=prec)
        lzb, mb = M.mar(prec=prec)
        np.testing.assert_array_equal(lza, lzb)
        np.testing.assert_array_equal(ma, mb)


def test_workload4_512_sets_against_oracle():
    """The batched benchmark at full size: 512 evidence sets (10% of the 200
    spins observed) on the random 3-regular graph, BF16 tensor-core GEMMs on
    the bisection tree, one tn_mar call (sub-batched under the device
    memory).  Against the oracle's stored values for eight seeded sets:
    log Z within 1e-4 relative and p(s_v | e) of three spins each within
    1e-3; the same sets in FP64 within 1e-10.  Every marginal row sums to
    one and observed spins get the indicator of their value."""
    g = _golden()["rrg200_batched"]
    w = synth.workload(4)
    m, ev = w.model, w.evid
    assert ev.shape[0] == 512
    M = tn.Model.from_synth(m)
    M.set_order(*M.optimize_order(3, 12, 2))
    rows = g["rows"]
    for prec, sub in (("bf16", None), ("fp64", rows)):
        e = ev if sub is None else ev[sub]
        lz, mg = M.mar(e, prec=prec)
        for i, b in enumerate(rows):
            r = b if sub is None else i
            ref = g["logz"][i]
            tol = 1e-10 if prec == "fp64" else 1e-4 * abs(ref)
            assert abs(lz[r] - ref) <= tol, (prec, b, lz[r] - ref)
            sp = M.split(mg[r])
            for v, p in zip(g["spins"][i], g["marg"][i]):
                err = np.max(np.abs(sp[v] - np.asarray(p)))
                assert err <= (1e-10 if prec == "fp64" else 1e-3), (prec, b, v, err)
        if sub is None:
            sums = mg.reshape(mg.shape[0], -1, 2).sum(axis=2)
            assert np.max(np.abs(sums - 1.0)) < 1e-6
            for b in (0, 511):
                row = M.split(mg[b])
                for v in np.nonzero(ev[b] >= 0)[0]:
                    assert row[v][ev[b][v]] == 1.0


def test_sampling_grid24_large_nodes():
    """Sampling on the 24 x 24 grid's benchmark tree, whose dense nodes sum
    4096 labels over 2^24-entry outputs (scanned per sample rather than
    tabulated): per-spin frequencies within 5 sigma of the FP64 marginals."""
    w = synth.workload(2)
    m = w.model
    M = tn.Model.from_synth(m)
    M.set_order(*M.reassociate(*M.optimize_order(0)))
    _, marg = M.mar(prec="fp64")
    p1 = np.array([x[1] for x in M.split(marg[0])])
    n = 20000
    s = M.sample(n, seed=3, prec="tf32")
    assert np.all(np.abs(s.mean(axis=0) - p1) < 5 * np.sqrt(p1 * (1 - p1) / n) + 2e-3)


def test_reassociated_tree_batched_evidence():
    """A re-associated tree (absorption runs contracted small-first) on a
    14 x 14 grid with a batch of evidence sets: the combined small tensors
    carry the batch label whenever an evidence vector joins them."""
    m = synth.grid_ising(14, 3)
    M = tn.Model.from_synth(m)
    l, r = M.reassociate(*M.optimize_order(0))
    M.set_order(l, r)
    ev = synth.evidence_batch(m, 6, 0.1, 17)
    for prec in ("fp64", "fp32"):
        lz, marg = M.mar(ev, prec=prec)
        for b in range(ev.shape[0]):
            lzr, mr = oracle.ve_mar(m, ev[b])
            tol = 1e-10 * max(1.0, abs(lzr)) if prec == "fp64" else 1e-4 * abs(lzr)
            assert abs(lz[b] - lzr) <= tol, (prec, b)
            _marg_close(M, marg[b], mr, 1e-10 if prec == "fp64" else 1e-3)


def test_slicing_pr_mar_matches_oracle():
    """PR / MAR over a sliced tree (Z-combination over slice assignments)
    equal the unsliced results and the oracle, with and without evidence on a
    sliced variable, for a batch of evidence sets."""
    m = synth.random_markov(12, 16, 3, 13, cards=(2, 3))
    M = tn.Model.from_synth(m)
    l, r = M.optimize_order(1, 4, 2)
    ev = synth.evidence_batch(m, 3, 0.2, 5)
    ev[1, 4] = 1                       # evidence on a sliced variable
    M.set_order(l, r, slice_vars=[4, 7])
    for prec in ("fp64", "fp32"):
        lz, marg = M.mar(ev, prec=prec)
        lzp = M.pr(ev, prec=prec)
        for b in range(ev.shape[0]):
            lzr, mr = oracle.brute_mar(m, ev[b])
            tol = 1e-10 if prec == "fp64" else 1e-4 * abs(lzr)
            assert abs(lz[b] - lzr) <= tol and abs(lzp[b] - lzr) <= tol
            _marg_close(M, marg[b], mr, 1e-10 if prec == "fp64" else 1e-3)
    with pytest.raises(tn.TNError):
        M.map(ev[0])


def test_sub_batching_under_budget():
    """A batch whose program exceeds the HBM budget runs in power-of-two
    sub-batches with the same results; a budget too small for one evidence
    set is TN_E_OOM."""
    m = synth.random_markov(12, 16, 3, 17, cards=(2, 3))
    ev = synth.evidence_batch(m, 13, 0.2, 3)
    ref_lz, ref_m = tn.Model.from_synth(m).mar(ev, prec="fp64")
    with pytest.raises(tn.TNError) as e:
        tn.Model.from_synth(m).mar(ev[:1], prec="fp64", budget=64)
    assert e.value.status == 4
    # smallest power-of-two budget that holds one evidence set
    b = 1024
    while True:
        try:
            tn.Model.from_synth(m).mar(ev[:1], prec="fp64", budget=b)
            break
        except tn.TNError:
            b *= 2
    M = tn.Model.from_synth(m)
    lz, mg = M.mar(ev, prec="fp64", budget=3 * b)
    np.testing.assert_allclose(lz, ref_lz, rtol=0, atol=1e-10)
    np.testing.assert_allclose(mg, ref_m, rtol=0, atol=1e-10)
    lzp = tn.Model.from_synth(m).pr(ev, prec="fp32", budget=3 * b)
    np.testing.assert_allclose(lzp, ref_lz, rtol=1e-4)


def test_mar_checkpointing_under_budget():
    """MAR under a memory budget below its forward cache (Sec. MAR: the
    reverse pass reads the forward intermediates): the largest ones are not
    kept and the reverse pass recomputes them.  At the smallest budget that
    runs (bisected to 1/256), FP64 marginals and log Z equal the unlimited
    run and the oracle within 1e-10, and the profile shows the recomputation
    as its own class (recomputation is chosen only when keeping every
    forward tensor does not fit)."""
    m = synth.grid_ising(16, 19)
    lz_ref, marg_ref = oracle.ve_mar(m)
    M = tn.Model.from_synth(m)
    tree = M.optimize_order(0)
    M.set_order(*tree)
    lz0, mg0 = M.mar(prec="fp64")

    def fresh():
        X = tn.Model.from_synth(m)
        X.set_order(*tree)
        return X

    def runs(b):
        try:
            fresh().mar(prec="fp64", budget=b)
            return True
        except tn.TNError as e:
            assert e.status == 4, e
            return False

    def smallest_budget():
        hi = 1 << 16
        while not runs(hi):
            hi *= 2
        lo = hi // 2
        while hi - lo > max(4096, hi // 256):
            mid = (lo + hi) // 2
            if runs(mid):
                hi = mid
            else:
                lo = mid
        return hi, fresh()
    b, X = smallest_budget()
    lz, mg = X.mar(prec="fp64", budget=b)
    assert abs(lz[0] - lz0[0]) < 1e-12 and abs(lz[0] - lz_ref) < 1e-10
    np.testing.assert_allclose(mg, mg0, rtol=0, atol=1e-12)
    _marg_close(X, mg[0], marg_ref, 1e-10)
    prof = fresh().profile("mar", prec="fp64", reps=1, budget=b)
    assert prof.get("recompute", {}).get("launches", 0) > 0, prof
    st = fresh().program_stats("mar", 1, "fp64", budget=b)
    assert st["recomputed"] > 0 and st["arena_bytes"] <= b < st["keep_all_bytes"], st
    # without recomputation the same tree needs more memory: the unlimited
    # program's profile has no recompute class, and at budget b the FP32
    # program (half the bytes) needs fewer recomputations or none
    assert "recompute" not in fresh().profile("mar", prec="fp64", reps=1)
    lz32, mg32 = fresh().mar(prec="fp32", budget=b)
    assert abs(lz32[0] - lz_ref) <= 1e-4 * abs(lz_ref)
    assert np.max(np.abs(mg32 - mg0)) < 1e-3


def test_autotuned_program_matches_default():
    """tn_options.autotune: the program built from the fastest of the timed
    candidate launch shapes (graph lanes x blocks per SM of the streaming
    kernels) computes the same FP64 values bit for bit as the default one
    (the shapes move work between streams and blocks, not its arithmetic),
    reports that it was tuned, and a second call reuses the choice."""
    m = synth.grid_ising(14, 3)
    ev = synth.evidence_batch(m, 6, 0.1, 17)
    M = tn.Model.from_synth(m)
    M.set_order(*M.reassociate(*M.optimize_order(0)))
    lz0, mg0 = M.mar(ev, prec="fp64")
    lz1, mg1 = M.mar(ev, prec="fp64", autotune=True)
    np.testing.assert_array_equal(lz1, lz0)
    np.testing.assert_array_equal(mg1, mg0)
    st = M.program_stats("mar", ev.shape[0], "fp64", autotune=True)
    assert st["tuned"] == 1 and st["lanes"] in (1, 2, 3, 4), st
    assert st["absorb_blocks_per_sm"] in (0, 2, 8), st
    assert M.program_stats("mar", ev.shape[0], "fp64")["tuned"] == 0
    lzt, mgt = M.mar(ev, prec="tf32", autotune=True)
    np.testing.assert_allclose(lzt, lz0, rtol=1e-4)
    assert np.max(np.abs(mgt - mg0)) < 1e-3
    lzp = M.pr(ev, prec="fp64", autotune=True)
    np.testing.assert_allclose(lzp, lz0, rtol=0, atol=1e-10)


def test_uai_files_through_tasks(tmp_path):
    """A model, its evidence sets and an MMAP query read from UAI-format
    files (tn_load_model, tn_read_evidence, tn_read_query) give the oracle's
    results: PR / MAR in FP64 within 1e-10 for every set, MAP and MMAP
    assignments exact; the 300-variable Bayesian network of the MAP workload
    read from files gives the oracle's MAP assignment."""
    m = synth.bayes_net(14, 21)
    ev = synth.evidence_batch(m, 4, 0.2, 5)
    q = synth.mmap_query(m, ev[0], 0.4, np.random.default_rng(3))
    pu, pe, pq = (str(tmp_path / x) for x in ("m.uai", "m.uai.evid", "m.uai.query"))
    synth.write_uai(m, pu)
    synth.write_evidence(ev, pe)
    synth.write_query(q, pq)
    M = tn.Model.from_uai(pu)
    E, Q = M.read_evidence(pe), M.read_query(pq)
    lz, mg = M.mar(E, prec="fp64")
    for b in range(E.shape[0]):
        lzr, mr = oracle.brute_mar(m, ev[b])
        assert abs(lz[b] - lzr) < 1e-10
        _marg_close(M, mg[b], mr, 1e-10)
    x, lp = M.map(E[0], prec="fp32")
    xb, lb = oracle.brute_map(m, ev[0])
    np.testing.assert_array_equal(x, xb)
    xq, lq = M.mmap(Q, E[0], prec="fp32")
    xqb, lqb = oracle.brute_mmap(m, q, ev[0])
    np.testing.assert_array_equal(xq, xqb)
    w = synth.workload(3)
    p3, e3 = str(tmp_path / "bn300.uai"), str(tmp_path / "bn300.uai.evid")
    synth.write_uai(w.model, p3)
    synth.write_evidence(w.evid, e3)
    M3 = tn.Model.from_uai(p3)
    x3, _ = M3.map(M3.read_evidence(e3)[0], prec="fp32")
    np.testing.assert_array_equal(x3, oracle.ve_map(w.model, w.evid[0])[0])


def test_multi_model_single_launch():
    """Models of uneven treewidth (grids, a 3-regular graph, a Bayesian
    network) solved by tn_solve_multi in one graph launch give the FP64
    results of separate tn_mar calls bit for bit, and the oracle's; PR in
    TF32 through the same launch within 1e-4."""
    ms = [synth.grid_ising(10, 31), synth.rrg3_ising(40, 32), synth.bayes_net(60, 33),
          synth.grid_ising(4, 34)]
    evs = [synth.evidence_batch(m, k, 0.2, 40 + i) for i, (m, k) in enumerate(zip(ms, [3, 2, 4, 5]))]
    Ms = [tn.Model.from_synth(m) for m in ms]
    res = tn.solve_multi(Ms, evs, "mar", "fp64")
    for M, e, (lz, mg) in zip(Ms, evs, res):
        lz1, mg1 = M.mar(e, prec="fp64")
        np.testing.assert_array_equal(lz, lz1)
        np.testing.assert_array_equal(mg, mg1)
    for b in range(evs[3].shape[0]):
        lzr, mr = oracle.brute_mar(ms[3], evs[3][b])
        assert abs(res[3][0][b] - lzr) < 1e-10
        _marg_close(Ms[3], res[3][1][b], mr, 1e-10)
    lzv, mv = oracle.ve_mar(ms[2], evs[2][1])
    assert abs(res[2][0][1] - lzv) < 1e-10
    _marg_close(Ms[2], res[2][1][1], mv, 1e-10)
    res32 = tn.solve_multi(Ms, evs, "pr", "tf32")
    for (lz, _), (lz64, _) in zip(res32, res):
        np.testing.assert_allclose(lz, lz64, rtol=1e-4)
    with pytest.raises(tn.TNError):
        tn.solve_multi([Ms[0], Ms[0]], [evs[0], evs[0]])


def test_workload4_batched_slice():
    """Workload 4 (3-regular, 200 spins, evidence sets with 10% observed) on
    its annealed tree: a batch of 16 evidence sets in BF16 and FP64 against
    the oracle's bucket elimination for two of them, and the batch against
    single-set runs."""
    w = synth.workload(4)
    m, ev = w.model, w.evid[:16]
    M = tn.Model.from_synth(m)
    M.set_order(*M.optimize_order(2, 6, 1))
    lz64, mg64 = M.mar(ev, prec="fp64")
    for b in (0, 9):
        assert abs(lz64[b] - oracle.ve_pr(m, ev[b])) < 1e-9
    lz1, mg1 = M.mar(ev[9:10], prec="fp64")
    assert abs(lz1[0] - lz64[9]) < 1e-9
    np.testing.assert_allclose(mg1[0], mg64[9], atol=1e-10)
    for prec in ("bf16", "tf32"):
        lz, mg = M.mar(ev, prec=prec)
        np.testing.assert_allclose(lz, lz64, rtol=1e-4)
        assert np.max(np.abs(mg - mg64)) < 1e-3
    # observed variables get the indicator of their value
    row = M.split(mg64[0])
    for v in np.nonzero(ev[0] >= 0)[0]:
        assert row[v][ev[0][v]] == 1.0


def test_workload4_partition_tree_batched():
    """Workload 4 on the bisection tree (order search method 3: space 2^25
    per evidence set instead of 2^28, read-write 16x lower): 64 evidence sets
    in BF16 and TF32 against the oracle's bucket elimination for two of them
    and against FP32 for all."""
    w = synth.workload(4)
    m, ev = w.model, w.evid[:64]
    M = tn.Model.from_synth(m)
    M.set_order(*M.optimize_order(3, 12, 2))
    assert M.tree_stats(1, "fp32")["sc"] <= 26
    lz32 = M.pr(ev, prec="fp32")
    for b in (0, 37):
        lz_ref = oracle.ve_pr(m, ev[b])
        assert abs(lz32[b] - lz_ref) <= 1e-4 * abs(lz_ref)
    for prec in ("bf16", "tf32"):
        lz, mg = M.mar(ev, prec=prec)
        np.testing.assert_allclose(lz, lz32, rtol=1e-4)
        for b in (0, 37):
            sp = M.split(mg[b])
            assert all(abs(sum(x) - 1.0) < 1e-6 for x in sp)


def test_workload4_annealed_tree_batched():
    """Workload 4 on the tree of order search method 4 (incremental
    annealing: about 10x fewer multiply-adds than method 2): 16 evidence sets,
    PR against the oracle's bucket elimination for two of them, TF32 MAR
    against FP32 PR, every marginal normalised."""
    w = synth.workload(4)
    m, ev = w.model, w.evid[:16]
    M = tn.Model.from_synth(m)
    M.set_order(*M.optimize_order(4, 4, 1))
    lz32 = M.pr(ev, prec="fp32")
    for b in (0, 9):
        lz_ref = oracle.ve_pr(m, ev[b])
        assert abs(lz32[b] - lz_ref) <= 1e-4 * abs(lz_ref)
    lz, mg = M.mar(ev, prec="tf32")
    np.testing.assert_allclose(lz, lz32, rtol=1e-4)
    for b in (0, 9):
        assert all(abs(sum(x) - 1.0) < 1e-6 for x in M.split(mg[b]))


def test_rrg3_sampling_statistics():
    """Backward sampling on a random 3-regular graph: per-spin frequencies
    within 5 sigma of the oracle's marginals and edge correlations
    E[s_i s_j] within 5 sigma of the exact ones (from brute force)."""
    m = synth.rrg3_ising(16, 31, field=True)
    M = tn.Model.from_synth(m)
    M.set_order(*M.optimize_order(1, 4, 2))
    n = 100000
    s = M.sample(n, seed=11, prec="fp32")
    _, marg = oracle.ve_mar(m)
    p1 = np.array([mv[1] for mv in marg])
    emp = s.mean(axis=0)
    sig = np.sqrt(p1 * (1 - p1) / n) + 1e-12
    assert np.all(np.abs(emp - p1) < 5 * sig + 1e-4)
    joint = oracle.brute_joint(m)
    X = ((np.arange(len(joint))[:, None] >> np.arange(m.nvars)[::-1]) & 1)
    S = 2 * X - 1
    Ss = 2 * s.astype(np.int64) - 1
    for sc in m.scopes:
        if len(sc) != 2:
            continue
        i, j = int(sc[0]), int(sc[1])
        exact = np.sum(joint * S[:, i] * S[:, j])
        empc = np.mean(Ss[:, i] * Ss[:, j])
        assert abs(empc - exact) < 5 * np.sqrt(max(1e-12, 1 - exact ** 2) / n) + 1e-4


def test_sampling_on_sliced_tree():
    """Sampling through a sliced tree (slice assignment drawn with
    probability Z_a / Z, then backward sampling within it): per-spin
    frequencies and edge correlations within 5 sigma of the exact values;
    observed variables (one of them sliced) keep their values."""
    m = synth.rrg3_ising(16, 33, field=True)
    M = tn.Model.from_synth(m)
    l, r = M.optimize_order(1, 4, 2)
    M.set_order(l, r, slice_vars=[3, 9])
    n = 100000
    s = M.sample(n, seed=5, prec="fp32")
    _, marg = oracle.ve_mar(m)
    p1 = np.array([mv[1] for mv in marg])
    emp = s.mean(axis=0)
    assert np.all(np.abs(emp - p1) < 5 * np.sqrt(p1 * (1 - p1) / n) + 1e-4)
    joint = oracle.brute_joint(m)
    S = 2 * ((np.arange(len(joint))[:, None] >> np.arange(m.nvars)[::-1]) & 1) - 1
    Ss = 2 * s.astype(np.int64) - 1
    for sc in m.scopes:
        if len(sc) == 2:
            i, j = int(sc[0]), int(sc[1])
            exact = np.sum(joint * S[:, i] * S[:, j])
            tol = 5 * np.sqrt(max(1e-12, 1 - exact ** 2) / n) + 1e-4
            assert abs(np.mean(Ss[:, i] * Ss[:, j]) - exact) < tol
    ev = np.full(m.nvars, -1, np.int32)
    ev[3], ev[5] = 1, 0
    n2 = 20000
    s2 = M.sample(n2, evid=ev, seed=6, prec="fp64")
    assert np.all(s2[:, 3] == 1) and np.all(s2[:, 5] == 0)
    _, marg_e = oracle.ve_mar(m, ev)
    p1e = np.array([mv[1] for mv in marg_e])
    assert np.all(np.abs(s2.mean(axis=0) - p1e) < 5 * np.sqrt(p1e * (1 - p1e) / n2) + 1e-4)


def test_workload5_sliced_pr_mar_and_sampling():
    """Workload 5 at full size (240-spin random 3-regular graph, no fields):
    annealed tree with re-associated chains, sliced to per-slice space 2^30
    (16 slice assignments).  PR + MAR in TF32: log Z within 1e-4 relative of
    the FP32 PR on the same tree; every marginal is 1/2 by the spin-flip
    symmetry of a field-free Ising model; 100000 samples whose spin
    frequencies are within 5 sigma of 1/2 and whose magnetisation per sample
    has zero mean within 5 sigma."""
    w = synth.workload(5)
    m = w.model
    M = tn.Model.from_synth(m)
    l, r = M.reassociate(*M.optimize_order(2, 20, 1))
    sl = M.choose_slices(30, 12, l, r)
    M.set_order(l, r, slice_vars=sl)
    assert M.tree_stats(1, "fp32")["sc"] <= 30
    lz_t, mg_t = M.mar(prec="tf32")
    lz_f = M.pr(prec="fp32")
    assert abs(lz_t[0] - lz_f[0]) <= 1e-4 * abs(lz_f[0])
    assert np.max(np.abs(mg_t - 0.5)) < 1e-3
    n = 100000
    s = M.sample(n, seed=7, prec="tf32")
    freq = s.mean(axis=0)
    assert np.all(np.abs(freq - 0.5) < 5 * np.sqrt(0.25 / n))
    mag = (2 * s.astype(np.int64) - 1).sum(axis=1)
    assert abs(mag.mean()) < 5 * mag.std() / np.sqrt(n)


def test_workload5_fp64_two_trees():
    """Workload 5 has no oracle value (its treewidth is beyond the CPU
    elimination).  Consistency instead: FP64 log Z on two different trees
    from the same annealing run (seed 1) -- absorption chains re-associated
    and sliced to per-slice space 2^30 (4 slice variables), and as found,
    sliced to 2^28 (7 slice variables) -- agree to 1e-11 relative.  Not an
    oracle check: both runs use this library's FP64 path."""
    w = synth.workload(5)
    M = tn.Model.from_synth(w.model)
    l0, r0 = M.optimize_order(2, 20, 1)
    lz, sets = [], []
    for (l, r), space in ((M.reassociate(l0, r0), 30), ((l0, r0), 28)):
        sl = M.choose_slices(space, 12, l, r)
        M.set_order(l, r, slice_vars=sl)
        sets.append(sorted(sl))
        lz.append(M.pr(prec="fp64")[0])
    assert sets[0] != sets[1]
    assert abs(lz[0] - lz[1]) <= 1e-11 * abs(lz[0]), lz

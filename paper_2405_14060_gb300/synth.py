"""Seeded synthetic graphical models and evidence, plus UAI-format text I/O.

This module only *builds inputs*: factor scopes and tables drawn from seeded
generators, evidence sets and query sets.  It performs no inference arithmetic
(no contraction, elimination, normalisation of results), so both the CUDA path
and the CPU oracle can take their inputs from here without sharing any of the
method's computation.

Conventions
-----------
* A model is a :class:`Model`: ``card[v]`` is the domain size of variable ``v``;
  factor ``f`` has scope ``scopes[f]`` (storage order) and a float64 table
  ``tables[f]`` in row-major order with the *last* scope variable fastest
  (the UAI convention).
* Binary Ising spins map index ``k in {0,1}`` to spin ``s = 2k - 1`` (index 0 is
  spin -1).  Couplings give the table ``exp(J s_i s_j)``, fields ``exp(h s_i)``.
* ``h ~ N(0, 0.5)`` reads 0.5 as the standard deviation.
* Evidence is an int32 vector over all variables, ``-1`` for unobserved.

Workloads (seed ``20240522 + k`` for workload ``k``)
----------------------------------------------------
1. 10x10 grid Ising, J~N(0,1), h~N(0,0.5), no evidence.
2. 24x24 grid Ising, same distributions, no evidence.
3. Bayesian network, 300 variables, domains U{2,3,4}, banded random DAG with
   up to 3 parents drawn from the previous ``W`` variables of a random
   topological order, CPT rows ~ Dirichlet(1); 20% observed, 30% of the
   remaining variables are the MMAP query.
4. Random 3-regular graph (pairing model), 200 binary variables, couplings
   J~N(0,1), no fields; 512 evidence sets with 10% of variables observed.
5. Random 3-regular graph, 240 binary variables, no evidence.
"""
from __future__ import annotations

import dataclasses
import io
from typing import List, Optional, Sequence

import numpy as np

BASE_SEED = 20240522
BN_WINDOW = 4


@dataclasses.dataclass
class Model:
    card: np.ndarray                 # int32 [nvars]
    scopes: List[np.ndarray]         # int32 [nv_f] each, storage order
    tables: List[np.ndarray]         # float64 [prod card] each, last var fastest
    kind: str = "MARKOV"             # "MARKOV" or "BAYES"
    name: str = ""

    @property
    def nvars(self) -> int:
        return int(self.card.shape[0])

    @property
    def nfactors(self) -> int:
        return len(self.scopes)

    def flat(self):
        """(card, scope_off, scope_vars, tables) as contiguous arrays, the
        layout taken by ``tn_load_model_arrays``."""
        off = np.zeros(self.nfactors + 1, dtype=np.int32)
        for i, s in enumerate(self.scopes):
            off[i + 1] = off[i] + len(s)
        sv = (np.concatenate(self.scopes).astype(np.int32)
              if self.nfactors else np.zeros(0, np.int32))
        tb = (np.concatenate(self.tables).astype(np.float64)
              if self.nfactors else np.zeros(0))
        return (np.ascontiguousarray(self.card, dtype=np.int32), off, sv, tb)


def _spin_pair_table(J: float) -> np.ndarray:
    s = np.array([-1.0, 1.0])
    return np.exp(J * np.outer(s, s)).reshape(-1)


def _spin_field_table(h: float) -> np.ndarray:
    return np.exp(h * np.array([-1.0, 1.0]))


def grid_ising(L: int, seed: int, W: Optional[int] = None,
               h_std: float = 0.5, field: bool = True) -> Model:
    """L x W grid (W defaults to L) of binary spins; variable ``r*W + c``.

    Edges are enumerated row-major: for each site, the edge to its right
    neighbour, then the edge to the site below.  Couplings are drawn first
    (one normal per edge, in edge order), then one field per site."""
    W = L if W is None else W
    rng = np.random.Generator(np.random.PCG64(seed))
    n = L * W
    edges = []
    for r in range(L):
        for c in range(W):
            i = r * W + c
            if c + 1 < W:
                edges.append((i, i + 1))
            if r + 1 < L:
                edges.append((i, i + W))
    J = rng.normal(0.0, 1.0, size=len(edges))
    h = rng.normal(0.0, h_std, size=n) if field else np.zeros(n)
    scopes, tables = [], []
    for (i, j), Jij in zip(edges, J):
        scopes.append(np.array([i, j], np.int32))
        tables.append(_spin_pair_table(Jij))
    if field:
        for i in range(n):
            scopes.append(np.array([i], np.int32))
            tables.append(_spin_field_table(h[i]))
    return Model(np.full(n, 2, np.int32), scopes, tables, "MARKOV",
                 f"grid{L}x{W}")


def random_regular3_edges(n: int, rng: np.random.Generator):
    """Random simple 3-regular graph on n vertices by the pairing model:
    3n half-edges are matched by a uniform shuffle; a matching with a loop or
    a repeated edge is rejected and redrawn."""
    if (3 * n) % 2:
        raise ValueError("3-regular graph needs an even number of vertices")
    while True:
        stubs = np.repeat(np.arange(n), 3)
        rng.shuffle(stubs)
        pairs = stubs.reshape(-1, 2)
        ok = True
        seen = set()
        for a, b in pairs:
            if a == b:
                ok = False
                break
            key = (min(a, b), max(a, b))
            if key in seen:
                ok = False
                break
            seen.add(key)
        if ok:
            return sorted(seen)


def rrg3_ising(n: int, seed: int, field: bool = False,
               h_std: float = 0.5) -> Model:
    """Random 3-regular graph Ising model, couplings J~N(0,1) drawn in
    sorted-edge order (then fields, if any)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    edges = random_regular3_edges(n, rng)
    J = rng.normal(0.0, 1.0, size=len(edges))
    scopes, tables = [], []
    for (i, j), Jij in zip(edges, J):
        scopes.append(np.array([i, j], np.int32))
        tables.append(_spin_pair_table(Jij))
    if field:
        h = rng.normal(0.0, h_std, size=n)
        for i in range(n):
            scopes.append(np.array([i], np.int32))
            tables.append(_spin_field_table(h[i]))
    return Model(np.full(n, 2, np.int32), scopes, tables, "MARKOV",
                 f"rrg3_{n}")


def tree_ising(n: int, seed: int, J_std: float = 1.0) -> Model:
    """Random recursive tree on n spins (vertex i>0 attaches to a uniform
    earlier vertex), couplings J~N(0, J_std), no fields."""
    rng = np.random.Generator(np.random.PCG64(seed))
    parents = [int(rng.integers(0, i)) for i in range(1, n)]
    J = rng.normal(0.0, J_std, size=n - 1)
    scopes, tables = [], []
    for i, (p, Jij) in enumerate(zip(parents, J), start=1):
        scopes.append(np.array([p, i], np.int32))
        tables.append(_spin_pair_table(Jij))
    return Model(np.full(n, 2, np.int32), scopes, tables, "MARKOV",
                 f"tree{n}")


def chain_model(n: int, card: Sequence[int], seed: int) -> Model:
    """Chain x0 - x1 - ... with positive random unary and pair tables
    (entries exp(N(0,1))): a hidden-Markov-like model for Viterbi pins."""
    rng = np.random.Generator(np.random.PCG64(seed))
    card = np.asarray(card, np.int32)
    scopes, tables = [], []
    for i in range(n):
        scopes.append(np.array([i], np.int32))
        tables.append(np.exp(rng.normal(size=card[i])))
    for i in range(n - 1):
        scopes.append(np.array([i, i + 1], np.int32))
        tables.append(np.exp(rng.normal(size=card[i] * card[i + 1])))
    return Model(card, scopes, tables, "MARKOV", f"chain{n}")


def random_markov(nvars: int, nfactors: int, max_scope: int, seed: int,
                  cards=(2, 3)) -> Model:
    """Small random Markov network: random scopes of 1..max_scope distinct
    variables, entries exp(N(0,1)).  Every variable appears in at least one
    factor (a unary factor is added for any that does not)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    card = rng.choice(np.asarray(cards), size=nvars).astype(np.int32)
    scopes, tables = [], []
    used = np.zeros(nvars, bool)
    for _ in range(nfactors):
        k = int(rng.integers(1, max_scope + 1))
        sc = rng.choice(nvars, size=min(k, nvars), replace=False).astype(np.int32)
        used[sc] = True
        scopes.append(sc)
        tables.append(np.exp(rng.normal(size=int(np.prod(card[sc])))))
    for v in np.nonzero(~used)[0]:
        scopes.append(np.array([v], np.int32))
        tables.append(np.exp(rng.normal(size=int(card[v]))))
    return Model(card, scopes, tables, "MARKOV", f"rand{nvars}")


def bayes_net(n: int, seed: int, window: int = BN_WINDOW, max_parents: int = 3,
              cards: Sequence[int] = (2, 3, 4)) -> Model:
    """Banded random DAG Bayesian network.

    Variable ids are placed in a uniformly random topological order.  The
    variable at topological position i draws u ~ U{0..max_parents} and takes
    min(u, available) distinct parents uniformly from the previous ``window``
    positions.  Domain sizes are uniform over ``cards``; every CPT row (one
    per parent configuration) is drawn from Dirichlet(1).  Factor scope is
    (parents in topological order..., child), child fastest."""
    rng = np.random.Generator(np.random.PCG64(seed))
    card = rng.choice(np.asarray(cards), size=n).astype(np.int32)
    topo = rng.permutation(n).astype(np.int32)
    scopes, tables = [], []
    for pos in range(n):
        child = int(topo[pos])
        lo = max(0, pos - window)
        avail = pos - lo
        u = int(rng.integers(0, max_parents + 1))
        k = min(u, avail)
        if k:
            ppos = np.sort(rng.choice(np.arange(lo, pos), size=k, replace=False))
            parents = topo[ppos]
        else:
            parents = np.zeros(0, np.int32)
        sc = np.concatenate([parents, [child]]).astype(np.int32)
        nrows = int(np.prod(card[parents])) if k else 1
        cpt = rng.dirichlet(np.ones(card[child]), size=nrows)
        scopes.append(sc)
        tables.append(cpt.reshape(-1))
    # keep factors in variable-id order of their child
    order = np.argsort([int(s[-1]) for s in scopes], kind="stable")
    scopes = [scopes[i] for i in order]
    tables = [tables[i] for i in order]
    return Model(card, scopes, tables, "BAYES", f"bn{n}")


def random_evidence(model: Model, frac: float, rng: np.random.Generator,
                    exclude: Optional[np.ndarray] = None) -> np.ndarray:
    """Observe round(frac * nvars) variables chosen uniformly (outside
    ``exclude``) at uniform random values; -1 marks unobserved."""
    n = model.nvars
    cand = np.arange(n) if exclude is None else np.setdiff1d(np.arange(n), exclude)
    k = int(round(frac * n))
    ev = np.full(n, -1, np.int32)
    if k:
        vs = rng.choice(cand, size=k, replace=False)
        for v in vs:
            ev[v] = int(rng.integers(0, model.card[v]))
    return ev


def evidence_batch(model: Model, batch: int, frac: float, seed: int) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.stack([random_evidence(model, frac, rng) for _ in range(batch)])


def mmap_query(model: Model, evid: np.ndarray, frac: float,
               rng: np.random.Generator) -> np.ndarray:
    """Query set: round(frac * #unobserved) unobserved variables, sorted."""
    free = np.nonzero(evid < 0)[0]
    k = int(round(frac * len(free)))
    return np.sort(rng.choice(free, size=k, replace=False)).astype(np.int32)


@dataclasses.dataclass
class Workload:
    index: int
    model: Model
    evid: np.ndarray                 # int32 [batch, nvars]
    query: Optional[np.ndarray] = None
    description: str = ""


def workload(k: int) -> Workload:
    """The five seeded workloads (see module docstring)."""
    seed = BASE_SEED + k
    if k == 1:
        m = grid_ising(10, seed)
        return Workload(1, m, np.full((1, m.nvars), -1, np.int32), None,
                        "10x10 grid Ising, PR+MAR, FP64")
    if k == 2:
        m = grid_ising(24, seed)
        return Workload(2, m, np.full((1, m.nvars), -1, np.int32), None,
                        "24x24 grid Ising, PR+MAR, TF32/FP32")
    if k == 3:
        m = bayes_net(300, seed)
        rng = np.random.Generator(np.random.PCG64(seed + 1000))
        ev = random_evidence(m, 0.2, rng)
        q = mmap_query(m, ev, 0.3, rng)
        return Workload(3, m, ev[None, :], q,
                        "300-var banded BN, MAP + MMAP, tropical FP32")
    if k == 4:
        m = rrg3_ising(200, seed)
        ev = evidence_batch(m, 512, 0.1, seed + 1000)
        return Workload(4, m, ev, None,
                        "3-regular 200 spins, 512 evidence sets, PR+MAR, BF16")
    if k == 5:
        m = rrg3_ising(240, seed)
        return Workload(5, m, np.full((1, m.nvars), -1, np.int32), None,
                        "3-regular 240 spins, PR+MAR TF32 + sampling")
    raise ValueError(k)


# ----------------------------------------------------------------- UAI text

def write_uai(model: Model, path_or_buf) -> None:
    """Write a model in UAI competition text format (tables to 17 digits)."""
    out = io.StringIO()
    out.write(f"{model.kind}\n{model.nvars}\n")
    out.write(" ".join(str(int(c)) for c in model.card) + "\n")
    out.write(f"{model.nfactors}\n")
    for s in model.scopes:
        out.write(f"{len(s)} " + " ".join(str(int(v)) for v in s) + "\n")
    out.write("\n")
    for t in model.tables:
        out.write(f"{len(t)}\n")
        out.write(" ".join(repr(float(x)) for x in t) + "\n\n")
    text = out.getvalue()
    if hasattr(path_or_buf, "write"):
        path_or_buf.write(text)
    else:
        with open(path_or_buf, "w") as f:
            f.write(text)


def write_evidence(evid, path) -> None:
    """Write evidence sets (int [nsets, nvars] or [nvars], -1 = unobserved) in
    the UAI multi-sample evidence format: "<nsets>" then, per set,
    "<nobs> v1 x1 v2 x2 ..."."""
    e = np.atleast_2d(np.asarray(evid))
    lines = [str(e.shape[0])]
    for row in e:
        obs = np.nonzero(row >= 0)[0]
        lines.append(" ".join([str(len(obs))] + [f"{int(v)} {int(row[v])}" for v in obs]))
    with open(path, "w") as f:
        f.write("\n".join(lines) + "\n")


def write_query(query, path) -> None:
    """Write an MMAP query in the UAI query format: "<nq> v1 ... vq"."""
    q = [int(v) for v in query]
    with open(path, "w") as f:
        f.write(" ".join([str(len(q))] + [str(v) for v in q]) + "\n")


def read_uai(path: str) -> Model:
    with open(path) as f:
        toks = f.read().split()
    kind = toks[0]
    p = 1
    n = int(toks[p]); p += 1
    card = np.array([int(t) for t in toks[p:p + n]], np.int32); p += n
    nf = int(toks[p]); p += 1
    scopes = []
    for _ in range(nf):
        k = int(toks[p]); p += 1
        scopes.append(np.array([int(t) for t in toks[p:p + k]], np.int32)); p += k
    tables = []
    for _ in range(nf):
        sz = int(toks[p]); p += 1
        tables.append(np.array([float(t) for t in toks[p:p + sz]])); p += sz
    return Model(card, scopes, tables, kind, path)

"""CPU FP64 oracle for exact inference (test infrastructure only).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA path:
the C library in ``tn_oracle.c`` implements the plain definitions of PR, MAR,
MPE, MMAP and sampling (paper Sec. "Tensor networks for probabilistic
modeling") by brute-force enumeration and by FP64 bucket elimination, and
``con.py`` implements the tensor-network contraction of Def. "Tensor Network"
(Eq. contraction-definition) and its tropical counterpart (Eq. tropical)
directly from those definitions.

Pins (tests/test_oracle.py): closed forms for tree Ising models and
zero-coupling models, Z = 1 for Bayesian networks without evidence, finite
differences of log Z for marginals, a textbook Viterbi recursion for MPE on
chains, agreement of brute force with elimination, order independence, and
the worked examples the paper prints for the contraction definition.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tn_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

E_ZERO = -4


class OracleError(RuntimeError):
    pass


def build(force: bool = False) -> str:
    """Compile tn_oracle.c with gcc (OpenMP) into oracle/_build/."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = ctypes.CDLL(_LIB_PATH)
            _lib.or_log_weight.restype = ctypes.c_double
        return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


class _M:
    """Contiguous arrays of a model for the C calls."""

    def __init__(self, model):
        card, off, sv, tab = model.flat()
        self.n = int(card.shape[0])
        self.card = np.ascontiguousarray(card, np.int32)
        self.nf = int(off.shape[0] - 1)
        self.off = np.ascontiguousarray(off, np.int32)
        self.sv = np.ascontiguousarray(sv, np.int32)
        self.tab = np.ascontiguousarray(tab, np.float64)

    def args(self):
        return (ctypes.c_int(self.n), _p(self.card), ctypes.c_int(self.nf),
                _p(self.off), _p(self.sv), _p(self.tab))


def _ev(model, evid):
    if evid is None:
        return np.full(model.nvars, -1, np.int32)
    return np.ascontiguousarray(evid, np.int32).reshape(-1)


def _check(rc, what):
    if rc == E_ZERO:
        raise ZeroDivisionError(f"{what}: p(e) = 0")
    if rc != 0:
        raise OracleError(f"{what} failed with code {rc}")


def num_threads() -> int:
    return int(_load().or_num_threads())


def set_num_threads(n: int) -> None:
    """Number of OpenMP threads the following oracle calls use."""
    L = _load()
    L.or_set_num_threads.restype = None
    L.or_set_num_threads(ctypes.c_int(int(n)))


# ------------------------------------------------------------ brute force

def brute_pr(model, evid=None) -> float:
    m, e = _M(model), _ev(model, evid)
    out = ctypes.c_double()
    _check(_load().or_brute_pr(*m.args(), _p(e), ctypes.byref(out)), "brute_pr")
    return out.value


def brute_mar(model, evid=None):
    """(log Z, marginals as a list of per-variable arrays)."""
    m, e = _M(model), _ev(model, evid)
    out = ctypes.c_double()
    marg = np.zeros(int(m.card.sum()))
    _check(_load().or_brute_mar(*m.args(), _p(e), ctypes.byref(out), _p(marg)),
           "brute_mar")
    return out.value, split_marginals(model, marg)


def brute_map(model, evid=None):
    m, e = _M(model), _ev(model, evid)
    x = np.zeros(m.n, np.int32)
    out = ctypes.c_double()
    _check(_load().or_brute_map(*m.args(), _p(e), _p(x), ctypes.byref(out)),
           "brute_map")
    return x, out.value


def brute_mmap(model, query, evid=None):
    m, e = _M(model), _ev(model, evid)
    q = np.ascontiguousarray(query, np.int32)
    x = np.zeros(len(q), np.int32)
    out = ctypes.c_double()
    _check(_load().or_brute_mmap(*m.args(), _p(e), ctypes.c_int(len(q)), _p(q),
                                 _p(x), ctypes.byref(out)), "brute_mmap")
    return x, out.value


def brute_joint(model, evid=None) -> np.ndarray:
    """p(free vars | e), free variables in increasing id, last fastest."""
    m, e = _M(model), _ev(model, evid)
    free = [v for v in range(m.n) if e[v] < 0]
    n = int(np.prod([m.card[v] for v in free])) if free else 1
    out = np.zeros(n)
    _check(_load().or_brute_joint(*m.args(), _p(e), _p(out)), "brute_joint")
    return out


# -------------------------------------------------------- elimination

def minfill_order(model, evid=None):
    """(order of the unobserved variables, log2 of the largest table)."""
    m, e = _M(model), _ev(model, evid)
    order = np.zeros(m.n, np.int32)
    lm = ctypes.c_double()
    _check(_load().or_minfill_order(*m.args(), _p(e), _p(order), ctypes.byref(lm)),
           "minfill_order")
    return order[order >= 0], lm.value


def ve_pr(model, evid=None, order=None) -> float:
    m, e = _M(model), _ev(model, evid)
    out = ctypes.c_double()
    if order is not None:
        o = np.full(m.n + 1, -1, np.int32)
        o[:len(order)] = order
        op = _p(o)
    else:
        op = None
    _check(_load().or_ve_pr(*m.args(), _p(e), op, ctypes.byref(out)), "ve_pr")
    return out.value


def ve_pr_prefix(model, order, nelim, evid=None):
    """Eliminate only the first ``nelim`` variables of ``order`` (a bounded
    sample of a PR elimination).  Returns (work of the prefix, work of the
    full order), both as the symbolic count of bucket entries visited."""
    m, e = _M(model), _ev(model, evid)
    o = np.full(m.n + 1, -1, np.int32)
    o[:len(order)] = order
    wp, wf = ctypes.c_double(), ctypes.c_double()
    _check(_load().or_ve_pr_prefix(*m.args(), _p(e), _p(o), ctypes.c_int(nelim),
                                   ctypes.byref(wp), ctypes.byref(wf)), "ve_pr_prefix")
    return wp.value, wf.value


def ve_mar(model, evid=None):
    m, e = _M(model), _ev(model, evid)
    out = ctypes.c_double()
    marg = np.zeros(int(m.card.sum()))
    _check(_load().or_ve_mar(*m.args(), _p(e), ctypes.byref(out), _p(marg)), "ve_mar")
    return out.value, split_marginals(model, marg)


def ve_map(model, evid=None, order=None):
    """(MAP assignment, its log weight) by max-sum bucket elimination;
    ``order`` (optional) is the elimination order (observed variables are
    skipped), else min-fill."""
    m, e = _M(model), _ev(model, evid)
    x = np.zeros(m.n, np.int32)
    out = ctypes.c_double()
    op = None
    if order is not None:
        o = np.full(m.n + 1, -1, np.int32)
        o[:len(order)] = order
        op = _p(o)
    _check(_load().or_ve_map(*m.args(), _p(e), op, _p(x), ctypes.byref(out)), "ve_map")
    return x, out.value


def map_gap(model, evid=None, order=None):
    """(MAP assignment x*, its log weight, gap): the gap is the log weight of
    x* minus that of the best assignment that differs from x* (in FP64).  The
    runner-up differs from x* in some free variable v, so it is the best of
    the MAP problems with v clamped to a value other than x*_v, taken over
    every v and value (Eq. log-map with extra evidence)."""
    e = _ev(model, evid).copy()
    x, lp = ve_map(model, e, order)
    best2 = -np.inf
    for v in range(model.nvars):
        if e[v] >= 0:
            continue
        for val in range(int(model.card[v])):
            if val == x[v]:
                continue
            e2 = e.copy()
            e2[v] = val
            try:
                best2 = max(best2, ve_map(model, e2, order)[1])
            except ZeroDivisionError:
                pass
    return x, lp, lp - best2


def ve_mmap(model, query, evid=None):
    m, e = _M(model), _ev(model, evid)
    q = np.ascontiguousarray(query, np.int32)
    x = np.zeros(len(q), np.int32)
    out = ctypes.c_double()
    _check(_load().or_ve_mmap(*m.args(), _p(e), ctypes.c_int(len(q)), _p(q), _p(x),
                              ctypes.byref(out)), "ve_mmap")
    return x, out.value


def ve_sample(model, n: int, uniforms: np.ndarray, evid=None) -> np.ndarray:
    """n exact samples; ``uniforms`` holds n * (#unobserved) values in [0,1)."""
    m, e = _M(model), _ev(model, evid)
    nfree = int((e < 0).sum())
    u = np.ascontiguousarray(uniforms, np.float64).reshape(-1)
    if u.shape[0] < n * nfree:
        raise ValueError("not enough uniforms")
    out = np.zeros((n, m.n), np.int8)
    _check(_load().or_ve_sample(*m.args(), _p(e), ctypes.c_int64(n), _p(u), _p(out)),
           "ve_sample")
    return out


def log_weight(model, x) -> float:
    """log prod_f T_f(x) at a full assignment x."""
    m = _M(model)
    xa = np.ascontiguousarray(x, np.int32)
    return float(_load().or_log_weight(*m.args(), _p(xa)))


def clamped_marginal(model, v: int, evid=None, order=None, logz=None):
    """p(v = x | e) for every x by conditioning: Z(e, v=x) / Z(e), each by
    bucket elimination (Eq. mar-prob written out).  ``order`` (optional) is
    the elimination order of every call (observed variables are skipped);
    ``logz`` (optional) is log Z(e) when already known."""
    e = _ev(model, evid).copy()
    lz = ve_pr(model, e, order) if logz is None else float(logz)
    out = np.zeros(int(model.card[v]))
    for x in range(int(model.card[v])):
        e2 = e.copy()
        e2[v] = x
        try:
            out[x] = np.exp(ve_pr(model, e2, order) - lz)
        except ZeroDivisionError:
            out[x] = 0.0
    return out


def brute_joint_marginal(model, query, evid=None) -> np.ndarray:
    """p(Q = q | e) for the variable set Q = query by summing the enumerated
    joint of the free variables over the others (the definition of a
    marginal); axes in the order of `query`.  Observed query variables take
    probability 1 at their value."""
    e = _ev(model, evid)
    free = [v for v in range(len(e)) if e[v] < 0]
    joint = brute_joint(model, e).reshape([int(model.card[v]) for v in free] or [1])
    keep = [free.index(v) for v in query if e[v] < 0]
    drop = tuple(i for i in range(len(free)) if i not in keep)
    sub = joint.sum(axis=drop) if free else joint.reshape(())
    # axes of `sub` follow increasing variable id; move them to query order
    free_q = sorted(v for v in query if e[v] < 0)
    if free_q:
        sub = np.transpose(sub, [free_q.index(v) for v in query if e[v] < 0])
    out = np.zeros([int(model.card[v]) for v in query])
    idx = tuple(slice(None) if e[v] < 0 else int(e[v]) for v in query)
    out[idx] = sub
    return out


def clamped_joint_marginal(model, query, evid=None) -> np.ndarray:
    """p(Q = q | e) = Z(e, Q = q) / Z(e), each Z by bucket elimination
    (Eq. mar-prob for a variable set, written out); axes in query order."""
    e = _ev(model, evid).copy()
    lz = ve_pr(model, e)
    shape = [int(model.card[v]) for v in query]
    out = np.zeros(shape)
    for q in np.ndindex(*shape):
        e2 = e.copy()
        if any(e[v] >= 0 and e[v] != x for v, x in zip(query, q)):
            continue
        for v, x in zip(query, q):
            e2[v] = x
        try:
            out[q] = np.exp(ve_pr(model, e2) - lz)
        except ZeroDivisionError:
            out[q] = 0.0
    return out


def split_marginals(model, flat):
    res, o = [], 0
    for c in model.card:
        res.append(np.array(flat[o:o + int(c)]))
        o += int(c)
    return res

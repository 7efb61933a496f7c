"""Thin ctypes binding of libtn (include/tn.h).

Argument marshalling only: every computation runs in libtn's CUDA kernels.
There is no fallback -- importing the binding without a built libtn raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

from . import build as _build

TN_FP64, TN_FP32, TN_TF32, TN_BF16 = 0, 1, 2, 3
PRECS = {"fp64": TN_FP64, "fp32": TN_FP32, "tf32": TN_TF32, "bf16": TN_BF16}
STATUS = {0: "TN_OK", 1: "TN_E_ARG", 2: "TN_E_PARSE", 3: "TN_E_ORDER", 4: "TN_E_OOM",
          5: "TN_E_CUDA", 6: "TN_E_TIMEOUT", 7: "TN_E_UNSUPPORTED"}

# Every symbol include/tn.h declares (checked by the CPU test suite).
EXPORTS = ["tn_load_model", "tn_load_model_arrays", "tn_free_model", "tn_set_order",
           "tn_tree_from_elimination", "tn_optimize_order", "tn_tree_stats", "tn_pr",
           "tn_mar", "tn_map", "tn_mmap", "tn_sample", "tn_pr_dev", "tn_mar_dev",
           "tn_last_device_ms", "tn_last_launch_count", "tn_last_error", "tn_contract_dev",
           "tn_profile", "tn_profile_steps", "tn_contract_dev_noalloc",
           "tn_reassociate", "tn_choose_slices", "tn_joint_mar", "tn_program_stats",
           "tn_read_evidence", "tn_read_query", "tn_solve_multi"]
PROFILE_CLASSES = ["small", "absorb", "reduce", "tcgemm", "simtgemm", "prep", "generic", "bgemm",
                   "recompute"]


class TNError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Options(ctypes.Structure):
    _fields_ = [("prec", ctypes.c_int), ("hbm_budget_bytes", ctypes.c_int64),
                ("max_slices", ctypes.c_int), ("autotune", ctypes.c_int),
                ("cuda_stream", ctypes.c_void_p)]


_lib = None
LIB_PATH = _build.LIB


def lib():
    """Load libtn.so (built in-tree by __graft_entry__.build() / build.py)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libtn.so is not built ({LIB_PATH}); run "
                              "python -c 'import __graft_entry__ as g; g.build()'")
        L = ctypes.CDLL(LIB_PATH)
        P, I, I64, D, U64 = (ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double,
                             ctypes.c_uint64)
        sig = {
            "tn_load_model": [ctypes.c_char_p, P],
            "tn_load_model_arrays": [I, P, I, P, P, P, P],
            "tn_set_order": [P, I, P, P, I, P],
            "tn_tree_from_elimination": [P, I, P, P, P],
            "tn_optimize_order": [P, I, I, U64, P, P],
            "tn_tree_stats": [P, I, I, P],
            "tn_pr": [P, I, P, P, P],
            "tn_mar": [P, I, P, P, P, P],
            "tn_map": [P, P, P, P, P],
            "tn_mmap": [P, P, I, P, P, P, P],
            "tn_sample": [P, P, U64, I64, P, P],
            "tn_pr_dev": [P, I, P, P, I, P, P],
            "tn_mar_dev": [P, I, P, P, I, P, P, P, P],
            "tn_contract_dev": [I, P, I, P, P, I, P, P, I, P, P, I, I, I, P, P],
            "tn_profile": [P, I, I, P, P, I, P],
            "tn_profile_steps": [P, I, I, P, P, I, P, P],
            "tn_contract_dev_noalloc": [I, P, I, P, P, I, P, P, I, P, P, I, I, P, P],
            "tn_reassociate": [P, P, P, P, P],
            "tn_choose_slices": [P, P, P, D, I, P, P],
            "tn_joint_mar": [P, P, I, P, P, P, P],
            "tn_program_stats": [P, I, I, P, P],
            "tn_read_evidence": [P, ctypes.c_char_p, I, P, P],
            "tn_read_query": [P, ctypes.c_char_p, I, P, P],
            "tn_solve_multi": [I, I, P, P, P, P, P, P],
        }
        for name, args in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = ctypes.c_int
        L.tn_free_model.argtypes = [P]
        L.tn_free_model.restype = None
        L.tn_last_error.restype = ctypes.c_char_p
        L.tn_last_device_ms.argtypes = [P]
        L.tn_last_device_ms.restype = D
        L.tn_last_launch_count.argtypes = [P]
        L.tn_last_launch_count.restype = I64
        _lib = L
    return _lib


def _ck(st: int):
    if st != 0:
        raise TNError(st, lib().tn_last_error().decode())


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _opts(prec="fp64", budget=0, stream=None, autotune=False) -> Options:
    o = Options()
    o.prec = PRECS[prec] if isinstance(prec, str) else int(prec)
    o.hbm_budget_bytes = int(budget)
    o.max_slices = 0
    o.autotune = 1 if autotune else 0
    o.cuda_stream = stream
    return o


class Model:
    """A graphical model held by libtn (one tn_model)."""

    def __init__(self, handle, nvars, card, nfactors, table_sizes):
        self._h = handle
        self.nvars = nvars
        self.card = np.asarray(card, np.int32)
        self.nfactors = nfactors
        self.table_sizes = np.asarray(table_sizes, np.int64)

    @property
    def nleaves(self):
        return self.nfactors + self.nvars

    @classmethod
    def from_arrays(cls, card, scopes, tables) -> "Model":
        card = np.ascontiguousarray(card, np.int32)
        off = np.zeros(len(scopes) + 1, np.int32)
        for i, s in enumerate(scopes):
            off[i + 1] = off[i] + len(s)
        sv = (np.ascontiguousarray(np.concatenate([np.asarray(s, np.int32) for s in scopes]))
              if scopes else np.zeros(1, np.int32))
        tb = (np.ascontiguousarray(np.concatenate([np.asarray(t, np.float64) for t in tables]))
              if tables else np.zeros(1))
        h = ctypes.c_void_p()
        _ck(lib().tn_load_model_arrays(len(card), _ptr(card), len(scopes), _ptr(off), _ptr(sv),
                                       _ptr(tb), ctypes.byref(h)))
        return cls(h, len(card), card, len(scopes), [len(t) for t in tables])

    @classmethod
    def from_synth(cls, m) -> "Model":
        return cls.from_arrays(m.card, m.scopes, m.tables)

    @classmethod
    def from_uai(cls, path: str) -> "Model":
        h = ctypes.c_void_p()
        _ck(lib().tn_load_model(path.encode(), ctypes.byref(h)))
        # read back sizes from the file header for convenience
        with open(path) as f:
            toks = f.read().split()
        n = int(toks[1])
        card = [int(t) for t in toks[2:2 + n]]
        nf = int(toks[2 + n])
        p = 3 + n
        sizes = []
        for _ in range(nf):
            k = int(toks[p]); p += 1
            sizes.append(int(np.prod([card[int(v)] for v in toks[p:p + k]])))
            p += k
        return cls(h, n, card, nf, sizes)

    def __del__(self):
        try:
            if self._h:
                lib().tn_free_model(self._h)
        except Exception:
            pass

    def read_evidence(self, path: str) -> np.ndarray:
        """Evidence sets of a UAI evidence file: int32 [nsets, nvars], -1 = free."""
        n = ctypes.c_int()
        _ck(lib().tn_read_evidence(self._h, path.encode(), 0, None, ctypes.byref(n)))
        out = np.zeros((max(1, n.value), self.nvars), np.int32)
        _ck(lib().tn_read_evidence(self._h, path.encode(), n.value, _ptr(out), ctypes.byref(n)))
        return out[:n.value]

    def read_query(self, path: str) -> np.ndarray:
        """Query variables of a UAI MMAP query file."""
        n = ctypes.c_int()
        _ck(lib().tn_read_query(self._h, path.encode(), 0, None, ctypes.byref(n)))
        out = np.zeros(max(1, n.value), np.int32)
        _ck(lib().tn_read_query(self._h, path.encode(), n.value, _ptr(out), ctypes.byref(n)))
        return out[:n.value]

    # ------------------------------------------------------------ orders
    def set_order(self, left=None, right=None, slice_vars: Sequence[int] = ()):
        sl = np.ascontiguousarray(slice_vars, np.int32) if len(slice_vars) else None
        if left is None:
            _ck(lib().tn_set_order(self._h, 0, None, None, 0, None))
            return
        l = np.ascontiguousarray(left, np.int32)
        r = np.ascontiguousarray(right, np.int32)
        _ck(lib().tn_set_order(self._h, len(l), _ptr(l), _ptr(r),
                               0 if sl is None else len(sl), None if sl is None else _ptr(sl)))

    def tree_from_elimination(self, order):
        o = np.ascontiguousarray(order, np.int32)
        l = np.zeros(self.nleaves - 1, np.int32)
        r = np.zeros(self.nleaves - 1, np.int32)
        _ck(lib().tn_tree_from_elimination(self._h, len(o), _ptr(o), _ptr(l), _ptr(r)))
        return l, r

    def optimize_order(self, method=1, restarts=8, seed=0):
        l = np.zeros(self.nleaves - 1, np.int32)
        r = np.zeros(self.nleaves - 1, np.int32)
        _ck(lib().tn_optimize_order(self._h, method, restarts, seed, _ptr(l), _ptr(r)))
        return l, r

    def reassociate(self, left, right):
        """Equivalent tree with runs of absorption steps re-associated (one
        pass over the large tensor per run instead of one per step)."""
        l = np.ascontiguousarray(left, np.int32)
        r = np.ascontiguousarray(right, np.int32)
        if l.shape != (self.nleaves - 1,) or r.shape != l.shape:
            raise TNError(1, "tree needs nleaves-1 entries per array")
        lo = np.zeros_like(l)
        ro = np.zeros_like(r)
        _ck(lib().tn_reassociate(self._h, _ptr(l), _ptr(r), _ptr(lo), _ptr(ro)))
        return lo, ro

    def choose_slices(self, target_sc_log2, max_vars=16, left=None, right=None):
        """Variables to slice so that every slice's largest intermediate holds
        at most 2**target_sc_log2 entries (greedy; at most max_vars)."""
        out = np.zeros(max(1, max_vars), np.int32)
        n = ctypes.c_int(0)
        lp = rp = None
        if left is not None:
            l = np.ascontiguousarray(left, np.int32)
            r = np.ascontiguousarray(right, np.int32)
            lp, rp = _ptr(l), _ptr(r)
        _ck(lib().tn_choose_slices(self._h, lp, rp, float(target_sc_log2), max_vars, _ptr(out),
                                   ctypes.byref(n)))
        return [int(v) for v in out[:n.value]]

    def tree_stats(self, batch=1, prec="fp64"):
        out = np.zeros(6)
        _ck(lib().tn_tree_stats(self._h, batch, PRECS[prec], _ptr(out)))
        return {"tc": out[0], "sc": out[1], "rw": out[2], "nodes": int(out[3]),
                "flops": out[4], "bytes": out[5]}

    # ------------------------------------------------------------ tasks
    def _evid(self, evid, batch=None):
        if evid is None:
            b = 1 if batch is None else batch
            return np.full((b, self.nvars), -1, np.int32)
        e = np.ascontiguousarray(evid, np.int32)
        return e.reshape(-1, self.nvars)

    def pr(self, evid=None, prec="fp64", budget=0, autotune=False):
        e = self._evid(evid)
        out = np.zeros(e.shape[0])
        o = _opts(prec, budget, None, autotune)
        _ck(lib().tn_pr(self._h, e.shape[0], _ptr(e), ctypes.byref(o), _ptr(out)))
        return out

    def mar(self, evid=None, prec="fp64", budget=0, autotune=False):
        e = self._evid(evid)
        lz = np.zeros(e.shape[0])
        marg = np.zeros((e.shape[0], int(self.card.sum())))
        o = _opts(prec, budget, None, autotune)
        _ck(lib().tn_mar(self._h, e.shape[0], _ptr(e), ctypes.byref(o), _ptr(lz), _ptr(marg)))
        return lz, marg

    def joint_mar(self, query, evid=None, prec="fp64", budget=0):
        """(log p(e), p(Q = q | e) as an array over the query's joint domain,
        axes in the order of `query`)."""
        e = self._evid(evid)
        q = np.ascontiguousarray(query, np.int32)
        shape = [int(self.card[v]) if 0 <= v < self.nvars else 1 for v in q] if q.size else [0]
        out = np.zeros(int(np.prod(shape)))
        lz = ctypes.c_double()
        o = _opts(prec, budget)
        _ck(lib().tn_joint_mar(self._h, _ptr(e[0]), len(q), _ptr(q), ctypes.byref(o),
                               ctypes.byref(lz), _ptr(out)))
        return lz.value, out.reshape(shape)

    def split(self, marg_row):
        out, p = [], 0
        for c in self.card:
            out.append(marg_row[p:p + int(c)])
            p += int(c)
        return out

    def map(self, evid=None, prec="fp64"):
        e = self._evid(evid)
        x = np.zeros(self.nvars, np.int32)
        lp = ctypes.c_double()
        o = _opts(prec)
        _ck(lib().tn_map(self._h, _ptr(e[0]), ctypes.byref(o), _ptr(x), ctypes.byref(lp)))
        return x, lp.value

    def mmap(self, query, evid=None, prec="fp64"):
        e = self._evid(evid)
        q = np.ascontiguousarray(query, np.int32)
        x = np.zeros(len(q), np.int32)
        lp = ctypes.c_double()
        o = _opts(prec)
        _ck(lib().tn_mmap(self._h, _ptr(e[0]), len(q), _ptr(q), ctypes.byref(o), _ptr(x),
                          ctypes.byref(lp)))
        return x, lp.value

    def sample(self, n, seed=0, evid=None, prec="fp64"):
        e = self._evid(evid)
        out = np.zeros((n, self.nvars), np.int8)
        o = _opts(prec)
        _ck(lib().tn_sample(self._h, _ptr(e[0]), seed, n, ctypes.byref(o), _ptr(out)))
        return out

    # ------------------------------------------------- device-pointer forms
    def pr_dev(self, evid, logz, tables=None, tables_are_log=False, prec="fp32", stream=None,
               autotune=False):
        """evid, logz (and tables) are torch CUDA tensors (int32 / float64)."""
        o = _opts(prec, 0, stream, autotune)
        _ck(lib().tn_pr_dev(self._h, int(evid.shape[0]), evid.data_ptr(),
                            None if tables is None else tables.data_ptr(),
                            1 if tables_are_log else 0, ctypes.byref(o), logz.data_ptr()))

    def mar_dev(self, evid, logz, marg, grad=None, tables=None, tables_are_log=False,
                prec="fp32", stream=None, autotune=False):
        o = _opts(prec, 0, stream, autotune)
        _ck(lib().tn_mar_dev(self._h, int(evid.shape[0]), evid.data_ptr(),
                             None if tables is None else tables.data_ptr(),
                             1 if tables_are_log else 0, ctypes.byref(o), logz.data_ptr(),
                             marg.data_ptr(), None if grad is None else grad.data_ptr()))

    def profile(self, task="mar", evid=None, batch=1, prec="tf32", reps=3, budget=0,
                autotune=False):
        """Per kernel class: ms, launches, FLOPs, bytes of one pass (averaged)."""
        e = None if evid is None else np.ascontiguousarray(evid, np.int32).reshape(-1, self.nvars)
        b = batch if e is None else e.shape[0]
        out = np.zeros(4 * len(PROFILE_CLASSES))
        o = _opts(prec, budget, None, autotune)
        _ck(lib().tn_profile(self._h, 0 if task == "pr" else 1, b,
                             None if e is None else _ptr(e), ctypes.byref(o), reps, _ptr(out)))
        res = {}
        for i, name in enumerate(PROFILE_CLASSES):
            ms, n, fl, by = out[4 * i:4 * i + 4]
            if n:
                res[name] = {"ms": ms, "launches": n, "flops": fl, "bytes": by}
        return res

    def profile_steps(self, task="mar", evid=None, batch=1, prec="tf32", cap=100000):
        """Per launch (launch order): class name, ms, FLOPs, bytes."""
        e = None if evid is None else np.ascontiguousarray(evid, np.int32).reshape(-1, self.nvars)
        b = batch if e is None else e.shape[0]
        out = np.zeros(cap * 4)
        n = ctypes.c_int()
        o = _opts(prec)
        _ck(lib().tn_profile_steps(self._h, 0 if task == "pr" else 1, b,
                                   None if e is None else _ptr(e), ctypes.byref(o), cap,
                                   _ptr(out), ctypes.byref(n)))
        k = min(n.value, cap)
        rows = out[:4 * k].reshape(k, 4)
        return [(PROFILE_CLASSES[int(r[0])], r[1], r[2], r[3]) for r in rows]

    def program_stats(self, task="mar", batch=1, prec="fp64", budget=0, autotune=False):
        """tn_program_stats: facts about the program a task call runs."""
        out = np.zeros(8)
        o = _opts(prec, budget, None, autotune)
        _ck(lib().tn_program_stats(self._h, 0 if task == "pr" else 1, batch, ctypes.byref(o),
                                   _ptr(out)))
        keys = ["arena_bytes", "keep_all_bytes", "recomputed", "launches", "lanes",
                "absorb_blocks_per_sm", "tuned", "sub_batch"]
        return {k: (float(v) if k.endswith("bytes") else int(v)) for k, v in zip(keys, out)}

    def last_device_ms(self) -> float:
        return float(lib().tn_last_device_ms(self._h))

    def last_launch_count(self) -> int:
        return int(lib().tn_last_launch_count(self._h))


def solve_multi(models, evids, task="mar", prec="fp64", autotune=False):
    """tn_solve_multi: PR ("pr") or PR + MAR ("mar") of several models in one
    graph launch.  evids[i]: int32 [batch, nvars] (or None: one set, no
    evidence).  Returns [(logz, marg or None) per model]."""
    n = len(models)
    evs = [m._evid(e) for m, e in zip(models, evids)]
    hs = (ctypes.c_void_p * n)(*[m._h for m in models])
    bt = np.array([e.shape[0] for e in evs], np.int32)
    ep = (ctypes.c_void_p * n)(*[e.ctypes.data for e in evs])
    lz = [np.zeros(e.shape[0]) for e in evs]
    mg = [np.zeros((e.shape[0], int(m.card.sum()))) for m, e in zip(models, evs)]
    lp = (ctypes.c_void_p * n)(*[a.ctypes.data for a in lz])
    mp = (ctypes.c_void_p * n)(*[a.ctypes.data for a in mg])
    o = _opts(prec, 0, None, autotune)
    _ck(lib().tn_solve_multi(1 if task == "mar" else 0, n, hs, _ptr(bt), ep, ctypes.byref(o),
                             lp, mp))
    return [(a, b if task == "mar" else None) for a, b in zip(lz, mg)]


def _contract_args(sizes, la, A, lb, B, lc, C, argmax):
    """Checks shared by the pairwise-contraction bindings: A, B and C are
    contiguous CUDA tensors on the current device with one dtype (float64 or
    float32) and the entry counts their labels give; argmax, when given, is a
    contiguous int32 CUDA tensor with one entry per output entry."""
    import torch
    sz = np.ascontiguousarray(sizes, np.int32)
    a = np.ascontiguousarray(la, np.int32)
    b = np.ascontiguousarray(lb, np.int32)
    c = np.ascontiguousarray(lc, np.int32)
    if A.dtype not in (torch.float64, torch.float32):
        raise TNError(1, "A must be float64 or float32")
    dev = torch.device("cuda", torch.cuda.current_device())
    for name, t in (("A", A), ("B", B), ("C", C)):
        if t.dtype != A.dtype:
            raise TNError(1, f"{name} has dtype {t.dtype}, A has {A.dtype}")
        if t.device != dev or not t.is_contiguous():
            raise TNError(1, f"{name} must be a contiguous tensor on {dev}")
    for name, t, l in (("A", A, a), ("B", B, b), ("C", C, c)):
        if np.any(l < 0) or np.any(l >= len(sz)):
            raise TNError(1, f"label of {name} out of range")
        want = int(np.prod([int(sz[v]) for v in l])) if len(l) else 1
        if t.numel() != want:
            raise TNError(1, f"{name} has {t.numel()} entries, its labels give {want}")
    if argmax is not None:
        if (argmax.dtype != torch.int32 or argmax.device != dev or
                not argmax.is_contiguous() or argmax.numel() != C.numel()):
            raise TNError(1, "argmax must be a contiguous int32 tensor with one entry "
                             "per output entry on the current device")
    dtype = 0 if A.dtype == torch.float64 else 1
    return sz, a, b, c, dtype


def contract_dev(sizes, la, A, lb, B, lc, C, semiring=0, argmax=None, prec="fp32",
                 stream=None):
    """One pairwise contraction on torch CUDA tensors (float64 or float32)."""
    sz, a, b, c, dtype = _contract_args(sizes, la, A, lb, B, lc, C, argmax)
    _ck(lib().tn_contract_dev(len(sz), _ptr(sz), len(a), _ptr(a), A.data_ptr(), len(b), _ptr(b),
                              B.data_ptr(), len(c), _ptr(c) if len(c) else None, C.data_ptr(),
                              semiring, dtype, PRECS[prec],
                              None if argmax is None else argmax.data_ptr(), stream))


def contract_dev_noalloc(sizes, la, A, lb, B, lc, C, semiring=0, argmax=None, stream=None):
    """tn_contract_dev_noalloc: the same contraction as contract_dev without
    any device allocation (split-K partials in the library's fixed scratch)."""
    sz, a, b, c, dtype = _contract_args(sizes, la, A, lb, B, lc, C, argmax)
    _ck(lib().tn_contract_dev_noalloc(len(sz), _ptr(sz), len(a), _ptr(a), A.data_ptr(), len(b),
                                      _ptr(b), B.data_ptr(), len(c), _ptr(c) if len(c) else None,
                                      C.data_ptr(), semiring, dtype,
                                      None if argmax is None else argmax.data_ptr(), stream))

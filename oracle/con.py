"""Tensor-network contraction by its definition (test infrastructure only).

``con(Lambda, T, V0)`` of Def. "Tensor Network" / Eq. contraction-definition:
sum, over every assignment of the labels not in V0, of the product of the
tensors sliced at that assignment.  ``tcon`` is the tropical contraction of
Def. "Tropical Tensor Network" (Eq. tropical): max over the assignments of
the sum of the sliced tensors.

Two forms of each: a pure-Python enumeration (``*_naive``, tiny inputs only)
and a vectorised numpy form that materialises the broadcast over the union of
all labels (``*_dense``, moderate inputs).  Labels are hashable names; each
tensor is an ndarray whose axes follow its label tuple.
"""
from __future__ import annotations

import itertools
from typing import Dict, Hashable, List, Sequence, Tuple

import numpy as np


def _sizes(labels: Sequence[Sequence[Hashable]], tensors) -> Dict[Hashable, int]:
    sz: Dict[Hashable, int] = {}
    for lab, t in zip(labels, tensors):
        t = np.asarray(t)
        if t.ndim != len(lab):
            raise ValueError("tensor rank does not match its labels")
        for l, d in zip(lab, t.shape):
            if sz.setdefault(l, d) != d:
                raise ValueError(f"label {l!r} has inconsistent sizes")
    return sz


def con_naive(labels, tensors, out_labels, sizes=None):
    """Eq. contraction-definition by explicit enumeration (FP64)."""
    sz = _sizes(labels, tensors)
    if sizes:
        sz.update(sizes)
    lam = list(dict.fromkeys([l for lab in labels for l in lab] + list(out_labels)))
    out = np.zeros([sz[l] for l in out_labels])
    for assign in itertools.product(*[range(sz[l]) for l in lam]):
        a = dict(zip(lam, assign))
        p = 1.0
        for lab, t in zip(labels, tensors):
            p *= float(np.asarray(t)[tuple(a[l] for l in lab)])
        out[tuple(a[l] for l in out_labels)] += p
    return out


def tcon_naive(labels, tensors, out_labels, sizes=None):
    """Tropical contraction by explicit enumeration: (values, argmax) where
    argmax holds, per output entry, the first maximising assignment of the
    eliminated labels in enumeration order (first eliminated label slowest),
    as a tuple."""
    sz = _sizes(labels, tensors)
    if sizes:
        sz.update(sizes)
    lam = list(dict.fromkeys([l for lab in labels for l in lab]))
    elim = [l for l in lam if l not in out_labels]
    out = np.full([sz[l] for l in out_labels], -np.inf)
    arg = {}
    for oa in itertools.product(*[range(sz[l]) for l in out_labels]):
        best, barg = -np.inf, None
        for ea in itertools.product(*[range(sz[l]) for l in elim]):
            a = dict(zip(out_labels, oa))
            a.update(zip(elim, ea))
            s = 0.0
            for lab, t in zip(labels, tensors):
                s += float(np.asarray(t)[tuple(a[l] for l in lab)])
            if s > best or barg is None:
                if s > best:
                    best, barg = s, ea
                elif barg is None:
                    barg = ea
        out[oa] = best
        arg[oa] = barg
    return out, arg


def _broadcast(labels, tensors, lam, sz, combine):
    acc = None
    for lab, t in zip(labels, tensors):
        t = np.asarray(t, dtype=np.float64)
        # move axes into the order of lam and insert singleton axes
        perm = [lab.index(l) for l in lam if l in lab]
        t = np.transpose(t, perm) if perm else t
        shape = [sz[l] if l in lab else 1 for l in lam]
        t = t.reshape(shape)
        acc = t if acc is None else combine(acc, t)
    return acc


def con_dense(labels, tensors, out_labels, sizes=None):
    """Eq. contraction-definition, vectorised: the product over the full
    union of labels, then a sum over the labels not in the output."""
    sz = _sizes(labels, tensors)
    if sizes:
        sz.update(sizes)
    lam = list(dict.fromkeys([l for lab in labels for l in lab] + list(out_labels)))
    prod = _broadcast(labels, tensors, lam, sz, np.multiply)
    prod = np.broadcast_to(prod, [sz[l] for l in lam])
    axes = tuple(i for i, l in enumerate(lam) if l not in out_labels)
    s = prod.sum(axis=axes) if axes else np.array(prod)
    kept = [l for l in lam if l in out_labels]
    return np.transpose(s, [kept.index(l) for l in out_labels]) if out_labels else s


def tcon_dense(labels, tensors, out_labels, sizes=None):
    """Eq. tropical, vectorised: (values, flat argmax over the eliminated
    labels taken in first-appearance order, first label slowest; the lowest
    flat index wins ties)."""
    sz = _sizes(labels, tensors)
    if sizes:
        sz.update(sizes)
    lam = list(dict.fromkeys([l for lab in labels for l in lab]))
    elim = [l for l in lam if l not in out_labels]
    full = list(out_labels) + elim
    s = _broadcast(labels, tensors, full, sz, np.add)
    s = np.broadcast_to(s, [sz[l] for l in full])
    no = int(np.prod([sz[l] for l in out_labels])) if out_labels else 1
    ne = int(np.prod([sz[l] for l in elim])) if elim else 1
    flat = np.asarray(s).reshape(no, ne)
    arg = np.argmax(flat, axis=1)           # first maximum = lowest index
    val = flat[np.arange(no), arg]
    shape = [sz[l] for l in out_labels]
    return val.reshape(shape), arg.reshape(shape)

"""Host interpreter for the library's tensor-program dumps (test infrastructure).

The CUDA library describes each program it runs (the residual and its
derivative programs) as text: tensor declarations ``T id name role classes``
and ops ``C out blk labels a blk labels b blk labels alpha`` (out += alpha *
einsum(a, b)) or ``A out blk labels a blk labels alpha`` (out += alpha * a,
permuted).  This module executes such a dump with numpy.einsum so the
program's algebra can be compared with the oracle without a GPU.
"""
from __future__ import annotations

import numpy as np
from numpy.lib.stride_tricks import as_strided


def parse(text: str):
    tensors, ops = {}, []
    for line in text.splitlines():
        f = line.split()
        if not f:
            continue
        lab = lambda s: "" if s == "-" else s
        if f[0] == "T":
            tensors[int(f[1])] = (f[2], int(f[3]), lab(f[4]))
        elif f[0] == "C":
            ops.append(("C", int(f[1]), lab(f[2]), lab(f[3]), int(f[4]), lab(f[5]), lab(f[6]),
                        int(f[7]), lab(f[8]), lab(f[9]), float(f[10])))
        elif f[0] == "A":
            ops.append(("A", int(f[1]), lab(f[2]), lab(f[3]), int(f[4]), lab(f[5]), lab(f[6]), float(f[7])))
    return tensors, ops


class Interp:
    def __init__(self, o, v, naux, nvec=1):
        self.o, self.v, self.naux, self.nvec = o, v, naux, nvec
        self.ext = {"o": o, "v": v, "n": o + v, "x": naux, "z": nvec}
        self.arr = {}      # name -> ndarray

    def shape(self, cls):
        return tuple(self.ext[c] for c in cls)

    def view(self, name, cls, blk):
        a = self.arr[name]
        if cls == "":
            return a
        sl = []
        for c, b in zip(cls, blk):
            if c == "n" and b == "o":
                sl.append(slice(0, self.o))
            elif c == "n" and b == "v":
                sl.append(slice(self.o, self.o + self.v))
            else:
                sl.append(slice(None))
        return a[tuple(sl)]

    @staticmethod
    def diag_view(a, labels):
        """View of `a` (labels may repeat) as an array over the distinct labels."""
        uniq = []
        for c in labels:
            if c not in uniq:
                uniq.append(c)
        if len(uniq) == len(labels):
            return a, labels
        shape, strides = [], []
        for c in uniq:
            pos = [k for k, x in enumerate(labels) if x == c]
            shape.append(a.shape[pos[0]])
            strides.append(sum(a.strides[k] for k in pos))
        return as_strided(a, shape=shape, strides=strides), "".join(uniq)

    def run(self, text):
        tensors, ops = parse(text)
        for tid, (name, role, cls) in tensors.items():
            if name not in self.arr:
                self.arr[name] = np.zeros(self.shape(cls))
        for op in ops:
            if op[0] == "C":
                _, to, bo, lo, ta, ba, la, tb, bb, lb, alpha = op
                out = self.view(tensors[to][0], tensors[to][2], bo)
                A = self.view(tensors[ta][0], tensors[ta][2], ba)
                B = self.view(tensors[tb][0], tensors[tb][2], bb)
                tgt, lo_u = self.diag_view(out, lo)
                tgt += alpha * np.einsum(f"{la},{lb}->{lo_u}", A, B)
            else:
                _, to, bo, lo, ta, ba, la, alpha = op
                out = self.view(tensors[to][0], tensors[to][2], bo)
                A = self.view(tensors[ta][0], tensors[ta][2], ba)
                tgt, lo_u = self.diag_view(out, lo)
                tgt += alpha * np.einsum(f"{la}->{lo_u}", A)
        return self

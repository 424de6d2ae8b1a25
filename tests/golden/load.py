"""Readers for the text fixtures in this folder (values printed in the paper)."""

import os

HERE = os.path.dirname(os.path.abspath(__file__))


def _lines(name):
    with open(os.path.join(HERE, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                yield line.split()


def fig1():
    out = {}
    for tok in _lines("fig1_formats.txt"):
        out[tok[0]] = tok[1:]
    return out


def compressed_dofs():
    out = {}
    for tok in _lines("compressed_dofs.txt"):
        out[tok[0]] = [int(t) for t in tok[1:]]
    return out


def structured_patterns():
    rows = []
    for tok in _lines("paper_structured_patterns.txt"):
        src, m, p, d, ndofs, nnz, nca = tok
        rows.append(dict(source=src, m=int(m), p=int(p), d=int(d), n_dofs=int(ndofs),
                         nnz=int(nnz), n_ca=None if nca == "-" else int(nca)))
    return rows


def unstructured_nca():
    return [tuple(int(t) for t in tok) for tok in _lines("paper_unstructured_nca.txt")]

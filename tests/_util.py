"""Test helpers: convert oracle-built H-matrices into block lists for the library's upload."""
import re
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def oracle_blocks(H):
    from oracle import hmatrix as ohm
    out = []
    for b in H.blocks:
        d = {"row0": b.row0, "nrows": b.nrows, "col0": b.col0, "ncols": b.ncols, "kind": b.kind}
        if b.kind == ohm.DENSE:
            d["D"] = b.D
        else:
            d.update(W=b.W, S=b.S, X=b.X)
        out.append(d)
    return out


def header_symbols():
    """Function names declared in include/hlr.h."""
    with open(os.path.join(ROOT, "include", "hlr.h")) as f:
        src = f.read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(hlr_[a-z_0-9]+)\s*\(", src, flags=re.M)
    return sorted(set(names))

"""Dof counting pinned to the sizes printed in Table tab:fom (Section 6.1):
N_V = d (n k + 1)^d and N_E = n^d k^d for the Q_k / Q_{k-1} pair."""
import os

import pytest

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "tab_fom.txt")


def _rows():
    out = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        name, dim, nx, ny, nz, k, nv, ne = line.split()
        out.append((name, int(dim), int(nx), int(ny), int(nz), int(k), int(nv), int(ne)))
    return out


@pytest.mark.parametrize("row", _rows(), ids=lambda r: r[0])
def test_table_fom_sizes(row):
    name, dim, nx, ny, nz, k, nv, ne = row
    o = O.Oracle(dim=dim, nx=nx, ny=ny, nz=nz, order=k, problem=O.UNIFORM)
    assert o.nv == nv
    assert o.ne == ne

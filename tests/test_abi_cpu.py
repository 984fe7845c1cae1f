"""CPU-only checks of the C ABI: the library builds and loads, exports every
symbol that include/lecqmc.h declares, and its host-side lattice builders give
the same bond lists and checkerboard families as the oracle's builders."""
import os
import re

import numpy as np
import pytest

import exact
from oracle import lattices

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lq():
    import paper_2601_08552_gb300 as p

    p.load()
    return p


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "lecqmc.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(lq_[a-z0-9_]+)\s*\(", txt)))


def test_every_declared_symbol_is_exported(lq):
    import ctypes

    lib = lq.load()
    syms = declared_symbols()
    assert len(syms) >= 30
    for s in syms:
        assert hasattr(lib, s), s
        assert isinstance(getattr(lib, s), ctypes._CFuncPtr)


def test_binding_lists_every_export(lq):
    from paper_2601_08552_gb300.lecqmc import EXPORTS

    assert sorted(EXPORTS) == declared_symbols()


@pytest.mark.parametrize("name,args", [("chain", (10,)), ("chain", (9, 1.0, False)), ("square", (4, 6)),
                                       ("square", (3, 5)), ("flatband", (7,)), ("flatband", (5, 0.3, -0.7, 1.1, 0.4)),
                                       ("cross_stitch", (6,))])
def test_builders_match_oracle_builders(lq, name, args):
    ref = getattr(lattices, name)(*args)
    L = getattr(lq.Lattice, name)(*args)
    bi, bj, k, fam = L.bonds()
    assert L.N == ref["N"]
    assert np.array_equal(bi, ref["bi"]) and np.array_equal(bj, ref["bj"])
    assert np.array_equal(k, ref["kb"])
    fam_ref, G = exact.families(ref)
    assert np.array_equal(fam, fam_ref) and L.n_families == G


def test_lattice_argument_errors(lq):
    with pytest.raises(lq.LqError):
        lq.Lattice.from_bonds(4, [0, 1], [1, 4], [-1.0, -1.0])
    with pytest.raises(lq.LqError):
        lq.Lattice.from_bonds(4, [0], [0], [-1.0])
    with pytest.raises(lq.LqError):
        lq.Lattice.chain(0)

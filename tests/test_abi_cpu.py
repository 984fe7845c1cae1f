"""CPU-only checks of the C ABI: the library builds and loads, exports every
symbol that include/lecqmc.h declares, the binding's ctypes structs have the
header's fields, sizes and offsets, and its host-side lattice builders give
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


def test_struct_layouts_match_header(tmp_path):
    """The binding's ctypes mirrors of the header's structs have the C sizes
    and field offsets (a small C program compiled against include/lecqmc.h
    prints them)."""
    import ctypes
    import shutil
    import subprocess

    from paper_2601_08552_gb300 import lecqmc as b

    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not available")
    mirrors = {"lq_params": b.Params, "lq_request": b.Request, "lq_result": b.Result,
               "lq_server_info": b.ServerStats, "lq_allocator": b.Allocator}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "lecqmc.h"', "int main(void) {"]
    for cname, py in mirrors.items():
        lines.append('  printf("%s sizeof %%zu\\n", sizeof(%s));' % (cname, cname))
        for fname, _ in py._fields_:
            lines.append('  printf("%s %s %%zu\\n", offsetof(%s, %s));' % (cname, fname, cname, fname))
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.check_call([gcc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    out = subprocess.check_output([str(exe)]).decode().split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for cname, py in mirrors.items():
        assert got[(cname, "sizeof")] == ctypes.sizeof(py), cname
        for fname, _ in py._fields_:
            assert got[(cname, fname)] == getattr(py, fname).offset, (cname, fname)
        # and every field the header declares, in order (padding can hide a missing last field)
        assert header_fields(cname) == [f for f, _ in py._fields_], cname


def header_fields(cname):
    """Field names of `typedef struct { ... } cname;` in include/lecqmc.h, in order."""
    txt = open(os.path.join(ROOT, "include", "lecqmc.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    m = re.search(r"typedef struct \{([^{}]*)\}\s*" + cname + r"\s*;", txt)
    assert m, cname
    names = []
    for decl in m.group(1).split(";"):
        decl = decl.strip()
        if not decl:
            continue
        fp = re.search(r"\(\s*\*\s*(\w+)\s*\)", decl)   # function pointer: ret (*name)(args)
        if fp:
            names.append(fp.group(1))
            continue
        first, *rest = decl.split(",")
        names.append(re.search(r"(\w+)\s*(\[[^\]]*\])?\s*$", first).group(1))
        names += [re.search(r"(\w+)\s*(\[[^\]]*\])?\s*$", r).group(1) for r in rest]
    return names


def test_noalloc_binding_rejects_bad_buffers_before_the_call(lq):
    """lq_sweep_noalloc receives raw device pointers: the binding checks each
    buffer's dtype, contiguity, element count and device first and raises
    ValueError, so a wrong buffer never reaches the kernels."""
    torch = pytest.importorskip("torch")
    from paper_2601_08552_gb300.lecqmc import sweep_noalloc

    lat = lq.Lattice.chain(8)
    params = dict(U=4.0, beta=1.0, dtau=0.1, n_up=2, n_dn=3, n_stab=4, precision=0, seed=1)
    L = 10
    good_f = torch.ones(L * 8, dtype=torch.int8)
    good_o = torch.arange(5, dtype=torch.int32)
    cases = [
        (torch.ones(L * 8, dtype=torch.int32), good_o, None, "dtype"),
        (torch.ones(L * 8 - 1, dtype=torch.int8), good_o, None, "elements"),
        (torch.ones((8, L), dtype=torch.int8).t(), good_o, None, "contiguous"),
        (good_f, torch.arange(4, dtype=torch.int32), None, "elements"),
        (good_f, torch.arange(5, dtype=torch.int64), None, "dtype"),
        (good_f, good_o, torch.zeros(3 * 9, dtype=torch.float32), "dtype"),
        (good_f, good_o, torch.zeros(2 * 9, dtype=torch.float64), "elements"),
        (good_f, good_o, None, "CUDA"),
        (good_f.numpy(), good_o, None, "torch tensor"),
    ]
    for f, o, r, what in cases:
        with pytest.raises(ValueError, match=what):
            sweep_noalloc(lat, params, 0, 0, f, o, 3, r)

"""Lattice builders for the oracle (test infrastructure only).

Each builder returns the hopping matrix K as an ordered bond list
``(bi, bj, kij)`` plus the onsite term ``eps`` and a two-valued sublattice
label per site.  The bond order fixes the checkerboard families (each bond
goes to the lowest family where neither site is used yet), so it is part of
the definition of e^{-dtau K}:

* ``chain``: bonds (i, i+1), even i then odd i; the periodic wrap (N-1, 0)
  falls into the odd group.  Hubbard hopping K_ij = -t (Eq. 5).
* ``square``: site x + Lx*y; x-bonds with even x, x-bonds with odd x, y-bonds
  with even y, y-bonds with odd y (each group row by row).  K_ij = -t (Eq. 5).
* ``flatband``: the one-dimensional BCL model after integrating out the B
  sublattice, H_eff(k) = S(k) S(k)^dagger with S1 = t1 + t2 e^{-ik},
  S2 = t3 + t4 e^{-ik} (SM Sec. III).  Real-space reading (Bloch convention
  c_k = N^{-1/2} sum_R e^{-ikR} c_R): onsite t1^2+t2^2 on A1 and t3^2+t4^2 on
  A2; A1_R-A1_{R+1}: t1 t2; A2_R-A2_{R+1}: t3 t4; A1_R-A2_R: t1 t3 + t2 t4;
  A1_R-A2_{R+1}: t1 t4; A1_R-A2_{R-1}: t2 t3.  Sites A1_R = 2R, A2_R = 2R+1.
* ``cross_stitch``: two legs a_R = 2R, b_R = 2R+1 with rung -t_intra,
  legs -t_leg and crossings a_R-b_{R+1}, b_R-a_{R+1} of -t_cross.
"""
import numpy as np


def _pack(N, bonds, eps=None, sub=None):
    bi = np.array([b[0] for b in bonds], dtype=np.int32)
    bj = np.array([b[1] for b in bonds], dtype=np.int32)
    kb = np.array([b[2] for b in bonds], dtype=np.float64)
    eps = np.zeros(N) if eps is None else np.asarray(eps, dtype=np.float64)
    sub = (np.arange(N) % 2).astype(np.int32) if sub is None else np.asarray(sub, dtype=np.int32)
    return dict(N=N, bi=bi, bj=bj, kb=kb, eps=eps, sub=sub)


def chain(N, t=1.0, periodic=True):
    bonds = []
    for parity in (0, 1):
        for i in range(parity, N - 1, 2):
            bonds.append((i, i + 1, -t))
        if periodic and N > 2 and (N - 1) % 2 == parity:
            bonds.append((N - 1, 0, -t))
    return _pack(N, bonds)


def square(Lx, Ly, t=1.0, periodic=True):
    N = Lx * Ly
    idx = lambda x, y: x + Lx * y  # noqa: E731
    bonds = []
    for parity in (0, 1):
        for y in range(Ly):
            for x in range(parity, Lx, 2):
                if x + 1 < Lx:
                    bonds.append((idx(x, y), idx(x + 1, y), -t))
                elif periodic and Lx > 2:
                    bonds.append((idx(x, y), idx(0, y), -t))
    for parity in (0, 1):
        for y in range(parity, Ly, 2):
            for x in range(Lx):
                if y + 1 < Ly:
                    bonds.append((idx(x, y), idx(x, y + 1), -t))
                elif periodic and Ly > 2:
                    bonds.append((idx(x, y), idx(x, 0), -t))
    sub = np.array([(x + y) % 2 for y in range(Ly) for x in range(Lx)], dtype=np.int32)
    return _pack(N, bonds, sub=sub)


def flatband(n_cells, t1=-0.2, t2=1.0, t3=1.0, t4=-0.2, periodic=True):
    N = 2 * n_cells
    A1 = lambda R: 2 * (R % n_cells)  # noqa: E731
    A2 = lambda R: 2 * (R % n_cells) + 1  # noqa: E731
    bonds = []
    nR = n_cells if periodic and n_cells > 2 else n_cells - 1
    for parity in (0, 1):
        for R in range(parity, nR, 2):
            bonds.append((A1(R), A1(R + 1), t1 * t2))
    for parity in (0, 1):
        for R in range(parity, nR, 2):
            bonds.append((A2(R), A2(R + 1), t3 * t4))
    for R in range(n_cells):
        bonds.append((A1(R), A2(R), t1 * t3 + t2 * t4))
    for R in range(n_cells):
        if R + 1 < n_cells or (periodic and n_cells > 2):
            bonds.append((A1(R), A2(R + 1), t1 * t4))
    for R in range(n_cells):
        if R - 1 >= 0 or (periodic and n_cells > 2):
            bonds.append((A1(R), A2(R - 1), t2 * t3))
    eps = np.array([t1 * t1 + t2 * t2, t3 * t3 + t4 * t4] * n_cells)
    bonds = [b for b in bonds if b[2] != 0.0]
    return _pack(N, bonds, eps=eps)


def cross_stitch(n_cells, t_intra=1.0, t_leg=1.0, t_cross=1.0, periodic=True):
    N = 2 * n_cells
    a = lambda R: 2 * (R % n_cells)  # noqa: E731
    b = lambda R: 2 * (R % n_cells) + 1  # noqa: E731
    nR = n_cells if periodic and n_cells > 2 else n_cells - 1
    bonds = []
    for R in range(n_cells):
        bonds.append((a(R), b(R), -t_intra))
    for leg in (a, b):
        for parity in (0, 1):
            for R in range(parity, nR, 2):
                bonds.append((leg(R), leg(R + 1), -t_leg))
    for parity in (0, 1):
        for R in range(parity, nR, 2):
            bonds.append((a(R), b(R + 1), -t_cross))
            bonds.append((b(R), a(R + 1), -t_cross))
    return _pack(N, bonds)


def dense_K(lat):
    """Dense hopping matrix K (N x N) of a bond list."""
    N = lat["N"]
    K = np.diag(lat["eps"]).astype(np.float64)
    for i, j, k in zip(lat["bi"], lat["bj"], lat["kb"]):
        K[i, j] += k
        K[j, i] += k
    return K

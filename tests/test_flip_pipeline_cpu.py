"""Host-side checks of the pipelined field-flip loop's design (no GPU).

The paired flip loop (up to 32 particles per spin) runs the serial chain of a
window of K = 4 sites on one leader warp while the other warps run one window
behind it.  Two facts make that correct, and both are checked here on the CPU:

1. The block recurrence.  The leader forms the next window's Green's block
   from three K x K blocks taken against the T before the current window
   (A1 = Z L~_{w+1}^T, A2 = X_w L~_{w+1}^T, B = Z L~_{w+1}^T, Z = R~_{w+1} T_w)
   and the current window's c-scaled factors, instead of recomputing it from
   the updated T.  A numpy model of both routes must agree to round-off on
   every window, including a short last window and rejected flips.
2. The barrier protocol.  The leader arrives at P (a window's factors stored)
   and waits at Q (the next blocks stored); the workers wait at P, meet among
   themselves at W, and arrive at Q; P and Q alternate between two ids by
   window parity.  A model of each warp's sequence of barrier operations, run
   under many orders of the warps, must never deadlock and never see more
   arrivals at a barrier than its count.
"""
import random

import numpy as np
import pytest

K = 4


def _window_chain(G, t0, kw, flip, delta):
    """The serial chain of one window on its K x K block G (modified in
    place): c_t for accepted sites, G[u][v] -= c G[u][t] G[t][v] (u, v > t)."""
    c = np.zeros(K)
    for t in range(kw):
        if flip[t0 + t]:
            c[t] = 1.0 / (1.0 / delta[t0 + t] + G[t, t])
            for u in range(t + 1, K):
                for v in range(t + 1, K):
                    G[u, v] -= c[t] * G[u, t] * G[t, v]
    return c


def _cg(G, c, kw):
    """c-scaled factors: CG[j][t] = c_t G[j][t] (j > t), CG[t][j] = c_t G[t][j]."""
    CG = np.zeros((K, K))
    for u in range(kw):
        for v in range(kw):
            if u > v:
                CG[u, v] = c[v] * G[u, v]
            elif u < v:
                CG[u, v] = c[u] * G[u, v]
    return CG


def _recur_xy(X, Y, CG, c, kw):
    X, Y = X.copy(), Y.copy()
    for t in range(kw - 1):
        for j in range(t + 1, kw):
            X[j] -= CG[j, t] * X[t]
            Y[j] -= CG[t, j] * Y[t]
    return X, c[:kw, None] * Y


def _unpipelined(T0, r, l, flip, delta):
    """Every window's block recomputed as X L~^T from the updated T."""
    T, blocks, n = T0.copy(), [], len(r)
    for t0 in range(0, n, K):
        kw = min(K, n - t0)
        X = r[t0:t0 + kw] @ T
        Y = (T @ l[t0:t0 + kw].T).T
        G = np.zeros((K, K))
        G[:kw, :kw] = X @ l[t0:t0 + kw].T
        blocks.append(G[:kw, :kw].copy())
        c = _window_chain(G, t0, kw, flip, delta)
        Xp, Ypp = _recur_xy(X, Y, _cg(G, c, kw), c, kw)
        T = T - Ypp.T @ Xp
    return blocks, T


def _pipelined(T0, r, l, flip, delta, scale_a1=True):
    """The leader's route: the next block from A1, A2, B and this window's
    factors; the workers' route: recurrences, T update and products one
    window behind.  scale_a1=False drops the c_t of the final sum (a planted
    mistake)."""
    T, blocks, n = T0.copy(), [], len(r)
    nw = (n + K - 1) // K

    def three_blocks(t0, kw, kz, X, T):
        Z = r[t0 + K:t0 + K + kz] @ T
        A1, A2, B = np.zeros((K, K)), np.zeros((K, K)), np.zeros((K, K))
        A1[:kz, :kw] = Z @ l[t0:t0 + kw].T
        A2[:kw, :kz] = X @ l[t0 + K:t0 + K + kz].T
        B[:kz, :kz] = Z @ l[t0 + K:t0 + K + kz].T
        return A1, A2, B

    kw0 = min(K, n)
    X = r[:kw0] @ T
    Y = (T @ l[:kw0].T).T
    Gn = np.zeros((K, K))
    Gn[:kw0, :kw0] = X @ l[:kw0].T
    blk = three_blocks(0, kw0, min(K, n - K) if nw > 1 else 0, X, T)
    for w in range(nw):
        t0, kw = w * K, min(K, n - w * K)
        G = Gn.copy()
        blocks.append(G[:kw, :kw].copy())
        c = _window_chain(G, t0, kw, flip, delta)
        CG = _cg(G, c, kw)
        if w + 1 < nw:  # leader: the next block
            A1, A2, B = [b.copy() for b in blk]
            for t in range(kw - 1):
                a1t, a2t = A1[:, t].copy(), A2[t, :].copy()
                for u in range(K):
                    for v in range(K):
                        if v > t:
                            A1[u, v] -= CG[t, v] * a1t[u]
                        if u > t:
                            A2[u, v] -= CG[u, t] * a2t[v]
            if scale_a1:
                A1 = A1 * c[None, :]
            Gn = B - A1[:, :kw] @ A2[:kw, :]
        # workers: window w's recurrences and T update, then window w + 1's products and blocks
        Xp, Ypp = _recur_xy(X, Y, CG, c, kw)
        T = T - Ypp.T @ Xp
        if w + 1 < nw:
            t1 = t0 + K
            kw1 = min(K, n - t1)
            X = r[t1:t1 + kw1] @ T
            Y = (T @ l[t1:t1 + kw1].T).T
            blk = three_blocks(t1, kw1, min(K, n - t1 - K) if w + 2 < nw else 0, X, T)
    return blocks, T


@pytest.mark.parametrize("m,n,p_flip,seed", [(8, 23, 0.7, 1), (16, 40, 1.0, 2), (4, 9, 0.3, 3), (8, 4, 0.9, 4),
                                             (2, 17, 0.5, 5)])
def test_block_recurrence_matches_unpipelined_update(m, n, p_flip, seed):
    rng = np.random.default_rng(seed)
    T0 = rng.normal(size=(m, m))
    r = rng.normal(size=(n, m))
    l = rng.normal(size=(n, m))
    delta = rng.choice([-0.33, 0.49], n) * rng.uniform(0.5, 1.5, n)
    flip = rng.random(n) < p_flip
    b0, T_a = _unpipelined(T0, r, l, flip, delta)
    b1, T_b = _pipelined(T0, r, l, flip, delta)
    assert len(b0) == len(b1) == (n + K - 1) // K
    scale = max(np.abs(b).max() for b in b0)
    assert max(np.abs(x - y).max() for x, y in zip(b0, b1)) < 1e-12 * scale
    assert np.abs(T_a - T_b).max() < 1e-12 * np.abs(T_a).max()


def test_block_recurrence_detects_a_dropped_factor():
    """The comparison above is sharp: the same model without the c_t of the
    final sum G_{w+1} = B - sum_t c_t A1[u][t] A2[t][v] fails it."""
    rng = np.random.default_rng(7)
    m, n = 8, 12
    T0, r, l = rng.normal(size=(m, m)), rng.normal(size=(n, m)), rng.normal(size=(n, m))
    delta, flip = np.full(n, 0.4), np.ones(n, dtype=bool)
    b0, _ = _unpipelined(T0, r, l, flip, delta)
    b1, _ = _pipelined(T0, r, l, flip, delta, scale_a1=False)
    assert max(np.abs(x - y).max() for x, y in zip(b0, b1)) > 1e-3 * max(np.abs(b).max() for b in b0)


# ---- barrier protocol -------------------------------------------------------
P0, Q0, W = 1, 3, 5  # ids: P = 1, 2 and Q = 3, 4 by window parity, W = 5


def _leader_ops(nw, ids=2):
    ops = []
    for w in range(nw):
        ops.append(("arrive", P0 + (w % ids)))
        if w + 1 < nw and w >= 1:  # window 1's blocks come with window 0's
            ops.append(("sync", Q0 + ((w + 1) % ids)))
    return ops


def _worker_ops(nw, ids=2):
    ops = []
    for w in range(1, nw):
        ops.append(("sync", P0 + ((w - 1) % ids)))  # factors of window w - 1
        ops.append(("sync", W))                     # recurrences done, then the T update
        ops.append(("sync", W))                     # T updated, then the products
        if w + 1 < nw:
            ops.append(("sync", W))                 # products done, then the blocks
            ops.append(("arrive", Q0 + ((w + 1) % ids)))
    ops.append(("sync", P0 + ((nw - 1) % ids)))
    ops.append(("sync", W))
    return ops


def _run(nw, n_workers, pick, ids=2):
    nthr = 32 * (n_workers + 1)
    need = {P0: nthr, P0 + 1: nthr, Q0: nthr, Q0 + 1: nthr, W: 32 * n_workers}
    warps = [_leader_ops(nw, ids)] + [_worker_ops(nw, ids) for _ in range(n_workers)]
    pc = [0] * len(warps)
    wait = [None] * len(warps)
    count = {b: 0 for b in need}
    gen = {b: 0 for b in need}
    while True:
        ready = [i for i in range(len(warps)) if pc[i] < len(warps[i]) and wait[i] is None]
        if not ready:
            assert all(pc[i] == len(warps[i]) for i in range(len(warps))), "deadlock"
            assert all(v == 0 for v in count.values())
            return
        i = pick(ready)
        op, b = warps[i][pc[i]]
        count[b] += 32
        assert count[b] <= need[b], "more arrivals at barrier %d than its count" % b
        pc[i] += 1
        if op == "sync":
            wait[i] = (b, gen[b])
        if count[b] == need[b]:
            count[b] = 0
            for j in range(len(warps)):
                if wait[j] == (b, gen[b]):
                    wait[j] = None
            gen[b] += 1


@pytest.mark.parametrize("n_workers", [3, 7])
def test_barrier_protocol_never_deadlocks_or_overfills(n_workers):
    for nw in range(1, 14):
        _run(nw, n_workers, lambda ready: ready[0])    # the leader whenever it can move
        _run(nw, n_workers, lambda ready: ready[-1])   # the workers first
        for seed in range(40):
            rng = random.Random(1000 * nw + seed)
            _run(nw, n_workers, lambda ready: rng.choice(ready))


def test_barrier_model_catches_a_single_id():
    """With one id each for P and Q instead of two, a leader that runs ahead
    arrives twice at P before every worker has passed it; the model fails."""
    with pytest.raises(AssertionError):
        _run(3, 3, lambda ready: ready[0], ids=1)

"""Exact Markov-chain enumeration of RSOS growth on tiny periodic lattices.

Test infrastructure only (see ``oracle/__init__.py``).  Independent of the
CUDA path.

The state of an L x L surface under the RSOS rule (Eq. 6) is its height
configuration modulo a global shift; we normalise every configuration so that
its minimum height is zero.  Starting from the flat surface (section II), the
reachable configurations are enumerated by breadth-first search over single
deposition attempts.

Two dynamics are built on the same attempt maps A_x ("attempt a deposit at
site x; keep the configuration if Eq. 6 rejects it"):

* random-sequential (RS): one attempt at a uniformly chosen site, L^2 attempts
  per Monte-Carlo step;
* double tiling (DT, section II): per sweep a uniformly random tiling origin
  (ox, oy) in [0,Tx) x [0,Ty) and an order of the four sub-tile sets (uniform
  over the 24 permutations, or fixed); within a phase every active sub-tile of
  a = (Tx/2)(Ty/2) sites receives 2a selections, each of a uniformly chosen
  site of the sub-tile, acted on with probability 1/2 (the random half mask).
  One selection is the kernel  1/2 I + 1/(2a) sum_{k in sub-tile} A_k.
* DT on a (+1) tiling (section III.C): tiles T or T + 1 wide (the first
  L mod T of the L div T tiles of an axis are the wider ones), each halved
  into floor(w/2) and w - floor(w/2) sites; the origin is uniform over one
  period of the pattern (T if T divides L, else L) and a sub-tile of a sites
  receives 2a selections with the kernel above for its own a.

From the stationary distribution pi of each chain we get the growth velocity
v (mean height gain per site per sweep / Monte-Carlo step) and the stationary
squared width E_pi[W^2] of Eq. 2.  Power iteration runs on probability
vectors; nothing here uses the Philox stream.
"""
from __future__ import annotations

import collections
import itertools

import numpy as np


def _neighbours(L: int):
    nb = []
    for y in range(L):
        for x in range(L):
            nb.append(((x + 1) % L + y * L, (x - 1) % L + y * L,
                       x + ((y - 1) % L) * L, x + ((y + 1) % L) * L))
    return nb


def enumerate_states(L: int, N: int):
    """All configurations reachable from the flat start, normalised to min 0.
    Returns (states as an int array [n_states, L*L], index dict)."""
    nb = _neighbours(L)
    start = tuple([0] * (L * L))
    index = {start: 0}
    order = [start]
    queue = collections.deque([start])
    while queue:
        s = queue.popleft()
        for x in range(L * L):
            if all(s[x] + 1 - s[n] <= N for n in nb[x]):
                h = list(s)
                h[x] += 1
                m = min(h)
                t = tuple(v - m for v in h)
                if t not in index:
                    index[t] = len(order)
                    order.append(t)
                    queue.append(t)
    return np.array(order, dtype=np.int64), index


def attempt_maps(L: int, N: int, states: np.ndarray, index: dict):
    """For every site x: target[x][s] (state after an attempt at x) and
    accepted[x][s] (1 if Eq. 6 accepts the deposit)."""
    nb = _neighbours(L)
    n = len(states)
    target = np.zeros((L * L, n), dtype=np.int64)
    accepted = np.zeros((L * L, n), dtype=np.float64)
    for si in range(n):
        s = states[si]
        for x in range(L * L):
            if all(s[x] + 1 - s[m] <= N for m in nb[x]):
                h = s.copy()
                h[x] += 1
                h -= h.min()
                target[x, si] = index[tuple(int(v) for v in h)]
                accepted[x, si] = 1.0
            else:
                target[x, si] = si
    return target, accepted


def width2_of_states(states: np.ndarray) -> np.ndarray:
    """Eq. 2 for every state (shift invariant)."""
    h = states.astype(np.float64)
    return (h * h).mean(axis=1) - h.mean(axis=1) ** 2


def _push(d: np.ndarray, target_x: np.ndarray) -> np.ndarray:
    """Distribution after applying the deterministic attempt map of one site."""
    out = np.zeros_like(d)
    np.add.at(out, target_x, d)
    return out


def _power(step, d0: np.ndarray, tol: float, max_iter: int) -> np.ndarray:
    d = d0
    for _ in range(max_iter):
        nd = step(d)
        if np.abs(nd - d).sum() < tol:
            return nd
        d = nd
    raise RuntimeError("power iteration did not converge")


def rs_chain(L: int, N: int, tol: float = 1e-14, max_iter: int = 200000):
    """Stationary RS growth velocity (per site per Monte-Carlo step) and E[W^2]."""
    states, index = enumerate_states(L, N)
    target, accepted = attempt_maps(L, N, states, index)
    area = L * L

    def step(d):
        out = np.zeros_like(d)
        for x in range(area):
            np.add.at(out, target[x], d / area)
        return out

    d0 = np.full(len(states), 1.0 / len(states))
    pi = _power(step, d0, tol, max_iter)
    n_acc = accepted.sum(axis=0)          # accepting sites per state
    velocity = float(pi @ n_acc) / area   # L^2 attempts per MCS, per site
    return {"L": L, "N": N, "n_states": len(states), "velocity": velocity,
            "w2": float(pi @ width2_of_states(states))}


def _dt_sequences(L: int, Tx: int, Ty: int, phase_order: int):
    """All (origin, permutation) pairs, each with equal weight, as lists of the
    sub-tiles (site lists) active in phases 0..3."""
    sx, sy = Tx // 2, Ty // 2
    perms = [tuple(range(4))] if phase_order == 1 else list(itertools.permutations(range(4)))
    seqs = []
    for oy in range(Ty):
        for ox in range(Tx):
            for perm in perms:
                phases = []
                for q in perm:
                    qx, qy = q & 1, q >> 1
                    subtiles = []
                    for ty in range(L // Ty):
                        for tx in range(L // Tx):
                            sites = []
                            for ky in range(sy):
                                for kx in range(sx):
                                    x = (ox + tx * Tx + qx * sx + kx) % L
                                    y = (oy + ty * Ty + qy * sy + ky) % L
                                    sites.append(y * L + x)
                            subtiles.append(sites)
                    phases.append(subtiles)
                seqs.append(phases)
    return seqs


def dt_chain(L: int, N: int, Tx: int, Ty: int, phase_order: int = 0,
             tol: float = 1e-14, max_iter: int = 100000):
    """Stationary DT growth velocity (per site per sweep) and E[W^2]."""
    assert Tx % 2 == 0 and Ty % 2 == 0 and L % Tx == 0 and L % Ty == 0
    states, index = enumerate_states(L, N)
    target, accepted = attempt_maps(L, N, states, index)
    seqs = _dt_sequences(L, Tx, Ty, phase_order)
    a = (Tx // 2) * (Ty // 2)

    def run(d, with_reward):
        total = np.zeros_like(d)
        reward = 0.0
        for phases in seqs:
            e = d.copy()
            for subtiles in phases:
                for sites in subtiles:
                    for _ in range(2 * a):
                        nxt = 0.5 * e
                        for k in sites:
                            if with_reward:
                                reward += float(e @ accepted[k]) / (2 * a) / len(seqs)
                            nxt += _push(e, target[k]) / (2 * a)
                        e = nxt
            total += e / len(seqs)
        return total, reward

    d0 = np.full(len(states), 1.0 / len(states))
    pi = _power(lambda d: run(d, False)[0], d0, tol, max_iter)
    _, reward = run(pi, True)
    return {"L": L, "N": N, "Tx": Tx, "Ty": Ty, "phase_order": phase_order,
            "n_states": len(states), "velocity": reward / (L * L),
            "w2": float(pi @ width2_of_states(states))}


def _halves(L: int, T: int):
    """Per tile of one axis of a (+1) tiling: the two halves as (start,
    width) in pattern coordinates."""
    n, r = L // T, L % T
    assert 1 <= n and r <= n
    out, x = [], 0
    for c in range(n):
        w = T + 1 if c < r else T
        out.append(((x, w // 2), (x + w // 2, w - w // 2)))
        x += w
    assert x == L
    return out


def _dt_sequences_general(L: int, Tx: int, Ty: int, phase_order: int):
    hx, hy = _halves(L, Tx), _halves(L, Ty)
    px = Tx if L % Tx == 0 else L
    py = Ty if L % Ty == 0 else L
    perms = [tuple(range(4))] if phase_order == 1 else list(itertools.permutations(range(4)))
    seqs = []
    for oy in range(py):
        for ox in range(px):
            for perm in perms:
                phases = []
                for q in perm:
                    qx, qy = q & 1, q >> 1
                    subtiles = []
                    for (ys, yw) in (h[qy] for h in hy):
                        for (xs, xw) in (h[qx] for h in hx):
                            subtiles.append([((oy + ys + j) % L) * L + (ox + xs + i) % L
                                             for j in range(yw) for i in range(xw)])
                    phases.append(subtiles)
                seqs.append(phases)
    return seqs


def dt_chain_general(L: int, N: int, Tx: int, Ty: int, phase_order: int = 0,
                     tol: float = 1e-14, max_iter: int = 100000):
    """Stationary DT growth velocity (per site per sweep) and E[W^2] on a (+1)
    tiling (section III.C)."""
    states, index = enumerate_states(L, N)
    target, accepted = attempt_maps(L, N, states, index)
    seqs = _dt_sequences_general(L, Tx, Ty, phase_order)

    def run(d, with_reward):
        total = np.zeros_like(d)
        reward = 0.0
        for phases in seqs:
            e = d.copy()
            for subtiles in phases:
                for sites in subtiles:
                    a = len(sites)
                    for _ in range(2 * a):
                        nxt = 0.5 * e
                        for k in sites:
                            if with_reward:
                                reward += float(e @ accepted[k]) / (2 * a) / len(seqs)
                            nxt += _push(e, target[k]) / (2 * a)
                        e = nxt
            total += e / len(seqs)
        return total, reward

    d0 = np.full(len(states), 1.0 / len(states))
    pi = _power(lambda d: run(d, False)[0], d0, tol, max_iter)
    _, reward = run(pi, True)
    return {"L": L, "N": N, "Tx": Tx, "Ty": Ty, "phase_order": phase_order, "tiling": 1,
            "n_states": len(states), "velocity": reward / (L * L),
            "w2": float(pi @ width2_of_states(states))}

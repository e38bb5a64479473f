"""Brute-force second quantisation on tiny systems (test helper, pure Python).

H = E_core + sum_{pq,s} h_pq a+_{ps} a_{qs}
      + 1/2 sum_{pqrs,s,t} (pq|rs) a+_{ps} a+_{rt} a_{st} a_{qs}
is applied term by term to each determinant, with the fermionic sign of
every creation/annihilation counted on the ordered product of creation
operators alpha_0 .. alpha_{N-1}, beta_0 .. beta_{N-1} acting on |0>.
No Slater-Condon rule is used, so the result pins the oracle's fast path.
"""
import itertools

import numpy as np


def _pos(p, spin, norb):
    return p + spin * norb


def _apply(state, pos, create):
    """state: int bit string over 2N spin orbitals.  Returns (sign, new) or None."""
    occ = (state >> pos) & 1
    if create == occ:
        return None
    sign = -1 if bin(state & ((1 << pos) - 1)).count("1") % 2 else 1
    return sign, state ^ (1 << pos)


def _apply_string(state, ops):
    """ops applied right to left: list of (pos, create) in written order."""
    sign = 1
    for pos, create in reversed(ops):
        r = _apply(state, pos, create)
        if r is None:
            return None
        s, state = r
        sign *= s
    return sign, state


def eri_full(norb, eri_packed):
    def pi(i, j):
        return i * (i + 1) // 2 + j if i >= j else j * (j + 1) // 2 + i
    g = np.zeros((norb,) * 4)
    for p, q, r, s in itertools.product(range(norb), repeat=4):
        g[p, q, r, s] = eri_packed[pi(pi(p, q), pi(r, s))]
    return g


def hamiltonian(norb, h, g, ecore, dets):
    """Dense <D_j|H|D_i> over ``dets`` = [(alpha, beta)] (absolute energies)."""
    index = {}
    states = []
    for k, (a, b) in enumerate(dets):
        st = a | (b << norb)
        index[st] = k
        states.append(st)
    n = len(dets)
    H = np.zeros((n, n))
    one = [(p, q, h[p, q]) for p in range(norb) for q in range(norb) if h[p, q] != 0.0]
    two = [(p, q, r, s, g[p, q, r, s]) for p, q, r, s in itertools.product(range(norb), repeat=4)
           if g[p, q, r, s] != 0.0]
    for i, st in enumerate(states):
        H[i, i] += ecore
        for p, q, v in one:
            for sp in (0, 1):
                res = _apply_string(st, [(_pos(p, sp, norb), 1), (_pos(q, sp, norb), 0)])
                if res is not None and res[1] in index:
                    H[index[res[1]], i] += v * res[0]
        for p, q, r, s, v in two:
            for s1 in (0, 1):
                for s2 in (0, 1):
                    ops = [(_pos(p, s1, norb), 1), (_pos(r, s2, norb), 1),
                           (_pos(s, s2, norb), 0), (_pos(q, s1, norb), 0)]
                    res = _apply_string(st, ops)
                    if res is not None and res[1] in index:
                        H[index[res[1]], i] += 0.5 * v * res[0]
    return H

"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and bench.py.

This module holds no FCIQMC arithmetic: it only draws integrals and lattice
descriptions from fixed seeds, in a fixed draw order, so that the oracle and
the GPU library receive bit-identical inputs.  The paper's own workloads
(FCIDUMP files for FeMoco, Cr2, butadiene, ...) are not available; these
stand in for their shape (an 8-fold symmetric ERI tensor, tens of orbitals,
Hubbard lattices at half filling).
"""
from __future__ import annotations


import numpy as np


def pair_index(i, j):
    i, j = max(i, j), min(i, j)
    return i * (i + 1) // 2 + j


def synthetic_abinitio(norb: int, n_chol: int, seed: int):
    """Synthetic ab initio integrals (chemist notation, FCIDUMP packing).

    h_pq: symmetric, diagonal linearly spaced in [-2, 2] Eh, off-diagonal
    N(0, 0.05^2).  (pq|rs) = sum_K L^K_pq L^K_rs with symmetric L^K whose
    upper-triangle entries are N(0, 0.1^2), plus 0.5 on each L^K_pp, which
    gives 8-fold symmetry and a positive semi-definite ERI matrix.  Drawn by
    numpy.random.Generator(Philox(seed)) in the order h, then L^1..L^K.
    Returns (h [norb, norb], eri_packed [npair*(npair+1)/2]).
    """
    rng = np.random.Generator(np.random.Philox(seed))
    h = np.zeros((norb, norb), np.float64)
    iu = np.triu_indices(norb, 1)
    h[iu] = rng.normal(0.0, 0.05, size=iu[0].size)
    h = h + h.T
    h[np.diag_indices(norb)] = np.linspace(-2.0, 2.0, norb)
    npair = norb * (norb + 1) // 2
    # packed pair order: index(p, q) = p(p+1)/2 + q for p >= q
    pp, qq = np.tril_indices(norb)
    Lp = np.zeros((n_chol, npair), np.float64)
    iu2 = np.triu_indices(norb)
    for k in range(n_chol):
        L = np.zeros((norb, norb), np.float64)
        L[iu2] = rng.normal(0.0, 0.1, size=iu2[0].size)
        L = np.triu(L) + np.triu(L, 1).T
        L[np.diag_indices(norb)] += 0.5
        Lp[k] = L[pp, qq]
    V = Lp.T @ Lp  # (npair, npair), V[pq, rs] = (pq|rs)
    r, c = np.tril_indices(npair)
    eri = np.ascontiguousarray(V[r, c])
    return h, eri


def hubbard_1d(L=8, t=1.0, U=4.0, periodic=True):
    """1D Hubbard ring at half filling: lx=L, ly=1."""
    return dict(kind="hubbard", lx=L, ly=1, periodic_x=periodic, periodic_y=False, t=t, U=U,
                n_alpha=L // 2, n_beta=L // 2)


def hubbard_2d(lx, ly, U, t=1.0):
    n = lx * ly
    return dict(kind="hubbard", lx=lx, ly=ly, periodic_x=True, periodic_y=True, t=t, U=U,
                n_alpha=n // 2, n_beta=n // 2)


def batched_hubbard_instances(count=64):
    """The batched 2D Hubbard set: lattice [3x4, 4x4, 4x5][k mod 3], U/t
    [2,4,8][(k div 3) mod 3], periodic, half filling, walker target
    10^(4 + 2k/63), tau 0.005, initiator threshold 3, seed 1000 + k."""
    lat = [(3, 4), (4, 4), (4, 5)]
    us = [2.0, 4.0, 8.0]
    out = []
    for k in range(count):
        lx, ly = lat[k % 3]
        sysd = hubbard_2d(lx, ly, us[(k // 3) % 3])
        params = dict(tau=0.005, initiator_threshold=3.0, seed=1000 + k,
                      target_walkers=float(10.0 ** (4.0 + 2.0 * k / 63.0)), initial_walkers=10.0,
                      shift_damping=0.1, shift_interval=10)
        out.append((sysd, params))
    return out


def serving_requests(n=200, rate=20.0, seed=5):
    """Poisson arrivals of mixed FCIQMC requests (times in seconds)."""
    rng = np.random.Generator(np.random.Philox(seed))
    t = 0.0
    reqs = []
    for i in range(n):
        t += rng.exponential(1.0 / rate)
        kind = int(rng.integers(0, 3))
        target = float(10.0 ** rng.uniform(4.0, 7.0))
        U = float(rng.integers(1, 9))
        if kind == 0:
            L = int(rng.choice([8, 10, 12, 14, 16, 18]))
            sysd = hubbard_1d(L, 1.0, U)
        elif kind == 1:
            lx, ly = [(3, 4), (4, 4), (3, 6), (4, 3)][int(rng.integers(0, 4))]
            sysd = hubbard_2d(lx, ly, U)
        else:
            norb = int(rng.integers(16, 41))
            ne = int(rng.choice([8, 10, 12, 14, 16]))
            sysd = dict(kind="abinitio", norb=norb, n_alpha=ne // 2, n_beta=ne // 2,
                        n_chol=2 * norb, integral_seed=int(rng.integers(0, 2 ** 31)))
        reqs.append(dict(id=i, arrival=t, system=sysd, target_walkers=target,
                         seed=int(rng.integers(1, 2 ** 62))))
    return reqs


def config_hubbard_ring():
    """8-site periodic ring, 4+4 electrons, t=1, U=4; tau 0.01, target 1e4,
    shift damping 0.1, reference = Neel determinant."""
    return hubbard_1d(8, 1.0, 4.0), dict(tau=0.01, target_walkers=1e4, shift_damping=0.1,
                                         shift_interval=10, initial_walkers=10.0,
                                         initiator_threshold=0.0, seed=1)


def config_abinitio_24():
    """24 orbitals, 6+6 electrons, 96 Cholesky vectors, seed 2; uniform
    generator, initiator threshold 3, tau 1e-3, target 1e6."""
    h, eri = synthetic_abinitio(24, 96, 2)
    sysd = dict(kind="abinitio", norb=24, n_alpha=6, n_beta=6, h1=h, eri=eri, ecore=0.0)
    return sysd, dict(tau=1e-3, target_walkers=1e6, initiator_threshold=3.0, p_single=0.1,
                      shift_damping=0.1, shift_interval=10, initial_walkers=10.0, seed=2)


def config_abinitio_50():
    """50 orbitals, 10+10 electrons, 200 Cholesky vectors, seed 4; initiator
    threshold 3, tau 5e-4, target 1e8, deterministic space of 1e4."""
    h, eri = synthetic_abinitio(50, 200, 4)
    sysd = dict(kind="abinitio", norb=50, n_alpha=10, n_beta=10, h1=h, eri=eri, ecore=0.0)
    return sysd, dict(tau=5e-4, target_walkers=1e8, initiator_threshold=3.0, p_single=0.1,
                      shift_damping=0.1, shift_interval=10, initial_walkers=10.0, seed=4,
                      semistoch_size=10000, semistoch_start=100)


def small_abinitio(norb=6, na=3, nb=3, n_chol=None, seed=7):
    n_chol = n_chol or 4 * norb
    h, eri = synthetic_abinitio(norb, n_chol, seed)
    return dict(kind="abinitio", norb=norb, n_alpha=na, n_beta=nb, h1=h, eri=eri, ecore=0.0)


def write_fcidump(path, h, eri_packed, n_alpha, n_beta, ecore=0.0):
    """Write integrals in FCIDUMP form (one entry per symmetry-unique index set)."""
    norb = h.shape[0]
    with open(path, "w") as f:
        f.write(" &FCI NORB=%d,NELEC=%d,MS2=%d,\n  ORBSYM=%s\n  ISYM=1,\n &END\n" %
                (norb, n_alpha + n_beta, n_alpha - n_beta, "1," * norb))
        for i in range(norb):
            for j in range(i + 1):
                ij = pair_index(i, j)
                for k in range(norb):
                    for l in range(k + 1):
                        kl = pair_index(k, l)
                        if kl > ij:
                            continue
                        v = eri_packed[ij * (ij + 1) // 2 + kl]
                        if v != 0.0:
                            f.write("%.17e %d %d %d %d\n" % (v, i + 1, j + 1, k + 1, l + 1))
        for i in range(norb):
            for j in range(i + 1):
                if h[i, j] != 0.0:
                    f.write("%.17e %d %d 0 0\n" % (h[i, j], i + 1, j + 1))
        f.write("%.17e 0 0 0 0\n" % ecore)

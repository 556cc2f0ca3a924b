"""Full-space brute force for small models (2-3 orbitals), independent of sectors.

Creation/annihilation operators are Kronecker products of 2x2 matrices with
Jordan-Wigner strings; H_loc of Eq. (H_loc) is assembled from those matrices by
matrix products; imaginary-time propagators are full-space matrix exponentials
(scipy's scaling-and-squaring Pade, or mpmath at extended precision). Nothing
here uses sectors, ranks or the oracle's code.
"""
from __future__ import annotations

import math
from functools import reduce

import numpy as np
import scipy.linalg


def fermion_ops(n_orb: int):
    """c[f] for f = 2a + s; basis index x = sum_f n_f 2^f; JW string over lower bits."""
    nf = 2 * n_orb
    a = np.array([[0.0, 1.0], [0.0, 0.0]])  # |1> -> |0>
    Z = np.diag([1.0, -1.0])
    I = np.eye(2)
    ops = []
    for f in range(nf):
        # Kronecker order: most significant bit first
        factors = [I] * (nf - 1 - f) + [a] + [Z] * f
        ops.append(reduce(np.kron, factors))
    return ops


def hamiltonian(n_orb, U, J, Up, mu, delta, density_only=False):
    c = fermion_ops(n_orb)
    cd = [m.T.copy() for m in c]
    nn = [cd[f] @ c[f] for f in range(2 * n_orb)]
    dim = 4 ** n_orb
    H = np.zeros((dim, dim))
    for a in range(n_orb):
        for s in range(2):
            H -= (mu + delta[a]) * nn[2 * a + s]
        H += U * nn[2 * a] @ nn[2 * a + 1]
    for a in range(n_orb):
        for b in range(a):
            for s in range(2):
                H += Up * nn[2 * a + s] @ nn[2 * b + 1 - s] + (Up - J) * nn[2 * a + s] @ nn[2 * b + s]
    if not density_only:
        for a in range(n_orb):
            for b in range(n_orb):
                if a == b:
                    continue
                H -= J * (cd[2 * a + 1] @ cd[2 * b] @ c[2 * b + 1] @ c[2 * a])
                H -= J * (cd[2 * b] @ cd[2 * b + 1] @ c[2 * a] @ c[2 * a + 1])
    return H


def trace_all_states(H, beta, ops_seq, n_orb):
    """Untruncated T = Tr[e^{-(beta-t_K)H} O_K ... O_1 e^{-t_1 H}] with shift E0 = min eig.

    Returns T~ = e^{beta E0} T (float) using scipy.linalg.expm on H - E0.
    """
    c = fermion_ops(n_orb)
    E0 = np.linalg.eigvalsh(H).min()
    Hs = H - E0 * np.eye(len(H))
    M = np.eye(len(H))
    t_prev = 0.0
    for (t, f, d) in ops_seq:
        M = scipy.linalg.expm(-(t - t_prev) * Hs) @ M
        M = (c[f].T if d else c[f]) @ M
        t_prev = t
    M = scipy.linalg.expm(-(beta - t_prev) * Hs) @ M
    return float(np.trace(M)), E0


def trace_all_states_mp(H, beta, ops_seq, n_orb, dps=40):
    """Same as trace_all_states in mpmath at `dps` digits (small models only)."""
    import mpmath as mp
    mp.mp.dps = dps
    c = fermion_ops(n_orb)
    Hm = mp.matrix(H.tolist())
    E, V = mp.eigsy(Hm)
    E0 = min(E)
    n = len(H)

    def prop(dt):
        D = mp.diag([mp.exp(-dt * (E[i] - E0)) for i in range(n)])
        return V * D * V.T

    M = mp.eye(n)
    t_prev = mp.mpf(0)
    for (t, f, d) in ops_seq:
        M = prop(mp.mpf(t) - t_prev) * M
        C = mp.matrix((c[f].T if d else c[f]).tolist())
        M = C * M
        t_prev = mp.mpf(t)
    M = prop(mp.mpf(beta) - t_prev) * M
    return sum(M[i, i] for i in range(n)), E0


def kept_projector(H, beta, trunc_eps, deg_tol=1e-9):
    """Projector on the kept multiplets of the full-space H (truncation type (i) of Sec. II):
    eigenvalues are grouped into multiplets of neighbours within deg_tol * max(1, |E|), and
    whole multiplets whose lowest member has exp(-beta (E - E0)) >= trunc_eps are kept.
    Returns (P, number of kept states)."""
    E, V = np.linalg.eigh(H)
    E0 = E[0]
    keep = 0
    i = 0
    while i < len(E):
        j = i + 1
        while j < len(E) and E[j] - E[j - 1] <= deg_tol * max(1.0, abs(E[j])):
            j += 1
        if math.exp(-beta * (E[i] - E0)) < trunc_eps:
            break
        keep = j
        i = j
    Vk = V[:, :keep]
    return Vk @ Vk.T, keep


def trace_projected(H, beta, ops_seq, n_orb, P):
    """T~ = e^{beta E0} Tr[P e^{-(beta-t_K)H} O_K ... O_1 e^{-t_1 H}] with full-space
    scaling-and-squaring exponentials of H - E0 (P commutes with H)."""
    c = fermion_ops(n_orb)
    E0 = np.linalg.eigvalsh(H).min()
    Hs = H - E0 * np.eye(len(H))
    M = P.copy()
    t_prev = 0.0
    for (t, f, d) in ops_seq:
        M = scipy.linalg.expm(-(t - t_prev) * Hs) @ M
        M = (c[f].T if d else c[f]) @ M
        t_prev = t
    M = scipy.linalg.expm(-(beta - t_prev) * Hs) @ M
    return float(np.trace(M)), E0

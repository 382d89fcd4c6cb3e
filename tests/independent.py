"""Independent numpy restatements used to pin the oracle (test helpers, no shared code).

Everything here is written from textbook geometry and the paper's equations, not from the oracle:
site positions come from the documented index layout, neighbours from Cartesian periodic images
and the textbook shell radii, alpha from Eq. sro and F^2 from Eq. fitness_function.
"""
import itertools

import numpy as np

FCC, BCC = 0, 1
FCC_BASIS = np.array([[0, 0, 0], [0, 1, 1], [1, 0, 1], [1, 1, 0]])
BCC_BASIS = np.array([[0, 0, 0], [1, 1, 1]])
# Textbook squared shell radii in half-lattice units (a/2)^2: fcc a/sqrt2, a, a*sqrt(3/2), a*sqrt2,
# a*sqrt(5/2); bcc a*sqrt3/2, a, a*sqrt2, a*sqrt(11)/2, a*sqrt3.
SHELL_R2 = {FCC: [2, 4, 6, 8, 10], BCC: [3, 4, 8, 11, 12]}
SHELL_Z = {FCC: [12, 6, 24, 12, 24], BCC: [8, 6, 12, 24, 8]}


def positions(kind, L):
    """Half-unit positions of sites in index order ((b * Lz + cz) * Ly + cy) * Lx + cx."""
    basis = FCC_BASIS if kind == FCC else BCC_BASIS
    Lx, Ly, Lz = L
    out = []
    for b in range(len(basis)):
        for cz in range(Lz):
            for cy in range(Ly):
                for cx in range(Lx):
                    out.append([2 * cx + basis[b][0], 2 * cy + basis[b][1], 2 * cz + basis[b][2]])
    return np.array(out, dtype=np.int64)


def shell_multiplicity(kind, L, M):
    """mult[k][s][t] = number of vectors d with |d|^2 = r2_k and P_s + d == P_t (mod 2L)."""
    P = positions(kind, L)
    N = len(P)
    period = 2 * np.array(L)
    mult = np.zeros((M, N, N), dtype=np.int64)
    delta = (P[None, :, :] - P[:, None, :]) % period  # [s, t, 3]
    for n in itertools.product(range(-2, 3), repeat=3):
        d = delta + np.array(n) * period
        r2 = (d * d).sum(axis=2)
        for k in range(M):
            mult[k] += (r2 == SHELL_R2[kind][k])
    return mult


def counts_by_images(kind, L, M, S, types):
    mult = shell_multiplicity(kind, L, M)
    onehot = np.eye(S, dtype=np.int64)[np.asarray(types)]
    return np.einsum("ksn,si,nj->kij", mult, onehot, onehot)


def alpha_eq_sro(kind, L, M, n_per, cnt):
    """alpha_ij^(k) = 1 - P_ij^(k) / c_j, P = N_ij / (N_i Z_k), c_j = N_j / N (Eq. sro)."""
    n = np.asarray(n_per, dtype=np.float64)
    N = n.sum()
    Z = np.array(SHELL_Z[kind][:M], dtype=np.float64)
    P = np.asarray(cnt, dtype=np.float64) / (n[None, :, None] * Z[:, None, None])
    c = n / N
    return 1.0 - P / c[None, None, :]


def f2_eq_fitness(alpha, target, w):
    """F^2 = sum_k w_k sum_ij (alpha - target)^2 (Eq. fitness_function, squared)."""
    d = np.asarray(alpha) - np.asarray(target)
    return float((np.asarray(w)[:, None, None] * d * d).sum())

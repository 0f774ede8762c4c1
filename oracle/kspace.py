"""k-space transforms of the block store, written from their definitions.

TEST INFRASTRUCTURE ONLY (like the rest of oracle/): plain numpy loops over the blocks, shared
with nothing on the CUDA path.

  folding     X_mu,nu(k) = Sum_R X_mu,nu(R) exp(i k.R)                  (Sec. IV.B, the
              "folding" of an operator into momentum space; R over all valid neighbouring cells)
  unfolding   X_mu,nu(R) = Re Sum_k w_k X_mu,nu(k) exp(-i k.R)            (Eq. density_matrix
              with X(k) = Sum_n f_nk c_n,mu,k c*_n,nu,k and w_k = 1/N_k)

Conventions: a block key (I, J, n1, n2, n3) couples orbital mu of atom I with orbital nu of atom
J shifted by R = n1 a1 + n2 a2 + n3 a3; k is given in fractional reciprocal coordinates kappa,
so k.R = 2 pi kappa.n.  Dense matrices use the atom-major orbital order (orbital offset of atom
I = Sum_{J<I} norb_J) and are returned as complex128 arrays [nk, nbasis, nbasis].
"""
from __future__ import annotations

import numpy as np


def orbital_offsets(norb_atom):
    norb_atom = np.asarray(norb_atom, np.int64)
    return np.concatenate([[0], np.cumsum(norb_atom)])


def fold(keys, offs, norb_atom, X, kfrac):
    keys = np.asarray(keys)
    kfrac = np.atleast_2d(np.asarray(kfrac, np.float64))
    o = orbital_offsets(norb_atom)
    n = int(o[-1])
    out = np.zeros((len(kfrac), n, n), np.complex128)
    for b, (I, J, n1, n2, n3) in enumerate(keys):
        blk = np.asarray(X[offs[b]:offs[b + 1]], np.float64).reshape(norb_atom[I], norb_atom[J])
        for q, kap in enumerate(kfrac):
            ph = np.exp(2j * np.pi * (kap[0] * n1 + kap[1] * n2 + kap[2] * n3))
            out[q, o[I]:o[I + 1], o[J]:o[J + 1]] += ph * blk
    return out


def unfold(keys, offs, norb_atom, Xk, kfrac, wk):
    keys = np.asarray(keys)
    kfrac = np.atleast_2d(np.asarray(kfrac, np.float64))
    o = orbital_offsets(norb_atom)
    out = np.zeros(int(offs[-1]), np.float64)
    for b, (I, J, n1, n2, n3) in enumerate(keys):
        acc = np.zeros((norb_atom[I], norb_atom[J]), np.complex128)
        for q, kap in enumerate(kfrac):
            ph = np.exp(-2j * np.pi * (kap[0] * n1 + kap[1] * n2 + kap[2] * n3))
            acc += wk[q] * ph * Xk[q, o[I]:o[I + 1], o[J]:o[J + 1]]
        out[offs[b]:offs[b + 1]] = acc.real.reshape(-1)
    return out


def monkhorst_pack(n1, n2, n3, shift=(0.0, 0.0, 0.0)):
    """Uniform k mesh kappa = (i + s)/n in fractional coordinates, equal weights."""
    g = np.array([(i + shift[0]) / n1 for i in range(n1)])
    h = np.array([(j + shift[1]) / n2 for j in range(n2)])
    l = np.array([(m + shift[2]) / n3 for m in range(n3)])
    k = np.array([[a, b, c] for a in g for b in h for c in l], np.float64)
    return k, np.full(len(k), 1.0 / len(k))


def density_matrix(keys, offs, norb_atom, C, f, kfrac, wk):
    """Eq. density_matrix: rho_mu,nu(R) = Re Sum_k w_k Sum_n f_nk c_n,mu,k c*_n,nu,k exp(-i k.R).

    C: complex [nk, nbasis, nbands] (row = orbital mu, column = band n); f: [nk, nbands]."""
    C = np.asarray(C, np.complex128)
    f = np.asarray(f, np.float64)
    rhok = np.einsum("qmn,qn,qvn->qmv", C, f, C.conj())
    return unfold(keys, offs, norb_atom, rhok, kfrac, wk)

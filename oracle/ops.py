"""Local spin operators written out from their definitions (oracle, test infrastructure only).

Spin-1/2 matrices in the local basis {|down> = 0, |up> = 1}; multi-site local
bases put the first listed site in the most significant position, matching the
global integer encoding (Eq. numberforspinconfig).

  bond(i, j)      = S_i . S_j = sum_a S^a_i S^a_j           (Eq. heisenbergallover)
  chirality(i,j,k)= S_i . (S_j x S_k) = sum_abc eps_abc S^a_i S^b_j S^c_k   (Eq. scalarchirality)
"""
from __future__ import annotations

import itertools

import numpy as np

# |0> = down, |1> = up
SZ = np.array([[-0.5, 0.0], [0.0, 0.5]], dtype=complex)
SP = np.array([[0.0, 0.0], [1.0, 0.0]], dtype=complex)   # S+ |down> = |up>
SM = SP.T.copy()
SX = 0.5 * (SP + SM)
SY = -0.5j * (SP - SM)
SPIN = (SX, SY, SZ)


def _kron(*ms):
    out = np.array([[1.0 + 0j]])
    for m in ms:
        out = np.kron(out, m)
    return out


def bond_matrix() -> np.ndarray:
    """4x4 matrix of S_i . S_j, local index 2*s_i + s_j."""
    return sum(_kron(S, S) for S in SPIN)


def levi_civita(a, b, c) -> int:
    return int(np.sign(np.linalg.det(np.eye(3)[[a, b, c]])))


def chirality_matrix() -> np.ndarray:
    """8x8 matrix of S_i . (S_j x S_k), local index 4*s_i + 2*s_j + s_k."""
    M = np.zeros((8, 8), dtype=complex)
    for a, b, c in itertools.permutations(range(3)):
        M += levi_civita(a, b, c) * _kron(SPIN[a], SPIN[b], SPIN[c])
    return M


def term_arrays(terms):
    """Flatten a Terms object into (nloc[T], sites[T][3], mats[T][8][8]) for the C oracle."""
    B = bond_matrix()
    C = chirality_matrix()
    nb, nt = len(terms.bonds), len(terms.tris)
    T = nb + nt
    nloc = np.zeros(T, dtype=np.int32)
    sites = np.zeros((T, 3), dtype=np.int32)
    mats = np.zeros((T, 8, 8), dtype=complex)
    for t in range(nb):
        nloc[t] = 2
        sites[t, :2] = terms.bonds[t]
        mats[t, :4, :4] = terms.J[t] * B
    for q in range(nt):
        t = nb + q
        nloc[t] = 3
        sites[t] = terms.tris[q]
        mats[t] = terms.Jchi[q] * C
    return nloc, sites, mats

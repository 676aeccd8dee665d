"""Ground-state observables from a symmetric-basis state.

A state psi of a one-dimensional irrep of the sector's group G satisfies
<psi| g O g^-1 |psi> = <psi|O|psi> for every g, so the spin correlation
<S_i . S_j> equals the expectation of the orbit average
(1/|orbit|) sum_{{i',j'} in orbit of {i,j}} S_i' . S_j', an operator that
commutes with G and is applied by the library's own H.x kernels
(ed_expectation).  From the correlations, the static structure factor of
Eq. structurefactor, S(k) = sum_j exp(i k.(r_j - r_0)) <S_j . S_0>, here
averaged over the reference site 0 (the same for a translation-invariant
state).  Scalar chiralities <S_i . (S_j x S_k)> of triangles follow the same
construction with the orbit-averaged triangle operator.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .ed import Hamiltonian


@dataclass
class _Bonds:
    """Terms-like container: bonds with couplings, no chirality terms."""
    bonds: np.ndarray
    J: np.ndarray
    tris: np.ndarray
    Jchi: np.ndarray


def pair_orbits(sector) -> list[np.ndarray]:
    """Orbits of the unordered site pairs {i, j}, i != j, under the sector's
    site permutations (spin flips leave S_i . S_j unchanged).  Every pair lies
    in exactly one orbit; each orbit is an int32 array [n][2] with i < j."""
    perm = np.asarray(sector.perm, dtype=np.int64)
    N = int(sector.n_sites)
    seen = np.zeros((N, N), dtype=bool)
    orbits = []
    for i in range(N):
        for j in range(i + 1, N):
            if seen[i, j]:
                continue
            a, b = perm[:, i], perm[:, j]
            lo, hi = np.minimum(a, b), np.maximum(a, b)
            pairs = np.unique(np.stack([lo, hi], axis=1), axis=0)
            seen[pairs[:, 0], pairs[:, 1]] = True
            orbits.append(pairs.astype(np.int32))
    return orbits


def correlations(basis, sector, psi, stream=None) -> np.ndarray:
    """C[i, j] = <psi| S_i . S_j |psi> / <psi|psi> for all site pairs (C[i, i] = 3/4),
    psi a torch CUDA tensor in the symmetric basis of `basis` (any dtype the
    library takes).  One ed_expectation per pair orbit."""
    N = int(sector.n_sites)
    C = np.full((N, N), np.nan)
    np.fill_diagonal(C, 0.75)
    for orb in pair_orbits(sector):
        terms = _Bonds(orb, np.full(len(orb), 1.0 / len(orb)), np.zeros((0, 3), np.int32), np.zeros(0))
        h = Hamiltonian(basis, terms)
        try:
            v = float(np.real(h.expectation(psi, stream=stream)[0]))
        finally:
            h.close()
        C[orb[:, 0], orb[:, 1]] = v
        C[orb[:, 1], orb[:, 0]] = v
    return C


def chiralities(basis, sector, psi, triangles, stream=None) -> np.ndarray:
    """<psi| S_i . (S_j x S_k) |psi> / <psi|psi> for each ordered triangle (i, j, k):
    the expectation of the orbit average (1/|G|) sum_g S_g(i) . (S_g(j) x S_g(k)),
    which commutes with G (a spin flip is a rotation by pi in spin space and
    leaves the scalar triple product unchanged)."""
    perm = np.asarray(sector.perm, dtype=np.int64)
    G = len(perm)
    out = np.empty(len(triangles))
    for n, (i, j, k) in enumerate(np.asarray(triangles, dtype=np.int64)):
        tris = np.stack([perm[:, i], perm[:, j], perm[:, k]], axis=1).astype(np.int32)
        terms = _Bonds(np.zeros((0, 2), np.int32), np.zeros(0), tris, np.full(G, 1.0 / G))
        h = Hamiltonian(basis, terms)
        try:
            out[n] = float(np.real(h.expectation(psi, stream=stream)[0]))
        finally:
            h.close()
    return out


def structure_factor(C: np.ndarray, positions: np.ndarray, ks: np.ndarray) -> np.ndarray:
    """S(k) = (1/N) sum_{i,j} exp(i k.(r_j - r_i)) C[i, j] for each row k of ks
    (Eq. structurefactor averaged over the reference site)."""
    r = np.asarray(positions, dtype=np.float64)
    ks = np.atleast_2d(np.asarray(ks, dtype=np.float64))
    N = len(r)
    out = np.empty(len(ks))
    for n, k in enumerate(ks):
        ph = np.exp(1j * (r @ k))
        out[n] = float(np.real(np.conj(ph) @ C @ ph)) / N
    return out

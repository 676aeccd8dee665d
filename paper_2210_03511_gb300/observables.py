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

Four- and six-spin order parameters (the nematic N of Eq.
nematicorderparameter and the chirality correlation X of Eq.
chiralityorderparameter) sum a product over the translates of a bond or a
triangle.  With B = sum_{t in T} t O t^-1 the translation sum of O, a state of
momentum k has <O B> = <B^2> / |T| (<psi|t A t^-1|psi> = <A> for every
translation t), and <B^2> = ||B psi||^2 because B is Hermitian.  B commutes
with the translations but not with the point group, so psi is first written in
the basis of its translation-only sector (ed_restrict, the characters of the
translations are those of psi's irrep) and B is applied there by the H.x
kernels.

The dynamical spin structure factor
S(q, w) = sum_n |<n|S^z(q)|0>|^2 delta(w - (E_n - E_0)), with
S^z(q) = N^-1/2 sum_i exp(i q.r_i) S^z_i, follows by the continued-fraction
expansion: phi = S^z(q)|0> is formed in the sector S^z(q) maps the ground
state into (ed_apply_sz: same group, characters times the operator's phases),
the Lanczos recursion from phi (ed_lanczos_tridiag) gives T, and
<phi|(z - H)^-1|phi> = |phi|^2 / (z - a_0 - b_0^2 / (z - a_1 - ...)), so that
S(q, w) = -Im G(w + E_0 + i eta) / pi, a sum of Lorentzians of width eta.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .ed import Basis, Hamiltonian


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


@dataclass
class SubSector:
    """Sector of a subgroup (the fields of ed_sector)."""
    n_sites: int
    n_up: int
    perm: np.ndarray
    spinflip: np.ndarray
    chi: np.ndarray
    n_sublat: int


def subgroup_sector(sector, elements) -> SubSector:
    """The sector of the subgroup formed by `elements` (indices into the
    sector's group, which must contain the identity, element 0) with the
    characters of the sector's irrep restricted to it.  The sublattice blocks
    are kept: a partition stable under a group is stable under its subgroups."""
    idx = [int(e) for e in elements]
    if 0 not in idx:
        raise ValueError("the subgroup must contain the identity (element 0)")
    idx = [0] + [e for e in idx if e != 0]
    return SubSector(int(sector.n_sites), int(sector.n_up), np.asarray(sector.perm)[idx].astype(np.int32),
                     np.asarray(sector.spinflip)[idx].astype(np.uint8), np.asarray(sector.chi)[idx].astype(complex),
                     int(sector.n_sublat))


class TranslationSector:
    """The translation-only sector of a state's sector, its basis, and the
    restriction of states to it (ed_restrict)."""

    def __init__(self, basis, sector, translations):
        self.basis = basis
        self.translations = [int(t) for t in translations]
        self.sector = subgroup_sector(sector, self.translations)
        self.sub = Basis(self.sector)
        self.perm = np.asarray(sector.perm, dtype=np.int64)[self.translations]

    @property
    def n_trans(self) -> int:
        return len(self.translations)

    def orbit_bonds(self, bond) -> np.ndarray:
        a, b = int(bond[0]), int(bond[1])
        return np.stack([self.perm[:, a], self.perm[:, b]], axis=1).astype(np.int32)

    def orbit_triangles(self, tri) -> np.ndarray:
        return np.stack([self.perm[:, int(v)] for v in tri], axis=1).astype(np.int32)

    def moments(self, psi, terms, stream=None):
        """(<B>, <B^2>) of the translation-invariant operator B given by `terms`
        in the state psi (torch CUDA tensor in the symmetric basis of `basis`)."""
        import torch
        h = Hamiltonian(self.sub, terms)
        try:
            x = psi
            if not h.is_real and not x.is_complex():
                x = x.to(torch.complex128)
            xs = self.basis.restrict_to(self.sub, x.contiguous(), stream=stream)
            phi = torch.empty_like(xs)
            h.apply(xs, phi, stream=stream)
            hx, nx = h.expectation(xs, stream=stream, raw=True)
            _, nphi = h.expectation(phi, stream=stream, raw=True)
        finally:
            h.close()
        return float(np.real(hx[0]) / nx[0]), float(nphi[0] / nx[0])

    def close(self):
        self.sub.close()


def nematic(ts: TranslationSector, psi, bond, stream=None) -> float:
    """N of Eq. nematicorderparameter for the bond (a, b): the sum over its
    translates (i, j) of the connected <(S_a.S_b)(S_i.S_j)> - <S_a.S_b><S_i.S_j>,
    = (<B^2> - <B>^2) / |T| with B = sum_t S_t(a).S_t(b)."""
    bonds = ts.orbit_bonds(bond)
    terms = _Bonds(bonds, np.ones(len(bonds)), np.zeros((0, 3), np.int32), np.zeros(0))
    b1, b2 = ts.moments(psi, terms, stream=stream)
    return (b2 - b1 * b1) / ts.n_trans


def chirality_correlation(ts: TranslationSector, psi, tri, stream=None) -> float:
    """X of Eq. chiralityorderparameter for the triangle (i, j, k): the sum over
    its translates t of <chi_(i,j,k) chi_t>, = <X^2> / |T| with X the
    translation sum of chi_(i,j,k) = S_i.(S_j x S_k)."""
    tris = ts.orbit_triangles(tri)
    terms = _Bonds(np.zeros((0, 2), np.int32), np.zeros(0), tris, np.ones(len(tris)))
    _, x2 = ts.moments(psi, terms, stream=stream)
    return x2 / ts.n_trans


# ---------------------------------------------------------------- dynamical structure factor
def szq_coefficients(positions, q) -> np.ndarray:
    """c_i = exp(i q.r_i) / sqrt(N): the site coefficients of S^z(q)."""
    r = np.asarray(positions, dtype=np.float64)
    return np.exp(1j * (r @ np.asarray(q, dtype=np.float64))) / np.sqrt(len(r))


def sz_target_sector(sector, c) -> SubSector:
    """The sector O = sum_i c_i S^z_i maps `sector` into: the same group, with
    characters lambda(g) chi(g), where s_g c_{g^-1(j)} = lambda(g) c_j (s_g = -1
    for an element with spin flip).  Raises if O is not mapped onto a multiple
    of itself by every element (e.g. a momentum not allowed on the torus)."""
    c = np.asarray(c, dtype=complex)
    perm = np.asarray(sector.perm, dtype=np.int64)
    N = perm.shape[1]
    j0 = int(np.argmax(np.abs(c)))
    lam = np.empty(len(perm), dtype=complex)
    for g, p in enumerate(perm):
        inv = np.empty(N, dtype=np.int64)
        inv[p] = np.arange(N)
        sg = -1.0 if np.asarray(sector.spinflip)[g] else 1.0
        lam[g] = sg * c[inv[j0]] / c[j0]
        if not np.allclose(sg * c[inv], lam[g] * c, atol=1e-9 * np.abs(c).max()):
            raise ValueError(f"element {g} does not map the operator onto a multiple of itself")
    chi = lam * np.asarray(sector.chi, dtype=complex)
    # exact roots of unity stay exact (real sectors keep real characters)
    chi = np.where(np.abs(chi.imag) < 1e-12, chi.real + 0j, chi)
    chi = np.where(np.abs(chi.real) < 1e-12, 1j * chi.imag, chi)
    return SubSector(int(sector.n_sites), int(sector.n_up), np.asarray(sector.perm, dtype=np.int32),
                     np.asarray(sector.spinflip, dtype=np.uint8), chi, int(sector.n_sublat))


def continued_fraction(alpha, beta, norm2, z) -> np.ndarray:
    """norm2 / (z - a_0 - b_0^2 / (z - a_1 - ... / (z - a_{m-1}))) for each z."""
    z = np.atleast_1d(np.asarray(z, dtype=complex))
    a = np.asarray(alpha, dtype=np.float64)
    b = np.asarray(beta, dtype=np.float64)
    d = z - a[-1]
    for n in range(len(a) - 2, -1, -1):
        d = z - a[n] - b[n] ** 2 / d
    return norm2 / d


def dynamical_structure_factor(h_target, phi, omegas, e0, eta, m=200, reorth=False, stream=None):
    """S(q, w) at the frequencies `omegas` with Lorentzian width eta, from
    phi = S^z(q)|0> in the target sector of the Hamiltonian h_target and the
    ground-state energy e0.  Returns (S, alpha, beta, |phi|^2)."""
    a, b, n2 = h_target.lanczos_tridiag(phi, m, reorth=reorth, stream=stream)
    G = continued_fraction(a, b, n2, np.asarray(omegas, dtype=np.float64) + e0 + 1j * eta)
    return -G.imag / np.pi, a, b, n2

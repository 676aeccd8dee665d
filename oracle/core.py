"""CPU FP64 oracle for symmetry-adapted ED (test infrastructure only).

Only the test suite, the smoke check and the benchmark's CPU-baseline arm use
this package.  It shares no code with the CUDA library.

What it computes (thesis chapter "Symmetries and Parallelization for
Large-Scale Exact Diagonalization" and the sections it builds on):
  * group action and representatives by applying every element
    (Eq. representativecondition, the naive search of the sublattice-coding
    section) -- `rep`, in C;
  * the basis: popcount-n_up states that are their own representative and
    whose projector (Eq. symmetryadaptedwavefunction1d) is non-zero, sorted
    (Alg. "Preparation of the distributed and symmetrized Hilbert space"
    without the distribution) -- `basis`;
  * the sparse matrix in that basis from local operators via
    Eq. matrixelementrepresentatives_lsed with the conj(chi) reading -- `csr`,
    or by column ranges on several threads for large sectors -- `csr_chunked`;
  * the dense matrix in the unsymmetrized fixed-Sz space -- `dense_sz`;
  * explicit symmetric vectors by the projector -- `projector_matrix`;
  * sector dimensions by the character formula (Eq. characterformula) --
    `sector_dim_formula`;
  * eigenvalues: dense LAPACK or ARPACK on the CSR -- `lowest_eigs`;
  * matrix-free sampled rows with keyed-random x -- `rows`;
  * spin correlations <S_i.S_j> of a symmetric-basis state, written out in the
    product basis (Eq. structurefactor) -- `correlation_matrix`; scalar
    chiralities <S_i.(S_j x S_k)> likewise -- `triangle_expectation`;
  * time evolution exp(-iHt) psi on the sparse matrix (library step) -- `evolve`;
  * a state written out in the product basis -- `plain_state`; its
    coefficients in a subgroup's sector -- `restrict`; products of two bond or
    triangle operators -- `product_expectation`; the nematic and chirality
    order parameters (Eqs. nematicorderparameter, chiralityorderparameter)
    term by term -- `nematic`, `chirality_sum`;
  * the dynamical structure factor of a one-site S^z sum as poles and weights
    from the dense eigendecomposition -- `sz_spectrum`, `lorentzians`.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from math import comb

import numpy as np
import scipy.sparse as sp

from . import ops

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = os.path.join(_HERE, "_liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    src = os.path.join(_HERE, "oracle.c")
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(src):
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c11", src, "-o", _LIB, "-lm"])
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        P = ctypes.POINTER
        L.orc_apply.restype = ctypes.c_uint64
        L.orc_apply.argtypes = [ctypes.c_uint64, ctypes.c_int, P(ctypes.c_int32), ctypes.c_int]
        L.orc_rep.restype = None
        L.orc_rep.argtypes = [ctypes.c_uint64, ctypes.c_int, ctypes.c_int, P(ctypes.c_int32), P(ctypes.c_uint8),
                              P(ctypes.c_double), P(ctypes.c_uint64), P(ctypes.c_int32), P(ctypes.c_int32),
                              P(ctypes.c_double), P(ctypes.c_double)]
        L.orc_basis.restype = ctypes.c_int64
        L.orc_basis.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, P(ctypes.c_int32), P(ctypes.c_uint8),
                                P(ctypes.c_double), P(ctypes.c_uint64), P(ctypes.c_int32), ctypes.c_int64]
        L.orc_coo.restype = ctypes.c_int64
        L.orc_coo.argtypes = [ctypes.c_int, ctypes.c_int, P(ctypes.c_int32), P(ctypes.c_uint8), P(ctypes.c_double),
                              P(ctypes.c_uint64), P(ctypes.c_int32), ctypes.c_int64,
                              ctypes.c_int, P(ctypes.c_int32), P(ctypes.c_int32), P(ctypes.c_double),
                              P(ctypes.c_int64), P(ctypes.c_int64), P(ctypes.c_double), ctypes.c_int64]
        L.orc_coo_cols.restype = ctypes.c_int64
        L.orc_coo_cols.argtypes = [ctypes.c_int, ctypes.c_int, P(ctypes.c_int32), P(ctypes.c_uint8),
                                   P(ctypes.c_double), P(ctypes.c_uint64), P(ctypes.c_int32), ctypes.c_int64,
                                   ctypes.c_int64, ctypes.c_int64,
                                   ctypes.c_int, P(ctypes.c_int32), P(ctypes.c_int32), P(ctypes.c_double),
                                   P(ctypes.c_int64), P(ctypes.c_int64), P(ctypes.c_double), ctypes.c_int64]
        L.orc_rows.restype = None
        L.orc_rows.argtypes = [ctypes.c_int, ctypes.c_int, P(ctypes.c_int32), P(ctypes.c_uint8), P(ctypes.c_double),
                               ctypes.c_int, P(ctypes.c_int32), P(ctypes.c_int32), P(ctypes.c_double),
                               P(ctypes.c_uint64), ctypes.c_int64, ctypes.c_uint64, ctypes.c_int, P(ctypes.c_double)]
        L.orc_num_threads.restype = ctypes.c_int
        L.orc_set_num_threads.restype = None
        L.orc_set_num_threads.argtypes = [ctypes.c_int]
        _lib = L
    return _lib


def _p(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


class _Sec:
    """Contiguous C views of a sector."""

    def __init__(self, sector):
        self.N = int(sector.n_sites)
        self.n_up = int(sector.n_up)
        self.G = int(sector.n_sym)
        self.perm = np.ascontiguousarray(sector.perm, dtype=np.int32)
        self.flip = np.ascontiguousarray(sector.spinflip, dtype=np.uint8)
        chi = np.asarray(sector.chi, dtype=complex)
        self.chi = np.ascontiguousarray(np.stack([chi.real, chi.imag], axis=1), dtype=np.float64)

    def args(self):
        return (self.N, self.G, _p(self.perm, ctypes.c_int32), _p(self.flip, ctypes.c_uint8),
                _p(self.chi, ctypes.c_double))


def apply(sector, g: int, state: int) -> int:
    s = _Sec(sector)
    return int(lib().orc_apply(state, s.N, _p(s.perm[g:g + 1].copy(), ctypes.c_int32), int(s.flip[g])))


def rep(sector, state: int):
    """(representative, first minimising element, |Stab(rep)|, sum_{Stab} chi)."""
    s = _Sec(sector)
    r = ctypes.c_uint64()
    g = ctypes.c_int32()
    n = ctypes.c_int32()
    sr = ctypes.c_double()
    si = ctypes.c_double()
    lib().orc_rep(state, s.N, s.G, _p(s.perm, ctypes.c_int32), _p(s.flip, ctypes.c_uint8), _p(s.chi, ctypes.c_double),
                  ctypes.byref(r), ctypes.byref(g), ctypes.byref(n), ctypes.byref(sr), ctypes.byref(si))
    return int(r.value), int(g.value), int(n.value), complex(sr.value, si.value)


def basis(sector):
    """Sorted representatives (uint64) and stabilizer orders (int32)."""
    s = _Sec(sector)
    D = lib().orc_basis(s.N, s.n_up, s.G, _p(s.perm, ctypes.c_int32), _p(s.flip, ctypes.c_uint8),
                        _p(s.chi, ctypes.c_double), None, None, 0)
    reps = np.zeros(max(D, 1), dtype=np.uint64)
    stab = np.zeros(max(D, 1), dtype=np.int32)
    D2 = lib().orc_basis(s.N, s.n_up, s.G, _p(s.perm, ctypes.c_int32), _p(s.flip, ctypes.c_uint8),
                         _p(s.chi, ctypes.c_double), _p(reps, ctypes.c_uint64), _p(stab, ctypes.c_int32), D)
    assert D2 == D
    return reps[:D], stab[:D]


def _terms_c(terms):
    nloc, sites, mats = ops.term_arrays(terms)
    m = np.ascontiguousarray(np.stack([mats.real, mats.imag], axis=-1), dtype=np.float64)
    return len(nloc), np.ascontiguousarray(nloc), np.ascontiguousarray(sites), m


def csr(problem, reps=None, stab=None) -> sp.csr_matrix:
    """Sparse H in the symmetric basis (complex128), duplicates summed."""
    sec, terms = problem.sector, problem.terms
    if reps is None:
        reps, stab = basis(sec)
    s = _Sec(sec)
    T, nloc, sites, mats = _terms_c(terms)
    D = len(reps)
    reps = np.ascontiguousarray(reps, dtype=np.uint64)
    stab = np.ascontiguousarray(stab, dtype=np.int32)
    args = s.args() + (_p(reps, ctypes.c_uint64), _p(stab, ctypes.c_int32), D, T, _p(nloc, ctypes.c_int32),
                       _p(sites, ctypes.c_int32), _p(mats, ctypes.c_double))
    n = lib().orc_coo(*args, None, None, None, 0)
    rows = np.zeros(max(n, 1), dtype=np.int64)
    cols = np.zeros(max(n, 1), dtype=np.int64)
    vals = np.zeros((max(n, 1), 2), dtype=np.float64)
    n2 = lib().orc_coo(*args, _p(rows, ctypes.c_int64), _p(cols, ctypes.c_int64), _p(vals, ctypes.c_double), n)
    assert n2 == n
    v = vals[:n, 0] + 1j * vals[:n, 1]
    H = sp.coo_matrix((v, (rows[:n], cols[:n])), shape=(D, D)).tocsr()
    H.sum_duplicates()
    return H


def csr_chunked(problem, reps=None, stab=None, chunk: int = 8192, workers: int | None = None,
                real: bool = False):
    """The matrix of `csr`, assembled by independent column ranges on several
    host threads (each range is the same column-wise assembly; duplicates are
    summed per range).  For sectors of millions of states.  Returned in CSC
    form (the columns are what is assembled); H is Hermitian, so H.T.conj()
    is the same matrix.  real=True keeps the real part only (for a real
    Hamiltonian in a sector with real characters; the imaginary parts are
    checked to be zero)."""
    from concurrent.futures import ThreadPoolExecutor
    sec, terms = problem.sector, problem.terms
    if reps is None:
        reps, stab = basis(sec)
    s = _Sec(sec)
    T, nloc, sites, mats = _terms_c(terms)
    D = len(reps)
    reps = np.ascontiguousarray(reps, dtype=np.uint64)
    stab = np.ascontiguousarray(stab, dtype=np.int32)
    per_col = int(sum(1 << int(n) for n in nloc))  # at most one entry per local image
    L = lib()

    def part(c0):
        c1 = min(D, c0 + chunk)
        cap = per_col * (c1 - c0)
        rows = np.empty(max(cap, 1), dtype=np.int64)
        cols = np.empty(max(cap, 1), dtype=np.int64)
        vals = np.empty((max(cap, 1), 2), dtype=np.float64)
        n = L.orc_coo_cols(*s.args(), _p(reps, ctypes.c_uint64), _p(stab, ctypes.c_int32), D, c0, c1, T,
                           _p(nloc, ctypes.c_int32), _p(sites, ctypes.c_int32), _p(mats, ctypes.c_double),
                           _p(rows, ctypes.c_int64), _p(cols, ctypes.c_int64), _p(vals, ctypes.c_double), cap)
        assert n >= 0
        if real:
            assert np.all(vals[:n, 1] == 0.0)
            v = vals[:n, 0].copy()
        else:
            v = vals[:n, 0] + 1j * vals[:n, 1]
        M = sp.coo_matrix((v, (rows[:n], cols[:n] - c0)), shape=(D, c1 - c0)).tocsc()
        M.sum_duplicates()
        return M

    workers = workers or os.cpu_count() or 1
    with ThreadPoolExecutor(workers) as ex:
        parts = list(ex.map(part, range(0, D, chunk)))
    return sp.hstack(parts, format="csc")


def rows(problem, states: np.ndarray, seed: int, is_complex: bool) -> np.ndarray:
    """Matrix-free y(sigma~) = sum_j H[sigma~, j] x(state_j) for the given representatives."""
    sec, terms = problem.sector, problem.terms
    s = _Sec(sec)
    T, nloc, sites, mats = _terms_c(terms)
    st = np.ascontiguousarray(states, dtype=np.uint64)
    y = np.zeros((len(st), 2), dtype=np.float64)
    lib().orc_rows(*s.args(), T, _p(nloc, ctypes.c_int32), _p(sites, ctypes.c_int32), _p(mats, ctypes.c_double),
                   _p(st, ctypes.c_uint64), len(st), seed, int(is_complex), _p(y, ctypes.c_double))
    return y[:, 0] + 1j * y[:, 1]


def num_threads() -> int:
    return int(lib().orc_num_threads())


def set_num_threads(n: int) -> None:
    """OpenMP threads of the C routines from now on."""
    lib().orc_set_num_threads(int(n))


# --------------------------------------------------------------------------
# unsymmetrized space and explicit projection (brute force, small N only)
# --------------------------------------------------------------------------
def sz_states(N: int, n_up: int) -> np.ndarray:
    """All popcount-n_up states in increasing order (N <= 20)."""
    a = np.arange(1 << N, dtype=np.uint64)
    pc = np.array([bin(int(x)).count("1") for x in a])
    return a[pc == n_up]


def dense_sz(problem) -> tuple[np.ndarray, np.ndarray]:
    """Dense H on the fixed-Sz space by applying each local operator to each state."""
    sec, terms = problem.sector, problem.terms
    N = sec.n_sites
    states = sz_states(N, sec.n_up)
    index = {int(s): i for i, s in enumerate(states)}
    H = np.zeros((len(states), len(states)), dtype=complex)
    nloc, sites, mats = ops.term_arrays(terms)
    for c, s in enumerate(states):
        s = int(s)
        for t in range(len(nloc)):
            nl = nloc[t]
            st = sites[t][:nl]
            a = 0
            for site in st:
                a = (a << 1) | ((s >> (N - 1 - site)) & 1)
            for ap in range(1 << nl):
                m = mats[t][ap, a]
                if m == 0:
                    continue
                tau = s
                for l, site in enumerate(st):
                    bit = 1 << (N - 1 - site)
                    if (ap >> (nl - 1 - l)) & 1:
                        tau |= bit
                    else:
                        tau &= ~bit
                H[index[tau], c] += m
    return H, states


def projector_matrix(sector, states: np.ndarray) -> tuple[np.ndarray, list[int]]:
    """Columns = normalised projections sum_g chi(g)^* g|sigma> of every state, one per orbit.

    Representatives are taken as the smallest integer in the explicitly
    enumerated orbit (independent of `rep`).  Returns (V, orbit minima kept)."""
    N, G = sec_N(sector), sector.n_sym
    index = {int(s): i for i, s in enumerate(states)}
    seen = set()
    cols, kept = [], []
    for s in states:
        s = int(s)
        if s in seen:
            continue
        orbit = []
        for g in range(G):
            t = 0
            for i in range(N):
                v = (s >> (N - 1 - i)) & 1
                if sector.spinflip[g]:
                    v ^= 1
                if v:
                    t |= 1 << (N - 1 - int(sector.perm[g][i]))
            orbit.append(t)
        seen.update(orbit)
        v = np.zeros(len(states), dtype=complex)
        for g, t in enumerate(orbit):
            v[index[t]] += np.conj(sector.chi[g])
        nrm = np.linalg.norm(v)
        if nrm > 1e-9:
            cols.append(v / nrm)
            kept.append(min(orbit))
    order = np.argsort(kept)
    V = np.array(cols).T[:, order] if cols else np.zeros((len(states), 0))
    # fix the phase convention of each column: the coefficient on the orbit
    # minimum is real positive in the symmetric-basis matrix of `csr`
    kept = [kept[i] for i in order]
    for c, m in enumerate(kept):
        ph = V[index[m], c]
        V[:, c] *= np.conj(ph) / abs(ph)
    return V, kept


def correlation_matrix(sector, psi: np.ndarray) -> np.ndarray:
    """C[i, j] = <phi|S_i . S_j|phi> / <phi|phi> for the state phi = sum_c psi_c v_c
    written out in the fixed-Sz product basis (v_c the explicit projections of
    `projector_matrix`, in basis order), each S_i . S_j applied through the
    4x4 matrix of its definition (ops.bond_matrix).  The spin correlation of
    Eq. structurefactor.  N <= 20."""
    N = sec_N(sector)
    states = sz_states(N, sector.n_up)
    V, kept = projector_matrix(sector, states)
    assert V.shape[1] == len(psi)
    phi = V @ np.asarray(psi, dtype=complex)
    nrm = float(np.real(np.vdot(phi, phi)))
    M = ops.bond_matrix()
    idx = {int(st): k for k, st in enumerate(states)}
    C = np.zeros((N, N))
    for i in range(N):
        for j in range(N):
            bi, bj = N - 1 - i, N - 1 - j
            out = np.zeros_like(phi)
            for k, st in enumerate(states):
                st = int(st)
                if i == j:
                    out[k] += 0.75 * phi[k]     # S_i . S_i = s(s+1) = 3/4
                    continue
                a = 2 * ((st >> bi) & 1) + ((st >> bj) & 1)
                for ap in range(4):
                    m = M[ap, a]
                    if m == 0:
                        continue
                    t = st & ~((1 << bi) | (1 << bj))
                    t |= ((ap >> 1) & 1) << bi
                    t |= (ap & 1) << bj
                    out[idx[t]] += m * phi[k]
            C[i, j] = float(np.real(np.vdot(phi, out))) / nrm
    return C


def triangle_expectation(sector, psi: np.ndarray, tri) -> float:
    """<phi|S_i . (S_j x S_k)|phi> / <phi|phi> for the ordered triangle (i, j, k),
    phi written out as in `correlation_matrix`, the scalar triple product
    applied through the 8x8 matrix of its definition (ops.chirality_matrix).
    N <= 20."""
    N = sec_N(sector)
    states = sz_states(N, sector.n_up)
    V, kept = projector_matrix(sector, states)
    phi = V @ np.asarray(psi, dtype=complex)
    M = ops.chirality_matrix()
    idx = {int(st): k for k, st in enumerate(states)}
    bits = [N - 1 - int(x) for x in tri]
    out = np.zeros_like(phi)
    for k, st in enumerate(states):
        st = int(st)
        a = 4 * ((st >> bits[0]) & 1) + 2 * ((st >> bits[1]) & 1) + ((st >> bits[2]) & 1)
        for ap in range(8):
            m = M[ap, a]
            if m == 0:
                continue
            t = st & ~((1 << bits[0]) | (1 << bits[1]) | (1 << bits[2]))
            t |= ((ap >> 2) & 1) << bits[0]
            t |= ((ap >> 1) & 1) << bits[1]
            t |= (ap & 1) << bits[2]
            out[idx[t]] += m * phi[k]
    return float(np.real(np.vdot(phi, out))) / float(np.real(np.vdot(phi, phi)))


def plain_state(sector, psi: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """(phi, states): the symmetric-basis state psi written out in the fixed-Sz
    product basis, phi = sum_c psi_c v_c with the explicit projections v_c of
    `projector_matrix` (Eq. symmetryadaptedwavefunction1d).  N <= 20."""
    states = sz_states(sec_N(sector), sector.n_up)
    V, _ = projector_matrix(sector, states)
    assert V.shape[1] == len(psi)
    return V @ np.asarray(psi, dtype=complex), states


def restrict(sector, psi: np.ndarray, sub_sector) -> np.ndarray:
    """Coefficients of the state of `psi` on the normalised projections of a
    subgroup's sector: V_H^dagger (V_G psi), both written out by
    `projector_matrix`.  N <= 20."""
    phi, states = plain_state(sector, psi)
    Vh, _ = projector_matrix(sub_sector, states)
    return Vh.conj().T @ phi


def _apply_local(N: int, states: np.ndarray, idx: dict, phi: np.ndarray, sites, M: np.ndarray) -> np.ndarray:
    """O phi for the operator with matrix M on `sites` (row/column index: the
    sites' bits, first site most significant) and the identity elsewhere."""
    bits = [N - 1 - int(x) for x in sites]
    k = len(bits)
    mask = 0
    for b in bits:
        mask |= 1 << b
    out = np.zeros_like(phi)
    for c, st in enumerate(states):
        st = int(st)
        a = 0
        for b in bits:
            a = (a << 1) | ((st >> b) & 1)
        for ap in range(1 << k):
            m = M[ap, a]
            if m == 0:
                continue
            t = st & ~mask
            for l, b in enumerate(bits):
                t |= ((ap >> (k - 1 - l)) & 1) << b
            out[idx[t]] += m * phi[c]
    return out


def product_expectation(sector, psi: np.ndarray, first, second) -> complex:
    """<phi| O_1 O_2 |phi> / <phi|phi> for two local operators, each given as
    ("bond", (i, j)) for S_i . S_j (ops.bond_matrix) or ("tri", (i, j, k)) for
    S_i . (S_j x S_k) (ops.chirality_matrix), phi written out as in
    `plain_state`.  Computed as <O_1 phi | O_2 phi> (O_1 is Hermitian)."""
    phi, states = plain_state(sector, psi)
    N = sec_N(sector)
    idx = {int(st): k for k, st in enumerate(states)}
    mats = {"bond": ops.bond_matrix(), "tri": ops.chirality_matrix()}
    u = _apply_local(N, states, idx, phi, first[1], mats[first[0]])
    v = _apply_local(N, states, idx, phi, second[1], mats[second[0]])
    return complex(np.vdot(u, v) / np.vdot(phi, phi))


def nematic(sector, psi: np.ndarray, bond, bonds) -> complex:
    """Eq. nematicorderparameter: sum over the bonds (i, j) of `bonds` (the
    bonds parallel to `bond`) of <(S_a.S_b)(S_i.S_j)> - <S_a.S_b><S_i.S_j>,
    each term computed directly on the written-out state.  Complex: the
    imaginary part of a sum over a whole translation class vanishes."""
    phi, states = plain_state(sector, psi)
    N = sec_N(sector)
    idx = {int(st): k for k, st in enumerate(states)}
    M = ops.bond_matrix()
    nrm = np.vdot(phi, phi)
    u = _apply_local(N, states, idx, phi, bond, M)
    ea = np.vdot(phi, u) / nrm
    total = 0j
    for b in bonds:
        v = _apply_local(N, states, idx, phi, b, M)
        total += np.vdot(u, v) / nrm - ea * (np.vdot(phi, v) / nrm)
    return complex(total)


def chirality_sum(sector, psi: np.ndarray, tri, tris) -> complex:
    """Eq. chiralityorderparameter: sum over the triangles t of `tris` of
    <chi_tri chi_t>, chi_(i,j,k) = S_i . (S_j x S_k), computed directly."""
    phi, states = plain_state(sector, psi)
    N = sec_N(sector)
    idx = {int(st): k for k, st in enumerate(states)}
    M = ops.chirality_matrix()
    nrm = np.vdot(phi, phi)
    u = _apply_local(N, states, idx, phi, tri, M)
    return complex(sum(np.vdot(u, _apply_local(N, states, idx, phi, t, M)) for t in tris) / nrm)


def sz_spectrum(problem, psi: np.ndarray, c) -> tuple[np.ndarray, np.ndarray, float]:
    """(poles E_n - E_0, weights |<n|O|0>|^2, E_0) for O = sum_i c_i S^z_i and
    the state |0> of `psi` in problem.sector (normalised here), from the
    eigenvectors of the dense fixed-Sz matrix (`dense_sz`).  The dynamical
    structure factor is sum_n w_n delta(w - pole_n); E_0 = <0|H|0>.  N <= 14."""
    phi, states = plain_state(problem.sector, psi)
    phi = phi / np.linalg.norm(phi)
    N = sec_N(problem.sector)
    c = np.asarray(c, dtype=complex)
    f = np.array([sum(c[i] * (0.5 if (int(s) >> (N - 1 - i)) & 1 else -0.5) for i in range(N)) for s in states])
    Hd, _ = dense_sz(problem)
    e0 = float(np.real(np.vdot(phi, Hd @ phi)))
    w, v = np.linalg.eigh(Hd)
    amp = v.conj().T @ (f * phi)
    return w - e0, np.abs(amp) ** 2, e0


def lorentzians(poles, weights, omegas, eta: float) -> np.ndarray:
    """sum_n w_n (eta/pi) / ((w - pole_n)^2 + eta^2) at each frequency w."""
    om = np.asarray(omegas, dtype=np.float64)[:, None]
    return (np.asarray(weights)[None, :] * (eta / np.pi) / ((om - np.asarray(poles)[None, :]) ** 2 + eta * eta)).sum(1)


def evolve(H, psi: np.ndarray, t: float) -> np.ndarray:
    """exp(-i H t) psi for the oracle's sparse matrix H (scipy's expm_multiply,
    the truncated Taylor method of Al-Mohy and Higham, as a library step)."""
    import scipy.sparse.linalg as sla
    return sla.expm_multiply(-1j * t * sp.csr_matrix(H), np.asarray(psi, dtype=complex))


def sec_N(sector) -> int:
    return int(sector.n_sites)


# --------------------------------------------------------------------------
# dimensions by the character formula
# --------------------------------------------------------------------------
def _fixed_count(perm_row, flip: int, n_up: int) -> int:
    """Number of popcount-n_up states fixed by one element, from its cycle structure."""
    N = len(perm_row)
    seen = [False] * N
    cycles = []
    for i in range(N):
        if seen[i]:
            continue
        L = 0
        j = i
        while not seen[j]:
            seen[j] = True
            j = int(perm_row[j])
            L += 1
        cycles.append(L)
    poly = np.zeros(N + 1, dtype=object)
    poly[0] = 1
    for L in cycles:
        new = np.zeros(N + 1, dtype=object)
        if flip:
            # spins alternate along the cycle: needs even length, two choices, L/2 up
            if L % 2:
                return 0
            for d in range(N + 1):
                if poly[d] and d + L // 2 <= N:
                    new[d + L // 2] += 2 * poly[d]
        else:
            for d in range(N + 1):
                if poly[d]:
                    new[d] += poly[d]
                    if d + L <= N:
                        new[d + L] += poly[d]
        poly = new
    return int(poly[n_up])


def sector_dim_formula(sector) -> int:
    """dim = (1/|G|) sum_g conj(chi(g)) Fix(g)  (Eq. characterformula for a 1-D irrep)."""
    tot = 0j
    for g in range(sector.n_sym):
        tot += np.conj(sector.chi[g]) * _fixed_count(sector.perm[g], int(sector.spinflip[g]), sector.n_up)
    d = tot / sector.n_sym
    r = int(round(d.real))
    if abs(d - r) > 1e-6:
        raise ValueError(f"non-integer dimension {d}")
    return r


def lowest_eigs(H, k: int = 1, tol: float = 1e-13) -> np.ndarray:
    """Lowest k eigenvalues: LAPACK for D <= 4000, ARPACK otherwise."""
    D = H.shape[0]
    if D <= 4000:
        A = H.toarray() if sp.issparse(H) else H
        return np.linalg.eigvalsh(A)[:k]
    import scipy.sparse.linalg as sla
    w = sla.eigsh(H, k=k, which="SA", tol=tol, return_eigenvectors=False, ncv=max(2 * k + 20, 40))
    return np.sort(w.real)[:k]


def binom(N: int, k: int) -> int:
    return comb(N, k)

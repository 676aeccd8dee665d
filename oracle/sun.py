"""CPU oracle for SU(N) exchange models in the d-ary encoding -- TEST
INFRASTRUCTURE ONLY (only tests/ use it; it shares no code with the CUDA
library).

What it computes, from the thesis:
  * a configuration of N sites with colours sigma_k in {0, ..., d-1} is the
    integer sum_k sigma_k d^(N-k), site 1 most significant (Eq.
    numberforspinconfig with local dimension d) -- `integer`, `digits`;
  * the colourings with given numbers of each colour, in increasing order
    (the SU(N) analogue of a fixed S^z sector) -- `states`;
  * the group acts actively on sites (the colour on site i moves to site
    perm[g][i]); the representative is the orbit's smallest integer (Eq.
    representativecondition), found by applying every element -- `rep`;
  * the basis: colourings that are their own representative with a non-zero
    projector sum_g conj(chi(g)) g (Eq. symmetryadaptedwavefunction1d) --
    `basis`;
  * H = sum_<ij> J_ij P_ij with P_ij the exchange of the colours of sites i and
    j (Eq. sunexchangeop; the model of Eq. sunheisenbergringex without the ring
    term) in that basis, with the element of Eq.
    matrixelementrepresentatives and the conj(chi) reading -- `csr`;
  * the same H on all colourings, without symmetry -- `dense`;
  * sector dimensions by the character formula (Eq. characterformula):
    dim = (1/|G|) sum_g conj(chi(g)) Fix(g), Fix(g) the colourings with the
    given counts that are constant on every cycle of g -- `sector_dim_formula`;
  * the library's packed form of a colouring (ceil(log2 d) bits per site,
    site 1 most significant; the same order as the d-ary integers) -- `packed`;
  * matrix-free rows of H for sampled representatives -- `rows`.
"""
from __future__ import annotations

from math import factorial

import numpy as np
import scipy.sparse as sp


def digits(state: int, N: int, d: int) -> list[int]:
    """Colours of sites 1..N (most significant first) of a d-ary integer."""
    out = [0] * N
    for k in range(N - 1, -1, -1):
        out[k] = state % d
        state //= d
    return out


def integer(dig, d: int) -> int:
    """sum_k sigma_k d^(N-k)."""
    v = 0
    for c in dig:
        v = v * d + int(c)
    return v


def states(N: int, d: int, counts) -> list[int]:
    """All colourings with counts[c] sites of colour c, as increasing d-ary integers
    (site by site from the most significant, colours in increasing order: the
    lexicographic order of the digit strings is the order of the integers)."""
    assert sum(int(c) for c in counts) == N
    left = [int(c) for c in counts]
    out, cur = [], []

    def extend():
        if len(cur) == N:
            out.append(integer(cur, d))
            return
        for c in range(d):
            if left[c]:
                left[c] -= 1
                cur.append(c)
                extend()
                cur.pop()
                left[c] += 1

    extend()
    return out


def apply(sector, g: int, state: int) -> int:
    """Integer of g applied to the colouring `state`: the colour on site i moves to perm[g][i]."""
    N, d = int(sector.n_sites), int(sector.n_colors)
    dig = digits(state, N, d)
    out = [0] * N
    for i in range(N):
        out[int(sector.perm[g][i])] = dig[i]
    return integer(out, d)


def rep(sector, state: int):
    """(representative, first minimising element, |Stab(rep)|, sum of chi over Stab(rep))."""
    G = sector.n_sym
    imgs = [apply(sector, g, state) for g in range(G)]
    r = min(imgs)
    g0 = imgs.index(r)
    stab = [h for h in range(G) if apply(sector, h, r) == r]
    return r, g0, len(stab), complex(sum(sector.chi[h] for h in stab))


def basis(sector):
    """Sorted representatives with a non-zero projector, and |Stab|."""
    out, st = [], []
    for s in states(sector.n_sites, sector.n_colors, sector.counts):
        r, g, n, ssum = rep(sector, int(s))
        if r == int(s) and abs(ssum) > 1e-9:
            out.append(r)
            st.append(n)
    return out, np.array(st, dtype=np.int64)


def _swap(state: int, N: int, d: int, i: int, j: int):
    dig = digits(state, N, d)
    if dig[i] == dig[j]:
        return None
    dig[i], dig[j] = dig[j], dig[i]
    return integer(dig, d)


def csr(problem, reps=None, stab=None) -> sp.csr_matrix:
    """H = sum_b J_b P_(i_b j_b) in the symmetric basis (complex128): column sigma~,
    image tau = P_ij sigma~ (or sigma~ itself when the colours agree) contributes
    J conj(chi(g_tau)) sqrt(|Stab tau~| / |Stab sigma~|) at row tau~."""
    sec, terms = problem.sector, problem.terms
    N, d = int(sec.n_sites), int(sec.n_colors)
    if reps is None:
        reps, stab = basis(sec)
    index = {int(r): i for i, r in enumerate(reps)}
    rows, cols, vals = [], [], []
    cache = {}
    for c, s in enumerate(reps):
        s = int(s)
        for (i, j), J in zip(terms.bonds, terms.J):
            t = _swap(s, N, d, int(i), int(j))
            if t is None:  # equal colours: P_ij acts as the identity
                rows.append(c)
                cols.append(c)
                vals.append(complex(J))
                continue
            if t not in cache:
                cache[t] = rep(sec, t)
            r, g, n, ssum = cache[t]
            if abs(ssum) < 1e-9:
                continue
            rows.append(index[r])
            cols.append(c)
            vals.append(J * np.conj(sec.chi[g]) * np.sqrt(n / stab[c]))
    D = len(reps)
    H = sp.coo_matrix((np.array(vals, dtype=complex), (rows, cols)), shape=(D, D)).tocsr()
    H.sum_duplicates()
    return H


def dense(problem):
    """H on all colourings with the sector's counts (no symmetry), and those colourings."""
    sec, terms = problem.sector, problem.terms
    N, d = int(sec.n_sites), int(sec.n_colors)
    st = states(N, d, sec.counts)
    index = {int(s): k for k, s in enumerate(st)}
    H = np.zeros((len(st), len(st)))
    for c, s in enumerate(st):
        s = int(s)
        for (i, j), J in zip(terms.bonds, terms.J):
            t = _swap(s, N, d, int(i), int(j))
            H[index[s if t is None else t], c] += J
    return H, st


def projector_matrix(sector, st):
    """Columns: normalised projections sum_g conj(chi(g)) g|sigma> (one per orbit with a
    non-zero projection), ordered by orbit minimum, phase fixed so that the coefficient
    on the minimum is real positive."""
    index = {int(s): k for k, s in enumerate(st)}
    seen, cols, kept = set(), [], []
    for s in st:
        s = int(s)
        if s in seen:
            continue
        orbit = [apply(sector, g, s) for g in range(sector.n_sym)]
        seen.update(orbit)
        v = np.zeros(len(st), dtype=complex)
        for g, t in enumerate(orbit):
            v[index[t]] += np.conj(sector.chi[g])
        nrm = np.linalg.norm(v)
        if nrm > 1e-9:
            cols.append(v / nrm)
            kept.append(min(orbit))
    order = np.argsort(kept)
    V = np.array(cols).T[:, order] if cols else np.zeros((len(st), 0))
    kept = [kept[i] for i in order]
    for c, m in enumerate(kept):
        ph = V[index[m], c]
        V[:, c] *= np.conj(ph) / abs(ph)
    return V, kept


def _fixed_count(perm_row, counts) -> int:
    """Colourings with the given counts that are constant on every cycle of the permutation:
    the coefficient of prod_c x_c^counts[c] in prod_cycles (sum_c x_c^len)."""
    N = len(perm_row)
    seen = [False] * N
    lens = []
    for i in range(N):
        if seen[i]:
            continue
        L, j = 0, i
        while not seen[j]:
            seen[j] = True
            j = int(perm_row[j])
            L += 1
        lens.append(L)
    poly = {tuple(0 for _ in counts): 1}
    for L in lens:
        new = {}
        for key, v in poly.items():
            for c in range(len(counts)):
                k2 = list(key)
                k2[c] += L
                if k2[c] <= counts[c]:
                    new[tuple(k2)] = new.get(tuple(k2), 0) + v
        poly = new
    return poly.get(tuple(int(c) for c in counts), 0)


def sector_dim_formula(sector) -> int:
    """dim = (1/|G|) sum_g conj(chi(g)) Fix(g) (Eq. characterformula for a 1-D irrep)."""
    tot = 0j
    for g in range(sector.n_sym):
        tot += np.conj(sector.chi[g]) * _fixed_count(sector.perm[g], [int(c) for c in sector.counts])
    v = tot / sector.n_sym
    r = int(round(v.real))
    if abs(v - r) > 1e-6:
        raise ValueError(f"non-integer dimension {v}")
    return r


def multinomial(counts) -> int:
    n = factorial(int(sum(counts)))
    for c in counts:
        n //= factorial(int(c))
    return n


def packed(state: int, N: int, d: int) -> int:
    """The library's packed colouring: site k's colour in bits [(N-1-k) b, (N-k) b), b = ceil(log2 d)."""
    b = max(1, int(np.ceil(np.log2(d))))
    v = 0
    for c in digits(state, N, d):
        v = (v << b) | int(c)
    return v


def rows(problem, reps, x_of):
    """Matrix-free rows for given representatives sigma~ (d-ary integers of compatible
    representatives): y(sigma~) = sum_j H[sigma~, j] x_j with H[i, j] = conj(H[j, i])
    (H Hermitian), the column of sigma~ formed as in `csr`, and x_j = x_of(tau~) for the
    representative tau~ (a d-ary integer) of index j."""
    sec, terms = problem.sector, problem.terms
    N, d = int(sec.n_sites), int(sec.n_colors)
    out = np.zeros(len(reps), dtype=complex)
    for q, s in enumerate(reps):
        s = int(s)
        r0, g0, n0, s0 = rep(sec, s)
        assert r0 == s and abs(s0) > 1e-9
        acc = 0j
        for (i, j), J in zip(terms.bonds, terms.J):
            t = _swap(s, N, d, int(i), int(j))
            if t is None:
                acc += J * x_of(s)
                continue
            r, g, n, ssum = rep(sec, t)
            if abs(ssum) < 1e-9:
                continue
            acc += np.conj(J * np.conj(sec.chi[g]) * np.sqrt(n / n0)) * x_of(r)
        out[q] = acc
    return out

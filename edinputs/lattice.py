"""Finite periodic clusters, their symmetry groups and 1-D irrep characters.

This module only states *the problem*: sites, bonds, triangles, the site
permutations of the space group (times an optional spin flip), the
characters of a one-dimensional irrep, and a sublattice-stable site
numbering.  It contains none of the exact-diagonalization arithmetic
(no representatives, no matrix elements); both the CUDA library and the
CPU oracle consume its output as plain arrays.

Conventions (thesis chapter "Large-Scale Exact Diagonalization"):
  * site s <-> bit (N-1-s) of the state integer, spin up = 1
    (Eq. numberforspinconfig: site 1 is the most significant digit);
  * the group acts actively: the spin on site i moves to site perm[g][i];
  * a space-group element is g = T_t R with R a point-group operation about
    the lattice's symmetry centre and t a Bravais translation; its character
    in the sector (k, rho_k) is exp(i k.t) chi_rho(R) (App. A, Eq. spacechars);
  * the direct product with spin flip multiplies characters (Eq. tensorchar);
  * sites are numbered so that sublattice X occupies the contiguous block
    [X*m, (X+1)*m) with sublattice 0 in the most significant bits
    (sublattice-coding section, "Generic sublattice coding algorithm").
"""
from __future__ import annotations

import itertools
import math
from dataclasses import dataclass, field

import numpy as np

_TOL = 1e-8


# --------------------------------------------------------------------------
# infinite lattices
# --------------------------------------------------------------------------
@dataclass
class Lattice:
    name: str
    A: np.ndarray            # rows: primitive vectors (Cartesian)
    basis: np.ndarray        # rows: basis-site offsets (Cartesian), origin at the point-group centre
    n_fold: int              # principal rotation order of the lattice's point group (4 or 6; 2 for a chain)

    @property
    def n_basis(self) -> int:
        return len(self.basis)


def square_lattice() -> Lattice:
    return Lattice("square", np.eye(2), np.zeros((1, 2)), 4)


def triangular_lattice() -> Lattice:
    A = np.array([[1.0, 0.0], [0.5, math.sqrt(3) / 2]])
    return Lattice("triangular", A, np.zeros((1, 2)), 6)


def kagome_lattice() -> Lattice:
    # Bravais vectors of length 2, sites at 0, A1/2, A2/2; origin moved to the
    # hexagon centre (A1+A2)/2 so that C6 and all reflections fix it.
    A = np.array([[2.0, 0.0], [1.0, math.sqrt(3)]])
    b = np.array([[0.0, 0.0], A[0] / 2, A[1] / 2]) - (A[0] + A[1]) / 2
    return Lattice("kagome", A, b, 6)


def chain_lattice() -> Lattice:
    # A 1-D chain embedded in 2-D with a huge rung so only x-bonds appear.
    return Lattice("chain", np.array([[1.0, 0.0], [0.0, 1000.0]]), np.zeros((1, 2)), 2)


def _point_ops(n_fold: int, chain: bool) -> list[tuple[str, np.ndarray, int, float]]:
    """Candidate orthogonal operations: (label, O, order-or-(-1 for mirror), angle)."""
    ops = []
    if chain:
        ops.append(("E", np.eye(2), 1, 0.0))
        ops.append(("sx", np.diag([-1.0, 1.0]), -1, math.pi / 2))
        return ops
    for k in range(n_fold):
        th = 2 * math.pi * k / n_fold
        c, s = math.cos(th), math.sin(th)
        ops.append((f"C{n_fold}^{k}" if k else "E", np.array([[c, -s], [s, c]]), k, th))
    for k in range(n_fold):
        ax = math.pi * k / n_fold  # mirror axis angle
        c, s = math.cos(2 * ax), math.sin(2 * ax)
        ops.append((f"m{k}", np.array([[c, s], [s, -c]]), -1, ax))
    return ops


# --------------------------------------------------------------------------
# finite clusters
# --------------------------------------------------------------------------
class Cluster:
    """Torus of a lattice spanned by integer periodicity vectors P (rows, lattice coords)."""

    def __init__(self, lattice: Lattice, P):
        self.lat = lattice
        self.P = np.array(P, dtype=np.int64)
        d = int(round(abs(np.linalg.det(self.P))))
        if d == 0:
            raise ValueError("degenerate periodicity vectors")
        self.n_cells = d
        cells = set()
        R = int(np.abs(self.P).sum()) + 2
        for a in range(-R, R + 1):
            for b in range(-R, R + 1):
                cells.add(self.reduce_cell((a, b)))
        self.cells = sorted(cells)
        if len(self.cells) != d:
            raise RuntimeError("cell enumeration failed")
        self.N = d * lattice.n_basis
        # default (unordered) site list: (cell, s)
        self.site_list = [(c, s) for c in self.cells for s in range(lattice.n_basis)]
        self.site_index = {cs: i for i, cs in enumerate(self.site_list)}
        self.pos = np.array([np.array(c) @ lattice.A + lattice.basis[s] for c, s in self.site_list])

    # integer cell reduction modulo the periodicity lattice
    def _hnf(self):
        """Row Hermite normal form [[a, b], [0, c]] of the periodicity lattice."""
        (p11, p12), (p21, p22) = self.P.tolist()
        def egcd(x, y):
            if y == 0:
                return (abs(x), 1 if x >= 0 else -1, 0)
            g, s, t = egcd(y, x % y)
            return (g, t, s - (x // y) * t)
        g, x, y = egcd(p11, p21)
        if g == 0:
            raise ValueError("degenerate periodicity vectors")
        r1 = (x * p11 + y * p21, x * p12 + y * p22)
        r2 = ((p21 // g) * p11 - (p11 // g) * p21, (p21 // g) * p12 - (p11 // g) * p22)
        a, c = r1[0], abs(r2[1])
        if a < 0:
            r1 = (-r1[0], -r1[1]); a = -a
        b = r1[1] % c
        return a, b, c, r1

    def reduce_cell(self, n):
        if not hasattr(self, "_h"):
            self._h = self._hnf()
        a, b, c, r1 = self._h
        n1, n2 = int(n[0]), int(n[1])
        q = n1 // a
        n1 -= q * r1[0]
        n2 -= q * r1[1]
        n2 %= c
        return (n1, n2)

    def locate(self, r: np.ndarray):
        """Site index at Cartesian position r (modulo the torus), or None."""
        Ainv = np.linalg.inv(self.lat.A)
        for s in range(self.lat.n_basis):
            f = (r - self.lat.basis[s]) @ Ainv
            fi = np.round(f)
            if np.all(np.abs(f - fi) < 1e-6):
                return self.site_index[(self.reduce_cell(fi.astype(np.int64)), s)]
        return None

    def cart_periods(self) -> np.ndarray:
        return self.P.astype(float) @ self.lat.A

    # ---------------- bonds -------------------------------------------------
    def neighbour_shells(self, n_shells: int):
        """Displacements from each basis site to the first n_shells distance shells."""
        lat = self.lat
        R = 6
        out = []  # per basis site: list of (dist, displacement)
        dists = set()
        for s in range(lat.n_basis):
            lst = []
            for a in range(-R, R + 1):
                for b in range(-R, R + 1):
                    for t in range(lat.n_basis):
                        d = np.array([a, b]) @ lat.A + lat.basis[t] - lat.basis[s]
                        L = float(np.hypot(*d))
                        if L < 1e-9:
                            continue
                        lst.append((L, d))
                        dists.add(round(L, 6))
            out.append(lst)
        shells = sorted(dists)[:n_shells]
        return shells, out

    def bonds(self, shell: int):
        """All bonds of the given distance shell (1 = nearest neighbours).

        Each bond appears once per lattice displacement, so bonds that wrap
        around the torus twice are counted twice (as in the infinite lattice).
        """
        shells, disp = self.neighbour_shells(shell)
        target = shells[shell - 1]
        out = []
        for i, (c, s) in enumerate(self.site_list):
            for L, d in disp[s]:
                if abs(round(L, 6) - target) > 1e-6:
                    continue
                j = self.locate(self.pos[i] + d)
                if j is None:
                    raise RuntimeError("neighbour not on lattice")
                if j == i:
                    raise ValueError("cluster too small: bond maps a site onto itself")
                if i < j:
                    out.append((i, j))
        return out

    def bonds_across_hexagons(self):
        """Kagome third neighbours across the hexagons (Eq. chiralhamiltonian's
        J3 term): pairs at twice the nearest-neighbour distance whose midpoint
        is a hexagon centre, not a site (the other pairs at that distance run
        along a line of sites through their middle site)."""
        shells, disp = self.neighbour_shells(1)
        d1 = shells[0]
        out = []
        for i, (c, s) in enumerate(self.site_list):
            for L, d in disp[s]:
                if abs(L - 2 * d1) > 1e-6:
                    continue
                if self.locate(self.pos[i] + d / 2) is not None:
                    continue
                j = self.locate(self.pos[i] + d)
                if j is None:
                    raise RuntimeError("neighbour not on lattice")
                if j == i:
                    raise ValueError("cluster too small: bond maps a site onto itself")
                if i < j:
                    out.append((i, j))
        return out

    def triangles(self):
        """Elementary nearest-neighbour triangles, vertices counter-clockwise."""
        shells, disp = self.neighbour_shells(1)
        d1 = shells[0]
        seen = set()
        out = []
        for i, (c, s) in enumerate(self.site_list):
            nn = [d for L, d in disp[s] if abs(L - d1) < 1e-6]
            for u, v in itertools.permutations(nn, 2):
                if abs(np.hypot(*(u - v)) - d1) > 1e-6:
                    continue
                if u[0] * v[1] - u[1] * v[0] <= 0:
                    continue  # keep the counter-clockwise ordering (i, i+u, i+v)
                cen = self.pos[i] + (u + v) / 3.0
                key = self._point_key(cen)
                if key in seen:
                    continue
                seen.add(key)
                j = self.locate(self.pos[i] + u)
                k = self.locate(self.pos[i] + v)
                out.append((i, j, k))
        return out

    def _point_key(self, r):
        f = r @ np.linalg.inv(self.lat.A)
        fp = f @ np.linalg.inv(self.P.astype(float))
        fp = fp - np.floor(fp + 1e-9)
        return tuple(np.round(fp, 6) % 1.0)

    # ---------------- symmetry ----------------------------------------------
    def point_group(self):
        """Point operations about the origin that map the infinite lattice and the torus onto themselves."""
        lat = self.lat
        res = []
        Ainv = np.linalg.inv(lat.A)
        Pc = self.cart_periods()
        Pinv = np.linalg.inv(Pc)
        for label, O, order, ang in _point_ops(lat.n_fold, lat.name == "chain"):
            ok = True
            for v in lat.A:
                f = (O @ v) @ Ainv
                if np.any(np.abs(f - np.round(f)) > 1e-6):
                    ok = False
            for b in lat.basis:
                if self._lattice_site_type(O @ b) is None:
                    ok = False
            for p in Pc:
                f = (O @ p) @ Pinv
                if np.any(np.abs(f - np.round(f)) > 1e-6):
                    ok = False
            if ok:
                res.append((label, O, order, ang))
        return res

    def _lattice_site_type(self, r):
        Ainv = np.linalg.inv(self.lat.A)
        for s in range(self.lat.n_basis):
            f = (r - self.lat.basis[s]) @ Ainv
            if np.all(np.abs(f - np.round(f)) < 1e-6):
                return s
        return None


# --------------------------------------------------------------------------
# symmetry groups and characters
# --------------------------------------------------------------------------
@dataclass
class SpaceGroup:
    perm: np.ndarray                 # [G][N] active permutation
    trans: np.ndarray                # [G][2] Cartesian translation part t
    pidx: np.ndarray                 # [G] index into point ops
    point_ops: list                  # (label, O, order, angle)


def space_group(cl: Cluster, point: str = "full", translations: bool = True) -> SpaceGroup:
    """All g = T_t R of the torus as site permutations.

    point: "full" (every point operation found), "rot" (proper rotations only),
           "none" (identity only), or an explicit list of operation labels.
    """
    ops = cl.point_group()
    if point == "none":
        ops = [o for o in ops if o[0] == "E"]
    elif point == "rot":
        ops = [o for o in ops if o[2] >= 0]
    elif isinstance(point, (list, tuple)):
        ops = [o for o in ops if o[0] in point]
    cells = cl.cells if translations else [(0, 0)]
    perms, trans, pidx = [], [], []
    seen = set()
    for oi, (label, O, order, ang) in enumerate(ops):
        for c in cells:
            t = np.array(c) @ cl.lat.A
            p = []
            for i in range(cl.N):
                j = cl.locate(O @ cl.pos[i] + t)
                if j is None:
                    raise RuntimeError("point operation does not map the lattice")
                p.append(j)
            key = tuple(p)
            if key in seen:
                continue
            seen.add(key)
            perms.append(p)
            trans.append(t)
            pidx.append(oi)
    perm = np.array(perms, dtype=np.int32)
    # identity first
    ident = np.arange(cl.N)
    k0 = [i for i in range(len(perm)) if np.array_equal(perm[i], ident)][0]
    order = [k0] + [i for i in range(len(perm)) if i != k0]
    return SpaceGroup(perm[order], np.array(trans)[order], np.array(pidx)[order], ops)


def one_d_irreps(ops) -> list[tuple[str, np.ndarray]]:
    """All one-dimensional irreps of a finite point group given as matrices.

    Found by brute force over assignments of roots of unity to the elements
    that are consistent with the multiplication table.  Returns
    (name, chi[op]) with Mulliken-style names: A/B by the character of the
    principal rotation (E<l> when complex), subscript 1/2 by the character of
    the mirror whose axis is at angle 0 when there is one.
    """
    mats = [o[1] for o in ops]
    n = len(mats)

    def find(M):
        for i, X in enumerate(mats):
            if np.allclose(X, M, atol=1e-8):
                return i
        raise RuntimeError("not closed")

    mul = np.array([[find(mats[a] @ mats[b]) for b in range(n)] for a in range(n)])
    # element orders
    e = find(np.eye(2))
    exps = []
    for a in range(n):
        k, x = 1, a
        while x != e:
            x = mul[x, a]
            k += 1
        exps.append(k)
    ex = int(np.lcm.reduce(exps))
    roots = [np.exp(2j * np.pi * q / ex) for q in range(ex)]
    # generators by greedy closure
    gens = []
    span = {e}
    for a in range(n):
        if a in span:
            continue
        gens.append(a)
        span = {e}
        frontier = [e]
        while frontier:
            x = frontier.pop()
            for g in gens:
                y = mul[x, g]
                if y not in span:
                    span.add(y)
                    frontier.append(y)
    chars = []
    for assign in itertools.product(range(ex), repeat=len(gens)):
        val = {e: 1.0 + 0j}
        frontier = [e]
        ok = True
        while frontier and ok:
            x = frontier.pop()
            for g, q in zip(gens, assign):
                y = mul[x, g]
                v = val[x] * roots[q]
                if y in val:
                    if abs(val[y] - v) > 1e-8:
                        ok = False
                        break
                else:
                    val[y] = v
                    frontier.append(y)
        if not ok or len(val) != n:
            continue
        chi = np.array([val[i] for i in range(n)])
        # full homomorphism check
        if all(abs(chi[mul[a, b]] - chi[a] * chi[b]) < 1e-8 for a in range(n) for b in range(n)):
            if not any(np.allclose(chi, c) for _, c in chars):
                chars.append(("", chi))
    # names
    rot = [i for i, o in enumerate(ops) if o[2] >= 0]
    prin = max(rot, key=lambda i: (exps[i], -ops[i][3])) if rot else e
    mir0 = [i for i, o in enumerate(ops) if o[2] == -1 and abs(o[3]) < 1e-9]
    if not mir0:
        mir0 = [i for i, o in enumerate(ops) if o[2] == -1]
    named = []
    for _, chi in chars:
        c = chi[prin]
        if abs(c - 1) < 1e-8:
            base = "A"
        elif abs(c + 1) < 1e-8:
            base = "B"
        else:
            l = int(round(np.angle(c) / (2 * np.pi / exps[prin]))) % exps[prin]
            base = f"E{l}"
        if mir0:
            base += "1" if abs(chi[mir0[0]] - 1) < 1e-8 else "2"
        named.append((base, chi))
    named.sort(key=lambda x: x[0])
    return named


@dataclass
class Sector:
    """One symmetry sector as plain arrays (the library's ed_sector)."""
    n_sites: int
    n_up: int
    perm: np.ndarray       # int32 [G][N]
    spinflip: np.ndarray   # uint8 [G]
    chi: np.ndarray        # complex128 [G]
    n_sublat: int
    label: str = ""

    @property
    def n_sym(self) -> int:
        return len(self.perm)

    @property
    def is_real(self) -> bool:
        return bool(np.all(np.abs(self.chi.imag) < 1e-12))


@dataclass
class SectorSUN:
    """One symmetry sector of an SU(N) model (the library's ed_sector_sun): sites
    carry one of n_colors colours, colour c occurs counts[c] times (the SU(N)
    analogue of a fixed S^z), and the group permutes sites (no colour change)."""
    n_sites: int
    n_colors: int
    counts: np.ndarray     # int32 [n_colors], summing to n_sites
    perm: np.ndarray       # int32 [G][N]
    chi: np.ndarray        # complex128 [G]
    n_sublat: int
    label: str = ""

    @property
    def n_sym(self) -> int:
        return len(self.perm)

    @property
    def is_real(self) -> bool:
        return bool(np.all(np.abs(self.chi.imag) < 1e-12))

    @property
    def bits(self) -> int:
        """Bits per site of the packed colour string: ceil(log2 n_colors)."""
        return max(1, int(np.ceil(np.log2(self.n_colors))))


@dataclass
class Terms:
    """Hamiltonian H = sum_b J_b S_i.S_j + sum_t Jchi_t S_i.(S_j x S_k)."""
    bonds: np.ndarray      # int32 [nb][2]
    J: np.ndarray          # float64 [nb]
    tris: np.ndarray       # int32 [nt][3] counter-clockwise
    Jchi: np.ndarray       # float64 [nt]

    @property
    def is_real(self) -> bool:
        return len(self.tris) == 0 or bool(np.all(self.Jchi == 0))

    def relabel(self, new_of_old: np.ndarray) -> "Terms":
        return Terms(new_of_old[self.bonds].astype(np.int32) if len(self.bonds) else self.bonds,
                     self.J, new_of_old[self.tris].astype(np.int32) if len(self.tris) else self.tris,
                     self.Jchi)


@dataclass
class Problem:
    name: str
    sector: Sector
    terms: Terms
    meta: dict = field(default_factory=dict)


# --------------------------------------------------------------------------
# sublattice decomposition and site ordering
# --------------------------------------------------------------------------
def _hnf_sublattices(index: int):
    """Integer lattices L' of Z^2 with [Z^2 : L'] = index, as HNF row bases."""
    out = []
    for a in range(1, index + 1):
        if index % a:
            continue
        c = index // a
        for b in range(a):
            out.append(np.array([[a, 0], [b, c]], dtype=np.int64))
    return out


def _in_lattice(v, B):
    f = np.array(v, dtype=float) @ np.linalg.inv(B.astype(float))
    return np.all(np.abs(f - np.round(f)) < 1e-6)


def sublattice_partitions(cl: Cluster, sg: SpaceGroup):
    """Candidate sublattice-stable partitions as lists of site blocks.

    A block is (coset of an invariant sub-Bravais lattice L', basis-site class);
    basis sites are either kept apart or merged.  Only partitions that every
    group element maps block-to-block are returned.
    """
    cands = []
    Ainv = np.linalg.inv(cl.lat.A)
    ops_used = sorted(set(sg.pidx.tolist()))
    for d in range(1, cl.n_cells + 1):
        if cl.n_cells % d:
            continue
        for B in _hnf_sublattices(d):
            if not all(_in_lattice(p, B) for p in cl.P):
                continue
            ok = True
            for oi in ops_used:
                O = sg.point_ops[oi][1]
                for v in B:
                    w = (O @ (v @ cl.lat.A)) @ Ainv
                    if not _in_lattice(np.round(w), B):
                        ok = False
            if not ok:
                continue
            for merge in (False, True):
                key = {}
                for i, (c, s) in enumerate(cl.site_list):
                    f = np.array(c, dtype=float) @ np.linalg.inv(B.astype(float))
                    f = f - np.floor(f + 1e-9)
                    coset = tuple(np.round(f, 6) % 1.0)
                    key[i] = (coset, 0 if merge else s)
                labels = sorted(set(key.values()))
                blocks = [[i for i in range(cl.N) if key[i] == lab] for lab in labels]
                if len({len(b) for b in blocks}) != 1:
                    continue
                if _stable(blocks, sg.perm):
                    cands.append(blocks)
    return cands


def _stable(blocks, perm) -> bool:
    where = {}
    for X, b in enumerate(blocks):
        for i in b:
            where[i] = X
    for p in perm:
        for b in blocks:
            if len({where[int(p[i])] for i in b}) != 1:
                return False
    return True


def _local_map_count(blocks, perm, flip) -> int:
    """Distinct (local position map, flip) pairs induced on the blocks by the group."""
    m = len(blocks[0])
    N = sum(len(b) for b in blocks)
    order = [i for b in blocks for i in b]
    new_of_old = np.empty(N, dtype=np.int64)
    new_of_old[order] = np.arange(N)
    pn = new_of_old[perm[:, order]]
    seen = set()
    for g in range(len(pn)):
        for X in range(len(blocks)):
            Z = pn[g, X * m] // m
            seen.add((tuple((pn[g, X * m:(X + 1) * m] - Z * m).tolist()), int(flip[g])))
    return len(seen)


def choose_partition(cands, perm, flip, max_table_bytes: int, max_block: int = 12):
    """Fewest sublattices (largest blocks, fewest representative candidates) whose
    SymmetryAction tables, stored once per distinct local map, fit the budget.

    A map costs 2^m bytes for m <= 8, else two uint16 chunk tables of
    2^(m - m//2) + 2^(m//2) entries."""
    best = None
    for blocks in cands:
        n_sub = len(blocks)
        m = len(blocks[0])
        if m > max_block:
            continue
        per_map = (1 << m) if m <= 8 else 2 * ((1 << (m - m // 2)) + (1 << (m // 2)))
        n_map = _local_map_count(blocks, perm, flip)
        size = n_map * per_map
        if size > max_table_bytes:
            continue
        key = (n_sub, size)
        if best is None or key < best[0]:
            best = (key, blocks)
    if best is None:
        raise ValueError("no sublattice partition fits the table budget")
    return best[1]


# --------------------------------------------------------------------------
# problem assembly
# --------------------------------------------------------------------------
def _snap_roots(chi: np.ndarray) -> np.ndarray:
    """Characters of 1-D irreps are roots of unity; exp(i k.t) evaluated in
    floating point carries errors of ~1e-14 (|k.t| up to tens of radians).
    Components within 1e-12 of 0, +-1/2 or +-1 are set to those values, so
    real characters are exactly +-1 and e.g. exp(2 pi i/3) = -1/2 + i sqrt(3)/2."""
    def snap(v):
        for c in (0.0, 0.5, -0.5, 1.0, -1.0):
            if abs(v - c) < 1e-12:
                return c
        return v
    return np.array([complex(snap(z.real), snap(z.imag)) for z in np.asarray(chi, dtype=complex)])


def build_problem(name: str, cl: Cluster, *, J: dict, Jchi: float = 0.0, J3_hex: float = 0.0, n_up: int | None = None,
                  point: str = "full", translations: bool = True, k=(0.0, 0.0), irrep: str = "A1",
                  spinflip: int | None = None, max_table_bytes: int = 96 * 1024,
                  n_sublat: int | None = None) -> Problem:
    """Assemble a sector of a cluster.

    J: {shell: coupling}.  J3_hex: coupling of the kagome third neighbours
    across the hexagons.  k: Cartesian momentum.  irrep: name of a 1-D irrep
    of the little group of k.  spinflip: None (no flip), +1 (even), -1 (odd).
    """
    N = cl.N
    if n_up is None:
        n_up = N // 2
    sg = space_group(cl, point=point, translations=translations)
    k = np.array(k, dtype=float)
    # little group of k: R^T-invariance modulo reciprocal Bravais vectors
    Bt = 2 * np.pi * np.linalg.inv(cl.lat.A).T  # rows: reciprocal vectors
    little = []
    for oi, (label, O, order, ang) in enumerate(sg.point_ops):
        dk = O @ k - k
        f = dk @ np.linalg.inv(Bt)
        if np.all(np.abs(f - np.round(f)) < 1e-6):
            little.append(oi)
    # momentum must be compatible with the torus
    for p in cl.cart_periods():
        ph = k @ p / (2 * np.pi)
        if abs(ph - round(ph)) > 1e-6:
            raise ValueError("momentum not allowed on this cluster")
    keep = np.isin(sg.pidx, little)
    perm = sg.perm[keep]
    trans = sg.trans[keep]
    pidx = sg.pidx[keep]
    lops = [sg.point_ops[i] for i in little]
    irr = one_d_irreps(lops)
    names = [n for n, _ in irr]
    if irrep not in names:
        raise ValueError(f"irrep {irrep} not among 1-D irreps {names} of the little group")
    chi_p = dict(zip(little, dict(irr)[irrep]))
    chi = _snap_roots(np.array([np.exp(1j * (k @ t)) * chi_p[int(pi)] for t, pi in zip(trans, pidx)]))
    flip = np.zeros(len(perm), dtype=np.uint8)
    if spinflip is not None:
        if 2 * n_up != N:
            raise ValueError("spin flip needs Sz = 0")
        perm = np.concatenate([perm, perm])
        flip = np.concatenate([flip, np.ones_like(flip)])
        chi = np.concatenate([chi, chi * float(spinflip)])
    sgk = SpaceGroup(perm, np.concatenate([trans] * (2 if spinflip is not None else 1)),
                     np.concatenate([pidx] * (2 if spinflip is not None else 1)), sg.point_ops)
    # terms in the cluster's native numbering
    bonds, Js = [], []
    for shell, Jv in sorted(J.items()):
        if Jv == 0:
            continue
        for b in cl.bonds(shell):
            bonds.append(b)
            Js.append(Jv)
    if J3_hex != 0.0:
        for b in cl.bonds_across_hexagons():
            bonds.append(b)
            Js.append(J3_hex)
    tris, Jc = [], []
    if Jchi != 0.0:
        for t in cl.triangles():
            tris.append(t)
            Jc.append(Jchi)
    terms = Terms(np.array(bonds, dtype=np.int32).reshape(-1, 2), np.array(Js, dtype=np.float64),
                  np.array(tris, dtype=np.int32).reshape(-1, 3), np.array(Jc, dtype=np.float64))
    # sublattice ordering
    cands = sublattice_partitions(cl, sgk)
    if n_sublat is not None:
        cands = [c for c in cands if len(c) == n_sublat]
    # blocks of up to 12 sites by default; an explicit block count may use up
    # to 16 (the library's limit; such tables are read from global memory)
    blocks = choose_partition(cands, perm, flip, max_table_bytes, max_block=16 if n_sublat is not None else 12)
    order = [i for b in blocks for i in b]         # new site -> old site
    new_of_old = np.empty(N, dtype=np.int64)
    new_of_old[order] = np.arange(N)
    perm_new = new_of_old[perm[:, order]].astype(np.int32)
    sector = Sector(N, n_up, perm_new, flip, chi, len(blocks), label=f"{name}")
    # elements that are pure translations (no point operation, no spin flip)
    tset = {tuple(r) for r in space_group(cl, point="none", translations=True).perm.tolist()}
    translations = [g for g in range(len(perm)) if not flip[g] and tuple(perm[g].tolist()) in tset]
    tri_all = np.array(cl.triangles(), dtype=np.int64).reshape(-1, 3)
    meta = dict(k=k.tolist(), irrep=irrep, spinflip=spinflip, n_cells=cl.n_cells,
                n_basis=cl.lat.n_basis, point_ops=[o[0] for o in lops], positions=cl.pos[order].tolist(),
                translations=translations, triangles=new_of_old[tri_all].astype(np.int32).tolist())
    return Problem(name, sector, terms.relabel(new_of_old), meta)


# --------------------------------------------------------------------------
# all sectors of a cluster
# --------------------------------------------------------------------------
def allowed_momenta(cl: Cluster) -> list[np.ndarray]:
    """Momenta k with k.p in 2 pi Z for the periodicity vectors, one per class
    modulo the reciprocal Bravais lattice (as many as unit cells)."""
    Pc = cl.cart_periods()
    Pinv = np.linalg.inv(Pc)
    Bt = 2 * np.pi * np.linalg.inv(cl.lat.A).T
    Btinv = np.linalg.inv(Bt)
    out = []
    R = cl.n_cells
    for n1 in range(-R, R + 1):
        for n2 in range(-R, R + 1):
            k = 2 * np.pi * (Pinv @ np.array([n1, n2], dtype=float))
            f = k @ Btinv
            f = f - np.floor(f + 1e-9)
            kk = f @ Bt
            if not any(np.allclose(kk, q, atol=1e-8) for q in out):
                out.append(kk)
    if len(out) != cl.n_cells:
        raise RuntimeError("momentum enumeration failed")
    return out


def little_group_irreps(cl: Cluster, k, point: str = "full") -> list[str]:
    """Names of the 1-D irreps of the little group of k (within the chosen point group)."""
    sg = space_group(cl, point=point, translations=True)
    sg.point_ops = [sg.point_ops[i] for i in sorted(set(sg.pidx.tolist()))]
    k = np.asarray(k, dtype=float)
    Bt = 2 * np.pi * np.linalg.inv(cl.lat.A).T
    little = []
    for oi, (label, O, order, ang) in enumerate(sg.point_ops):
        f = (O @ k - k) @ np.linalg.inv(Bt)
        if np.all(np.abs(f - np.round(f)) < 1e-6):
            little.append(sg.point_ops[oi])
    return [n for n, _ in one_d_irreps(little)]

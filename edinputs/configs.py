"""Named synthetic workloads shaped like the thesis's ED benchmarks.

The thesis's clusters exist only in its (missing) figures, so each workload is
a concrete periodic cluster chosen here; its periodicity vectors are stated in
the docstring of each function.
"""
from __future__ import annotations

import math

import numpy as np

from .lattice import (Cluster, Problem, SectorSUN, Terms, build_problem, chain_lattice, kagome_lattice,
                      square_lattice, triangular_lattice)

PI = math.pi


def chain(N: int, J1: float = 1.0, J2: float = 0.0, *, translations=False, reflection=False,
          k: int = 0, irrep: str = "A1", spinflip=None, n_up=None, n_sublat=None, max_table_bytes=96 * 1024):
    """Periodic chain of N sites; momentum 2*pi*k/N."""
    cl = Cluster(chain_lattice(), [[N, 0], [0, 1]])
    J = {1: J1}
    if J2:
        J[2] = J2
    point = "full" if reflection else "none"
    if not reflection and irrep == "A1":
        irrep = "A"
    return build_problem(f"chain{N}", cl, J=J, n_up=n_up, point=point, translations=translations,
                         k=(2 * PI * k / N, 0.0), irrep=irrep, spinflip=spinflip, n_sublat=n_sublat,
                         max_table_bytes=max_table_bytes)


def square(P, J1=1.0, J2=0.0, *, k=(0.0, 0.0), irrep="A1", point="full", spinflip=None, n_up=None,
           n_sublat=None, max_table_bytes=96 * 1024, translations=True):
    cl = Cluster(square_lattice(), P)
    J = {1: J1}
    if J2:
        J[2] = J2
    return build_problem(f"square{cl.N}", cl, J=J, n_up=n_up, point=point, k=k, irrep=irrep,
                         spinflip=spinflip, n_sublat=n_sublat, max_table_bytes=max_table_bytes,
                         translations=translations)


def triangular(P, J1=1.0, J2=0.0, *, k=(0.0, 0.0), irrep="A1", point="full", spinflip=None, n_up=None,
               n_sublat=None, max_table_bytes=96 * 1024, translations=True):
    cl = Cluster(triangular_lattice(), P)
    J = {1: J1}
    if J2:
        J[2] = J2
    return build_problem(f"triangular{cl.N}", cl, J=J, n_up=n_up, point=point, k=k, irrep=irrep,
                         spinflip=spinflip, n_sublat=n_sublat, max_table_bytes=max_table_bytes,
                         translations=translations)


def kagome(P, J1=1.0, J2=0.0, Jchi=0.0, *, J3=0.0, k=(0.0, 0.0), irrep="A", point="rot", spinflip=None,
           n_up=None, n_sublat=None, max_table_bytes=96 * 1024, translations=True):
    """Kagome cluster (Eq. chiralhamiltonian: J1, J2, J3 across the hexagons, J_chi on
    every triangle); the scalar chirality breaks mirrors, so the default point group is C6."""
    cl = Cluster(kagome_lattice(), P)
    J = {1: J1}
    if J2:
        J[2] = J2
    return build_problem(f"kagome{cl.N}", cl, J=J, Jchi=Jchi, J3_hex=J3, n_up=n_up, point=point, k=k, irrep=irrep,
                         spinflip=spinflip, n_sublat=n_sublat, max_table_bytes=max_table_bytes,
                         translations=translations)


# ---------------------------------------------------------------------------
# the five workloads
# ---------------------------------------------------------------------------
def chain16():
    """Heisenberg chain N=16, periodic, J1=1, Sz=0, no spatial symmetry (dim 12870)."""
    return chain(16, 1.0)


def square32(irrep="A1", momentum="Gamma", n_sublat=2):
    """32-site tilted square cluster a1=(4,4), a2=(4,-4); J1=1, J2=0.5; T32 x C4v, Sz=0.
    Two sublattice blocks of 16 sites (the checkerboard) by default: 8-site
    blocks have a 64-element block group acting on 256 substates, so images
    typically have 4-16 representative candidates; 16-site blocks have 1-2."""
    k = (0.0, 0.0) if momentum == "Gamma" else (PI, PI)
    return square([[4, 4], [4, -4]], 1.0, 0.5, k=k, irrep=irrep, n_sublat=n_sublat, max_table_bytes=4 << 20)


def kagome36(spinflip=1, irrep="A"):
    """36-site kagome, Bravais a1=2A1+2A2, a2=-2A1+4A2 (12 cells); J1=1, J2=0.2, Jchi=0.3
    on every triangle; T12 x C6 x Z2 (144 elements), Gamma sector, Sz=0."""
    return kagome([[2, 2], [-2, 4]], 1.0, 0.2, 0.3, irrep=irrep, spinflip=spinflip)


def triangular24(k=(0.0, 0.0), irrep="A1"):
    """24-site triangular torus a1=(5,1), a2=(4,-4) in lattice coordinates; J1=1, J2=0.125.

    No 24-site triangular torus has a sixfold axis (24 is not a^2+ab+b^2); this
    one keeps the largest point group available at N=24, C2v, so T24 x C2v = 96.
    """
    return triangular([[5, 1], [4, -4]], 1.0, 0.125, k=k, irrep=irrep)


def square40(spinflip=1, irrep="A"):
    """40-site square cluster a1=(6,2), a2=(-2,6); J1=1, J2=0.55; T40 x C4 x Z2 (320)."""
    return square([[6, 2], [-2, 6]], 1.0, 0.55, irrep=irrep, point="full", spinflip=spinflip)


def all_sectors(kind: str, P, J1=1.0, J2=0.0, *, n_sublat: int, n_up=None, point="full", max_table_bytes=96 * 1024):
    """Every (k, rho_k) sector of a square or triangular torus: each allowed
    momentum with every 1-D irrep of its little group.  Sectors share one site
    numbering (the sublattice count is fixed)."""
    from .lattice import allowed_momenta, little_group_irreps
    lat = {"square": square_lattice, "triangular": triangular_lattice}[kind]()
    make = {"square": square, "triangular": triangular}[kind]
    cl = Cluster(lat, P)
    out = []
    for k in allowed_momenta(cl):
        for irr in little_group_irreps(cl, k, point=point):
            p = make(P, J1, J2, k=tuple(k), irrep=irr, n_sublat=n_sublat, n_up=n_up, point=point,
                     max_table_bytes=max_table_bytes)
            p.meta["sector"] = f"k=({k[0]:.3f},{k[1]:.3f}) {irr}"
            out.append(p)
    return out


def triangular24_sectors(J2=0.125, max_table_bytes=96 * 1024):
    """Every (k, rho_k) sector of the 24-site triangular torus (a1=(5,1), a2=(4,-4)),
    J1=1, J2=0.125, Sz=0: 24 momenta, each with the 1-D irreps of its little
    group inside C2v (36 sectors).  Every sector uses the same site numbering
    (2 blocks of 12 sites)."""
    return all_sectors("triangular", [[5, 1], [4, -4]], 1.0, J2, n_sublat=2, max_table_bytes=max_table_bytes)


# ---------------------------------------------------------------------------
# SU(N) models: H = sum_<ij> J_ij P_ij with P_ij the exchange of the colours
# of sites i and j (the thesis's SU(N) Heisenberg model, chapter on the SU(N)
# chiral spin liquid), colours in the d-ary encoding of Eq. numberforspinconfig
# ---------------------------------------------------------------------------
def sun(kind: str, P, n_colors: int, counts, J1: float = 1.0, J2: float = 0.0, *, k=(0.0, 0.0), irrep=None,
        point="full", n_sublat: int, translations=True):
    """SU(n_colors) exchange model on a chain, square or triangular cluster with
    periodicity P (for a chain P = [[N, 0], [0, 1]]); `counts` colours of each
    kind.  The site numbering is sublattice-stable with n_sublat blocks (the
    library packs a site into ceil(log2 n_colors) bits, and a block must fit 16
    bits)."""
    lat = {"chain": chain_lattice, "square": square_lattice, "triangular": triangular_lattice}[kind]()
    cl = Cluster(lat, P)
    J = {1: J1}
    if J2:
        J[2] = J2
    if irrep is None:
        irrep = "A" if (kind == "chain" and point == "none") else "A1"
    if kind == "chain" and point == "none" and irrep == "A1":
        irrep = "A"
    spin = build_problem(f"{kind}{cl.N}_su{n_colors}", cl, J=J, point=point, k=k, irrep=irrep, n_sublat=n_sublat,
                         translations=translations, max_table_bytes=1 << 30)
    counts = np.asarray(counts, dtype=np.int32)
    if len(counts) != n_colors or int(counts.sum()) != cl.N:
        raise ValueError("counts must give one number per colour, summing to the number of sites")
    s = spin.sector
    sec = SectorSUN(cl.N, n_colors, counts, s.perm, s.chi, s.n_sublat, label=spin.name)
    terms = Terms(spin.terms.bonds, spin.terms.J, np.zeros((0, 3), np.int32), np.zeros(0))
    return Problem(spin.name, sec, terms, dict(spin.meta, counts=counts.tolist(), n_colors=n_colors))


def sun_chain(N: int, n_colors: int, counts, J1=1.0, J2=0.0, *, k: int = 0, reflection=False, n_sublat=2,
              irrep=None):
    """SU(n_colors) chain of N sites, periodic, momentum 2 pi k / N (with the reflection
    when `reflection`, irrep of the little group as named by one_d_irreps)."""
    return sun("chain", [[N, 0], [0, 1]], n_colors, counts, J1, J2, k=(2 * PI * k / N, 0.0),
               point="full" if reflection else "none", n_sublat=n_sublat, irrep=irrep)


def sun_triangular21():
    """SU(3) Heisenberg model (J1 = 1) on the 21-site triangular torus a1=(4,1), a2=(-1,5)
    (21 = 4^2 + 4 + 1: the torus keeps the sixfold axis but, being chiral, no mirror),
    7 sites of each colour, Gamma, fully symmetric irrep of T21 x C6 (126 elements);
    three blocks of 7 sites (14 bits each)."""
    return sun("triangular", [[4, 1], [-1, 5]], 3, [7, 7, 7], 1.0, 0.0, irrep="A", n_sublat=3)

"""Checks of the problem generator (clusters, groups, characters, site ordering)."""
import numpy as np
import pytest

from edinputs import configs as C
from edinputs.lattice import Cluster, kagome_lattice, one_d_irreps, triangular_lattice


def _closed(perm):
    S = {tuple(p) for p in perm}
    for a in perm:
        for b in perm:
            if tuple(a[b]) not in S:  # (a o b)[i] = a[b[i]]
                return False
    return True


@pytest.mark.parametrize("make", [C.chain16, C.square32, C.kagome36, C.triangular24, C.square40])
def test_workload_groups(make):
    p = make()
    s = p.sector
    N = s.n_sites
    assert np.array_equal(s.perm[0], np.arange(N)) and s.spinflip[0] == 0
    assert abs(s.chi[0] - 1) < 1e-12
    # group closure and character homomorphism on the (perm, flip) pairs
    key = {(tuple(p_), int(f)): g for g, (p_, f) in enumerate(zip(s.perm, s.spinflip))}
    G = s.n_sym
    rng = np.random.default_rng(0)
    pairs = [(a, b) for a in range(G) for b in range(G)] if G <= 64 else \
        [tuple(x) for x in rng.integers(0, G, size=(4000, 2))]
    for a, b in pairs:
        comp = (tuple(s.perm[a][s.perm[b]]), int(s.spinflip[a] ^ s.spinflip[b]))
        assert comp in key
        assert abs(s.chi[key[comp]] - s.chi[a] * s.chi[b]) < 1e-9
    # bonds and triangles map onto themselves
    bonds = {tuple(sorted(b)) for b in p.terms.bonds.tolist()}
    for g in range(G):
        pm = s.perm[g]
        assert {tuple(sorted((pm[i], pm[j]))) for i, j in bonds} == bonds
    # sublattice stability of the contiguous blocks
    m = N // s.n_sublat
    for g in range(G):
        for X in range(s.n_sublat):
            dest = {int(s.perm[g][i]) // m for i in range(X * m, (X + 1) * m)}
            assert len(dest) == 1


def test_workload_sizes():
    assert C.chain16().sector.n_sym == 1
    assert C.square32().sector.n_sym == 256 and len(C.square32().terms.bonds) == 128
    k = C.kagome36()
    assert k.sector.n_sym == 144 and len(k.terms.tris) == 24 and len(k.terms.bonds) == 144
    assert C.triangular24().sector.n_sym == 96
    assert C.square40().sector.n_sym == 320


def test_d6_character_table():
    """1-D irreps of the hexagonal point group reproduce rows A1, A2, B1, B2 of Tab. d6chartable.

    Classes of the table: 1, 2C6, 2C3, C2, 3 sigma_d, 3 sigma_v.  The two mirror
    classes are told apart by which of them contains the mirror along a1; the
    table's B1/B2 rows differ only by that assignment, so the set of rows is
    compared with both mirror classes kept separate."""
    cl = Cluster(triangular_lattice(), [[2, 2], [-2, 4]])
    ops = cl.point_group()
    assert len(ops) == 12
    irr = one_d_irreps(ops)
    assert len(irr) == 4
    lab = [o[0] for o in ops]
    c6 = lab.index("C6^1")
    c3 = lab.index("C6^2")
    c2 = lab.index("C6^3")
    mA = lab.index("m0")   # mirror axis at 0 degrees
    mB = lab.index("m1")   # mirror axis at 30 degrees (the other class)
    rows = {tuple(np.round([chi[0], chi[c6], chi[c3], chi[c2], chi[mA], chi[mB]], 9).real) for _, chi in irr}
    table = {(1, 1, 1, 1, 1, 1), (1, 1, 1, 1, -1, -1), (1, -1, 1, -1, 1, -1), (1, -1, 1, -1, -1, 1)}
    assert rows == {tuple(float(v) for v in r) for r in table}
    # class structure: the mirrors at 0 and 60 degrees are conjugate
    m2 = lab.index("m2")
    for _, chi in irr:
        assert abs(chi[mA] - chi[m2]) < 1e-12


def test_kagome_triangles_orientation():
    cl = Cluster(kagome_lattice(), [[2, 0], [0, 2]])
    tris = cl.triangles()
    assert len(tris) == 2 * cl.n_cells
    for i, j, k in tris:
        u = cl.pos[j] - cl.pos[i]
        v = cl.pos[k] - cl.pos[i]
        # minimal images
        assert u[0] * v[1] - u[1] * v[0] != 0


def test_square32_all_sectors_partition_the_sz0_space():
    """Every (k, rho_k) sector of the 32-site square cluster under translations x C4
    (1-D irreps of each little group; C4v's 2-D irrep E appears through the C4 characters
    +-i, i.e. complex sectors): the character-formula dimensions add up to C(32, 16)."""
    import oracle
    ps = C.all_sectors("square", [[4, 4], [4, -4]], 1.0, 0.5, n_sublat=4, point="rot")
    assert sum(oracle.sector_dim_formula(p.sector) for p in ps) == oracle.binom(32, 16)
    assert any(not p.sector.is_real for p in ps)

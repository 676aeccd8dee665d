"""The largest state word: N = 64 sites, so every bit of the 64-bit word is a
site (site 0 is bit 63).  Ring of 64 sites with J1 = 1, J2 = 0.3 and
translations (8 sublattice blocks of 8 sites), one to three up spins.

Against the oracle: the basis bit-exact, the representative search on random
states (half of them with site 0, the sign bit of the word, up), H.x element
by element within the FP64 bound, and the Lanczos ground energy.
"""
import numpy as np
import pytest

import oracle
from edinputs import configs as C
from edinputs.vectors import state_vector

pytestmark = pytest.mark.gpu

EPS64 = np.finfo(np.float64).eps


@pytest.fixture(scope="module")
def P():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2210_03511_gb300 import build
    build.build()
    import paper_2210_03511_gb300 as pkg
    return pkg


@pytest.mark.parametrize("k,n_up", [(0, 2), (5, 2), (0, 3)])
def test_chain64(P, k, n_up):
    import torch
    p = C.chain(64, 1.0, 0.3, translations=True, k=k, n_up=n_up)
    assert p.sector.n_sites == 64
    reps, stab = oracle.basis(p.sector)
    b = P.Basis(p.sector)
    greps, gstab = b.export()
    assert np.array_equal(greps, reps) and np.array_equal(gstab.astype(np.int32), stab)
    rng = np.random.default_rng(64 + k + n_up)
    states = []
    for t in range(200):
        sites = rng.choice(64, n_up, replace=False)
        if t % 2 == 0 and 0 not in sites:
            sites[0] = 0
        states.append(sum(1 << (63 - int(s)) for s in sites))
    states = np.array(states, dtype=np.uint64)
    assert np.any(states >> np.uint64(63))
    rep, g, ns, cp = P.representatives(p.sector, states)
    for i, st in enumerate(states):
        r0, g0, n0, ssum = oracle.rep(p.sector, int(st))
        assert int(rep[i]) == r0 and ns[i] == n0 and bool(cp[i]) == (abs(ssum) > 1e-9)
    H = oracle.csr(p, reps, stab)
    h = P.Hamiltonian(b, p.terms)
    cplx = not h.is_real
    X = state_vector(7, reps, complex_=cplx)
    x = torch.tensor(X, dtype=torch.complex128 if cplx else torch.float64, device="cuda")
    y = torch.empty_like(x)
    h.apply(x, y)
    torch.cuda.synchronize()
    bound = 64 * EPS64 * (abs(H) @ np.abs(X)) + 1e-300
    assert np.all(np.abs(y.cpu().numpy() - H @ X) <= bound)
    e_ref = np.linalg.eigvalsh(H.toarray())[0]
    vals, _ = h.lanczos(n_eig=1, tol=1e-12, max_iter=300)
    assert vals[0] == pytest.approx(e_ref, abs=1e-10 * max(1.0, abs(e_ref)))

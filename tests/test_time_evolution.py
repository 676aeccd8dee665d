"""Krylov time evolution psi <- exp(-i H dt) psi (ed_time_evolve).

CPU: the oracle's propagator (scipy's expm_multiply on its sparse matrix) is
pinned to closed forms: an eigenvector only acquires the phase exp(-i E t);
two sites prepared in |up down> oscillate into |down up> with probability
sin^2(J t / 2) (the singlet and triplet split by J); the norm is conserved.

GPU: repeated Krylov steps against the oracle on the same start vector,
for a real Hamiltonian with complex vectors and a complex (chiral) one.
Tolerance: the steps' own error estimates are below 1e-12 for m = 30 and
dt = 0.2; the comparison allows 1e-9 (rounding of ~30 FP64 steps of
|H| ~ 10 and of the oracle's Taylor method).
"""
import numpy as np
import pytest

import oracle
from edinputs import configs as C
from edinputs.lattice import Sector, Terms
from edinputs.vectors import state_vector


def test_oracle_eigenvector_phase():
    p = C.chain(10, 1.0, 0.3, translations=True)
    reps, stab = oracle.basis(p.sector)
    H = oracle.csr(p, reps, stab)
    w, v = np.linalg.eigh(H.toarray())
    for k in (0, 3):
        out = oracle.evolve(H, v[:, k], 0.7)
        assert np.allclose(out, np.exp(-1j * w[k] * 0.7) * v[:, k], atol=1e-12)


def test_oracle_two_site_oscillation():
    s = Sector(2, 1, np.array([[0, 1]], np.int32), np.zeros(1, np.uint8), np.ones(1, complex), 1)
    t = Terms(np.array([[0, 1]], np.int32), np.array([1.0]), np.zeros((0, 3), np.int32), np.zeros(0))

    class Prob:
        sector, terms = s, t
    H = oracle.csr(Prob)
    psi0 = np.array([0.0, 1.0])          # basis |01>, |10>: start in |10> (site 0 up)
    for tt in (0.3, 1.1, 2.5):
        out = oracle.evolve(H, psi0, tt)
        assert abs(out[0]) ** 2 == pytest.approx(np.sin(tt / 2) ** 2, abs=1e-12)
        assert np.linalg.norm(out) == pytest.approx(1.0, abs=1e-12)


CASES = {
    "chain14": lambda: C.chain(14, 1.0, 0.4, translations=True, reflection=True, spinflip=-1, irrep="A2"),
    "kagome12_E1": lambda: C.kagome([[2, 0], [0, 2]], 1.0, 0.2, 0.3, irrep="E1"),
}


@pytest.mark.gpu
@pytest.mark.parametrize("name", sorted(CASES))
def test_gpu_krylov_steps_match_oracle(name):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2210_03511_gb300 import build
    build.build()
    import paper_2210_03511_gb300 as P
    p = CASES[name]()
    reps, stab = oracle.basis(p.sector)
    H = oracle.csr(p, reps, stab)
    b = P.Basis(p.sector)
    h = P.Hamiltonian(b, p.terms)
    X = state_vector(13, reps, complex_=True)
    X = X / np.linalg.norm(X)
    psi = torch.tensor(X, dtype=torch.complex128, device="cuda")
    e_start = np.real(h.expectation(psi)[0])
    ref = X.copy()
    for step in range(5):
        err, mu = h.evolve(psi, 0.2, m=30)
        assert err < 1e-12 and mu == 30
        ref = oracle.evolve(H, ref, 0.2)
    got = psi.cpu().numpy()
    assert np.abs(got - ref).max() < 1e-9, np.abs(got - ref).max()
    assert np.linalg.norm(got) == pytest.approx(1.0, abs=1e-12)
    assert np.real(h.expectation(psi)[0]) == pytest.approx(e_start, abs=1e-10)
    # an invariant subspace: an eigenvector takes a pure phase with a short Krylov space
    ev = torch.zeros((1, b.dim), dtype=torch.complex128, device="cuda")
    vals, _ = h.lanczos(n_eig=1, tol=1e-13, max_iter=300, evecs=ev, dtype=P.ED_C128)
    v0 = ev[0].clone()
    h.evolve(ev[0], 0.5, m=30)
    ph = torch.vdot(v0, ev[0]).item()
    assert abs(ph - np.exp(-1j * vals[0] * 0.5)) < 1e-6

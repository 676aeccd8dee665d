"""Lanczos vectors of the plain recursion kept in host memory (host_vectors = 1)
or in device memory (host_vectors = 2): the Ritz vectors and the
mixed-precision refinement come from the stored vectors instead of a second
pass, with the same results (the second pass regenerates the same vectors bit
for bit)."""
import numpy as np
import pytest

import oracle
from edinputs import configs as C

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2210_03511_gb300 import build
    build.build()
    import paper_2210_03511_gb300 as pkg
    return pkg


@pytest.mark.parametrize("make", [lambda: C.chain(14, 1.0, 0.4, translations=True, reflection=True, spinflip=-1,
                                                  irrep="A2"),
                                  lambda: C.kagome([[2, 0], [0, 2]], 1.0, 0.2, 0.3, irrep="E1")])
def test_host_vectors_match_second_pass(P, make):
    import torch
    p = make()
    H = oracle.csr(p)
    ref = np.linalg.eigvalsh(H.toarray())[:2]
    b = P.Basis(p.sector)
    h = P.Hamiltonian(b, p.terms)
    h.store()
    real = h.is_real
    d64, d32 = (P.ED_F64, P.ED_F32) if real else (P.ED_C128, P.ED_C64)
    t64 = torch.float64 if real else torch.complex128
    out = {}
    for hv in (0, 1, 2):
        # mixed precision, plain recursion: refined energy
        ev, rep = h.lanczos(n_eig=1, tol=1e-10, max_iter=300, dtype=d32, reorth=False, refine=True, host_vectors=hv)
        assert abs(ev[0] - ref[0]) <= 1e-10 * abs(ref[0]), (hv, ev[0], ref[0])
        out[("mixed", hv)] = (ev[0], rep.n_apply)
        # FP64 eigenvectors from the plain recursion
        V = torch.empty((2, b.dim), dtype=t64, device="cuda")
        ev, rep = h.lanczos(n_eig=2, tol=1e-12, max_iter=300, dtype=d64, reorth=False, evecs=V, host_vectors=hv)
        assert np.all(np.abs(ev - ref) <= 1e-10 * np.abs(ref))
        out[("evec", hv)] = (V.cpu().numpy(), rep.n_apply, rep.iters)
        # each Ritz vector is an eigenvector of the oracle's matrix
        for k in range(2):
            v = out[("evec", hv)][0][k].astype(np.complex128)
            r = H @ v - ev[k] * v
            assert np.linalg.norm(r) <= 1e-6 * abs(ev[k]) * np.linalg.norm(v)
    for kept in (1, 2):
        assert out[("mixed", kept)][0] == pytest.approx(out[("mixed", 0)][0], rel=1e-13, abs=0)
        # no second pass: one H.x per step instead of two
        assert out[("evec", kept)][1] == out[("evec", kept)][2]
        assert np.allclose(out[("evec", kept)][0], out[("evec", 0)][0], rtol=0, atol=1e-9)
    assert out[("evec", 0)][1] > out[("evec", 0)][2]
    # the same vectors, whether kept on the host or on the device
    assert np.array_equal(out[("evec", 1)][0], out[("evec", 2)][0])

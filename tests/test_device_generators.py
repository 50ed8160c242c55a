"""The device ensemble generators (workloads/device.py), run on the CPU: the
Gram-Schmidt Haar draw gives the unique Q of Z = QR with a positive diagonal
R (the host recipe's factor: library QR, then R's diagonal phases folded into
Q), Q is unitary to working precision, and every ensemble has the shape,
dtype and symmetry its recipe states."""
import numpy as np
import pytest
import torch

from workloads.device import _q_positive_r, batch


@pytest.mark.parametrize("cplx", [True, False])
@pytest.mark.parametrize("n", [1, 2, 7, 23])
def test_gram_schmidt_equals_qr_with_positive_r(cplx, n):
    g = torch.Generator().manual_seed(100 + n)
    Z = torch.randn((64, n, n), generator=g, dtype=torch.float64)
    if cplx:
        Z = torch.complex(Z, torch.randn((64, n, n), generator=g, dtype=torch.float64))
    Q = _q_positive_r(Z)
    Qr, R = torch.linalg.qr(Z)
    d = torch.diagonal(R, dim1=-2, dim2=-1)
    Qref = Qr * (d / d.abs()).unsqueeze(-2)
    assert float((Q - Qref).abs().max()) < 1e-12
    eye = torch.eye(n, dtype=Q.dtype)
    assert float((Q.conj().transpose(-1, -2) @ Q - eye).abs().max()) < 1e-13
    # R = Q^H Z is upper triangular with a positive real diagonal
    Rq = Q.conj().transpose(-1, -2) @ Z
    assert float(torch.tril(Rq, diagonal=-1).abs().max()) < 1e-12 if n > 1 else True
    assert bool((torch.diagonal(Rq, dim1=-2, dim2=-1).real > 0).all())


def test_every_ensemble_shape_dtype_and_symmetry():
    for name, dt in (("haar_u", torch.complex128), ("haar_o", torch.float64), ("gue", torch.complex128),
                     ("goe", torch.float64), ("ginibre_c", torch.complex128), ("ginibre_r", torch.float64)):
        A = batch(name, 9, 16, seed=3, device="cpu")
        assert A.shape == (16, 9, 9) and A.dtype == dt and A.is_contiguous()
        again = batch(name, 9, 16, seed=3, device="cpu")
        assert torch.equal(A, again)                      # seeded
        if name in ("gue", "goe"):
            assert torch.equal(A, A.conj().transpose(-1, -2))
        if name.startswith("haar"):
            eye = torch.eye(9, dtype=dt)
            assert float((A.conj().transpose(-1, -2) @ A - eye).abs().max()) < 1e-13
    # complex Ginibre entries are CN(0, 1): E|a|^2 = 1, E a^2 = 0
    G = batch("ginibre_c", 16, 2000, seed=4, device="cpu").reshape(-1).numpy()
    assert abs(np.mean(np.abs(G) ** 2) - 1) < 0.01 and abs(np.mean(G ** 2)) < 0.01

"""The adjoint's matrix-free MINRES on CPU tensors (CPU only).

The implicit step of the adjoint solves A z = qbar with A = M + h^2 (hess Phi + H_c),
symmetric and, away from the converged state, possibly indefinite.  The matrix-free path
runs MINRES (Paige and Saunders, 1975) on Hessian-vector products.  Here the routine is
checked against a dense solve on symmetric matrices with known spectra.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _sym(rng, n, lam):
    Q, _ = np.linalg.qr(rng.normal(size=(n, n)))
    A = Q @ np.diag(lam) @ Q.T
    return 0.5 * (A + A.T)


@pytest.mark.parametrize("kind", ["spd", "indefinite", "clustered"])
def test_minres_matches_a_dense_solve(kind):
    from paper_2409_16385_gb300.adjoint import _minres
    rng = np.random.default_rng({"spd": 0, "indefinite": 1, "clustered": 2}[kind])
    n = 80
    lam = rng.uniform(1.0, 100.0, n)
    if kind == "indefinite":
        lam *= rng.choice([-1.0, 1.0], n)
    if kind == "clustered":
        lam = np.repeat([2.0, -5.0, 40.0], [30, 20, 30])      # converges in 3 iterations
    A = _sym(rng, n, lam)
    b = rng.normal(size=n)
    At, bt = torch.tensor(A), torch.tensor(b)
    calls = []

    def apply(v):
        calls.append(1)
        return At @ v

    x = _minres(apply, bt).numpy()
    xr = np.linalg.solve(A, b)
    assert np.abs(x - xr).max() <= 1e-10 * np.abs(xr).max()
    assert np.linalg.norm(A @ x - b) <= 1e-11 * np.linalg.norm(b)
    assert len(calls) <= 2 * n          # Lanczos loses orthogonality in floating point
    if kind == "clustered":
        assert len(calls) <= 4          # Krylov space of three distinct eigenvalues


def test_minres_zero_right_hand_side_and_shape():
    from paper_2409_16385_gb300.adjoint import _minres
    A = torch.eye(6, dtype=torch.float64) * 3.0
    b = torch.zeros((2, 3), dtype=torch.float64)
    x = _minres(lambda v: (A @ v.reshape(-1)).reshape(v.shape), b)
    assert x.shape == b.shape and float(x.abs().max()) == 0.0
    b = torch.arange(6, dtype=torch.float64).reshape(2, 3)
    x = _minres(lambda v: (A @ v.reshape(-1)).reshape(v.shape), b)
    assert torch.allclose(x, b / 3.0, rtol=1e-14, atol=0)

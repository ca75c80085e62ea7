"""The first-order (Daleckii-Krein) correction behind the eigensolvers' early stop, checked on
the CPU against an exact eigendecomposition: for A = Lambda + E with ||E||_F <= d / 4, d the
distance of diag(Lambda) from zero, V (f(Lambda) + L o E) V^H is within ||E||_F^2 / d (plus
rounding) of the PSD projection of V A V^H, f(x) = max(x, 0)."""
import numpy as np
import pytest


def _proj(A):
    w, V = np.linalg.eigh(A)
    return (V * np.maximum(w, 0)) @ V.conj().T


def _weight(li, lj):
    if li >= 0 and lj >= 0:
        return 1.0
    if li < 0 and lj < 0:
        return 0.0
    lp, lm = (li, lj) if li >= 0 else (lj, li)
    return lp / (lp - lm)


@pytest.mark.parametrize("complex_", [False, True])
def test_first_order_correction_meets_its_bound(complex_):
    rng = np.random.default_rng(20210604 + complex_)
    n, accepted = 16, 0
    for _ in range(400):
        lam = rng.normal(size=n)
        lam[rng.random(n) < 0.3] *= 10 ** rng.uniform(-4, -1)   # eigenvalues near zero
        E = rng.normal(size=(n, n)) + (1j * rng.normal(size=(n, n)) if complex_ else 0)
        E = 0.5 * (E + E.conj().T)
        np.fill_diagonal(E, 0)
        E *= 10 ** rng.uniform(-8, -2) / np.linalg.norm(E)
        d = np.min(np.abs(lam))
        if np.linalg.norm(E) > d / 4:
            continue
        accepted += 1
        Z = rng.normal(size=(n, n)) + (1j * rng.normal(size=(n, n)) if complex_ else 0)
        V, _ = np.linalg.qr(Z)
        L = np.array([[_weight(a, b) for b in lam] for a in lam])
        M = np.diag(np.maximum(lam, 0)) + L * E
        A = np.diag(lam) + E
        err = np.linalg.norm(V @ M @ V.conj().T - _proj(V @ A @ V.conj().T))
        assert err <= np.linalg.norm(E) ** 2 / d + 64 * n * 2.0 ** -53 * np.linalg.norm(A)
    assert accepted > 100

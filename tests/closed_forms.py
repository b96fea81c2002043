"""Closed-form spectra used as pins (not part of the method)."""
import numpy as np


def laplacian5_eigs(N: int, eps: float = 1.0) -> np.ndarray:
    """All eigenvalues of workloads.laplacian5(N, eps), ascending, in the
    cancellation-free form 4/h^2 [eps sin^2(k pi h / 2) + sin^2(l pi h / 2)]."""
    h = 1.0 / (N + 1)
    k = np.arange(1, N + 1)
    s = np.sin(k * np.pi * h / 2.0) ** 2
    lam = 4.0 * (N + 1) ** 2 * (eps * s[:, None] + s[None, :])
    return np.sort(lam.ravel())


def gradient_singular_values(N: int) -> np.ndarray:
    """Singular values of workloads.gradient(N): sqrt of the Laplacian's."""
    return np.sqrt(laplacian5_eigs(N))

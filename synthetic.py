"""Seeded synthetic inputs shaped like the paper's workloads.

This module is shared by the tests, the benchmark and the oracle's callers.  It holds no
arithmetic of the method itself: it only draws matrices.

Entries follow the random-matrix generator of Section 3.2 (eq. random-matrix-generation):
    a_ij = (rand - 0.5) * exp(phi * randn),
with rand uniform on [0, 1) and randn standard normal.  phi sets the spread of magnitudes.

Storage convention: every matrix is column-major (BLAS).  A column-major rows x cols matrix
with leading dimension ld = rows is held as a C-contiguous array of shape (cols, rows).
The helpers below return that array; `colmajor_view` turns it into the mathematical matrix.
"""
from __future__ import annotations

import numpy as np


def paper_matrix(rows: int, cols: int, phi: float, seed: int) -> np.ndarray:
    """Column-major rows x cols FP64 matrix from the paper's generator (host, numpy PCG64).

    Returns the storage array of shape (cols, rows), C-contiguous, so ld = rows.
    """
    g = np.random.Generator(np.random.PCG64(seed))
    u = g.random((cols, rows), dtype=np.float64)
    z = g.standard_normal((cols, rows), dtype=np.float64)
    return np.ascontiguousarray((u - 0.5) * np.exp(phi * z))


def paper_matrix_torch(rows: int, cols: int, phi: float, seed: int, device="cuda"):
    """Same distribution drawn on a torch device (Philox on CUDA), for sizes where host
    generation would be slow.  Storage shape (cols, rows), contiguous, so ld = rows."""
    import torch

    g = torch.Generator(device=device)
    g.manual_seed(seed)
    u = torch.rand((cols, rows), generator=g, dtype=torch.float64, device=device)
    z = torch.randn((cols, rows), generator=g, dtype=torch.float64, device=device)
    u.sub_(0.5)
    z.mul_(phi).exp_()
    u.mul_(z)
    return u


def ones_matrix(rows: int, cols: int, value: float = 1.0) -> np.ndarray:
    """All-equal column-major matrix (the all-ones example of Section 3.1), storage (cols, rows)."""
    return np.full((cols, rows), value, dtype=np.float64)


def colmajor_view(storage: np.ndarray) -> np.ndarray:
    """The mathematical rows x cols matrix of a column-major storage array (cols, rows)."""
    return storage.T


def seed_for(config: int, phi_index: int, operand: int) -> int:
    """Fixed seed per matrix: config number, phi index, operand (1 = A, 2 = B)."""
    return 1000 * config + 10 * phi_index + operand

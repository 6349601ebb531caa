"""Test helper: dense matrices from the library's exported block-CSR."""
import numpy as np


def bsr_to_dense(rp, col, vals):
    """Dense matrix from an exported block-CSR (row_ptr, col, vals[nnzb, b, b])."""
    N = len(rp) - 1
    b = vals.shape[1] if vals.ndim == 3 else 0
    D = np.zeros((N * b, N * b))
    for i in range(N):
        for z in range(rp[i], rp[i + 1]):
            j = col[z]
            D[i * b:(i + 1) * b, j * b:(j + 1) * b] += vals[z]
    return D

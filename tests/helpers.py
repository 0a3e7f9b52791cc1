"""Shared helpers for the GPU parity tests (test infrastructure)."""

import numpy as np

from oracle import gp_oracle as O


def canonical_gpu_csr(csr):
    """(orig_row, orig_col, value) triples of the GPU's active block, sorted."""
    rows = np.repeat(np.arange(len(csr.perm)), np.diff(csr.row_ptr))
    r = csr.perm[rows].astype(np.int64)
    c = csr.perm[csr.col].astype(np.int64)
    order = np.lexsort((c, r))
    return r[order], c[order], csr.val[order]


def canonical_oracle_csr(x, h, dim, n1, n2, beta=1.0):
    """Same triples from the oracle's brute force, restricted to active rows."""
    rp, col, val = O.assemble_csr(x, h, dim, n1, n2, beta)
    _, mask = O.bump_table(x, h, dim, n1, n2, beta)
    rows = np.repeat(np.arange(len(rp) - 1), np.diff(rp))
    keep = mask[rows] != 0
    return rows[keep], col[keep], val[keep], mask


def value_tol_ok(v_gpu, v_ref, diag, r, c, rtol, stol):
    """|dK_ij| <= rtol |K_ij| + stol sqrt(K_ii K_jj): relative error with a
    floor on the scale of the entry's Cauchy-Schwarz bound (K is PSD)."""
    scale = np.sqrt(diag[r] * diag[c])
    err = np.abs(v_gpu - v_ref)
    bound = rtol * np.abs(v_ref) + stol * scale
    return bool(np.all(err <= bound)), float(np.max(err / (np.abs(v_ref) + scale)))

"""Shared helpers for the GPU parity tests (test infrastructure)."""

import numpy as np

from oracle import gp_oracle as O

# One unit of the smallest spacing of each stored format (its denormal step):
# an entry of the Jacobi-scaled matrix below the normal range cannot be held
# to a relative tolerance in that format, only to this absolute resolution.
DENORMAL_STEP = {"fp32": 2.0 ** -149, "fp64": 2.0 ** -1074}
NORMAL_MIN = {"fp32": 2.0 ** -126, "fp64": 2.0 ** -1022}

_ORACLE_CSR = {}


def canonical_gpu_csr(csr):
    """(orig_row, orig_col, value) triples of the GPU's active block, sorted."""
    rows = np.repeat(np.arange(len(csr.perm)), np.diff(csr.row_ptr))
    r = csr.perm[rows].astype(np.int64)
    c = csr.perm[csr.col].astype(np.int64)
    order = np.lexsort((c, r))
    return r[order], c[order], csr.val[order]


def canonical_oracle_csr(x, h, dim, n1, n2, beta=1.0, key=None):
    """Same triples from the oracle's brute force, restricted to active rows:
    the pattern of the float64 support predicates, each entry's value
    evaluated to full accuracy (oracle.entries_hp).  `key` caches the result
    for repeated use within a session."""
    if key is not None and key in _ORACLE_CSR:
        return _ORACLE_CSR[key]
    rp, col, _ = O.assemble_csr(x, h, dim, n1, n2, beta)
    _, mask = O.bump_table(x, h, dim, n1, n2, beta)
    rows = np.repeat(np.arange(len(rp) - 1), np.diff(rp))
    keep = mask[rows] != 0
    r, c = rows[keep], col[keep]
    v = O.entries_hp(x, h, dim, n1, n2, r, c, beta)
    out = (r, c, v, mask)
    if key is not None:
        _ORACLE_CSR[key] = out
    return out


def value_tol_ok(v_gpu, v_ref, diag, r, c, rtol, prec):
    """|dK_ij| <= rtol |K_ij| + step sqrt(K_ii K_jj) with `step` one unit of the
    stored format's denormal spacing: the GPU stores Khat = D^-1/2 K D^-1/2
    (D = diag K), whose entries below the format's normal range carry only
    that absolute resolution; unscaled, it is step sqrt(K_ii K_jj).
    Returns (ok, worst relative error over the entries whose Khat value is in
    the format's normal range)."""
    scale = np.sqrt(diag[r] * diag[c])
    err = np.abs(v_gpu - v_ref)
    floor = DENORMAL_STEP[prec] * scale
    bound = rtol * np.abs(v_ref) + floor
    normal = np.abs(v_ref) > NORMAL_MIN[prec] * scale   # Khat entry in the format's normal range
    worst = float(np.max(err[normal] / np.abs(v_ref[normal]))) if np.any(normal) else 0.0
    return bool(np.all(err <= bound)), worst


def grad_solver_bound(info_ref, eps, safety):
    """Per-component bound on a gradient computed from solves that stopped at
    relative residual eps: safety * eps * (sens_quad + sens_trace / 2), the
    first-order change of the estimator (oracle.lml_grad_same_probes with
    with_bounds=True).  `safety` covers what the first-order residual model
    leaves out: FP32 rounding of the stored entries and of the CG vectors acts
    as an extra residual well below eps at rtol 1e-6 (measured: every
    component within 0.15 of the bound at safety 1 on the parity workloads)."""
    return safety * eps * (info_ref["grad_sens_quad"] + 0.5 * info_ref["grad_sens_trace"])


def grad_ok(g_gpu, g_ref, info_ref, eps, safety):
    """(ok, worst ratio |dg| / bound) for grad_solver_bound; components whose
    bound is zero (no entry depends on them) must agree exactly."""
    bound = grad_solver_bound(info_ref, eps, safety)
    err = np.abs(np.asarray(g_gpu) - np.asarray(g_ref))
    ok = bool(np.all((err <= bound) | ((bound == 0) & (err == 0))))
    ratio = np.where(bound > 0, err / np.where(bound > 0, bound, 1.0), 0.0)
    return ok, float(np.max(ratio)) * safety

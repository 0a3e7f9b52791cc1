"""Plain FP64 CPU oracle for the sparse exact-GP hot path of arXiv 2205.09070.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import, call or
execute this module: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline / reference arm of ``bench.py`` use it.  It shares no code, constants
or helpers with the CUDA library; the two meet only through the seeded input
generators, which hold none of the method's arithmetic.

Everything is float64 numpy, written for a reader to check against the paper
by eye: brute-force O(N^2) pair enumeration, dense matrices, dense Cholesky.

Paper sections used (arXiv 2205.09070):
  * Sec. 2.1, Eq. (eqn:log_likelihood): ln L = -1/2 y^T K^-1 y - 1/2 ln|K|
    (additive constant dropped, prior mean m = 0).
  * Sec. 2.2, Eq. (eq:bump_kernel): k_s = k~(x1,x2) * sum_i f_i(x1) f_i(x2).
  * Sec. 2.2, Eq. (eq:bump): f_i(x) = sum_j a_ij exp[beta - beta/(1-|x-x0|^2/r^2)]
    times the indicator of the bump's support.
  * Sec. 2.2, Eq. (eq:kstat): the compactly supported stationary kernel k~.
  * Sec. 2.2, Eq. (eq:sparsity_estimate) and the two equations after it: the
    sparsity upper bound used as a statistical check.
  * Sec. 2.4, Eqs. (eq:constrained) and (eq:augmented): the training
    objectives, driven by Adam (a reading: Sec. 4 names gradient-based
    training as future work without a method).
  * Sec. 2.5: CG for K x = y and a randomized log-determinant (the cited
    estimator of Boutsidis et al., truncated Taylor series of ln(I - C) with
    Hutchinson probes, beside stochastic Lanczos quadrature).

Readings where the paper is silent, garbled or inconsistent:
  * Eq. (eq:bump) prints the indicator as chi(r < |x - x0|); the text calls the
    bumps compactly supported, so the support is the open ball |x - x0| < r.
  * beta is a fixed shape constant (default 1), not a hyperparameter: the
    climate example counts 42 hyperparameters for n1=2, n2=4 in 3-D
    (Sec. 3), which is 2*4*(3+2) + 2 with no beta.
  * K carries a stationary amplitude A and observation noise sigma_n^2 on the
    diagonal: K = A * k~ * sum_m f_m f_m^T + sigma_n^2 I  (V = sigma_n^2 I of
    Eq. eq:likelihoodGP folded into K, m = 0).
  * The stationary support test is strict (d < r), as printed in Eq. (eq:kstat).
  * The sparsity pattern is the support predicate {i == j} union
    {d_ij < r_s and x_i, x_j share the support of some f_m}; entries whose
    value cancels to zero are still part of the pattern.
  * The log-determinant estimator is stochastic Lanczos quadrature (SLQ) on the
    Jacobi-scaled active block, with Rademacher probes from a counter-based
    SplitMix64 stream; inactive rows (outside every bump) are exact.

Hyperparameter vector layout, P = n1*n2*(dim+2) + 3 doubles:
  for m < n1, b < n2: [centre_mb[0..dim-1], r_mb, a_mb]; then r_s, A, sigma_n^2.
  A vector with one more entry carries the length scale l of a squared-
  exponential core kernel k_c = exp(-|x1 - x2|^2 / (2 l^2)) multiplying k_s
  (Sec. 2.2: kernels can be multiplied, k_c * k_s, with no restriction on the
  core; the paper's kernel figure shows a squared-exponential core).

Parity pins (tests/test_oracle_pins.py) tie every function here to something
other than itself: an independently derived power series and its derivative,
closed-form special values, brute-force properties (symmetry, PSD, exact zeros
for disjoint supports), Euler homogeneity identities, central finite
differences, eigen-decomposition special cases and the published SplitMix64
output sequence.
"""

from __future__ import annotations

import math
from decimal import Decimal, getcontext, localcontext

import numpy as np

# Prefactor of Eq. (eq:kstat): sqrt(2) / (3 sqrt(pi)); it is also k~(0).
KSTAT_PREFACTOR = math.sqrt(2.0) / (3.0 * math.sqrt(math.pi))


# ----------------------------------------------------------------------------
# hyperparameters
# ----------------------------------------------------------------------------

def n_params(dim: int, n1: int, n2: int, core: bool = False) -> int:
    """Number of hyperparameters: per bump a centre, a radius and an amplitude
    (Eq. eq:bump), then the stationary radius r_s, amplitude A and noise, and
    the core length scale l when there is a core kernel."""
    return n1 * n2 * (dim + 2) + 3 + (1 if core else 0)


def unpack_h(h, dim: int, n1: int, n2: int):
    """Split the flat hyperparameter vector into its named parts; "ell" is the
    core kernel's length scale, or None without a core kernel."""
    h = np.asarray(h, dtype=np.float64)
    if h.shape not in ((n_params(dim, n1, n2),), (n_params(dim, n1, n2, True),)):
        raise ValueError("hyperparameter vector has the wrong length")
    nb = n1 * n2 * (dim + 2)
    b = h[:nb].reshape(n1, n2, dim + 2)
    return {
        "centres": b[:, :, :dim],
        "radii": b[:, :, dim],
        "amps": b[:, :, dim + 1],
        "r_s": float(h[nb]),
        "A": float(h[nb + 1]),
        "sigma2": float(h[nb + 2]),
        "ell": float(h[nb + 3]) if h.shape[0] == nb + 4 else None,
    }


def core_kernel(d2, ell):
    """k_c at squared distance d2: exp(-d2 / (2 l^2)), or 1 without a core."""
    d2 = np.asarray(d2, dtype=np.float64)
    return np.ones_like(d2) if ell is None else np.exp(-d2 / (2.0 * ell * ell))


# ----------------------------------------------------------------------------
# Eq. (eq:kstat): compactly supported stationary kernel
# ----------------------------------------------------------------------------

def kstat(rho):
    """k~ as a function of rho = d / r, exactly as printed in Eq. (eq:kstat):

        sqrt(2)/(3 sqrt(pi)) * (3 rho^2 log(rho / (1 + sqrt(1 - rho^2)))
                                 + (2 rho^2 + 1) sqrt(1 - rho^2))   if rho < 1
        0                                                          otherwise.

    At rho = 0 the term rho^2 log(rho) is taken at its limit, 0.
    """
    rho = np.asarray(rho, dtype=np.float64)
    out = np.zeros_like(rho)
    inside = rho < 1.0
    r = rho[inside]
    s = np.sqrt(1.0 - r * r)
    with np.errstate(divide="ignore", invalid="ignore"):
        log_term = np.where(r > 0.0, 3.0 * r * r * np.log(r / (1.0 + s)), 0.0)
    out[inside] = KSTAT_PREFACTOR * (log_term + (2.0 * r * r + 1.0) * s)
    return out


def kstat_drho(rho):
    """d k~ / d rho for Eq. (eq:kstat), differentiated by hand.

    With s = sqrt(1 - rho^2) and ds/drho = -rho/s, the derivative of the
    bracket collapses to 6 rho log(rho/(1+s)) + 6 rho s; since
    rho/(1+s) = sqrt((1-s)/(1+s)), log(rho/(1+s)) = -atanh(s), so
    d k~/d rho = 6 C rho (s - atanh(s)) for rho < 1 and 0 outside.
    """
    rho = np.asarray(rho, dtype=np.float64)
    out = np.zeros_like(rho)
    inside = rho < 1.0
    r = rho[inside]
    s = np.sqrt(1.0 - r * r)
    with np.errstate(divide="ignore", invalid="ignore"):
        # at rho = 0, rho * atanh(1) is taken at its limit, 0
        out[inside] = np.where(r > 0.0, 6.0 * KSTAT_PREFACTOR * r * (s - np.arctanh(s)), 0.0)
    return out


# ----------------------------------------------------------------------------
# Eq. (eq:bump): bump functions
# ----------------------------------------------------------------------------

def bump_phi(x, centre, radius, amp, beta=1.0):
    """One bump a * exp(beta - beta / (1 - |x - c|^2 / r^2)) on the open ball
    |x - c| < r, zero elsewhere (Eq. eq:bump with the support reading above).
    Returns (phi, inside) for points x of shape (N, dim)."""
    x = np.asarray(x, dtype=np.float64)
    q = np.sum((x - centre) ** 2, axis=1) / (radius * radius)
    inside = q < 1.0
    phi = np.zeros(x.shape[0])
    u = 1.0 - q[inside]
    phi[inside] = amp * np.exp(beta - beta / u)
    return phi, inside


def bump_phi_grads(x, centre, radius, amp, beta=1.0):
    """Partial derivatives of one bump w.r.t. its centre (N, dim), radius (N,)
    and amplitude (N,), differentiated by hand from Eq. (eq:bump):
    with q = |x-c|^2/r^2 and u = 1-q, d phi/d q = -beta phi / u^2, so
      d phi / d c_k = 2 beta phi (x_k - c_k) / (r^2 u^2)
      d phi / d r   = 2 beta phi q / (r u^2)
      d phi / d a   = phi / a  (= exp(beta - beta/u)).
    All three vanish outside the support."""
    x = np.asarray(x, dtype=np.float64)
    n, dim = x.shape
    diff = x - centre
    q = np.sum(diff ** 2, axis=1) / (radius * radius)
    inside = q < 1.0
    d_c = np.zeros((n, dim))
    d_r = np.zeros(n)
    d_a = np.zeros(n)
    u = 1.0 - q[inside]
    e = np.exp(beta - beta / u)
    phi = amp * e
    d_c[inside] = (2.0 * beta * phi / (radius * radius * u * u))[:, None] * diff[inside]
    d_r[inside] = 2.0 * beta * phi * q[inside] / (radius * u * u)
    d_a[inside] = e
    return d_c, d_r, d_a


def bump_table(x, h, dim, n1, n2, beta=1.0):
    """F[i, m] = f_m(x_i) (Eq. eq:bump) and the support mask
    M_i = sum over m of 2^m [x_i lies in the support of some bump of f_m]."""
    p = unpack_h(h, dim, n1, n2)
    x = np.asarray(x, dtype=np.float64)
    n = x.shape[0]
    F = np.zeros((n, n1))
    mask = np.zeros(n, dtype=np.int64)
    for m in range(n1):
        in_m = np.zeros(n, dtype=bool)
        for b in range(n2):
            phi, inside = bump_phi(x, p["centres"][m, b], p["radii"][m, b], p["amps"][m, b], beta)
            F[:, m] += phi
            in_m |= inside
        mask |= in_m.astype(np.int64) << m
    return F, mask


# ----------------------------------------------------------------------------
# Eq. (eq:bump_kernel) with Eq. (eq:kstat): the covariance matrix K
# ----------------------------------------------------------------------------

def pair_rows(x, h, dim, n1, n2, rows, beta=1.0, table=None):
    """Brute force over all N columns for the given rows (original order).
    `table` may pass a precomputed (F, mask) = bump_table(x, h, ...).

    Returns (pattern, values) of shape (len(rows), N):
      pattern[a, j] = (j == rows[a]) or (d^2 < r_s^2 and M_i & M_j != 0)
      values[a, j]  = A k~(d / r_s) sum_m F_im F_jm + sigma_n^2 [j == rows[a]]
    """
    p = unpack_h(h, dim, n1, n2)
    x = np.asarray(x, dtype=np.float64)
    rows = np.asarray(rows, dtype=np.int64)
    F, mask = table if table is not None else bump_table(x, h, dim, n1, n2, beta)
    d2 = np.sum((x[rows, None, :] - x[None, :, :]) ** 2, axis=2)
    diag = rows[:, None] == np.arange(x.shape[0])[None, :]
    pattern = diag | ((d2 < p["r_s"] ** 2) & ((mask[rows, None] & mask[None, :]) != 0))
    rho = np.sqrt(d2) / p["r_s"]
    S = np.zeros(d2.shape)
    for m in range(n1):                       # sum_m f_m(x_i) f_m(x_j), term by term
        S += F[rows, m][:, None] * F[:, m][None, :]
    vals = p["A"] * kstat(rho) * core_kernel(d2, p["ell"]) * S + p["sigma2"] * diag
    vals = np.where(pattern, vals, 0.0)
    return pattern, vals


def assemble_csr(x, h, dim, n1, n2, beta=1.0, chunk=512):
    """CSR of K in original point order with ascending columns, by brute force
    over all N^2 pairs (chunked over rows to bound memory).
    Returns (row_ptr int64 [N+1], col int64 [nnz], val float64 [nnz])."""
    x = np.asarray(x, dtype=np.float64)
    n = x.shape[0]
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    cols, vals = [], []
    table = bump_table(x, h, dim, n1, n2, beta)
    for start in range(0, n, chunk):
        rows = np.arange(start, min(n, start + chunk))
        pat, v = pair_rows(x, h, dim, n1, n2, rows, beta, table)
        r_idx, c_idx = np.nonzero(pat)
        cols.append(c_idx.astype(np.int64))
        vals.append(v[r_idx, c_idx])
        row_ptr[rows + 1] = np.sum(pat, axis=1)
    row_ptr = np.cumsum(row_ptr)
    col = np.concatenate(cols) if cols else np.zeros(0, np.int64)
    val = np.concatenate(vals) if vals else np.zeros(0)
    return row_ptr, col, val


def dense_K(x, h, dim, n1, n2, beta=1.0, chunk=1024):
    """Dense K (N x N) by brute force; entries outside the pattern are zero.
    Rows are filled in chunks to bound the temporaries."""
    x = np.asarray(x, dtype=np.float64)
    n = x.shape[0]
    table = bump_table(x, h, dim, n1, n2, beta)
    K = np.zeros((n, n))
    for start in range(0, n, chunk):
        rows = np.arange(start, min(n, start + chunk))
        _, K[rows] = pair_rows(x, h, dim, n1, n2, rows, beta, table)
    return K


# ----------------------------------------------------------------------------
# The same entries to full accuracy (decimal arithmetic)
# ----------------------------------------------------------------------------
#
# Evaluated in float64, the printed Eq. (eq:kstat) cancels as rho -> 1: its
# two terms are of order s = sqrt(1 - rho^2) while their sum is of order s^5,
# so an entry near the edge of the stationary support keeps only a few
# correct digits.  A bump of Eq. (eq:bump) is steep near its own edge, and a
# sum over bumps or functions may cancel as well.  The functions below take
# every float64 input as the exact number it represents, evaluate the same
# printed expressions with HP_DIGITS significant decimal digits (Python's
# decimal module), and round only the finished entry to float64.  They are the
# reference for element-wise value parity.  Which pairs are stored is still
# decided by the float64 predicates above (support tests d^2 < r_s^2 and
# |x - c|^2 / r^2 < 1), exactly as the plain definition is written.

HP_DIGITS = 60


def _hp_pi():
    """pi to the working precision by Machin's formula
    pi = 16 arctan(1/5) - 4 arctan(1/239), arctan(1/q) = sum_k (-1)^k / ((2k+1) q^(2k+1))."""
    def arctan_inv(q):
        q = Decimal(q)
        total, power, k = Decimal(0), 1 / q, 0
        eps = Decimal(10) ** (-(getcontext().prec + 5))
        while power > eps:
            term = power / (2 * k + 1)
            total += term if k % 2 == 0 else -term
            power /= q * q
            k += 1
        return total
    return 16 * arctan_inv(5) - 4 * arctan_inv(239)


def _hp_constants():
    """C = sqrt(2) / (3 sqrt(pi)) of Eq. (eq:kstat) at the working precision."""
    return Decimal(2).sqrt() / (3 * _hp_pi().sqrt())


def kstat_hp(rho2, C=None):
    """Eq. (eq:kstat) exactly as printed, as a function of rho^2 = d^2 / r^2
    (a Decimal), evaluated at the context's precision:
        C (3 rho^2 log(rho / (1 + s)) + (2 rho^2 + 1) s),  s = sqrt(1 - rho^2),
    for rho < 1, and 0 otherwise; at rho = 0 the term rho^2 log(rho) is taken
    at its limit, 0."""
    C = _hp_constants() if C is None else C
    if rho2 >= 1:
        return Decimal(0)
    s = (1 - rho2).sqrt()
    if rho2 == 0:
        return C * s
    rho = rho2.sqrt()
    return C * (3 * rho2 * (rho / (1 + s)).ln() + (2 * rho2 + 1) * s)


def _hp_candidate_bumps(x, h, dim, n1, n2):
    """For each point of x, the bumps (m, b) whose float64 support test is
    close to passing (q < 1 + 1e-9); the exact evaluation then decides with
    u > 0.  Returns (unpacked h, list of bump lists, one per point)."""
    p = unpack_h(h, dim, n1, n2)
    x = np.asarray(x, dtype=np.float64).reshape(-1, dim)
    near = np.zeros((x.shape[0], n1 * n2), dtype=bool)
    for m in range(n1):
        for b in range(n2):
            q = np.sum((x - p["centres"][m, b]) ** 2, axis=1) / (p["radii"][m, b] ** 2)
            near[:, m * n2 + b] = q < 1.0 + 1e-9
    return p, [[(int(t) // n2, int(t) % n2) for t in np.nonzero(row)[0]] for row in near]


def bump_sums_hp(point, p, dim, n1, n2, beta, bumps):
    """f_m(point) for m < n1 (Eq. eq:bump) in decimal: the sum over the listed
    bumps (m, b) of a exp(beta - beta / u), u = 1 - |x - c|^2 / r^2 > 0."""
    f = [Decimal(0)] * n1
    xb = [Decimal(float(point[k])) for k in range(dim)]
    B = Decimal(float(beta))
    for m, b in bumps:
        c = p["centres"][m, b]
        d2 = sum((xb[k] - Decimal(float(c[k]))) ** 2 for k in range(dim))
        u = 1 - d2 / Decimal(float(p["radii"][m, b])) ** 2
        if u > 0:
            f[m] += Decimal(float(p["amps"][m, b])) * (B - B / u).exp()
    return f


def entries_hp(x, h, dim, n1, n2, rows, cols, beta=1.0, digits=HP_DIGITS):
    """K_ij = A k~(|x_i - x_j| / r_s) k_c(x_i, x_j) sum_m f_m(x_i) f_m(x_j)
    + sigma_n^2 [i = j] (Eq. eq:bump_kernel with Eq. eq:kstat and Eq. eq:bump;
    k_c = 1 without a core kernel) for the listed pairs
    (i, j) = (rows[t], cols[t]), evaluated to `digits` significant digits and
    rounded to float64.  The caller lists pairs of the pattern; a pair whose
    exact distance reaches r_s (possible only at a float64 tie) gets k~ = 0."""
    x = np.asarray(x, dtype=np.float64)
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    out = np.empty(rows.shape[0])
    pts = np.unique(np.concatenate([rows, cols]))      # only the points the pairs touch
    with localcontext() as ctx:
        ctx.prec = digits
        p, cand = _hp_candidate_bumps(x[pts], h, dim, n1, n2)
        slot = {int(i): t for t, i in enumerate(pts)}
        C = _hp_constants()
        A = Decimal(p["A"])
        s2 = Decimal(p["sigma2"])
        rs2 = Decimal(p["r_s"]) ** 2
        ell = Decimal(p["ell"]) if p["ell"] is not None else None
        fcache, memo = {}, {}

        def F(i):
            if i not in fcache:
                fcache[i] = bump_sums_hp(x[i], p, dim, n1, n2, beta, cand[slot[i]])
            return fcache[i]

        for t in range(rows.shape[0]):
            i, j = int(rows[t]), int(cols[t])
            key = (min(i, j), max(i, j))
            if key not in memo:
                Fi, Fj = F(i), F(j)
                S = sum(Fi[m] * Fj[m] for m in range(n1))
                if i == j:
                    v = A * C * S + s2
                else:
                    d2 = sum((Decimal(float(x[i, k])) - Decimal(float(x[j, k]))) ** 2 for k in range(dim))
                    v = A * kstat_hp(d2 / rs2, C) * S
                    if ell is not None:
                        v *= (-d2 / (2 * ell * ell)).exp()
                memo[key] = float(v)
            out[t] = memo[key]
    return out


def cross_K_hp(xs, x, h, dim, n1, n2, beta=1.0, digits=HP_DIGITS):
    """kappa[a, i] = k(xs_a, x_i) as cross_K computes it, with every pair in
    support (float64 test d^2 < r_s^2) evaluated by the decimal route of
    entries_hp; pairs out of support are exactly 0."""
    p = unpack_h(h, dim, n1, n2)
    xs = np.asarray(xs, dtype=np.float64).reshape(-1, dim)
    x = np.asarray(x, dtype=np.float64)
    d2 = np.sum((xs[:, None, :] - x[None, :, :]) ** 2, axis=2)
    insup = d2 < p["r_s"] ** 2
    kappa = np.zeros(d2.shape)
    if not np.any(insup):
        return kappa
    with localcontext() as ctx:
        ctx.prec = digits
        pq, cand_q = _hp_candidate_bumps(xs, h, dim, n1, n2)
        touched = np.nonzero(np.any(insup, axis=0))[0]
        _, cand_x = _hp_candidate_bumps(x[touched], h, dim, n1, n2)
        slot = {int(i): t for t, i in enumerate(touched)}
        C = _hp_constants()
        A = Decimal(p["A"])
        rs2 = Decimal(p["r_s"]) ** 2
        fx = {}
        for a in np.nonzero(np.any(insup, axis=1))[0]:
            fq = bump_sums_hp(xs[a], pq, dim, n1, n2, beta, cand_q[a])
            if all(v == 0 for v in fq):
                continue
            for i in np.nonzero(insup[a])[0]:
                if i not in fx:
                    fx[i] = bump_sums_hp(x[i], pq, dim, n1, n2, beta, cand_x[slot[int(i)]])
                S = sum(fq[m] * fx[i][m] for m in range(n1))
                if S == 0:
                    continue
                dd = sum((Decimal(float(xs[a, k])) - Decimal(float(x[i, k]))) ** 2 for k in range(dim))
                v = A * kstat_hp(dd / rs2, C) * S
                if p["ell"] is not None:
                    v *= (-dd / (2 * Decimal(p["ell"]) ** 2)).exp()
                kappa[a, i] = float(v)
    return kappa


# ----------------------------------------------------------------------------
# Sec. 2.1: posterior mean at test points, kappa^T (K + V)^-1 y (prior mean 0)
# ----------------------------------------------------------------------------

def cross_K(xs, x, h, dim, n1, n2, beta=1.0):
    """kappa[a, i] = k(xs_a, x_i) = A k~(|xs_a - x_i| / r_s) sum_m f_m(xs_a) f_m(x_i)
    by brute force over all pairs (Eq. eq:bump_kernel with Eq. eq:kstat).  A
    test point is not an observation, so no noise term enters."""
    p = unpack_h(h, dim, n1, n2)
    xs = np.asarray(xs, dtype=np.float64).reshape(-1, dim)
    x = np.asarray(x, dtype=np.float64)
    Fq, _ = bump_table(xs, h, dim, n1, n2, beta)
    F, _ = bump_table(x, h, dim, n1, n2, beta)
    d2 = np.sum((xs[:, None, :] - x[None, :, :]) ** 2, axis=2)
    S = np.zeros(d2.shape)
    for m in range(n1):
        S += Fq[:, m][:, None] * F[:, m][None, :]
    return np.where(d2 < p["r_s"] ** 2, p["A"] * kstat(np.sqrt(d2) / p["r_s"]) * core_kernel(d2, p["ell"]) * S,
                    0.0)


def predict_mean(x, y, h, xs, dim, n1, n2, beta=1.0):
    """Posterior mean m(xs) = kappa^T K^-1 y (Sec. 2.1, with V = sigma_n^2 I
    inside K and prior mean 0): dense K, dense solve, brute-force kappa."""
    K = dense_K(x, h, dim, n1, n2, beta)
    alpha = np.linalg.solve(K, np.asarray(y, dtype=np.float64))
    return cross_K(xs, x, h, dim, n1, n2, beta) @ alpha


def prior_var(xs, h, dim, n1, n2, beta=1.0):
    """k(x*, x*) = A k~(0) k_c(0) sum_m f_m(x*)^2 = A C sum_m f_m(x*)^2
    (Eq. eq:bump_kernel at d = 0; a test point carries no noise)."""
    p = unpack_h(h, dim, n1, n2)
    Fq, _ = bump_table(np.asarray(xs, dtype=np.float64).reshape(-1, dim), h, dim, n1, n2, beta)
    return p["A"] * KSTAT_PREFACTOR * np.sum(Fq * Fq, axis=1)


def prior_var_hp(xs, h, dim, n1, n2, beta=1.0, digits=HP_DIGITS):
    """prior_var with f_m(x*) from the decimal route (bump_sums_hp), rounded
    once: accurate where the float64 bumps lose digits near their edges."""
    xs = np.asarray(xs, dtype=np.float64).reshape(-1, dim)
    out = np.zeros(xs.shape[0])
    with localcontext() as ctx:
        ctx.prec = digits
        p, cand = _hp_candidate_bumps(xs, h, dim, n1, n2)
        AC = Decimal(p["A"]) * _hp_constants()
        for a in range(xs.shape[0]):
            if cand[a]:
                f = bump_sums_hp(xs[a], p, dim, n1, n2, beta, cand[a])
                out[a] = float(AC * sum(v * v for v in f))
    return out


def dense_K_hp(x, h, dim, n1, n2, beta=1.0):
    """dense_K with every stored entry from the decimal route (entries_hp)."""
    x = np.asarray(x, dtype=np.float64)
    rp, col, _ = assemble_csr(x, h, dim, n1, n2, beta)
    rows = np.repeat(np.arange(x.shape[0]), np.diff(rp))
    K = np.zeros((x.shape[0], x.shape[0]))
    K[rows, col] = entries_hp(x, h, dim, n1, n2, rows, col, beta)
    return K


def predict_var(x, h, xs, dim, n1, n2, beta=1.0, kappa=None, prior=None, K=None):
    """Posterior variance of the latent function at test points (Sec. 2.1,
    Eq. eq:pred_distr): k(x*, x*) - kappa^T (K + V)^-1 kappa, V = sigma_n^2 I
    inside K; dense K and a dense solve.  `kappa`, `prior` and `K` may pass the
    cross-covariance, k(x*, x*) and K (for example the full-accuracy ones)."""
    K = dense_K(x, h, dim, n1, n2, beta) if K is None else K
    kap = cross_K(xs, x, h, dim, n1, n2, beta) if kappa is None else kappa
    pri = prior_var(xs, h, dim, n1, n2, beta) if prior is None else prior
    return pri - np.sum(kap * np.linalg.solve(K, kap.T).T, axis=1)


def predict_var_sensitivity(x, h, xs, dim, n1, n2, beta=1.0, kappa=None):
    """Per test point, what bounds the variance's change when the solve of
    Khat u = D^-1/2 kappa stops at relative residual eps: to first order
    kappa^T K^-1 kappa moves by r^T Khat^-1 khat, at most
    eps |khat| |Khat^-1 khat| (khat = D^-1/2 kappa on the active rows), and by
    |khat|^T |Khat^-1 khat| times the relative rounding of the entries.
    Returns (|khat| |Khat^-1 khat|, |khat|^T |Khat^-1 khat|)."""
    K = dense_K(x, h, dim, n1, n2, beta)
    _, mask = bump_table(x, h, dim, n1, n2, beta)
    act = np.nonzero(mask != 0)[0]
    kap = cross_K(xs, x, h, dim, n1, n2, beta) if kappa is None else kappa
    if act.size == 0:
        return np.zeros(kap.shape[0]), np.zeros(kap.shape[0])
    Ka = K[np.ix_(act, act)]
    Dm = 1.0 / np.sqrt(np.diag(Ka))
    Khat = Ka * Dm[:, None] * Dm[None, :]
    kh = kap[:, act] * Dm[None, :]
    u = np.linalg.solve(Khat, kh.T).T
    return np.linalg.norm(kh, axis=1) * np.linalg.norm(u, axis=1), np.sum(np.abs(kh) * np.abs(u), axis=1)


# ----------------------------------------------------------------------------
# Eq. (eqn:log_likelihood): exact LML and its exact gradient
# ----------------------------------------------------------------------------

def lml_exact(K, y):
    """-1/2 y^T K^-1 y - 1/2 ln|K| by dense Cholesky (Sec. 2.1, Sec. 2.5)."""
    L = np.linalg.cholesky(K)
    w = np.linalg.solve(L, y)
    return -0.5 * float(w @ w) - float(np.sum(np.log(np.diag(L))))


def dK_dtheta_all(x, h, dim, n1, n2, beta=1.0):
    """Yield (index, dK) for every hyperparameter, dK dense N x N, from the
    chain rule on K = A k~(d/r_s) sum_m F_m F_m^T + sigma_n^2 I."""
    p = unpack_h(h, dim, n1, n2)
    x = np.asarray(x, dtype=np.float64)
    n = x.shape[0]
    F, _ = bump_table(x, h, dim, n1, n2, beta)
    d2 = np.sum((x[:, None, :] - x[None, :, :]) ** 2, axis=2)
    d = np.sqrt(d2)
    rho = d / p["r_s"]
    kc = core_kernel(d2, p["ell"])
    kt = kstat(rho) * kc          # the core multiplies every term
    A = p["A"]
    idx = 0
    for m in range(n1):
        for b in range(n2):
            d_c, d_r, d_a = bump_phi_grads(x, p["centres"][m, b], p["radii"][m, b], p["amps"][m, b], beta)
            for dphi in [d_c[:, k] for k in range(dim)] + [d_r, d_a]:
                dS = np.outer(dphi, F[:, m]) + np.outer(F[:, m], dphi)
                yield idx, A * kt * dS
                idx += 1
    S = np.zeros((n, n))
    for m in range(n1):
        S += np.outer(F[:, m], F[:, m])
    yield idx, A * (kstat_drho(rho) * (-rho / p["r_s"])) * kc * S  # r_s
    yield idx + 1, kt * S                                          # A
    yield idx + 2, np.eye(n)                                       # sigma_n^2
    if p["ell"] is not None:                                       # l: d k_c / d l = k_c d^2 / l^3
        yield idx + 3, A * kt * S * d2 / p["ell"] ** 3


def lml_grad_exact(x, y, h, dim, n1, n2, beta=1.0):
    """Exact ln L and d ln L / d theta = 1/2 alpha^T K_theta alpha
    - 1/2 tr(K^-1 K_theta), alpha = K^-1 y, via a dense Cholesky inverse."""
    K = dense_K(x, h, dim, n1, n2, beta)
    y = np.asarray(y, dtype=np.float64)
    L = np.linalg.cholesky(K)
    Linv = np.linalg.solve(L, np.eye(K.shape[0]))
    Kinv = Linv.T @ Linv
    alpha = Kinv @ y
    lml = -0.5 * float(y @ alpha) - float(np.sum(np.log(np.diag(L))))
    grad = np.zeros(len(np.asarray(h)))
    for i, dK in dK_dtheta_all(x, h, dim, n1, n2, beta):
        grad[i] = 0.5 * float(alpha @ (dK @ alpha)) - 0.5 * float(np.sum(Kinv * dK))
    return lml, grad


# ----------------------------------------------------------------------------
# Probes: SplitMix64 (Steele, Lea & Flood, OOPSLA 2014) as a counter stream
# ----------------------------------------------------------------------------

_SM_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_SM_M1 = np.uint64(0xBF58476D1CE4E5B9)
_SM_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed, k):
    """k-th output (k = 0, 1, ...) of the SplitMix64 stream whose state starts
    at `seed`: the state after k+1 increments by the golden gamma, pushed
    through the published 30/27/31 xor-shift-multiply finaliser."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + (np.asarray(k, dtype=np.uint64) + np.uint64(1)) * _SM_GAMMA
        z = (z ^ (z >> np.uint64(30))) * _SM_M1
        z = (z ^ (z >> np.uint64(27))) * _SM_M2
        return z ^ (z >> np.uint64(31))


def rademacher(seed, n_probes, orig_index):
    """Rademacher probe matrix Z (len(orig_index) x n_probes) with
    Z[i, l] = +1 if bit 63 of splitmix64(seed, l * 2^40 + orig_index[i]) is 0
    and -1 otherwise."""
    idx = np.asarray(orig_index, dtype=np.uint64)
    out = np.empty((idx.shape[0], n_probes))
    for l in range(n_probes):
        z = splitmix64(seed, np.uint64(l) * np.uint64(1 << 40) + idx)
        out[:, l] = np.where((z >> np.uint64(63)) == 0, 1.0, -1.0)
    return out


# ----------------------------------------------------------------------------
# Stochastic estimators on the same probes as the GPU path
# ----------------------------------------------------------------------------

def active_split(K, mask):
    """Rows with mask 0 lie outside every bump: their row of K is sigma_n^2 on
    the diagonal only.  Returns (active index array, inactive index array)."""
    mask = np.asarray(mask)
    return np.nonzero(mask != 0)[0], np.nonzero(mask == 0)[0]


def lanczos_quadrature(Khat, z, m):
    """Gauss quadrature estimate of z^T log(Khat) z from m Lanczos steps
    started at z/|z|, with full re-orthogonalisation (Golub & Meurant):
    T = Q Theta Q^T, estimate = |z|^2 sum_k Q[0,k]^2 log theta_k.
    Stops early if the Krylov space is exhausted."""
    n = Khat.shape[0]
    nz = float(np.linalg.norm(z))
    V = np.zeros((n, m + 1))
    V[:, 0] = z / nz
    a, b = [], []
    for j in range(m):
        w = Khat @ V[:, j]
        if j > 0:
            w = w - b[-1] * V[:, j - 1]
        a.append(float(V[:, j] @ w))
        w = w - a[-1] * V[:, j]
        for _ in range(2):
            w = w - V[:, : j + 1] @ (V[:, : j + 1].T @ w)
        beta = float(np.linalg.norm(w))
        if j == m - 1 or beta <= 1e-12 * max(1.0, abs(a[-1])):
            break
        b.append(beta)
        V[:, j + 1] = w / beta
    k = len(a)
    T = np.diag(a) + np.diag(b[: k - 1], 1) + np.diag(b[: k - 1], -1)
    theta, Q = np.linalg.eigh(T)
    return nz * nz * float(np.sum(Q[0, :] ** 2 * np.log(theta)))


def gershgorin_bound(A):
    """max_i sum_j |A_ij|: an upper bound on every eigenvalue of A (Gershgorin)."""
    return float(np.max(np.sum(np.abs(A), axis=1))) if A.shape[0] else 0.0


def taylor_logdet_terms(Khat, Z, m, a):
    """Per-probe terms of the randomized log-determinant of Boutsidis et al.
    (the estimator Sec. 2.5 uses): with C = I - Khat / a (a >= lambda_max),
      ln|Khat| = N ln a + ln|I - C| = N ln a - sum_{k>=1} tr(C^k) / k,
    truncated after m terms, each trace replaced by z^T C^k z for one probe:
      Gamma_l = N ln a - sum_{k=1}^{m} z_l^T C^k z_l / k.
    For Rademacher probes E[z z^T] = I, so the mean of Gamma_l is the
    truncated series.  Z may hold any probe columns."""
    n = Khat.shape[0]
    V = np.array(Z, dtype=np.float64, copy=True)
    acc = np.zeros(V.shape[1])
    for k in range(1, m + 1):
        V = V - (Khat @ V) / a                     # V = C^k Z
        acc += np.sum(Z * V, axis=0) / k           # z^T C^k z / k, per column
    return n * math.log(a) - acc


def logdet_taylor_same_probes(x, h, dim, n1, n2, n_probes, m, seed, beta=1.0):
    """ln|K| by the truncated-Taylor randomized estimator on the same split and
    probes as the GPU path: ln|K| = sum_act ln D + mean_l Gamma_l(Khat)
    + N_inact ln sigma_n^2, Khat = D^-1/2 K_act D^-1/2, a = gershgorin_bound(Khat).
    Returns (logdet, per-probe Gamma, a)."""
    p = unpack_h(h, dim, n1, n2)
    x = np.asarray(x, dtype=np.float64)
    K = dense_K(x, h, dim, n1, n2, beta)
    _, mask = bump_table(x, h, dim, n1, n2, beta)
    act, inact = active_split(K, mask)
    Ka = K[np.ix_(act, act)]
    D = np.diag(Ka).copy()
    Dm = 1.0 / np.sqrt(D)
    Khat = Ka * Dm[:, None] * Dm[None, :]
    if act.size == 0:
        return inact.size * math.log(p["sigma2"]), np.zeros(n_probes), 0.0
    a = gershgorin_bound(Khat)
    gam = taylor_logdet_terms(Khat, rademacher(seed, n_probes, act), m, a)
    logdet = float(np.sum(np.log(D))) + float(np.mean(gam)) + inact.size * math.log(p["sigma2"])
    return logdet, gam, a


def lml_grad_same_probes(x, y, h, dim, n1, n2, n_probes, lanczos_steps, seed,
                         beta=1.0, with_grad=True, with_bounds=False):
    """The stochastic LML and gradient the GPU path estimates, computed densely.

    K splits into the active block K_a (rows inside some bump) and
    sigma_n^2 I on the inactive rows.  With D = diag(K_a) and
    Khat = D^-1/2 K_a D^-1/2, and Rademacher probes z_l on the active rows
    (SplitMix64, original point index as counter):
      ln|K|  ~  sum log D + (1/nv) sum_l SLQ_m(Khat, z_l) + N_inact log sigma_n^2
      y^T K^-1 y exact (dense solve)
      tr(K^-1 K_theta) ~ (1/nv) sum_l z_l^T Khat^-1 Khat_theta z_l
                         + [inactive rows, exact: N_inact / sigma_n^2 for noise]
    where Khat_theta = D^-1/2 K_theta D^-1/2 (D held fixed).
    Returns (lml, grad or None, info dict with the pieces).

    with_bounds=True adds, per parameter, what bounds the gradient's change
    when the solves stop early.  If ahat = Khat^-1 yhat is replaced by
    ahat + Khat^-1 r (residual r) and u_l = Khat^-1 z_l by u_l + Khat^-1 r_l,
    the gradient moves, to first order, by
      r^T Khat^-1 Khat_theta ahat  -  (1/2nv) sum_l r_l^T Khat^-1 Khat_theta z_l,
    so with |r| <= eps |yhat| and |r_l| <= eps |z_l| its change is at most
      eps * (sens_quad + sens_trace / 2),
      sens_quad  = |yhat| |Khat^-1 Khat_theta ahat|,
      sens_trace = (1/nv) sum_l |z_l| |Khat^-1 Khat_theta z_l|.
    It also adds the standard error of the Hutchinson trace over the probes
    (sample standard deviation of z_l^T Khat^-1 Khat_theta z_l over l, / sqrt(nv)),
    which bounds the distance to the exact gradient statistically (the
    estimate's trace part enters the gradient with weight 1/2)."""
    p = unpack_h(h, dim, n1, n2)
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    K = dense_K(x, h, dim, n1, n2, beta)
    _, mask = bump_table(x, h, dim, n1, n2, beta)
    act, inact = active_split(K, mask)
    s2 = p["sigma2"]
    Ka = K[np.ix_(act, act)]
    D = np.diag(Ka).copy()
    Dm = 1.0 / np.sqrt(D)
    Khat = Ka * Dm[:, None] * Dm[None, :]
    Z = rademacher(seed, n_probes, act)
    quad = np.array([lanczos_quadrature(Khat, Z[:, l], lanczos_steps) for l in range(n_probes)]) \
        if act.size else np.zeros(n_probes)
    logdet = float(np.sum(np.log(D))) + (float(np.mean(quad)) if act.size else 0.0) \
        + inact.size * math.log(s2)
    alpha = np.zeros_like(y)
    if act.size:
        alpha[act] = np.linalg.solve(Ka, y[act])
    alpha[inact] = y[inact] / s2
    quad_form = float(y @ alpha)
    lml = -0.5 * quad_form - 0.5 * logdet
    info = {"logdet": logdet, "quad_form": quad_form, "slq_terms": quad, "n_active": int(act.size),
            "alpha": alpha}
    if not with_grad:
        return lml, None, info
    # U_hat = Khat^-1 Z; the estimator per parameter is (1/nv) tr(U_hat^T Khat_theta Z).
    Uhat = np.linalg.solve(Khat, Z) if act.size else np.zeros((0, n_probes))
    npar = len(np.asarray(h))
    grad = np.zeros(npar)
    if with_bounds:
        Kinv = np.linalg.inv(Khat) if act.size else np.zeros((0, 0))
        yhat = y[act] * Dm
        ahat = Kinv @ yhat
        sens_q, sens_t, tr_se = np.zeros(npar), np.zeros(npar), np.zeros(npar)
    for i, dK in dK_dtheta_all(x, h, dim, n1, n2, beta):
        dKa = dK[np.ix_(act, act)]
        dKhat = dKa * Dm[:, None] * Dm[None, :]
        tr_act = float(np.sum(Uhat * (dKhat @ Z))) / n_probes if act.size else 0.0
        tr_inact = float(np.sum(np.diag(dK)[inact])) / s2
        grad[i] = 0.5 * float(alpha @ (dK @ alpha)) - 0.5 * (tr_act + tr_inact)
        if with_bounds and act.size:
            W = Kinv @ (dKhat @ np.column_stack([ahat, Z]))
            sens_q[i] = float(np.linalg.norm(yhat) * np.linalg.norm(W[:, 0]))
            sens_t[i] = float(np.mean(np.linalg.norm(Z, axis=0) * np.linalg.norm(W[:, 1:], axis=0)))
            per_probe = np.sum(Uhat * (dKhat @ Z), axis=0)
            tr_se[i] = float(np.std(per_probe, ddof=1) / math.sqrt(n_probes)) if n_probes > 1 else 0.0
    if with_bounds:
        info.update({"grad_sens_quad": sens_q, "grad_sens_trace": sens_t, "grad_trace_se": tr_se})
    return lml, grad, info


# ----------------------------------------------------------------------------
# Sparsity estimate (Eq. eq:sparsity_estimate and the two equations after it)
# ----------------------------------------------------------------------------

def ball_volume(dim, r):
    """Volume of a dim-dimensional ball: pi^(dim/2) / Gamma(dim/2 + 1) r^dim."""
    return math.pi ** (dim / 2.0) / math.gamma(dim / 2.0 + 1.0) * r ** dim


def sparsity_upper_bound(h, dim, n1, n2, domain_volume=1.0):
    """sum_i sum_j sum_k Vol(r_ij) Vol(r_ik) / Vol(X)^2: the upper bound on the
    fraction of non-zero covariances for uniformly distributed points."""
    p = unpack_h(h, dim, n1, n2)
    total = 0.0
    for i in range(n1):
        v = [ball_volume(dim, r) for r in p["radii"][i]]
        total += sum(v) ** 2
    return total / domain_volume ** 2


def sparsity_upper_bound_grad(h, dim, n1, n2, domain_volume=1.0):
    """d s / d h for the bound above, differentiated by hand: only the bump
    radii enter, with d Vol(dim, r) / d r = dim Vol(dim, r) / r, so
      d s / d r_ij = 2 (sum_k Vol(r_ik)) dim Vol(r_ij) / r_ij / Vol(X)^2."""
    p = unpack_h(h, dim, n1, n2)
    g = np.zeros(len(np.asarray(h)))        # a core length scale, if any, does not enter the bound
    for i in range(n1):
        v = [ball_volume(dim, r) for r in p["radii"][i]]
        tot = sum(v)
        for j in range(n2):
            r = p["radii"][i, j]
            g[(i * n2 + j) * (dim + 2) + dim] = 2.0 * tot * dim * v[j] / r / domain_volume ** 2
    return g


def augmented_objective(lml, grad_lml, h, dim, n1, n2, domain_volume=1.0):
    """Eq. (eq:augmented): ln L + (1 - s) ln L = (2 - s(h)) ln L(h) with s the
    sparsity bound above, and its gradient by the product rule:
      (2 - s) d ln L / d h - ln L d s / d h.
    Returns (value, gradient, s)."""
    s = sparsity_upper_bound(h, dim, n1, n2, domain_volume)
    ds = sparsity_upper_bound_grad(h, dim, n1, n2, domain_volume)
    return (2.0 - s) * lml, (2.0 - s) * np.asarray(grad_lml, dtype=np.float64) - lml * ds, s


# ----------------------------------------------------------------------------
# gradient-based training on the objectives of Sec. 2.4 (Sec. 4 names
# gradient-based optimisation of the hyperparameters as future work and fixes
# no method: the reading here is Adam, Kingma and Ba 2015, Algorithm 1)
# ----------------------------------------------------------------------------
def positive_entries(n_params, dim, n1, n2):
    """Entries of h that must stay positive and are stepped in ln h: every bump
    radius, then r_s, A, sigma_n^2 (and the core length scale, if present)."""
    pos = np.zeros(n_params, dtype=bool)
    for b in range(n1 * n2):
        pos[b * (dim + 2) + dim] = True
    pos[n1 * n2 * (dim + 2):] = True
    return pos


def adam_ascent(objective, h0, positive, n_steps, lr, beta1=0.9, beta2=0.999, eps=1e-8, feasible=None,
                max_halvings=30):
    """Adam ascending objective(h) -> (value, d value / d h, extra) over
    theta = ln h on the positive entries and theta = h elsewhere, so that
    d value / d theta = h * d value / d h there.  Step t = 1, 2, ...:
      m = beta1 m + (1 - beta1) g,  v = beta2 v + (1 - beta2) g^2,
      theta <- theta + lr * (m / (1 - beta1^t)) / (sqrt(v / (1 - beta2^t)) + eps).
    With feasible(h) given (the constraint of Eq. eq:constrained), a step whose
    end is infeasible is halved until it is feasible and not taken after
    max_halvings halvings.  Returns (h_n, [(value, extra) at h_0 .. h_n])."""
    h = np.array(h0, dtype=np.float64)
    m = np.zeros_like(h)
    v = np.zeros_like(h)
    trace = []
    for t in range(1, n_steps + 2):
        value, grad_h, extra = objective(h)
        trace.append((value, extra))
        if t == n_steps + 1:
            break
        g = np.where(positive, h * grad_h, grad_h)
        m = beta1 * m + (1.0 - beta1) * g
        v = beta2 * v + (1.0 - beta2) * g * g
        step = lr * (m / (1.0 - beta1 ** t)) / (np.sqrt(v / (1.0 - beta2 ** t)) + eps)
        f = 1.0
        for _ in range(max_halvings + 1):
            h_new = h + f * step
            h_new[positive] = np.exp(np.log(h[positive]) + f * step[positive])
            if feasible is None or feasible(h_new):
                break
            f *= 0.5
        else:
            h_new = h.copy()
        h = h_new
    return h, trace


def train_same_probes(x, y, h0, dim, n1, n2, n_probes, lanczos_steps, seed, objective, n_steps, lr,
                      beta1=0.9, beta2=0.999, eps=1e-8, domain_volume=1.0, s_max=None, max_halvings=30,
                      beta=1.0):
    """Adam on one of the Sec. 2.4 objectives with the same-probe estimator of
    ln L and its gradient (lml_grad_same_probes) and the sparsity bound s(h):
      "lml"          ln L
      "augmented"    (2 - s) ln L, Eq. eq:augmented
      "constrained"  ln L with every iterate kept at s(h) < s_max, Eq. eq:constrained.
    Returns (h_n, trace rows (objective, ln L, s) at h_0 .. h_n)."""
    h0 = np.asarray(h0, dtype=np.float64)

    def obj(h):
        lml, g, _ = lml_grad_same_probes(x, y, h, dim, n1, n2, n_probes, lanczos_steps, seed, beta=beta)
        if objective == "augmented":
            value, grad, s = augmented_objective(lml, g, h, dim, n1, n2, domain_volume)
        else:
            value, grad, s = lml, g, sparsity_upper_bound(h, dim, n1, n2, domain_volume)
        return value, grad, (lml, s)

    feasible = None
    if objective == "constrained":
        def feasible(h):
            return sparsity_upper_bound(h, dim, n1, n2, domain_volume) < s_max
    h, trace = adam_ascent(obj, h0, positive_entries(len(h0), dim, n1, n2), n_steps, lr, beta1, beta2, eps,
                           feasible, max_halvings)
    return h, np.array([[value, lml, s] for value, (lml, s) in trace])

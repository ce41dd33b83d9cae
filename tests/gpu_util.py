"""Shared helpers of the GPU parity tests (tolerances written out here)."""
import numpy as np

# FP32 overlap: 1e-5 relative on pairs whose FP32 evaluation is well
# conditioned (kappa * 2^-23 * 8 <= 1e-5, f >= 1e-30); every other pair must
# stay within a few times the oracle's FP32 error scale sum (|arg|+4) 2^-23 e.
OVERLAP_RTOL = 1e-5
OVERLAP_BOUND_FACTOR = 3.0
# split-BF16 and FP32 Pearson: absolute error per correlation at the workload
# sizes (long vectors)
PEARSON_ATOL = 1e-6


def shifted_rows(X):
    """The rows as the vector pipeline feeds them to the Gram: centred on a
    per-row shift s_i (the mean of min(D, 1024) values at stride
    floor(D / count)), not on the mean; the exact mean enters afterwards as
    r_ij = (G_ij - D delta_i delta_j) / sqrt(ss_i ss_j), delta = mean - s.
    Rows with D delta^2 > ss / 64 are centred again on their mean.  The
    products whose rounding the allowances bound are those of these rows."""
    X = np.asarray(X, np.float64)
    D = X.shape[1]
    count = min(D, 1024)
    s = X[:, : count * (D // count): D // count].mean(1, keepdims=True)
    mu = X.mean(1, keepdims=True)
    ss = ((X - mu) ** 2).sum(1, keepdims=True)
    again = D * (mu - s) ** 2 > ss / 64
    return X - np.where(again, mu, s)


def pearson_tolerance(X, pi, pj, prec):
    """Per-pair error allowance of the GPU paths for short vectors.

    split-BF16: c = hi + lo + d with |d| <= 2^-16 |c| (two round-to-nearest
    steps at unit roundoff 2^-8), and the dropped lo*lo term is <= 2^-16
    |c_i c_j|, so each product is off by at most 3 * 2^-16 |c_i c_j|; with
    independent signs the sum's error stays within 6 * 2^-16 *
    sqrt(sum_k c_ik^2 c_jk^2), divided by sqrt(ss_i ss_j).  It falls like
    1/sqrt(D) and is far below 1e-6 at D = 2^20.
    FP32: round-to-nearest accumulation over D terms, a random walk of
    relative size ~2^-24 sqrt(D); allowance 2^-22 sqrt(D) |G_ij| /
    sqrt(ss_i ss_j) (|r| for rows centred on their exact means).
    c here are the shifted rows (see shifted_rows); ss the centred sums.
    """
    X = np.asarray(X, np.float64)
    C = X - X.mean(1, keepdims=True)
    ss = (C * C).sum(1)
    Cs = shifted_rows(X)
    D = X.shape[1]
    if prec == 1:
        S2 = Cs * Cs
        num = np.sqrt(np.einsum("pk,pk->p", S2[pi], S2[pj]))
        return PEARSON_ATOL + 6 * 2.0 ** -16 * num / np.sqrt(ss[pi] * ss[pj])
    g = np.einsum("pk,pk->p", Cs[pi], Cs[pj]) / np.sqrt(ss[pi] * ss[pj])
    return PEARSON_ATOL + 2.0 ** -22 * np.sqrt(D) * np.abs(g)
def regroup_tolerance(X, pi, pj, chain=256):
    """Allowance between two split-BF16 results that differ only in how the
    same products are grouped into tensor-core chains (whole tiles against
    split-K units, resident against out-of-core).

    A chain adds at most 3 * chain products in FP32; each partial sum rounds
    with relative error <= 2^-23 (2^-24 round-to-nearest, 2^-23 if the
    accumulator truncates), a random walk of about 2^-23 sqrt(3 chain) S_c
    for a chain whose |products| sum to S_c.  Chains round independently, so
    one result is off by about 2^-23 sqrt(3 chain) sqrt(sum_c S_c^2); two
    results, and a factor 4 for the tail: 8 * 2^-23 sqrt(3 chain)
    sqrt(sum_c S_c^2) / sqrt(ss_i ss_j), the products those of the shifted
    rows (see shifted_rows).  A lost or doubled 64-column range
    moves r by about its share of sum |c_i c_j|, orders of magnitude more.
    """
    X = np.asarray(X, np.float64)
    C = np.abs(shifted_rows(X))
    n, D = C.shape
    Cm = X - X.mean(1, keepdims=True)
    ss = (Cm * Cm).sum(1)
    nc = (D + chain - 1) // chain
    Cp = np.zeros((n, nc * chain))
    Cp[:, :D] = C
    out = np.empty(len(pi))
    m = max(1, (1 << 24) // (nc * chain))
    for a in range(0, len(pi), m):
        b = min(len(pi), a + m)
        S = (Cp[pi[a:b]] * Cp[pj[a:b]]).reshape(b - a, nc, chain).sum(-1)
        out[a:b] = np.sqrt((S * S).sum(1))
    return 1e-12 + 8 * 2.0 ** -23 * np.sqrt(3 * chain) * out / np.sqrt(ss[pi] * ss[pj])

# adjoint: norm-wise, |g - g_ref|_inf <= 1e-4 max(|g_ref|_inf, 1e-6 sum w w)
GRAD_RTOL = 1e-4


def check_overlap(f_gpu, f_ref, kappa, bound, what=""):
    f_gpu = np.asarray(f_gpu, np.float64)
    err = np.abs(f_gpu - f_ref)
    good = (kappa * 2.0 ** -23 * 8 <= 1e-5) & (f_ref >= 1e-30)
    rel = err[good] / np.abs(f_ref[good])
    assert good.mean() > 0.5, f"{what}: too few well-conditioned pairs ({good.mean():.3f})"
    assert rel.max(initial=0.0) <= OVERLAP_RTOL, \
        f"{what}: max rel err {rel.max():.3e} at {np.argmax(rel)}"
    bad = ~good
    if bad.any():
        lim = np.maximum(OVERLAP_BOUND_FACTOR * bound[bad], OVERLAP_RTOL * np.abs(f_ref[bad]))
        over = err[bad] > lim + 1e-37
        assert not over.any(), f"{what}: {over.sum()} ill-conditioned pairs beyond bound"
    return float(rel.max(initial=0.0))


def check_grad(g_gpu, g_ref, wsum):
    g_gpu = np.asarray(g_gpu, np.float64)
    scale = np.maximum(np.abs(g_ref).max(1), 1e-6 * wsum)
    err = np.abs(g_gpu - g_ref).max(1)
    worst = float((err / scale).max())
    assert worst <= GRAD_RTOL, f"grad norm-wise rel err {worst:.3e}"
    return worst


def cloud_wsum(c, pi, pj):
    off = c["offsets"]
    w = c.get("weight")
    if w is None:
        sz = np.diff(off)
        return sz[pi] * sz[pj]
    cs = np.concatenate([[0.0], np.cumsum(np.asarray(w, np.float64))])
    ws = cs[off[1:]] - cs[off[:-1]]
    return ws[pi] * ws[pj]

"""Seeded synthetic inputs for the all-pairs workloads.

This module only draws random inputs; it holds none of the method's
arithmetic.  Both the CUDA path (through the binding) and the FP64 oracle are
fed the very same arrays produced here.

Point clouds use numpy's counter-based Philox generator; dense vectors are
drawn with torch's seeded generator on the device they are needed on (the
large vector sets are generated directly in GPU memory; the oracle then reads
back the rows it checks).  The shapes and distributions stand in for the
paper's data sets, which are not available: localisation-microscopy particles
(Sec. V-C), irregular comparison costs (Sec. VII, Fig. 6) and dense FP32 noise
patterns as in the forensics application (Sec. V-A).
"""
from __future__ import annotations

import numpy as np


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(int(seed)))


def _clouds_from_sizes(rng, sizes, dim, coord, sigma):
    sizes = np.asarray(sizes, np.int64)
    off = np.zeros(len(sizes) + 1, np.int64)
    np.cumsum(sizes, out=off[1:])
    tot = int(off[-1])
    pts = rng.uniform(coord[0], coord[1], size=(tot, dim)).astype(np.float32)
    sig = rng.uniform(sigma[0], sigma[1], size=tot).astype(np.float32)
    out = {"dim": dim, "offsets": off, "x": np.ascontiguousarray(pts[:, 0]),
           "y": np.ascontiguousarray(pts[:, 1]), "sigma": sig,
           "weight": np.ones(tot, np.float32)}
    out["z"] = np.ascontiguousarray(pts[:, 2]) if dim == 3 else None
    return out


def clouds_uniform(n: int = 256, dim: int = 2, size=(64, 128), coord=(-1.0, 1.0),
                   sigma=(0.02, 0.05), seed: int = 0) -> dict:
    """n clouds, sizes uniform in [size[0], size[1]], points uniform in the box,
    per-point sigma uniform, weights 1 (the small plain workload: 256 2-D clouds
    of 64-128 points, sigma in [0.02, 0.05])."""
    rng = _rng(seed)
    sizes = rng.integers(size[0], size[1] + 1, size=n)
    return _clouds_from_sizes(rng, sizes, dim, coord, sigma)


def lognormal_sizes(n: int, median: float = 300.0, shape: float = 1.0,
                    clip=(50, 5000), seed: int = 0) -> np.ndarray:
    rng = _rng(seed)
    s = np.exp(np.log(median) + shape * rng.standard_normal(n))
    return np.clip(np.rint(s), clip[0], clip[1]).astype(np.int64)


def clouds_lognormal(n: int = 20000, dim: int = 3, median: float = 300.0,
                     shape: float = 1.0, clip=(50, 5000), coord=(-1.0, 1.0),
                     sigma=(0.01, 0.05), seed: int = 0) -> dict:
    """Uneven clouds for the batching workload: sizes lognormal (median 300,
    log-sd 1.0) clipped to [50, 5000], 3-D points uniform in [-1, 1]^3,
    sigma uniform in [0.01, 0.05], weights 1."""
    sizes = lognormal_sizes(n, median, shape, clip, seed)
    rng = _rng(seed + 7919)
    return _clouds_from_sizes(rng, sizes, dim, coord, sigma)


def clouds_templates(n: int = 1024, n_templates: int = 8, template_pts: int = 400,
                     size=(100, 400), jitter: float = 0.01, sigma=(0.02, 0.05),
                     seed: int = 0) -> dict:
    """Registration workload: cloud i keeps n_i ~ U{100..400} points of template
    (i mod 8) (400 points uniform in [-0.5, 0.5]^2), drawn without replacement,
    moved by a random rotation theta ~ U[-pi, pi) and translation
    t ~ U[-0.5, 0.5]^2, plus N(0, jitter^2) noise; sigma ~ U[0.02, 0.05].
    Also returns the generating poses (``theta``, ``t``) and template ids."""
    rng = _rng(seed)
    templ = rng.uniform(-0.5, 0.5, size=(n_templates, template_pts, 2))
    sizes = rng.integers(size[0], size[1] + 1, size=n)
    theta = rng.uniform(-np.pi, np.pi, size=n)
    trans = rng.uniform(-0.5, 0.5, size=(n, 2))
    off = np.zeros(n + 1, np.int64)
    np.cumsum(sizes, out=off[1:])
    xs = np.empty(int(off[-1]), np.float64)
    ys = np.empty(int(off[-1]), np.float64)
    for i in range(n):
        pick = rng.choice(template_pts, size=int(sizes[i]), replace=False)
        p = templ[i % n_templates, pick]
        c, s = np.cos(theta[i]), np.sin(theta[i])
        px = c * p[:, 0] - s * p[:, 1] + trans[i, 0]
        py = s * p[:, 0] + c * p[:, 1] + trans[i, 1]
        px = px + jitter * rng.standard_normal(len(pick))
        py = py + jitter * rng.standard_normal(len(pick))
        xs[off[i]:off[i + 1]] = px
        ys[off[i]:off[i + 1]] = py
    sig = rng.uniform(sigma[0], sigma[1], size=int(off[-1])).astype(np.float32)
    return {"dim": 2, "offsets": off, "x": xs.astype(np.float32),
            "y": ys.astype(np.float32), "z": None, "sigma": sig,
            "weight": np.ones(int(off[-1]), np.float32), "theta": theta,
            "t": trans, "template": np.arange(n) % n_templates}


def group_ids(n: int, group: int = 16, seed: int = 0) -> np.ndarray:
    """A seeded permutation of 0..n-1 cut into consecutive groups of ``group``:
    returns the group id of every item."""
    perm = _rng(seed + 104729).permutation(n)
    gid = np.empty(n, np.int64)
    gid[perm] = np.arange(n) // group
    return gid


def vectors_grouped(n: int, D: int, group: int = 16, shared_weight: float = 0.05,
                    seed: int = 0, device="cpu", chunk_rows: int = 512):
    """Dense FP32 noise vectors: x_i = eps_i + w * g_{group(i)}, eps and g i.i.d.
    N(0, 1), groups of 16 from a seeded permutation (the correlation workloads).
    Returns a torch tensor [n, D] float32 on ``device`` (generated there)."""
    import torch

    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    n_groups = (n + group - 1) // group
    X = torch.randn(n, D, generator=gen, device=device, dtype=torch.float32)
    shared = torch.randn(n_groups, D, generator=gen, device=device, dtype=torch.float32)
    gid = torch.from_numpy(group_ids(n, group, seed)).to(device)
    for r0 in range(0, n, chunk_rows):
        r1 = min(n, r0 + chunk_rows)
        X[r0:r1].add_(shared.index_select(0, gid[r0:r1]), alpha=shared_weight)
    del shared
    return X


def sparse_cv(n: int, dim: int = 20 ** 6, nnz=(100_000, 1_800_000), common: int = 4_000_000,
              common_boost: float = 8.0, shared_weight: float = 0.6, seed: int = 0,
              device="cpu", sizes=None, as_torch: bool = False):
    """Synthetic composition vectors (the bioinformatics workload's shape):
    sparse rows over a k-mer index space of ``dim`` codes (20^6 for k = 6),
    nnz_i ~ U[nnz[0], nnz[1]] (or ``sizes``), indices drawn per code with a
    probability ``common_boost`` times higher in the first ``common`` codes
    (frequent k-mers shared by most species), values v = shared_weight *
    g[code] + N(0, 1) with one global g ~ N(0, 1), so rows correlate on the
    codes they share.  Returns (offsets int64 [n+1], indices int32 [nnz]
    sorted per row, values float32 [nnz]) as numpy arrays; the draws run on
    ``device`` with torch's seeded generator (``as_torch``: indices and values
    stay torch tensors on ``device``)."""
    import torch

    rng = _rng(seed + 15485863)
    if sizes is None:
        sizes = rng.integers(nnz[0], nnz[1] + 1, size=n)
    sizes = np.asarray(sizes, np.int64)
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    common = min(common, dim)
    w_common = common_boost
    w_rest = (dim - common * common_boost / 1.0) / max(dim - common, 1) if dim > common else 0.0
    w_rest = max(w_rest, 0.05)
    g = torch.randn(dim, generator=gen, device=device, dtype=torch.float32)
    off = np.zeros(n + 1, np.int64)
    idx_parts, val_parts = [], []
    for i in range(n):
        p = float(sizes[i]) / dim
        u = torch.rand(dim, generator=gen, device=device)
        thr = torch.full((dim,), p * w_rest, device=device)
        thr[:common] = min(1.0, p * w_common)
        ids = torch.nonzero(u < thr).flatten()
        vals = shared_weight * g[ids] + torch.randn(len(ids), generator=gen, device=device)
        if as_torch:
            idx_parts.append(ids.to(torch.int32))
            val_parts.append(vals.float())
        else:
            idx_parts.append(ids.to(torch.int32).cpu().numpy())
            val_parts.append(vals.float().cpu().numpy())
        off[i + 1] = off[i] + len(ids)
    if as_torch:
        return (off, torch.cat(idx_parts) if n else torch.zeros(0, dtype=torch.int32),
                torch.cat(val_parts) if n else torch.zeros(0))
    return (off, np.concatenate(idx_parts) if n else np.zeros(0, np.int32),
            np.concatenate(val_parts) if n else np.zeros(0, np.float32))


# Workload shapes (seed 0 unless stated)
WORKLOADS = {
    "overlap2d_n256": dict(kind="clouds_uniform", n=256, dim=2, size=(64, 128),
                           sigma=(0.02, 0.05)),
    "pearson_n8192_d1m": dict(kind="vectors", n=8192, D=1 << 20),
    "overlap3d_n20000_lognormal": dict(kind="clouds_lognormal", n=20000),
    "register2d_n1024": dict(kind="clouds_templates", n=1024),
}

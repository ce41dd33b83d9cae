"""Parity at the full workload sizes, in the launch configuration the
benchmark uses (tuned plan, graph replay), on sampled outputs the FP64
oracle computes one by one:

* 20,000 lognormal 3-D clouds (2e8 pairs): every pair among the 32 largest
  clouds, the first and last rows, and random pairs;
* 1024 template clouds, 20 ascent steps, teacher-forced: at every step the
  GPU's f and update on sampled pairs equal the oracle's at the GPU's own
  parameters;
* the out-of-core correlation, 8192 x 3*2^20 FP32 in page-locked host memory
  through a 48 GiB slot cache, on sampled pairs.
"""
import numpy as np
import pytest

import synth
from gpu_util import PEARSON_ATOL, check_overlap

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ap():
    import paper_2009_04755_gb300 as ap
    ap.lib()
    return ap


def _pidx(pi, pj, n):
    pi = np.asarray(pi, np.int64)
    pj = np.asarray(pj, np.int64)
    return pi * n - pi * (pi + 1) // 2 + (pj - pi - 1)


def test_overlap3d_n20000_sampled(ap, oracle_lib):
    n = 20000
    c = synth.clouds_lognormal(n=n, dim=3, seed=0)
    sizes = np.diff(c["offsets"])
    big = np.sort(np.argsort(sizes)[-32:])
    pi, pj = [], []
    for x in range(len(big)):
        for y in range(x + 1, len(big)):
            pi.append(big[x]); pj.append(big[y])
    for j in range(1, n, 997):
        pi.append(0); pj.append(j)
    pi.append(n - 2); pj.append(n - 1)
    rng = np.random.default_rng(0)
    a = rng.integers(0, n - 1, 800)
    b = rng.integers(0, n, 800)
    keep = a < b
    pi = np.concatenate([pi, a[keep]]).astype(np.int64)
    pj = np.concatenate([pj, b[keep]]).astype(np.int64)
    with ap.Items.from_clouds(c) as it:
        it.tune(0)
        f = it.run_pairs()
        torch.cuda.synchronize()
        assert it.last_device_error() == 0
        got = f[torch.from_numpy(_pidx(pi, pj, n)).cuda()].double().cpu().numpy()
        assert torch.isfinite(f).all() and float(f.min()) >= 0.0
    ref, kappa, bound = oracle_lib.overlap(c, pi, pj, with_cond=True)
    check_overlap(got, ref, kappa, bound, "3d n20000")


def test_register2d_n1024_teacher_forced(ap, oracle_lib):
    n, steps, eta = 1024, 20, 1e-3
    c = synth.clouds_templates(n=n, seed=0)
    rng = np.random.default_rng(1)
    a = rng.integers(0, n - 1, 600)
    b = rng.integers(0, n, 600)
    keep = a < b
    pi, pj = a[keep][:250], b[keep][:250]
    sel = torch.from_numpy(_pidx(pi, pj, n)).cuda()
    P = n * (n - 1) // 2
    with ap.Items.from_clouds(c) as it:
        it.tune(1)
        p = torch.zeros(P, 3, device="cuda")
        for _ in range(steps):
            pk = p[sel].double().cpu().numpy()
            f_ref, g_ref = oracle_lib.overlap_grad(c, pi, pj, pk)
            p, f, flags = it.ascent(p, 1, eta)
            fk = f[sel].double().cpu().numpy()
            step = p[sel].double().cpu().numpy() - pk
            assert np.all(np.abs(fk - f_ref) <= 1e-5 * f_ref + 1e-30)
            want = eta * g_ref / f_ref[:, None]
            scale = np.maximum(np.abs(want).max(1), 1e-7)
            ulp = np.abs(pk).max(1) * 2.0 ** -23 / scale
            assert np.all(np.abs(step - want).max(1) / scale <= 1e-4 + 2 * ulp)
            assert not bool(flags.any())
        assert it.last_device_error() == 0


def test_pearson_out_of_core_8192x3m_sampled(ap, oracle_lib):
    n, D, cache = 8192, 3 << 20, 48 << 30
    Xh = torch.empty(n, D, dtype=torch.float32, pin_memory=True)
    chunk = 1024
    for r0 in range(0, n, chunk):
        Xd = synth.vectors_grouped(chunk, D, seed=1000 + r0 // chunk, device="cuda")
        Xh[r0:r0 + chunk].copy_(Xd)
        del Xd
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    rng = np.random.default_rng(5)
    rows = np.sort(rng.choice(n, 48, replace=False))
    pi, pj = np.triu_indices(len(rows), 1)
    gi, gj = rows[pi], rows[pj]
    with ap.Items.from_vectors(Xh, slot_cache_bytes=cache) as it:
        r = it.run_pairs()
        torch.cuda.synchronize()
        st = it.stats()
        assert it.last_device_error() == 0
        got = r[torch.from_numpy(_pidx(gi, gj, n)).cuda()].cpu().numpy()
    sub = Xh.numpy()[rows]
    ref = oracle_lib.pearson(sub, pi, pj)
    assert np.abs(got - ref).max() <= PEARSON_ATOL
    assert abs(st["reuse_R"] - 1.625) < 1e-9
    assert st["h2d_bytes"] == int(1.625 * n) * D * 4
    del Xh

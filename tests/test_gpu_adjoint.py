"""GPU parity of the overlap adjoint, the autograd wrapper and the fused
batched ascent step against the FP64 oracle (analytic gradient, and the
oracle's own pin to central finite differences)."""
import numpy as np
import pytest

import synth
from gpu_util import check_grad, check_overlap, cloud_wsum

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ap():
    import paper_2009_04755_gb300 as ap
    ap.lib()
    return ap


def _params(P, seed, spread=0.3):
    rng = np.random.default_rng(seed)
    return np.stack([rng.uniform(-np.pi, np.pi, P), rng.uniform(-spread, spread, P),
                     rng.uniform(-spread, spread, P)], 1).astype(np.float32)


def test_backward_matches_oracle_gradient(ap, oracle_lib):
    n = 48
    c = synth.clouds_templates(n=n, seed=7)
    pi, pj = oracle_lib.all_pairs(n)
    prm = _params(len(pi), 1)
    f_ref, g_ref = oracle_lib.overlap_grad(c, pi, pj, prm.astype(np.float64))
    _, kappa, bound = oracle_lib.overlap(c, pi, pj, params=prm.astype(np.float64), with_cond=True)
    with ap.Items.from_clouds(c) as it:
        g, f = it.backward(params=torch.from_numpy(prm).cuda())
        g, f = g.cpu().numpy(), f.cpu().numpy()
        go = torch.full((len(pi),), 2.0, device="cuda")
        g2, _ = it.backward(params=torch.from_numpy(prm).cuda(), grad_out=go)
    check_overlap(f, f_ref, kappa, bound, "adjoint f")
    check_grad(g, g_ref, cloud_wsum(c, pi, pj))
    np.testing.assert_allclose(g2.cpu().numpy(), 2 * g, rtol=1e-6, atol=0)


def test_backward_at_identity(ap, oracle_lib):
    n = 20
    c = synth.clouds_templates(n=n, seed=2)
    pi, pj = oracle_lib.all_pairs(n)
    f_ref, g_ref = oracle_lib.overlap_grad(c, pi, pj, None)
    with ap.Items.from_clouds(c) as it:
        g, f = it.backward(params=None)
    check_grad(g.cpu().numpy(), g_ref, cloud_wsum(c, pi, pj))


def test_autograd_function(ap, oracle_lib):
    from paper_2009_04755_gb300.autograd import overlap_align
    n = 24
    c = synth.clouds_templates(n=n, seed=5)
    pi, pj = oracle_lib.all_pairs(n)
    prm = _params(len(pi), 3)
    w = np.random.default_rng(0).uniform(0.5, 1.5, len(pi))
    f_ref, g_ref = oracle_lib.overlap_grad(c, pi, pj, prm.astype(np.float64))
    with ap.Items.from_clouds(c) as it:
        p = torch.from_numpy(prm).cuda().requires_grad_(True)
        f = overlap_align(it, p)
        (f * torch.from_numpy(w).float().cuda()).sum().backward()
        grad = p.grad.cpu().numpy()
    check_grad(grad, g_ref * w[:, None], cloud_wsum(c, pi, pj) * w)


def test_ascent_teacher_forced(ap, oracle_lib):
    """At every step the GPU's update from its own parameters p_k must equal
    the oracle's eta * grad f / f evaluated at p_k."""
    n = 32
    c = synth.clouds_templates(n=n, seed=11)
    pi, pj = oracle_lib.all_pairs(n)
    eta = 1e-3
    with ap.Items.from_clouds(c) as it:
        p = torch.zeros(len(pi), 3, device="cuda")
        for _ in range(3):
            pk = p.cpu().numpy().astype(np.float64)
            f_ref, g_ref = oracle_lib.overlap_grad(c, pi, pj, pk)
            p, f, flags = it.ascent(p, 1, eta, fmin=1e-30)
            step = p.cpu().numpy().astype(np.float64) - pk
            want = eta * g_ref / f_ref[:, None]
            scale = np.maximum(np.abs(want).max(1), 1e-7)
            err = np.abs(step - want).max(1) / scale
            # the step is formed in FP32 from p_k: allow for the rounding of p_k + step
            ulp = np.abs(pk).max(1) * 2.0 ** -23 / scale
            assert np.all(err <= 1e-4 + 2 * ulp), float((err - 2 * ulp).max())
            assert not flags.any()


def test_ascent_20_steps_increases_cost(ap):
    n = 64
    c = synth.clouds_templates(n=n, seed=13)
    with ap.Items.from_clouds(c) as it:
        p = torch.zeros(n * (n - 1) // 2, 3, device="cuda")
        f0 = it.run_pairs(params=p).clone()
        p, f, flags = it.ascent(p, 20, 1e-3)
        f1 = it.run_pairs(params=p)
    # ascent on log f: the mean log-cost goes up
    assert float(torch.log(f1).mean()) > float(torch.log(f0).mean())

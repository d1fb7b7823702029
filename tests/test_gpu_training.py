"""Training-loop options around the hot path, through the C ABI, against the
oracle: local-energy clipping in the VMC gradient (per-geometry median and
mean absolute deviation on the device) and proposal-width adaptation from the
acceptance fraction (width kept in device memory)."""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_2011_07125_gb300 import synth
from helpers import setup

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_GRAD_FP32 = 1e-3


def make(wl, P, precision="fp32"):
    from paper_2011_07125_gb300.binding import FermiNet
    fn = FermiNet(wl.net, wl.geoms, counts=wl.counts, precision=precision)
    fn.set_params(torch.from_numpy(P).cuda())
    return fn


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _energies(B, seed):
    e = (np.random.default_rng(seed).standard_normal(B) * 2 - 7).astype(np.float32)
    e[::7] += 300.0   # outliers above and below the band
    e[3::11] -= 500.0
    return e


@pytest.mark.parametrize("name,counts", [("li", [33]), ("c4h4x8", [3, 4, 5, 2, 6, 1, 7, 8])])
@pytest.mark.parametrize("scale", [5.0, 0.7])
def test_clipped_gradient_matches_oracle(name, counts, scale):
    """Odd and even per-geometry counts (medians of one and of two middle
    values), outliers on both sides."""
    wl = dataclasses.replace(synth.workload(name), counts=counts)
    lay = oracle.layout(wl.net)
    P = synth.init_params(lay)
    x = synth.init_walkers(wl)
    geo = synth.geometry_of_walkers(counts)
    eloc = _energies(len(x), 4)
    fn = make(wl, P)
    fn.set_train_opts(clip_scale=scale)
    em, g = fn.energy_grad(cuda(x), cuda(eloc))
    assert fn.sync() == "FN_OK"
    em_o, g_o = oracle.energy_grad_clipped(wl.net, P, wl.geoms, x, eloc, scale, geo=geo)
    np.testing.assert_allclose(em.cpu().numpy(), em_o, rtol=1e-12, atol=1e-12)
    err = np.linalg.norm(g.cpu().numpy() - g_o) / np.linalg.norm(g_o)
    print(name, scale, "clipped gradient rel L2", err)
    assert err < TOL_GRAD_FP32
    # clipping changes the gradient here (the outliers are outside the band)
    _, g_plain = oracle.energy_grad(wl.net, P, wl.geoms, x, eloc, geo=geo)
    assert np.linalg.norm(g_plain - g_o) > 10 * TOL_GRAD_FP32 * np.linalg.norm(g_o)
    # the replica form refuses clipping
    from paper_2011_07125_gb300.binding import FermiNetError
    with pytest.raises(FermiNetError):
        fn.energy_grad_partial(cuda(x), cuda(eloc), fn.energy_sums(cuda(eloc)), fn.walker_counts(len(x)))
    fn.close()


def test_wide_clip_band_is_the_plain_gradient():
    wl, lay, P, x, geo = setup("li", 24)
    eloc = (np.random.default_rng(5).standard_normal(24) - 7).astype(np.float32)
    fn = make(wl, P)
    em0, g0 = fn.energy_grad(cuda(x), cuda(eloc))
    fn.set_train_opts(clip_scale=1e6)
    em1, g1 = fn.energy_grad(cuda(x), cuda(eloc))
    assert fn.sync() == "FN_OK"
    assert torch.equal(em0, em1)
    assert float((g1 - g0).norm() / g0.norm()) < 1e-6


@pytest.mark.parametrize("width0", [0.02, 0.6])
def test_width_adaptation_matches_oracle(width0):
    """Moves with the width in device memory equal moves with the same width
    passed by value (same Philox streams), and the width afterwards is the
    oracle's adaptation of it from the accepted counts."""
    wl, lay, P, x, geo = setup("li", 64)
    fn = make(wl, P)
    xa, xb = cuda(x), cuda(x)
    la = fn.logpsi(xa, with_sign=False)
    lb = la.clone()
    acc_a = fn.mcmc_step(xa, la, 5, width0, 9, 40)
    w = torch.tensor([width0], dtype=torch.float32, device="cuda")
    fn.set_train_opts(width=w, accept_lo=0.5, accept_hi=0.55, width_factor=1.1)
    acc_b = fn.mcmc_step(xb, lb, 5, 123.0, 9, 40)  # the width argument is ignored
    assert fn.sync() == "FN_OK"
    assert torch.equal(xa, xb) and torch.equal(la, lb) and torch.equal(acc_a, acc_b)
    # the library holds the band and the factor as float32
    lo, hi, fac = (float(np.float32(v)) for v in (0.5, 0.55, 1.1))
    want = oracle.adapt_width(np.float32(width0), int(acc_b.sum()), 64 * 5, lo, hi, fac)
    assert float(w.item()) == float(np.float32(want))
    # without an accepted-count buffer the library counts internally
    w2 = w.clone()
    fn.set_train_opts(width=w2, accept_lo=0.5, accept_hi=0.55, width_factor=1.1)
    acc_c = fn.mcmc_step(xa, la, 3, 0.0, 9, 50)
    fn.set_train_opts(width=w, accept_lo=0.5, accept_hi=0.55, width_factor=1.1)
    fn.lib.ferminet_mcmc_step(fn.ctx, xb.data_ptr(), lb.data_ptr(), 64, 3, 0.0, 9, 50, None)
    assert fn.sync() == "FN_OK"
    assert torch.equal(xa, xb) and torch.equal(w, w2)
    want = oracle.adapt_width(float(np.float32(want)), int(acc_c.sum()), 64 * 3, lo, hi, fac)
    assert float(w.item()) == float(np.float32(want))
    fn.close()


def test_adaptation_drives_acceptance_into_the_band():
    """Repeated calls move the acceptance fraction towards [0.4, 0.6]."""
    wl, lay, P, x, geo = setup("ne", 256)
    fn = make(wl, P)
    xx = cuda(x)
    lp = fn.logpsi(xx, with_sign=False)
    w = torch.tensor([2.0], dtype=torch.float32, device="cuda")  # far too wide: nearly nothing accepted
    fn.set_train_opts(width=w, accept_lo=0.4, accept_hi=0.6, width_factor=1.25)
    fracs = []
    for k in range(40):
        acc = fn.mcmc_step(xx, lp, 5, 0.0, 3, 5 * k)
        fracs.append(float(acc.sum()) / (256 * 5))
    assert fn.sync() == "FN_OK"
    print("acceptance", fracs[0], "->", fracs[-5:], "width", float(w.item()))
    assert fracs[0] < 0.2
    assert 0.3 < np.mean(fracs[-5:]) < 0.7
    fn.close()


@pytest.mark.parametrize("prec", ["fp32", "mixed"])
def test_training_step_graph_matches_calls(prec):
    """ferminet_step with clipping and width adaptation, replayed from its
    CUDA graph, equals the separate calls bit for bit over two steps."""
    wl, lay, P, x, geo = setup("c4h4x8", 3)
    fn = make(wl, P, prec)
    xa, xb = cuda(x), cuda(x)
    la = fn.logpsi(xa, with_sign=False)
    lb = la.clone()
    wa = torch.tensor([0.3], dtype=torch.float32, device="cuda")
    wb = wa.clone()
    for k in range(2):
        ctr = 100 + 7 * k
        fn.set_train_opts(clip_scale=3.0, width=wa)
        acc = fn.mcmc_step(xa, la, 3, 0.0, 9, ctr)
        e = fn.local_energy(xa)["eloc"]
        em, g = fn.energy_grad(xa, e)
        fn.set_train_opts(clip_scale=3.0, width=wb)
        o = fn.step(xb, lb, 3, 0.0, 9, ctr, use_graph=True)
        assert fn.sync() == "FN_OK"
        assert torch.equal(xa, xb) and torch.equal(la, lb) and torch.equal(wa, wb)
        assert torch.equal(acc, o["accepted"])
        assert torch.equal(e, o["eloc"]) and torch.equal(em, o["emean"]) and torch.equal(g, o["grad"])
    fn.close()

"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Every comparison uses the same seeded float32 inputs on both sides.  FP32-path
bars: log|psi| within 1e-5 relative (to max(|log psi|, 1)) and the local energy
within 1e-4 Ha per walker and 1e-5 Ha on the batch mean, each widened by the
FP32 rounding term of helpers.py where the walker sits near a node of psi;
parameter gradients within 1e-3 relative L2 (FP32 accumulation over walkers
whose orbital matrices may be ill-conditioned).
"""
import os

import numpy as np
import pytest

import oracle
from paper_2011_07125_gb300 import synth
from helpers import (TOL_ELOC_ABS, TOL_LOGPSI_REL, U32, U_MIXED, conditioning, gamma, eloc_bound, emean_bound,
                     equilibrated, logpsi_bound, rel_err, setup)

TOL_GRAD_FP32 = 1e-3

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = [("li", None), ("ne", 24), ("ar", 6), ("c4h6", 4), ("c4h4x8", 2), ("kr", 3)]


def make(wl, P, precision="fp32"):
    from paper_2011_07125_gb300.binding import FermiNet
    fn = FermiNet(wl.net, wl.geoms, counts=wl.counts, precision=precision)
    fn.set_params(torch.from_numpy(P).cuda())
    return fn


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("name,per", CASES)
def test_logpsi(name, per):
    wl, lay, P, x, geo = setup(name, per)
    fn = make(wl, P)
    lp, sg = fn.logpsi(cuda(x))
    ref = oracle.local_energy(wl.net, P, wl.geoms, x, geo=geo) if per else None
    lp_o, sg_o = oracle.logpsi(wl.net, P, wl.geoms, x, geo=geo)
    assert fn.sync() == "FN_OK"
    d = np.abs(lp.cpu().numpy() - lp_o)
    print(name, "logpsi max rel err", rel_err(lp.cpu().numpy(), lp_o).max())
    assert np.array_equal(sg.cpu().numpy(), sg_o)
    bound = logpsi_bound(wl.net, ref) if ref is not None else TOL_LOGPSI_REL * np.maximum(np.abs(lp_o), 1)
    assert np.all(d <= bound), (d / bound).max()


@pytest.mark.parametrize("name,per", CASES)
def test_local_energy(name, per):
    wl, lay, P, x, geo = setup(name, per)
    fn = make(wl, P)
    out = fn.local_energy(cuda(x))
    ref = oracle.local_energy(wl.net, P, wl.geoms, x, geo=geo)
    assert fn.sync() == "FN_OK"
    e = out["eloc"].cpu().numpy().astype(np.float64)
    de = np.abs(e - ref["eloc"])
    print(name, "E_L max abs err", de.max(), "mean err", abs(e.mean() - ref["eloc"].mean()),
          "kinetic err", np.abs(out["kinetic"].cpu().numpy() - ref["kinetic"]).max(),
          "|E_L| max", np.abs(ref["eloc"]).max())
    S, _ = conditioning(ref)
    strict = gamma(wl.net) * U32 * S < 0.1 * TOL_ELOC_ABS  # rounding floor well below the bar
    print(name, "walkers", len(e), "well-conditioned", int(strict.sum()),
          "max err there", de[strict].max() if strict.any() else None)
    assert np.all(np.abs(out["logpsi"].cpu().numpy() - ref["logpsi"]) <= logpsi_bound(wl.net, ref))
    assert np.array_equal(out["sign"].cpu().numpy(), ref["sign"])
    bound = eloc_bound(wl.net, ref)
    assert np.all(de <= bound), (de / bound).max()
    assert abs(e.mean() - ref["eloc"].mean()) <= emean_bound(wl.net, ref)
    if strict.any():
        assert de[strict].max() < TOL_ELOC_ABS


@pytest.mark.parametrize("name", ["ne", "ar", "c4h6"])
def test_fp32_unwidened_bars_on_sampled_walkers(name):
    """On 48 walkers sampled from |psi|^2, the share of walkers inside the
    unwidened FP32 bars (1e-4 Ha per walker, 1e-5 relative on log|psi|) is
    gated, besides every walker inside its widened bar (measured shares on
    GB300: 0.88 to 1.0 for E_L, 1.0 for log|psi|)."""
    wl, P, xs = equilibrated(name, 48)
    ref = oracle.local_energy(wl.net, P, wl.geoms[:1], xs)
    from paper_2011_07125_gb300.binding import FermiNet
    fn = FermiNet(wl.net, wl.geoms[:1], counts=[len(xs)], precision="fp32")
    fn.set_params(torch.from_numpy(P).cuda())
    out = fn.local_energy(cuda(xs))
    assert fn.sync() == "FN_OK"
    de = np.abs(out["eloc"].cpu().numpy().astype(np.float64) - ref["eloc"])
    rl = rel_err(out["logpsi"].cpu().numpy(), ref["logpsi"])
    f_e, f_l = np.mean(de <= TOL_ELOC_ABS), np.mean(rl <= TOL_LOGPSI_REL)
    print(name, "share within 1e-4 Ha", f_e, "share within 1e-5 rel", f_l, "batch-mean err",
          abs(de.mean()))
    assert f_e >= 0.8 and f_l >= 0.95
    assert np.all(de <= eloc_bound(wl.net, ref))
    assert abs((out["eloc"].cpu().numpy() - ref["eloc"]).mean()) <= emean_bound(wl.net, ref)


def test_chunked_equals_unchunked(monkeypatch):
    """A ragged split of the batch into chunks changes no bit of any output."""
    wl, lay, P, x, geo = setup("ne", 23)
    fn = make(wl, P)
    xx = cuda(x)
    a = fn.local_energy(xx)
    la = fn.logpsi(xx)[0]
    ga = fn.logpsi_vjp(xx, torch.linspace(-1, 1, 23, device="cuda"))
    monkeypatch.setenv("FERMINET_CHUNK", "5")
    b = fn.local_energy(xx)
    lb = fn.logpsi(xx)[0]
    gb = fn.logpsi_vjp(xx, torch.linspace(-1, 1, 23, device="cuda"))
    assert torch.equal(a["eloc"], b["eloc"]) and torch.equal(la, lb)
    # the FP64 gradient reduction sums per-chunk FP32 partials in another order
    assert float((ga - gb).norm() / ga.norm()) < 1e-5


@pytest.mark.parametrize("name,per", [("li", 16), ("ne", 8), ("c4h6", 2), ("c4h4x8", 1)])
def test_logpsi_vjp(name, per):
    wl, lay, P, x, geo = setup(name, per)
    fn = make(wl, P)
    seeds = np.random.default_rng(3).standard_normal(x.shape[0]).astype(np.float32)
    g = fn.logpsi_vjp(cuda(x), cuda(seeds)).cpu().numpy().astype(np.float64)
    g_o = oracle.logpsi_vjp(wl.net, P, wl.geoms, x, seeds, geo=geo)
    err = np.linalg.norm(g - g_o) / np.linalg.norm(g_o)
    print(name, "vjp rel L2", err)
    for e in lay:  # block by block, so a misplaced block is named
        sl = slice(e.offset, e.offset + e.count)
        nb = np.linalg.norm(g_o[sl])
        if nb > 1e-6 * np.linalg.norm(g_o):
            assert np.linalg.norm(g[sl] - g_o[sl]) / nb < 1e-2, e.name
    assert err < TOL_GRAD_FP32


@pytest.mark.parametrize("name,per", [("li", 32), ("c4h4x8", 2)])
def test_energy_grad(name, per):
    wl, lay, P, x, geo = setup(name, per)
    fn = make(wl, P)
    eloc = (np.random.default_rng(4).standard_normal(x.shape[0]) * 2 - 7).astype(np.float32)
    em, g = fn.energy_grad(cuda(x), cuda(eloc))
    em_o, g_o = oracle.energy_grad(wl.net, P, wl.geoms, x, eloc, geo=geo)
    np.testing.assert_allclose(em.cpu().numpy(), em_o, rtol=1e-12, atol=1e-12)
    err = np.linalg.norm(g.cpu().numpy() - g_o) / np.linalg.norm(g_o)
    print(name, "energy grad rel L2", err)
    assert err < TOL_GRAD_FP32


def test_autograd_function():
    from paper_2011_07125_gb300.binding import logpsi_autograd
    wl, lay, P, x, geo = setup("li", 16)
    fn = make(wl, P)
    p = cuda(P).requires_grad_(True)
    xx = cuda(x)
    lp = logpsi_autograd(fn, p, xx)
    w = torch.linspace(0.5, 1.5, 16, device="cuda")
    (lp * w).sum().backward()
    g_o = oracle.logpsi_vjp(wl.net, P, wl.geoms, x, w.cpu().numpy())
    err = np.linalg.norm(p.grad.cpu().numpy() - g_o) / np.linalg.norm(g_o)
    assert err < TOL_GRAD_FP32


@pytest.mark.parametrize("steps,width", [(1, 0.02), (4, 0.4)])
def test_mcmc(steps, width):
    """Same Philox streams on both sides: identical decisions except where the
    acceptance margin |2 dlogpsi - log u| is below 1e-4 (precision-dependent
    near-ties), identical positions for the rest."""
    wl, lay, P, x, geo = setup("li")
    fn = make(wl, P)
    xx = cuda(x)
    lp = fn.logpsi(xx)[0]
    lp0 = lp.cpu().numpy().astype(np.float64)
    acc = fn.mcmc_step(xx, lp, steps, width, synth.SEED_MCMC, 7)
    xo, lpo, acco, margin = oracle.mcmc(wl.net, P, wl.geoms, x, lp0, steps, width, synth.SEED_MCMC, 7)
    assert fn.sync() == "FN_OK"
    ok = margin > 1e-4
    assert ok.mean() > 0.95
    a = acc.cpu().numpy()
    assert np.array_equal(a[ok], acco[ok])
    dx = np.abs(xx.cpu().numpy() - xo).reshape(len(x), -1).max(axis=1)
    assert dx[ok].max() < 1e-5
    assert 0 < a.sum() < steps * len(x) or width < 0.05
    assert rel_err(lp.cpu().numpy()[ok], lpo[ok]).max() < TOL_LOGPSI_REL


def test_hydrogen_exact_on_gpu():
    net = synth.Net(2, 8, 4, 1, 1, 0, 1)
    lay = oracle.layout(net)
    P = synth.init_params(lay, 3)
    for e in lay:
        if e.name.startswith("w_orb"):
            P[e.offset:e.offset + e.count] = 0
        if e.name.startswith("g_orb"):
            P[e.offset:e.offset + e.count] = 1
    wl = synth.Workload("h", net, [synth.atom(1)], [64], 1.0, 1, 0.1, "fp32", True)
    fn = make(wl, P)
    x = synth.init_walkers(wl, 5)
    out = fn.local_energy(cuda(x))
    assert fn.sync() == "FN_OK"
    np.testing.assert_allclose(out["eloc"].cpu().numpy(), -0.5, atol=2e-5)
    em, g = fn.energy_grad(cuda(x), out["eloc"])
    assert abs(em.item() + 0.5) < 2e-5
    assert float(g.abs().max()) < 1e-4


def test_empty_batch_and_bad_batch():
    from paper_2011_07125_gb300.binding import FermiNetError
    wl, lay, P, x, geo = setup("c4h4x8", 2)
    fn = make(wl, P)
    with pytest.raises(FermiNetError):
        fn.logpsi(cuda(x[:5]))
    wl1, _, P1, x1, _ = setup("li", 4)
    fn1 = make(wl1, P1)
    lp, sg = fn1.logpsi(cuda(x1[:0]))
    assert lp.numel() == 0
    # an empty batch of a one-geometry context whose table lists walkers
    e0 = torch.zeros(0, device="cuda")
    em, g = fn1.energy_grad(cuda(x1[:0]), e0)
    assert float(em[0]) == 0.0 and float(g.abs().max()) == 0.0
    assert float(fn1.energy_sums(e0)[0]) == 0.0
    assert fn1.sync() == "FN_OK"


@pytest.mark.parametrize("name,per", [("li", 32), ("c4h4x8", 2)])
def test_replica_calls_reproduce_energy_grad(name, per):
    """One replica: energy sums + gradient share with the batch's own mean and
    count give ferminet_energy_grad's result (same seeds, same FP64 sums)."""
    from paper_2011_07125_gb300 import replicas
    wl, lay, P, x, geo = setup(name, per)
    fn = make(wl, P)
    eloc = (np.random.default_rng(4).standard_normal(x.shape[0]) * 2 - 7).astype(np.float32)
    xx, ee = cuda(x), cuda(eloc)
    sums = fn.energy_sums(ee).cpu().numpy()
    ref = np.array([eloc[geo == g].astype(np.float64).sum() for g in range(len(wl.geoms))])
    np.testing.assert_allclose(sums, ref, rtol=1e-13, atol=1e-12)
    em, g = fn.energy_grad(xx, ee)
    em_r, g_r = replicas.energy_grad(fn, xx, ee)
    np.testing.assert_allclose(em_r.cpu().numpy(), em.cpu().numpy(), rtol=1e-15, atol=0)
    np.testing.assert_allclose(g_r.float().cpu().numpy(), g.cpu().numpy(), rtol=1e-6, atol=1e-7)
    assert fn.sync() == "FN_OK"


@pytest.mark.parametrize("name,per", [("li", 32), ("c4h4x8", 3)])
def test_two_replicas_add_to_whole_batch(name, per):
    """Two replicas, each with its own context and half of every geometry's
    walkers, run one after the other on this GPU; their shares, added on the
    host as the all-reduces would, equal the oracle's whole-batch gradient."""
    wl, lay, P, x, geo = setup(name, per)
    eloc = (np.random.default_rng(4).standard_normal(x.shape[0]) * 2 - 7).astype(np.float32)
    G = len(wl.geoms)
    halves = []
    for r in range(2):
        idx, cnt, off = [], [], 0
        for c in wl.counts:
            lo, hi = off + (0 if r == 0 else c // 2), off + (c // 2 if r == 0 else c)
            idx.extend(range(lo, hi))
            cnt.append(hi - lo)
            off += c
        halves.append((np.array(idx), cnt))
    fns = []
    for idx, cnt in halves:
        from paper_2011_07125_gb300.binding import FermiNet
        f = FermiNet(wl.net, wl.geoms, counts=cnt, precision="fp32")
        f.set_params(cuda(P))
        fns.append((f, cuda(x[idx]), cuda(eloc[idx])))
    sums = sum(f.energy_sums(e) for f, _, e in fns)
    cnts = sum(f.walker_counts(xr.shape[0]) for f, xr, _ in fns)
    parts = [f.energy_grad_partial(xr, e, sums, cnts) for f, xr, e in fns]
    emean = parts[0][0]
    assert torch.equal(emean, parts[1][0])
    grad = sum(g for _, g in parts)
    em_o, g_o = oracle.energy_grad(wl.net, P, wl.geoms, x, eloc, geo=geo)
    np.testing.assert_allclose(emean.cpu().numpy(), em_o, rtol=1e-12, atol=1e-12)
    err = np.linalg.norm(grad.cpu().numpy() - g_o) / np.linalg.norm(g_o)
    print(name, "two-replica energy grad rel L2", err)
    assert err < TOL_GRAD_FP32
    for f, _, _ in fns:
        assert f.sync() == "FN_OK"


def test_singular_walker_reported():
    """Two up electrons at the same point make every up determinant vanish:
    log|psi| = -inf, sign 0, and the status word reports it."""
    wl, lay, P, x, geo = setup("li", 4)
    x = x.copy()
    x[1, 1] = x[1, 0]
    fn = make(wl, P)
    lp, sg = fn.logpsi(cuda(x))
    st = fn.sync()
    lp = lp.cpu().numpy()
    assert st == "FN_ESINGULAR"
    assert np.isneginf(lp[1]) and sg.cpu().numpy()[1] == 0
    assert np.all(np.isfinite(lp[[0, 2, 3]]))


@pytest.mark.parametrize("name,per,prec", [("ne", 32, "fp32"), ("c4h4x8", 4, "mixed")])
def test_step_graph_matches_calls(name, per, prec):
    """ferminet_step replayed from its CUDA graph (two steps, new counter each)
    equals the same step issued as separate calls, bit for bit."""
    wl, lay, P, x, geo = setup(name, per)
    fn = make(wl, P, prec)
    xa = cuda(x)
    xb = cuda(x)
    la = fn.logpsi(xa, with_sign=False)
    lb = la.clone()
    for k in range(2):
        ctr = 100 + 7 * k
        acc = fn.mcmc_step(xa, la, 3, 0.1, 9, ctr)
        e = fn.local_energy(xa)["eloc"]
        em, g = fn.energy_grad(xa, e)
        o = fn.step(xb, lb, 3, 0.1, 9, ctr, use_graph=True)
        assert fn.sync() == "FN_OK"
        assert torch.equal(xa, xb) and torch.equal(la, lb)
        assert torch.equal(acc, o["accepted"])
        assert torch.equal(e, o["eloc"]) and torch.equal(em, o["emean"])
        assert torch.equal(g, o["grad"])


@pytest.mark.parametrize("name,per,prec", [("li", 16, "fp32"), ("ne", 6, "fp32"), ("c4h6", 3, "mixed"),
                                           ("c4h4x8", 2, "mixed")])
def test_pair_fused_matches_separate(name, per, prec):
    """The fused two-electron layer + spin-mean kernel against the separate
    kernels on the value pass, the local-energy pass and the adjoint (whose
    forward stores every layer).  Same arithmetic in the same order, except
    the value rows of 32 -> 32 layers in the mixed path: the fused kernel
    contracts them on warp MMAs with BF16 hi + lo operands (about 16
    significant bits), the separate kernel in FP32; there both log|psi| stay
    within the mixed log|psi| bar of the oracle and the gradients agree to
    1e-3 (the mixed gradient bar is 1e-2)."""
    wl, lay, P, x, geo = setup(name, per)
    fn = make(wl, P, precision=prec)
    xx = cuda(x)
    seeds = torch.linspace(-1.0, 1.0, x.shape[0], device="cuda")
    res = []
    for unfused in (0, 1):
        fn.set_tuning(pair_unfused=unfused)
        lp = fn.logpsi(xx)[0]
        out = fn.local_energy(xx)
        g = fn.logpsi_vjp(xx, seeds)
        res.append((lp, out["eloc"], out["logpsi"], g))
        assert fn.sync() == "FN_OK"
    (lp0, e0, l0, g0), (lp1, e1, l1, g1) = res
    torch.testing.assert_close(l0, l1, rtol=1e-6, atol=1e-6)
    torch.testing.assert_close(e0, e1, rtol=1e-4, atol=1e-4)
    if prec == "fp32":
        torch.testing.assert_close(lp0, lp1, rtol=1e-6, atol=1e-6)
        assert float((g0 - g1).norm() / g1.norm()) < 1e-5
    else:
        ref = oracle.local_energy(wl.net, P, wl.geoms, x, geo=geo)
        bound = logpsi_bound(wl.net, ref, u=U_MIXED)
        for lp in (lp0, lp1):
            assert np.all(np.abs(lp.cpu().numpy() - ref["logpsi"]) <= bound)
        assert np.all(np.abs((lp0 - lp1).cpu().numpy()) <= bound)
        assert float((g0 - g1).norm() / g1.norm()) < 1e-3
    print(name, prec, "fused vs separate: max |dE|", float((e0 - e1).abs().max()),
          "bitwise" if torch.equal(e0, e1) and torch.equal(lp0, lp1) else "not bitwise")


def test_two_electron_width_outside_fused_kernel():
    """d2 = 12 is not covered by the fused pair kernel: the separate kernels
    run, and log|psi| and E_L still match the oracle."""
    from paper_2011_07125_gb300.binding import FermiNet
    net = synth.Net(3, 32, 12, 2, 3, 2, 2)
    geoms = [synth.Geometry(np.array([[0.0, 0.0, -0.8], [0.0, 0.0, 0.8]]), np.array([3.0, 2.0]))]
    wl = synth.Workload("two-centre", net, geoms, [12], 1.0, 1, 0.02, "fp32", True)
    P = synth.init_params(oracle.layout(net), seed=3)
    x = synth.init_walkers(wl, seed=4)
    fn = FermiNet(net, geoms, counts=[12], precision="fp32")
    fn.set_params(cuda(P))
    out = fn.local_energy(cuda(x))
    ref = oracle.local_energy(net, P, geoms, x)
    assert fn.sync() == "FN_OK"
    assert np.all(np.abs(out["logpsi"].cpu().numpy() - ref["logpsi"]) <= logpsi_bound(net, ref))
    de = np.abs(out["eloc"].cpu().numpy().astype(np.float64) - ref["eloc"])
    bound = eloc_bound(net, ref)
    assert np.all(de <= bound), (de / bound).max()


def test_pair_fused_large_groups():
    """56 electrons: one (walker, electron) group of the local-energy pass's
    32 -> 32 two-electron layer needs the shared-memory share of two blocks, so
    the fused kernel runs its two-block instance; it matches the separate
    kernels like the three-block instance does on smaller systems."""
    from paper_2011_07125_gb300.binding import FermiNet
    net = synth.Net(3, 32, 32, 1, 28, 28, 1)
    geoms = [synth.atom(56)]
    wl = synth.Workload("z56", net, geoms, [3], 1.0, 1, 0.02, "fp32", True)
    P = synth.init_params(oracle.layout(net), seed=3)
    x = synth.init_walkers(wl, seed=4)
    fn = FermiNet(net, geoms, counts=[3], precision="fp32")
    fn.set_params(cuda(P))
    xx = cuda(x)
    seeds = torch.linspace(-1.0, 1.0, 3, device="cuda")
    res = []
    for unfused in (0, 1):
        fn.set_tuning(pair_unfused=unfused)
        out = fn.local_energy(xx)
        g = fn.logpsi_vjp(xx, seeds)
        assert fn.sync() == "FN_OK"
        res.append((out["logpsi"], out["eloc"], g))
    (l0, e0, g0), (l1, e1, g1) = res
    torch.testing.assert_close(l0, l1, rtol=1e-6, atol=1e-6)
    torch.testing.assert_close(e0, e1, rtol=1e-4, atol=1e-4)
    assert float((g0 - g1).norm() / g1.norm()) < 1e-5


@pytest.mark.parametrize("env", [{"FERMINET_PIVOT_TAU": "0.999"}, {"FERMINET_DET64": "1"}])
def test_fp64_determinant_redo(monkeypatch, env):
    """Every orbital matrix goes through the FP64 redo (flagged by the pivot
    ratio, or forced), in the tangent pass and in the value pass: E_L and
    log|psi| still match the oracle, and the flagged count reports the matrices
    when flagging is by ratio."""
    for k, v in env.items():
        monkeypatch.setenv(k, v)
    wl, lay, P, x, geo = setup("c4h6", 3)
    fn = make(wl, P)
    out = fn.local_energy(cuda(x))
    assert fn.sync() == "FN_OK"
    ref = oracle.local_energy(wl.net, P, wl.geoms, x, geo=geo)
    de = np.abs(out["eloc"].cpu().numpy().astype(np.float64) - ref["eloc"])
    bound = eloc_bound(wl.net, ref)
    assert np.all(de <= bound), (de / bound).max()
    assert np.all(np.abs(out["logpsi"].cpu().numpy() - ref["logpsi"]) <= logpsi_bound(wl.net, ref))
    # the value pass takes the same route (its pairs redone by the list kernel)
    lp, sg = fn.logpsi(cuda(x))
    assert fn.sync() == "FN_OK"
    assert np.all(np.abs(lp.cpu().numpy() - ref["logpsi"]) <= logpsi_bound(wl.net, ref))
    assert np.array_equal(sg.cpu().numpy(), ref["sign"])
    if "FERMINET_PIVOT_TAU" in env:
        fn.local_energy(cuda(x))
        assert fn.flagged_matrices() > 0


def test_singular_walker_in_tangent_pass():
    """The singular walker of the value-pass test, through the local-energy
    pass: status FN_ESINGULAR, log|psi| = -inf there, the others finite."""
    wl, lay, P, x, geo = setup("li", 4)
    x = x.copy()
    x[1, 1] = x[1, 0]
    fn = make(wl, P)
    out = fn.local_energy(cuda(x))
    assert fn.sync() == "FN_ESINGULAR"
    lp = out["logpsi"].cpu().numpy()
    assert np.isneginf(lp[1])
    assert np.all(np.isfinite(out["eloc"].cpu().numpy()[[0, 2, 3]]))

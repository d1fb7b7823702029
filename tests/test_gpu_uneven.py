"""The multi-geometry batch with uneven walker counts against the FP64 oracle.

Eight C4H4-shaped geometries whose walker counts keep the ratios of the full
batch (256 ... 4096 scaled by 1/128: 2, 4, 6, 8, 12, 16, 24, 32 walkers), all
in one context and one launch per kernel, so every kernel meets the ragged
walker-to-geometry mapping.  The walkers are first moved towards |psi|^2 (the
distribution the VMC estimator averages over) by FP32 Metropolis moves on the
GPU.  Checked: per-walker log|psi| and E_L under the parity bars of each
precision, and the batch-mean E_L of every geometry (1e-3 Ha for the mixed
path, the FP32 bar for the FP32 path), and the VMC gradient.  A geometry's
mean over its few sampled walkers estimates the mean over its full batch with
a sampling error, so each per-geometry bar adds three standard errors of the
sample; the mean over all sampled walkers (the bias) takes the bar alone.
"""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_2011_07125_gb300 import synth
from helpers import (TOL_EMEAN_ABS, TOL_GRAD_MIXED, TOL_EMEAN_MIXED, U_MIXED, eloc_bound, emean_bound,
                     logpsi_bound, mixed_eloc_bound, sample_mean_bound)

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _uneven():
    wl = synth.workload("c4h4x8")
    counts = [c // 128 for c in wl.counts]
    assert counts == [2, 4, 6, 8, 12, 16, 24, 32]
    return dataclasses.replace(wl, counts=counts)


@pytest.fixture(scope="module")
def sampled():
    from paper_2011_07125_gb300.binding import FermiNet
    wl = _uneven()
    lay = oracle.layout(wl.net)
    P = synth.init_params(lay)
    x = synth.init_walkers(wl)
    geo = synth.geometry_of_walkers(wl.counts)
    fn = FermiNet(wl.net, wl.geoms, counts=wl.counts, precision="fp32")
    fn.set_params(torch.from_numpy(P).cuda())
    xx = torch.from_numpy(x).cuda()
    lp = fn.logpsi(xx, with_sign=False)
    for k in range(30):
        fn.mcmc_step(xx, lp, 10, 0.15, 5, 10 * k)
    assert fn.sync() == "FN_OK"
    fn.close()
    xs = np.ascontiguousarray(xx.cpu().numpy())
    ref = oracle.local_energy(wl.net, P, wl.geoms, xs, geo=geo)
    return wl, P, xs, geo, ref


@pytest.mark.parametrize("prec", ["fp32", "mixed"])
def test_uneven_geometries_local_energy(sampled, prec):
    from paper_2011_07125_gb300.binding import FermiNet
    wl, P, xs, geo, ref = sampled
    fn = FermiNet(wl.net, wl.geoms, counts=wl.counts, precision=prec)
    fn.set_params(torch.from_numpy(P).cuda())
    out = fn.local_energy(torch.from_numpy(xs).cuda())
    assert fn.sync() == "FN_OK"
    e = out["eloc"].cpu().numpy().astype(np.float64)
    de = e - ref["eloc"]
    dl = np.abs(out["logpsi"].cpu().numpy() - ref["logpsi"])
    per_geo = np.array([de[geo == g].mean() for g in range(len(wl.geoms))])
    print(prec, "per-geometry mean E_L error", per_geo, "max |dE|", np.abs(de).max(),
          "fraction within 1e-4 Ha", np.mean(np.abs(de) <= 1e-4))
    assert np.array_equal(out["sign"].cpu().numpy(), ref["sign"])
    cnt = np.array(wl.counts)
    if prec == "fp32":
        assert np.all(np.abs(de) <= eloc_bound(wl.net, ref)), (np.abs(de) / eloc_bound(wl.net, ref)).max()
        assert np.all(dl <= logpsi_bound(wl.net, ref))
        assert abs(de.mean()) <= emean_bound(wl.net, ref)
        assert np.all(np.abs(per_geo) <= sample_mean_bound(de, cnt, TOL_EMEAN_ABS)), per_geo
        assert np.mean(np.abs(de) <= 1e-4) >= 0.8
    else:
        assert np.all(np.abs(de) <= mixed_eloc_bound(wl.net, ref)), \
            (np.abs(de) / mixed_eloc_bound(wl.net, ref)).max()
        assert np.all(dl <= logpsi_bound(wl.net, ref, u=U_MIXED))
        assert abs(de.mean()) < TOL_EMEAN_MIXED
        assert np.all(np.abs(per_geo) <= sample_mean_bound(de, cnt, TOL_EMEAN_MIXED)), per_geo
    fn.close()


def test_uneven_geometries_gradient(sampled):
    """Mixed context: E_L from the tensor-core pass, per-geometry means and the
    VMC gradient over the uneven batch against the oracle's gradient computed
    with the oracle's own local energies."""
    from paper_2011_07125_gb300.binding import FermiNet
    wl, P, xs, geo, ref = sampled
    fn = FermiNet(wl.net, wl.geoms, counts=wl.counts, precision="mixed")
    fn.set_params(torch.from_numpy(P).cuda())
    xx = torch.from_numpy(xs).cuda()
    out = fn.local_energy(xx)
    em, g = fn.energy_grad(xx, out["eloc"])
    assert fn.sync() == "FN_OK"
    em_o, g_o = oracle.energy_grad(wl.net, P, wl.geoms, xs, ref["eloc"], geo=geo)
    de = out["eloc"].cpu().numpy().astype(np.float64) - ref["eloc"]
    assert np.all(np.abs(em.cpu().numpy() - em_o) <= sample_mean_bound(de, np.array(wl.counts), TOL_EMEAN_MIXED))
    err = np.linalg.norm(g.cpu().numpy() - g_o) / np.linalg.norm(g_o)
    print("uneven mixed gradient rel L2", err)
    assert err < TOL_GRAD_MIXED
    fn.close()

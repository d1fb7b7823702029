"""KFAC (the optimiser Sec. 1 credits for FermiNet's accuracy) through the C
ABI against the oracle: the Kronecker factors of a mixed-precision context
(tensor-core Gram products of the stored rows and of the adjoint's
pre-activation gradients) and the damped preconditioned update (FP64
Gauss-Jordan inverses on the device)."""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_2011_07125_gb300 import synth
from helpers import setup

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _make(wl, P, prec="mixed"):
    from paper_2011_07125_gb300.binding import FermiNet
    fn = FermiNet(wl.net, wl.geoms, counts=wl.counts, precision=prec)
    fn.set_params(torch.from_numpy(P).cuda())
    return fn


@pytest.mark.parametrize("name,per", [("li", 16), ("ne", 6), ("c4h6", 2), ("c4h4x8", 1)])
def test_kfac_factors_match_oracle(name, per):
    wl, lay, P, x, geo = setup(name, per)
    fn = _make(wl, P)
    F = fn.kfac_factors(torch.from_numpy(x).cuda()).cpu().numpy()
    assert fn.sync() == "FN_OK"
    F_o = oracle.kfac_factors(wl.net, P, wl.geoms, x, geo=geo)
    blocks, nb = oracle.kfac_blocks(wl.net)
    assert F.shape == F_o.shape
    for bname, off, d in blocks:
        a, b = F[off:off + d * d], F_o[off:off + d * d]
        err = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)
        print(name, bname, "rel Frobenius err", err)
        assert err < 2e-2, bname
    d_err = np.linalg.norm(F[nb:] - F_o[nb:]) / np.linalg.norm(F_o[nb:])
    print(name, "envelope diagonal rel err", d_err)
    assert d_err < 2e-2


@pytest.mark.parametrize("name,per,lam", [("li", 16, 1e-3), ("c4h6", 2, 1e-2)])
def test_kfac_precondition_matches_oracle(name, per, lam):
    """The device preconditioner on the oracle's own factors and a random
    gradient, against the oracle's FP64 update."""
    wl, lay, P, x, geo = setup(name, per)
    fn = _make(wl, P)
    F_o = oracle.kfac_factors(wl.net, P, wl.geoms, x, geo=geo)
    g = np.random.default_rng(9).standard_normal(P.shape[0]).astype(np.float32)
    out = fn.kfac_precondition(torch.from_numpy(F_o).cuda(), torch.from_numpy(g).cuda(), lam).cpu().numpy()
    assert fn.sync() == "FN_OK"
    want = oracle.kfac_precondition(wl.net, F_o, g.astype(np.float64), lam)
    err = np.linalg.norm(out - want) / np.linalg.norm(want)
    print(name, "KFAC update rel L2", err)
    assert err < 1e-4
    for e in lay:
        sl = slice(e.offset, e.offset + e.count)
        assert np.linalg.norm(out[sl] - want[sl]) <= 1e-3 * np.linalg.norm(want[sl]) + 1e-30, e.name


def test_kfac_step_matches_oracle_and_needs_mixed():
    """Factors and update of the VMC gradient, end to end on the device,
    against the oracle's pipeline; an FP32 context refuses the factors."""
    from paper_2011_07125_gb300.binding import FermiNetError
    wl, lay, P, x, geo = setup("c4h4x8", 2)  # two walkers per geometry: a non-zero gradient
    fn = _make(wl, P)
    xx = torch.from_numpy(x).cuda()
    eloc = (np.random.default_rng(4).standard_normal(len(x)) * 2 - 7).astype(np.float32)
    em, g = fn.energy_grad(xx, torch.from_numpy(eloc).cuda())
    F = fn.kfac_factors(xx)
    d = fn.kfac_precondition(F, g, 1e-2).cpu().numpy()
    assert fn.sync() == "FN_OK"
    _, g_o = oracle.energy_grad(wl.net, P, wl.geoms, x, eloc, geo=geo)
    d_o = oracle.kfac_precondition(wl.net, oracle.kfac_factors(wl.net, P, wl.geoms, x, geo=geo), g_o, 1e-2)
    err = np.linalg.norm(d - d_o) / np.linalg.norm(d_o)
    print("KFAC step rel L2", err)
    assert err < 5e-2
    f32 = _make(wl, P, "fp32")
    with pytest.raises(FermiNetError):
        f32.kfac_factors(xx)

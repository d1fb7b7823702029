"""Shared helpers of the test suite (seeded inputs, oracle calls, tolerances).

Tolerances.  The local energy is a small difference of large terms: with
S_w = |grad log psi|^2 + |lap log psi| (from the oracle), an evaluation whose
operands carry unit roundoff u has an error floor of about u * S_w per walker,
amplified by the depth of the network.  Each per-walker bound is therefore the
stated bar plus gamma * u * S_w: it reduces to the bar on well-conditioned
walkers and widens only near nodes of psi, where S_w is large.

- FP32 path (u = 2^-24): gamma = L * sqrt(d1 + 2 d2) (L layers of dot products
  of length d1 + 2 d2, random-walk rounding growth).  Measured on GB300 over
  initial and |psi|^2-sampled walkers of every workload, the largest
  (error - 1e-4 Ha) / (u S_w) is 0.64 gamma (8 C4H4 geometries): 1.6x headroom.
- Mixed path (BF16 hi + lo operands, about 16 significant bits, u = 2^-17):
  the same form with the measured constant G_MIXED_ELOC = 20 (largest measured
  ratio 5.3, Li initial walkers: 3.8x headroom) over a 1e-4 Ha base.
- log|psi|: 1e-5 relative to max(|log psi|, 1) plus G * u * |grad log psi|
  (one bohr of distance), with measured constants G_LOGPSI_FP32 = 50 (largest
  measured ratio 15.8, Ar) and G_LOGPSI_MIXED = 100 (largest 30.8, C4H4).
- Batch mean: the stated bar plus gamma * u * mean(S_w).
Besides these bars, the parity tests gate the fraction of |psi|^2-sampled
walkers that meet the unwidened bars (1e-4 Ha, 1e-5 relative).
"""
import math

import numpy as np

import oracle
from paper_2011_07125_gb300 import synth

U32 = 2.0 ** -24
TOL_LOGPSI_REL = 1e-5
TOL_ELOC_ABS = 1e-4
TOL_EMEAN_ABS = 1e-5


def setup(name, per_geom=None, seed_params=synth.SEED_PARAMS, seed_walkers=synth.SEED_WALKERS):
    """Workload, layout, float32 parameters and float32 walkers."""
    wl = synth.workload(name)
    if per_geom is not None:
        wl = synth.subset(wl, per_geom)
    lay = oracle.layout(wl.net)
    P = synth.init_params(lay, seed_params)
    x = synth.init_walkers(wl, seed_walkers)
    geo = synth.geometry_of_walkers(wl.counts)
    return wl, lay, P, x, geo


def rel_err(a, b):
    return np.abs(a - b) / np.maximum(np.abs(b), 1.0)


def gamma(net):
    return net.n_layers * math.sqrt(net.d1 + 2 * net.d2)


def conditioning(ref):
    """S_w = |grad log psi|^2 + |lap log psi| and |grad log psi| from oracle output."""
    g2 = (ref["grad"] ** 2).sum(axis=1)
    lap = np.abs(ref["d2"].sum(axis=1))
    return g2 + lap, np.sqrt(g2)


def eloc_bound(net, ref, u=U32, base=TOL_ELOC_ABS):
    S, _ = conditioning(ref)
    return base + gamma(net) * u * S


G_LOGPSI_FP32 = 50.0
G_LOGPSI_MIXED = 100.0
G_MIXED_ELOC = 20.0


def logpsi_bound(net, ref, u=U32, base=TOL_LOGPSI_REL):
    _, g = conditioning(ref)
    G = G_LOGPSI_FP32 if u == U32 else G_LOGPSI_MIXED
    return base * np.maximum(np.abs(ref["logpsi"]), 1.0) + G * u * g


def emean_bound(net, ref, u=U32, base=TOL_EMEAN_ABS):
    S, _ = conditioning(ref)
    return base + gamma(net) * u * S.mean()


# Mixed path (BF16 hi + lo operands, about 16 significant bits: u = 2^-17).
U_MIXED = 2.0 ** -17
TOL_EMEAN_MIXED = 1e-3
TOL_GRAD_MIXED = 1e-2


def mixed_eloc_bound(net, ref):
    """Per-walker E_L bound of the mixed path: 1e-4 Ha plus the measured
    G_MIXED_ELOC * u * S_w rounding term."""
    S, _ = conditioning(ref)
    return TOL_ELOC_ABS + G_MIXED_ELOC * U_MIXED * S


def sample_mean_bound(de, counts_sel, base):
    """Bound of a mean error over n walkers drawn from a larger batch: the
    batch bar plus three standard errors of the sample (pooled spread)."""
    sd = float(np.sqrt(np.mean(np.asarray(de) ** 2)))
    return base + 3.0 * sd / np.sqrt(np.maximum(counts_sel, 1))


def equilibrated(name, sample, moves=300, width=0.15):
    """`sample` walkers of the workload's full batch after `moves` FP32
    Metropolis moves on the GPU (towards |psi|^2, the distribution the VMC
    estimator averages over).  Returns (workload, params, walkers)."""
    import torch
    from paper_2011_07125_gb300.binding import FermiNet
    wl, lay, P, x, geo = setup(name)
    fn = FermiNet(wl.net, wl.geoms, counts=wl.counts, precision="fp32")
    fn.set_params(torch.from_numpy(P).cuda())
    xx = torch.from_numpy(x).cuda()
    lp = fn.logpsi(xx, with_sign=False)
    for k in range(moves // 10):
        fn.mcmc_step(xx, lp, 10, width, 5, 10 * k)
    assert fn.sync() == "FN_OK"
    fn.close()
    idx = np.linspace(0, wl.batch - 1, sample).astype(int) if len(wl.geoms) == 1 else np.arange(sample)
    return wl, P, np.ascontiguousarray(xx.cpu().numpy()[idx])

"""Shared helpers of the test suite (seeded inputs, oracle calls, tolerances).

Tolerances of the FP32 path.  The local energy is a small difference of large
terms: with S_w = |grad log psi|^2 + |lap log psi| (from the oracle), the FP32
forward-Laplacian evaluation has a rounding floor of about u * S_w per walker
(u = 2^-24), amplified by the depth of the network.  The per-walker bound is
therefore the stated 1e-4 Ha plus gamma * u * S_w with gamma = L * sqrt(d1 + 2 d2)
(L layers of dot products of length d1 + 2 d2, random-walk rounding growth);
it reduces to 1e-4 Ha on well-conditioned walkers and widens only near nodes of
psi, where S_w is large.  log|psi| gets 1e-5 relative plus 2 gamma u |grad log psi|
(one bohr of distance).  The batch mean gets 1e-5 Ha plus the mean of the
per-walker rounding terms.
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


def logpsi_bound(net, ref, u=U32, base=TOL_LOGPSI_REL):
    _, g = conditioning(ref)
    return base * np.maximum(np.abs(ref["logpsi"]), 1.0) + 2 * gamma(net) * u * g


def emean_bound(net, ref, u=U32, base=TOL_EMEAN_ABS):
    S, _ = conditioning(ref)
    return base + gamma(net) * u * S.mean()


# Mixed path (BF16 hi + lo operands, about 16 significant bits: u = 2^-17).
U_MIXED = 2.0 ** -17
TOL_EMEAN_MIXED = 1e-3
TOL_GRAD_MIXED = 1e-2
TOL_ELOC_ABS_MIXED = 1e-3


def mixed_eloc_bound(net, ref):
    """Per-walker E_L bound of the mixed path: the rounding model above with
    the mixed unit roundoff."""
    return eloc_bound(net, ref, u=U_MIXED, base=TOL_ELOC_ABS_MIXED)

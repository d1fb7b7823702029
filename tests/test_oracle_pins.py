"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test targets a class of plausible mistakes (dropped term, wrong sign or
index, transposed operand, wrong factor) that would otherwise go unnoticed.
None of them compares the oracle with itself through the same code path.
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_2011_07125_gb300 import synth


def _params(net, seed=0):
    lay = oracle.layout(net)
    return lay, synth.init_params(lay, seed).astype(np.float64)


def _set(lay, P, prefix, value):
    for e in lay:
        if e.name.startswith(prefix):
            P[e.offset:e.offset + e.count] = value


def _block(lay, P, name):
    e = next(e for e in lay if e.name == name)
    return P[e.offset:e.offset + e.count]


# ---------------------------------------------------------------------------
# Exact states inside the Ansatz (Eq. 1, Eq. 4)
# ---------------------------------------------------------------------------

def test_hydrogen_exact_local_energy_and_zero_gradient():
    """n_up=1, n_down=0, Z=1, K=1, w=0, g=1, pi=1, sigma=1 gives psi=exp(-r):
    E_L = -1/2 at every point, and the VMC gradient vanishes (zero variance)."""
    net = synth.Net(2, 8, 4, 1, 1, 0, 1)
    lay, P = _params(net, seed=3)
    _set(lay, P, "w_orb", 0.0)
    _set(lay, P, "g_orb", 1.0)
    x = np.random.default_rng(0).standard_normal((16, 1, 3)) * 1.5
    out = oracle.local_energy(net, P, [synth.atom(1)], x)
    np.testing.assert_allclose(out["eloc"], -0.5, atol=1e-12)
    np.testing.assert_allclose(out["logpsi"], -np.linalg.norm(x[:, 0], axis=1), atol=1e-12)
    em, g = oracle.energy_grad(net, P, [synth.atom(1)], x, out["eloc"])
    assert abs(em[0] + 0.5) < 1e-12
    assert np.max(np.abs(g)) < 1e-10


@pytest.mark.parametrize("Z,zeta", [(2.0, 1.6875), (3.0, 2.0), (1.0, 0.7)])
def test_hydrogenic_two_electron_closed_form(Z, zeta):
    """n_up=n_down=1, w=0, g=1, sigma=zeta: psi = exp(-zeta(r1+r2)) and
    E_L = sum_i(-zeta^2/2 + (zeta - Z)/r_i) + 1/r12 (textbook helium-like)."""
    net = synth.Net(2, 8, 4, 2, 1, 1, 1)
    lay, P = _params(net, seed=1)
    _set(lay, P, "w_orb", 0.0)
    _set(lay, P, "g_orb", 1.0)
    _set(lay, P, "sigma", zeta)
    # two identical determinants: psi = 2 exp(-zeta(r1+r2))
    x = np.random.default_rng(1).standard_normal((8, 2, 3))
    out = oracle.local_energy(net, P, [synth.atom(Z)], x)
    r = np.linalg.norm(x, axis=2)
    r12 = np.linalg.norm(x[:, 0] - x[:, 1], axis=1)
    want = (-zeta ** 2 / 2 + (zeta - Z) / r).sum(axis=1) + 1.0 / r12
    np.testing.assert_allclose(out["eloc"], want, rtol=1e-11, atol=1e-11)
    np.testing.assert_allclose(out["logpsi"], math.log(2.0) - zeta * r.sum(axis=1), atol=1e-12)


def test_two_centre_envelope_closed_form():
    """One electron, two nuclei, w=0, g=1, pi=(1, c), sigma=(a, b):
    psi = exp(-a r_A) + c exp(-b r_B), and
    -1/2 lap psi / psi = sum_m p_m (-s_m^2/2 + s_m / r_m) / psi."""
    net = synth.Net(2, 8, 4, 1, 1, 0, 2)
    lay, P = _params(net, seed=2)
    _set(lay, P, "w_orb", 0.0)
    _set(lay, P, "g_orb", 1.0)
    a, b, c = 1.3, 0.8, 0.6
    _block(lay, P, "sigma_up")[:] = [a, b]
    _block(lay, P, "pi_up")[:] = [1.0, c]
    geom = synth.Geometry(R=np.array([[0.0, 0.0, -0.7], [0.2, 0.1, 0.9]]), Z=np.array([1.0, 2.0]))
    x = np.random.default_rng(2).standard_normal((8, 1, 3))
    out = oracle.local_energy(net, P, [geom], x)
    rA = np.linalg.norm(x[:, 0] - geom.R[0], axis=1)
    rB = np.linalg.norm(x[:, 0] - geom.R[1], axis=1)
    tA, tB = np.exp(-a * rA), c * np.exp(-b * rB)
    psi = tA + tB
    T = (tA * (-a * a / 2 + a / rA) + tB * (-b * b / 2 + b / rB)) / psi
    V = -1.0 / rA - 2.0 / rB + 2.0 / np.linalg.norm(geom.R[0] - geom.R[1])
    np.testing.assert_allclose(out["eloc"], T + V, rtol=1e-11, atol=1e-11)
    np.testing.assert_allclose(out["logpsi"], np.log(psi), atol=1e-12)


# ---------------------------------------------------------------------------
# Structure of Eq. 3
# ---------------------------------------------------------------------------

def test_antisymmetry_same_spin_swap():
    """Swapping two same-spin electrons flips the sign of psi and leaves
    log|psi| and E_L unchanged; swapping across spins is not a symmetry."""
    wl = synth.workload("li")
    net = synth.Net(2, 16, 8, 3, 3, 2, 1)
    lay, P = _params(net)
    x = np.random.default_rng(4).standard_normal((6, 5, 3))
    lp, s = oracle.logpsi(net, P, wl.geoms, x)
    for (i, j) in [(0, 1), (0, 2), (3, 4)]:
        y = x.copy()
        y[:, [i, j]] = y[:, [j, i]]
        lp2, s2 = oracle.logpsi(net, P, wl.geoms, y)
        np.testing.assert_allclose(lp2, lp, atol=1e-11)
        np.testing.assert_array_equal(s2, -s)
    e1 = oracle.local_energy(net, P, wl.geoms, x[:2])["eloc"]
    y = x[:2].copy()
    y[:, [3, 4]] = y[:, [4, 3]]
    e2 = oracle.local_energy(net, P, wl.geoms, y)["eloc"]
    np.testing.assert_allclose(e2, e1, rtol=1e-10)
    y = x.copy()
    y[:, [0, 3]] = y[:, [3, 0]]
    lp3, _ = oracle.logpsi(net, P, wl.geoms, y)
    assert np.max(np.abs(lp3 - lp)) > 1e-6


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6])
def test_lu_determinant_matches_leibniz(n):
    rng = np.random.default_rng(n)
    for _ in range(5):
        A = rng.standard_normal((n, n))
        s, la = oracle.slogdet(A)
        d = oracle.det_leibniz(A)
        assert np.sign(d) == s
        assert abs(la - math.log(abs(d))) < 1e-11
    # singular matrix: two equal rows
    A = rng.standard_normal((n, n))
    if n > 1:
        A[1] = A[0]
        s, la = oracle.slogdet(A)
        assert s == 0.0 or la < -25
    s, la = oracle.slogdet(np.zeros((0, 0)))
    assert s == 1.0 and la == 0.0


def test_identical_determinants_add_log_k():
    """K identical determinants: log|psi_K| = log K + log|psi_1|."""
    K = 4
    net1 = synth.Net(2, 16, 8, 1, 2, 2, 1)
    netK = synth.Net(2, 16, 8, K, 2, 2, 1)
    lay1, P1 = _params(net1, seed=5)
    layK, PK = _params(netK, seed=6)
    for e1 in lay1:
        eK = next(e for e in layK if e.name == e1.name)
        blk1 = P1[e1.offset:e1.offset + e1.count]
        if eK.count == e1.count:
            PK[eK.offset:eK.offset + eK.count] = blk1
        else:  # per-determinant block: replicate determinant 0
            PK[eK.offset:eK.offset + eK.count] = np.tile(blk1, K)
    x = np.random.default_rng(7).standard_normal((5, 4, 3))
    g = [synth.atom(4)]
    l1, s1 = oracle.logpsi(net1, P1, g, x)
    lK, sK = oracle.logpsi(netK, PK, g, x)
    np.testing.assert_allclose(lK, l1 + math.log(K), atol=1e-11)
    np.testing.assert_array_equal(sK, s1)


def test_translation_invariance_molecule():
    """Shifting all electrons and nuclei together changes neither psi nor E_L."""
    wl = synth.workload("c4h6")
    net = synth.Net(2, 16, 8, 2, 3, 3, 10)
    lay, P = _params(net, seed=8)
    geom = wl.geoms[0]
    x = geom.R[np.arange(6) % 10][None] + np.random.default_rng(9).standard_normal((2, 6, 3))
    shift = np.array([0.7, -1.3, 2.1])
    g2 = synth.Geometry(R=geom.R + shift, Z=geom.Z)
    a = oracle.local_energy(net, P, [geom], x)
    b = oracle.local_energy(net, P, [g2], x + shift)
    np.testing.assert_allclose(b["logpsi"], a["logpsi"], atol=1e-10)
    np.testing.assert_allclose(b["eloc"], a["eloc"], rtol=1e-9, atol=1e-9)


# ---------------------------------------------------------------------------
# Derivatives
# ---------------------------------------------------------------------------

def test_coordinate_derivatives_match_central_differences():
    """Jet first and second derivatives vs central differences (h = 1e-4)."""
    net = synth.Net(3, 16, 8, 2, 2, 2, 2)
    lay, P = _params(net, seed=10)
    geom = synth.Geometry(R=np.array([[0.0, 0.0, 0.0], [1.4, 0.0, 0.0]]), Z=np.array([1.0, 3.0]))
    x = np.random.default_rng(11).standard_normal((1, 4, 3))
    out = oracle.local_energy(net, P, [geom], x)
    h = 1e-4
    lp0, _ = oracle.logpsi(net, P, [geom], x)
    for c in range(12):
        xp = x.copy().reshape(-1)
        xm = x.copy().reshape(-1)
        xp[c] += h
        xm[c] -= h
        lpp, _ = oracle.logpsi(net, P, [geom], xp.reshape(1, 4, 3))
        lpm, _ = oracle.logpsi(net, P, [geom], xm.reshape(1, 4, 3))
        fd1 = (lpp[0] - lpm[0]) / (2 * h)
        fd2 = (lpp[0] - 2 * lp0[0] + lpm[0]) / h ** 2
        assert abs(fd1 - out["grad"][0, c]) < 1e-6 * max(1, abs(fd1))
        assert abs(fd2 - out["d2"][0, c]) < 1e-3 * max(1, abs(fd2))
    # kinetic energy assembled from the per-coordinate pieces
    T = -0.5 * (out["d2"][0] + out["grad"][0] ** 2).sum()
    assert abs(T - out["kinetic"][0]) < 1e-10 * max(1, abs(T))


def test_parameter_gradient_matches_directional_differences():
    """sum_w seed_w d log|psi_w| / d theta . v vs central differences along v."""
    net = synth.Net(3, 16, 8, 3, 3, 2, 2)
    lay, P = _params(net, seed=12)
    rng = np.random.default_rng(13)
    # non-trivial envelopes and orbital biases so every block gets exercised
    for e in lay:
        if e.name.startswith(("pi_", "sigma_", "g_orb")):
            P[e.offset:e.offset + e.count] = 0.5 + rng.random(e.count)
        if e.name.startswith(("b", "c")) and e.name[1:].isdigit():
            P[e.offset:e.offset + e.count] = 0.1 * rng.standard_normal(e.count)
    geom = synth.Geometry(R=np.array([[0.0, 0.0, 0.0], [0.0, 1.1, 0.3]]), Z=np.array([2.0, 3.0]))
    x = rng.standard_normal((3, 5, 3))
    seeds = np.array([0.7, -1.2, 0.4])
    g = oracle.logpsi_vjp(net, P, [geom], x, seeds)
    for trial in range(3):
        v = rng.standard_normal(P.shape[0])
        eps = 1e-6
        lpp, _ = oracle.logpsi(net, P + eps * v, [geom], x)
        lpm, _ = oracle.logpsi(net, P - eps * v, [geom], x)
        fd = seeds @ ((lpp - lpm) / (2 * eps))
        assert abs(fd - g @ v) < 1e-6 * max(1.0, abs(fd))
    # each block separately (catches a transposed or misplaced block)
    for e in lay:
        v = np.zeros(P.shape[0])
        v[e.offset:e.offset + e.count] = rng.standard_normal(e.count)
        eps = 1e-6
        lpp, _ = oracle.logpsi(net, P + eps * v, [geom], x)
        lpm, _ = oracle.logpsi(net, P - eps * v, [geom], x)
        fd = seeds @ ((lpp - lpm) / (2 * eps))
        assert abs(fd - g @ v) < 2e-6 * max(1.0, abs(fd)), e.name


def test_vmc_gradient_is_derivative_of_reweighted_energy():
    """The VMC gradient of Eq. 2 (E_L held fixed) is the derivative at eps=0 of
    the importance-reweighted estimate sum_w r_w E_w / sum_w r_w with
    r_w = |psi_{theta+eps v}(x_w)|^2 / |psi_theta(x_w)|^2."""
    net = synth.Net(2, 16, 8, 2, 2, 1, 1)
    lay, P = _params(net, seed=14)
    rng = np.random.default_rng(15)
    geoms = [synth.atom(3), synth.Geometry(R=np.array([[0.1, 0.0, 0.0]]), Z=np.array([3.0]))]
    x = rng.standard_normal((7, 3, 3))
    geo = np.array([0, 0, 0, 1, 1, 1, 1], np.int32)
    E = rng.standard_normal(7) * 3 - 7
    em, g = oracle.energy_grad(net, P, geoms, x, E, geo=geo)
    for gi in range(2):
        np.testing.assert_allclose(em[gi], E[geo == gi].mean(), rtol=1e-14)
    v = rng.standard_normal(P.shape[0])
    lp0, _ = oracle.logpsi(net, P, geoms, x, geo=geo)

    def F(eps):
        lp, _ = oracle.logpsi(net, P + eps * v, geoms, x, geo=geo)
        r = np.exp(2 * (lp - lp0))
        return sum((r[geo == k] * E[geo == k]).sum() / r[geo == k].sum() for k in range(2))

    eps = 1e-5
    fd = (F(eps) - F(-eps)) / (2 * eps)
    assert abs(fd - g @ v) < 1e-6 * max(1, abs(fd))


# ---------------------------------------------------------------------------
# Coulomb terms of Eq. 1
# ---------------------------------------------------------------------------

def test_coulomb_hand_cases():
    # helium-like: nucleus Z=2 at origin, electrons at +-x: 1/2 - 2 - 2
    R = np.zeros((1, 3))
    Z = np.array([2.0])
    x = np.array([[1.0, 0, 0], [-1.0, 0, 0]])
    assert abs(oracle.potential(R, Z, x) - (0.5 - 4.0)) < 1e-15
    # H2 at 1.4 bohr with electrons at the midpoint and 1 bohr above it
    R = np.array([[0, 0, -0.7], [0, 0, 0.7]])
    Z = np.array([1.0, 1.0])
    x = np.array([[0.0, 0, 0], [0.0, 1.0, 0]])
    rb = math.sqrt(1 + 0.49)
    want = 1.0 - 2 / 0.7 - 2 / rb + 1 / 1.4
    assert abs(oracle.potential(R, Z, x) - want) < 1e-14
    # 3-4-5 triangle of nuclei
    R = np.array([[0.0, 0, 0], [3.0, 0, 0], [0.0, 4.0, 0]])
    Z = np.array([1.0, 2.0, 3.0])
    assert abs(oracle.nuclear_repulsion(R, Z) - (2 / 3 + 3 / 4 + 6 / 5)) < 1e-15


def test_square_c4h4_nuclear_repulsion_symmetry():
    """The (a, b) = (2.7, 2.7) C4H4 geometry is a square: its repulsion is
    unchanged by a 90-degree rotation and by relabelling the nuclei."""
    g = synth.c4h4_geometries(8)[0]
    e = oracle.nuclear_repulsion(g.R, g.Z)
    rot = np.array([[0, -1, 0], [1, 0, 0], [0, 0, 1.0]])
    assert abs(oracle.nuclear_repulsion(g.R @ rot.T, g.Z) - e) < 1e-12
    p = np.random.default_rng(0).permutation(8)
    assert abs(oracle.nuclear_repulsion(g.R[p], g.Z[p]) - e) < 1e-12
    # hand value: carbons on a square of side 2.7 (4 sides, 2 diagonals)
    s = 2.7
    cc = 36 * (4 / s + 2 / (s * math.sqrt(2)))
    assert e > cc


# ---------------------------------------------------------------------------
# Random numbers and Metropolis (Sec. 1, Eq. 2: sampling |psi|^2)
# ---------------------------------------------------------------------------

def test_mcmc_normals_are_standard_normal():
    n3 = 30
    zs = []
    us = []
    for w in range(400):
        z, u = oracle.mcmc_randoms(n3, w, 2, 5)
        zs.append(z)
        us.append(u)
    z = np.concatenate(zs)
    u = np.array(us)
    assert abs(z.mean()) < 0.03 and abs(z.var() - 1) < 0.04
    # fourth moment of a standard normal is 3
    assert abs((z ** 4).mean() - 3) < 0.3
    assert 0 < u.min() and u.max() < 1 and abs(u.mean() - 0.5) < 0.05
    # different walkers / steps / seeds give different streams
    a, _ = oracle.mcmc_randoms(n3, 0, 2, 5)
    b, _ = oracle.mcmc_randoms(n3, 1, 2, 5)
    c, _ = oracle.mcmc_randoms(n3, 0, 2, 6)
    d, _ = oracle.mcmc_randoms(n3, 0, 3, 5)
    for o in (b, c, d):
        assert abs(np.corrcoef(a, o)[0, 1]) < 0.6 and np.max(np.abs(a - o)) > 0.1
    # Philox is a bijection for a fixed key: distinct counters, distinct blocks
    seen = {tuple(oracle.philox4x32_10([i, 0, 0, 0], [1, 2])) for i in range(2000)}
    assert len(seen) == 2000


def test_philox_known_answer_vectors():
    """Philox4x32-10 against the published known-answer vectors
    (tests/golden/philox4x32_10_kat.txt): a swapped output word, a wrong round
    or Weyl constant, or a missing round changes every vector."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "philox4x32_10_kat.txt")
    rows = [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(t, 16) for t in r]
        assert oracle.philox4x32_10(v[0:4], v[4:6]) == v[6:10]


def test_mcmc_hydrogen_samples_psi_squared():
    """|psi|^2 = exp(-2r) has <r> = 3/2 bohr; sampling |psi| instead (a dropped
    factor of 2 in the acceptance) would give <r> = 3."""
    net = synth.Net(1, 4, 4, 1, 1, 0, 1)
    lay, P = _params(net)
    _set(lay, P, "w_orb", 0.0)
    _set(lay, P, "g_orb", 1.0)
    B = 2000
    x = np.random.default_rng(16).standard_normal((B, 1, 3))
    lp, _ = oracle.logpsi(net, P, [synth.atom(1)], x)
    x, lp, acc, _ = oracle.mcmc(net, P, [synth.atom(1)], x, lp, 100, 0.8, 2, 0)
    rs = []
    for k in range(10):
        x, lp, acc, _ = oracle.mcmc(net, P, [synth.atom(1)], x, lp, 10, 0.8, 2, 1000 + 10 * k)
        rs.append(np.linalg.norm(x[:, 0], axis=1).mean())
    r = float(np.mean(rs))
    assert abs(r - 1.5) < 0.05, r
    np.testing.assert_allclose(lp, -np.linalg.norm(x[:, 0], axis=1), atol=1e-12)


def test_clip_seeds_reduce_to_plain_estimator_and_vanish_at_zero_width():
    """Clipping (the training-loop option around the gradient): with a band
    wide enough to clip nothing, the clipped gradient is the plain VMC
    gradient of oracle_energy_grad; with a zero-width band every energy is
    clipped to the median and the gradient vanishes."""
    net = synth.Net(2, 8, 4, 2, 2, 1, 1)
    lay, P = _params(net, 7)
    x = np.random.default_rng(21).standard_normal((9, 3, 3))
    eloc = np.random.default_rng(22).standard_normal(9) * 3 - 7
    em, g = oracle.energy_grad(net, P, [synth.atom(3)], x, eloc)
    em_c, g_c = oracle.energy_grad_clipped(net, P, [synth.atom(3)], x, eloc, 1e9)
    np.testing.assert_allclose(em_c, em, rtol=1e-15)
    np.testing.assert_allclose(g_c, g, rtol=1e-9, atol=1e-12 * np.abs(g).max())
    em0, g0 = oracle.energy_grad_clipped(net, P, [synth.atom(3)], x, eloc, 0.0)
    np.testing.assert_allclose(em0, em, rtol=1e-15)
    assert np.abs(g0).max() == 0.0


@pytest.mark.parametrize("B", [1, 2, 7, 10, 101])
def test_clip_seeds_median_spread_band_and_centering(B):
    rng = np.random.default_rng(23 + B)
    e = rng.standard_normal(B) * 2 - 5
    if B > 3:
        e[1] = 400.0   # outliers on both sides
        e[2] = -900.0
    scale = 1.5
    seeds, st = oracle.clip_seeds(e, scale)
    m, tv, cbar = st[0]
    # median and mean absolute deviation against the library routines
    assert m == np.median(e)
    np.testing.assert_allclose(tv, np.mean(np.abs(e - np.median(e))), rtol=1e-14)
    # the clipped energy behind every seed lies in the band and equals E_L inside it
    c = seeds * B / 2 + cbar
    lo, hi = m - scale * tv, m + scale * tv
    assert np.all(c >= lo - 1e-12) and np.all(c <= hi + 1e-12)
    inside = (e > lo) & (e < hi)
    np.testing.assert_allclose(c[inside], e[inside], rtol=1e-13, atol=1e-12)
    if B > 3:
        np.testing.assert_allclose(c[[1, 2]], [hi, lo], rtol=1e-13)
    # centred seeds; invariant under a permutation of the walkers
    assert abs(seeds.sum()) < 1e-12 * max(1.0, np.abs(seeds).max() * B)
    perm = rng.permutation(B)
    s2, _ = oracle.clip_seeds(e[perm], scale)
    np.testing.assert_allclose(s2, seeds[perm], rtol=1e-14, atol=1e-15)


def test_clip_seeds_geometries_are_independent():
    rng = np.random.default_rng(31)
    e = rng.standard_normal(12)
    geo = np.array([0, 1, 0, 1, 1, 0, 0, 1, 0, 0, 1, 1], np.int32)
    seeds, st = oracle.clip_seeds(e, 2.0, geo=geo, n_geo=2)
    for g in range(2):
        sg, stg = oracle.clip_seeds(e[geo == g], 2.0)
        np.testing.assert_allclose(seeds[geo == g], sg, rtol=1e-15)
        np.testing.assert_allclose(st[g], stg[0], rtol=1e-15)


def test_adapt_width_cases():
    assert oracle.adapt_width(0.02, 60, 100, 0.5, 0.55, 1.1) == pytest.approx(0.022, rel=1e-15)
    assert oracle.adapt_width(0.02, 40, 100, 0.5, 0.55, 1.1) == pytest.approx(0.02 / 1.1, rel=1e-15)
    assert oracle.adapt_width(0.02, 52, 100, 0.5, 0.55, 1.1) == 0.02
    assert oracle.adapt_width(0.02, 0, 0, 0.5, 0.55, 1.1) == 0.02


# ---------------------------------------------------------------------------
# Full-covariance envelope (Eq. 4: one 3x3 Sigma per orbital and nucleus)
# ---------------------------------------------------------------------------

def _rotation(rng):
    q, r = np.linalg.qr(rng.standard_normal((3, 3)))
    return q * np.sign(np.diag(r))


def test_full_covariance_with_scaled_rotations_is_isotropic():
    """Sigma = s Q with Q orthogonal gives |Sigma d| = |s| |d|: the
    full-covariance network equals the isotropic one with sigma = s in log|psi|,
    its derivatives and E_L, and its Sigma gradient contracted with Q is the
    isotropic sigma gradient (chain rule through Sigma = s Q)."""
    rng = np.random.default_rng(41)
    iso = synth.Net(2, 12, 6, 2, 2, 1, 2)
    full = synth.Net(2, 12, 6, 2, 2, 1, 2, envelope=1)
    lay_i, P_i = _params(iso, 42)
    lay_f = oracle.layout(full)
    assert [e.name for e in lay_i] == [e.name for e in lay_f]
    P_f = np.zeros(sum(e.count for e in lay_f))
    Qs = {}
    for ei, ef in zip(lay_i, lay_f):
        blk = P_i[ei.offset:ei.offset + ei.count]
        if ei.name.startswith("sigma_"):
            blk[:] = 0.4 + rng.random(ei.count)
            P_i[ei.offset:ei.offset + ei.count] = blk
            Q = np.stack([_rotation(rng) for _ in range(ei.count)])
            Qs[ei.name] = Q
            P_f[ef.offset:ef.offset + ef.count] = (blk[:, None, None] * Q).reshape(-1)
        else:
            assert ei.count == ef.count
            P_f[ef.offset:ef.offset + ef.count] = blk
    geom = synth.Geometry(R=np.array([[0.0, 0.0, 0.0], [0.3, 1.2, -0.4]]), Z=np.array([2.0, 1.0]))
    x = rng.standard_normal((4, 3, 3))
    oi = oracle.local_energy(iso, P_i, [geom], x)
    of = oracle.local_energy(full, P_f, [geom], x)
    for k in ("logpsi", "sign", "eloc", "kinetic"):
        np.testing.assert_allclose(of[k], oi[k], rtol=1e-10, atol=1e-10)
    np.testing.assert_allclose(of["grad"], oi["grad"], rtol=1e-9, atol=1e-9)
    seeds = np.array([0.3, -0.8, 1.1, 0.5])
    gi = oracle.logpsi_vjp(iso, P_i, [geom], x, seeds)
    gf = oracle.logpsi_vjp(full, P_f, [geom], x, seeds)
    for ei, ef in zip(lay_i, lay_f):
        a = gi[ei.offset:ei.offset + ei.count]
        b = gf[ef.offset:ef.offset + ef.count]
        if ei.name.startswith("sigma_"):
            b = (b.reshape(-1, 3, 3) * Qs[ei.name]).sum(axis=(1, 2))
        np.testing.assert_allclose(b, a, rtol=1e-9, atol=1e-12 * max(1.0, np.abs(gi).max()), err_msg=ei.name)


def test_full_covariance_hydrogen_closed_form():
    """psi = exp(-|S r|) (one electron, Z = 1, w = 0, g = 1, pi = 1): with
    M = S^T S, u = M r and rho = |S r|, the Laplacian of psi over psi is
    |u|^2 / rho^2 - tr(M) / rho + |u|^2 / rho^3, so
    E_L = -1/2 (that) - 1/|r| at every point."""
    net = synth.Net(1, 4, 4, 1, 1, 0, 1, envelope=1)
    lay, P = _params(net, 43)
    _set(lay, P, "w_orb", 0.0)
    _set(lay, P, "g_orb", 1.0)
    S = np.array([[1.3, 0.2, -0.1], [0.0, 0.7, 0.4], [0.3, -0.2, 1.9]])
    _block(lay, P, "sigma_up")[:] = S.reshape(-1)
    x = np.random.default_rng(44).standard_normal((16, 1, 3))
    out = oracle.local_energy(net, P, [synth.atom(1)], x)
    r = x[:, 0]
    M = S.T @ S
    u = r @ M.T
    rho = np.linalg.norm(r @ S.T, axis=1)
    uu = (u ** 2).sum(axis=1)
    lap = uu / rho ** 2 - np.trace(M) / rho + uu / rho ** 3
    want = -0.5 * lap - 1.0 / np.linalg.norm(r, axis=1)
    np.testing.assert_allclose(out["eloc"], want, rtol=1e-10, atol=1e-10)
    np.testing.assert_allclose(out["logpsi"], -rho, rtol=1e-12)


def test_full_covariance_derivatives_and_parameter_gradient_by_differences():
    """Jets and the reverse pass of a full-covariance network against central
    differences (coordinates and random parameter directions, block by block)."""
    net = synth.Net(2, 10, 6, 2, 2, 2, 2, envelope=1)
    lay, P = _params(net, 45)
    rng = np.random.default_rng(46)
    for e in lay:
        if e.name.startswith("sigma_"):
            P[e.offset:e.offset + e.count] += 0.3 * rng.standard_normal(e.count)
        if e.name.startswith(("pi_", "g_orb")):
            P[e.offset:e.offset + e.count] = 0.5 + rng.random(e.count)
    geom = synth.Geometry(R=np.array([[0.0, 0.0, 0.0], [1.0, 0.5, 0.2]]), Z=np.array([2.0, 2.0]))
    x = rng.standard_normal((2, 4, 3))
    out = oracle.local_energy(net, P, [geom], x[:1])
    h = 1e-4
    lp0, _ = oracle.logpsi(net, P, [geom], x[:1])
    for c in range(12):
        xp = x[:1].copy().reshape(-1)
        xm = x[:1].copy().reshape(-1)
        xp[c] += h
        xm[c] -= h
        lpp, _ = oracle.logpsi(net, P, [geom], xp.reshape(1, 4, 3))
        lpm, _ = oracle.logpsi(net, P, [geom], xm.reshape(1, 4, 3))
        assert abs((lpp[0] - lpm[0]) / (2 * h) - out["grad"][0, c]) < 1e-6 * max(1, abs(out["grad"][0, c]))
        fd2 = (lpp[0] - 2 * lp0[0] + lpm[0]) / h ** 2
        assert abs(fd2 - out["d2"][0, c]) < 1e-3 * max(1, abs(fd2))
    seeds = np.array([0.9, -0.6])
    g = oracle.logpsi_vjp(net, P, [geom], x, seeds)
    for e in lay:
        v = np.zeros(P.shape[0])
        v[e.offset:e.offset + e.count] = rng.standard_normal(e.count)
        eps = 1e-6
        lpp, _ = oracle.logpsi(net, P + eps * v, [geom], x)
        lpm, _ = oracle.logpsi(net, P - eps * v, [geom], x)
        fd = seeds @ ((lpp - lpm) / (2 * eps))
        assert abs(fd - g @ v) < 2e-6 * max(1.0, abs(fd)), e.name


# ---------------------------------------------------------------------------
# KFAC factors and preconditioner (Sec. 1: the optimiser behind FermiNet)
# ---------------------------------------------------------------------------

def _kfac_block(net, F, name):
    blocks, _ = oracle.kfac_blocks(net)
    _, off, d = next(b for b in blocks if b[0] == name)
    return F[off:off + d * d].reshape(d, d)


def test_kfac_single_row_factors_are_rank_one_gradient_pieces():
    """One walker with one electron: every one-electron layer and the orbital
    layer see a single row, so A = a a^T and G = d d^T with grad = d a^T
    ([W b] of the reverse pass, seed 1): grad grad^T = tr(A) G and
    grad^T grad = tr(G) A."""
    net = synth.Net(3, 10, 6, 3, 1, 0, 2)
    lay, P = _params(net, 51)
    rng = np.random.default_rng(52)
    for e in lay:
        if e.name.startswith(("b", "g_orb", "pi_", "sigma_")):
            P[e.offset:e.offset + e.count] = 0.3 + rng.random(e.count)
    geom = synth.Geometry(R=np.array([[0.0, 0.0, 0.0], [0.4, 1.1, -0.2]]), Z=np.array([1.0, 1.0]))
    x = rng.standard_normal((1, 1, 3))
    F = oracle.kfac_factors(net, P, [geom], x)
    g = oracle.logpsi_vjp(net, P, [geom], x, np.ones(1))
    for l in range(net.n_layers):
        wV = 3 * (4 * net.n_nuc if l == 0 else net.d1) + 2 * (4 if l == 0 else net.d2)
        W = np.concatenate([_block(lay, g, f"V{l}").reshape(net.d1, wV), _block(lay, g, f"b{l}")[:, None]], axis=1)
        A, G = _kfac_block(net, F, f"A1_{l}"), _kfac_block(net, F, f"G1_{l}")
        np.testing.assert_allclose(W @ W.T, np.trace(A) * G, rtol=1e-10, atol=1e-12)
        np.testing.assert_allclose(W.T @ W, np.trace(G) * A, rtol=1e-10, atol=1e-12)
    W = np.concatenate([_block(lay, g, "w_orb_up").reshape(-1, net.d1), _block(lay, g, "g_orb_up")[:, None]], axis=1)
    A, G = _kfac_block(net, F, "Ao_0"), _kfac_block(net, F, "Go_0")
    np.testing.assert_allclose(W @ W.T, np.trace(A) * G, rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(W.T @ W, np.trace(G) * A, rtol=1e-10, atol=1e-12)


def test_kfac_envelope_diagonal_and_batch_averaging():
    """D is the mean squared per-walker gradient of the envelope parameters
    (against per-walker reverse passes), and every factor of a batch is the
    walker-weighted mean of the factors of its parts."""
    net = synth.Net(2, 8, 4, 2, 2, 1, 2)
    lay, P = _params(net, 53)
    geom = synth.Geometry(R=np.array([[0.0, 0.0, 0.0], [0.0, 0.0, 1.3]]), Z=np.array([2.0, 1.0]))
    x = np.random.default_rng(54).standard_normal((5, 3, 3))
    F = oracle.kfac_factors(net, P, [geom], x)
    _, nb = oracle.kfac_blocks(net)
    p0 = next(e.offset for e in lay if e.name == "pi_up")
    gw = np.stack([oracle.logpsi_vjp(net, P, [geom], x, np.eye(5)[w]) for w in range(5)])
    np.testing.assert_allclose(F[nb:], (gw[:, p0:] ** 2).mean(axis=0), rtol=1e-10, atol=1e-14)
    F1 = oracle.kfac_factors(net, P, [geom], x[:2])
    F2 = oracle.kfac_factors(net, P, [geom], x[2:])
    np.testing.assert_allclose(F, (2 * F1 + 3 * F2) / 5, rtol=1e-10, atol=1e-14)
    for name, off, d in oracle.kfac_blocks(net)[0]:  # symmetric positive semidefinite
        M = F[off:off + d * d].reshape(d, d)
        np.testing.assert_allclose(M, M.T, rtol=0, atol=1e-12 * max(1.0, np.abs(M).max()))
        assert np.linalg.eigvalsh(M).min() > -1e-10 * max(1.0, np.abs(M).max()), name


def test_kfac_precondition_against_library_solves():
    """Each layer block of the update is (G + sqrt(l) I)^-1 [W b] (A + sqrt(l) I)^-1
    (checked against numpy's dense solves), envelope entries grad / (D + l), and
    a huge damping reduces the update to grad / l."""
    net = synth.Net(2, 8, 4, 2, 2, 1, 2)
    lay, P = _params(net, 55)
    geom = synth.Geometry(R=np.array([[0.0, 0.0, 0.0], [0.0, 0.0, 1.3]]), Z=np.array([2.0, 1.0]))
    x = np.random.default_rng(56).standard_normal((4, 3, 3))
    F = oracle.kfac_factors(net, P, [geom], x)
    grad = np.random.default_rng(57).standard_normal(P.shape[0])
    lam = 1e-2
    out = oracle.kfac_precondition(net, F, grad, lam)
    g = np.sqrt(lam)
    for l in range(net.n_layers):
        wV = 3 * (4 * net.n_nuc if l == 0 else net.d1) + 2 * (4 if l == 0 else net.d2)
        M = np.concatenate([_block(lay, grad, f"V{l}").reshape(net.d1, wV), _block(lay, grad, f"b{l}")[:, None]], 1)
        A, G = _kfac_block(net, F, f"A1_{l}"), _kfac_block(net, F, f"G1_{l}")
        want = np.linalg.solve(G + g * np.eye(len(G)), M) @ np.linalg.inv(A + g * np.eye(len(A)))
        got = np.concatenate([_block(lay, out, f"V{l}").reshape(net.d1, wV), _block(lay, out, f"b{l}")[:, None]], 1)
        np.testing.assert_allclose(got, want, rtol=1e-8, atol=1e-10 * np.abs(want).max())
    M = np.concatenate([_block(lay, grad, "w_orb_down").reshape(-1, net.d1), _block(lay, grad, "g_orb_down")[:, None]], 1)
    A, G = _kfac_block(net, F, "Ao_1"), _kfac_block(net, F, "Go_1")
    want = np.linalg.solve(G + g * np.eye(len(G)), M) @ np.linalg.inv(A + g * np.eye(len(A)))
    got = np.concatenate([_block(lay, out, "w_orb_down").reshape(-1, net.d1), _block(lay, out, "g_orb_down")[:, None]], 1)
    np.testing.assert_allclose(got, want, rtol=1e-8, atol=1e-10 * np.abs(want).max())
    _, nb = oracle.kfac_blocks(net)
    p0 = next(e.offset for e in lay if e.name == "pi_up")
    np.testing.assert_allclose(out[p0:], grad[p0:] / (F[nb:] + lam), rtol=1e-12)
    big = oracle.kfac_precondition(net, F, grad, 1e16)
    np.testing.assert_allclose(big * 1e16, grad, rtol=1e-4, atol=1e-6 * np.abs(grad).max())

"""Seeded synthetic inputs for the FermiNet VMC hot path.

This module holds no arithmetic of the method itself: it builds nuclear
geometries, walker positions and a flat initial parameter buffer from seeds.
Both the CUDA path and the FP64 oracle consume what it produces, so the two
sides always see bit-identical inputs.

The paper (arXiv:2011.07125) ships no datasets and no trained weights; its
systems (Ne and Ar atoms, Sec. 2 / Table 1; bicyclobutane-sized C4H6 and
cyclobutadiene-sized C4H4 molecules, Sec. 3 / Table 2 / Fig. 2) are stood in
for by the seeded shapes below.

Parameter buffers are generated from a *layout* (a list of entries with
``count``, ``fan_in`` and ``kind``) supplied by the caller, so this module does
not need to know how either implementation orders its parameters.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Sequence

import numpy as np

# Init kinds shared by both layouts (values match the C enums on both sides).
INIT_NORMAL = 0   # N(0, 1/fan_in)
INIT_ZERO = 1     # biases
INIT_ONE = 2      # envelope weights pi and exponents sigma ("exponents 1.0")
INIT_EYE3 = 3     # full-covariance envelope matrices: 3x3 identities (row-major)

# Seeds of the standard workloads: parameters 0, walkers 1, Metropolis 2.
SEED_PARAMS = 0
SEED_WALKERS = 1
SEED_MCMC = 2


@dataclasses.dataclass
class Net:
    """Network shape: L layers, one-/two-electron widths, K determinants."""
    n_layers: int
    d1: int
    d2: int
    n_det: int
    n_up: int
    n_down: int
    n_nuc: int
    envelope: int = 0  # 0: isotropic sigma (Sec. 3); 1: full 3x3 covariance (Eq. 4)

    @property
    def n_elec(self) -> int:
        return self.n_up + self.n_down


@dataclasses.dataclass
class Geometry:
    """One nuclear geometry: positions R [N,3] (bohr), charges Z [N]."""
    R: np.ndarray
    Z: np.ndarray


@dataclasses.dataclass
class Workload:
    name: str
    net: Net
    geoms: List[Geometry]
    counts: List[int]          # walkers per geometry, in batch order
    walker_var: float          # per-coordinate variance of the initial walkers
    mcmc_steps: int            # Metropolis moves per step
    mcmc_width: float          # proposal standard deviation (bohr)
    precision: str             # "fp32" or "mixed"
    with_grad: bool            # whether a step includes the VMC gradient

    @property
    def batch(self) -> int:
        return int(sum(self.counts))


def init_params(layout: Sequence, seed: int = SEED_PARAMS) -> np.ndarray:
    """Flat float32 parameter buffer in the order of ``layout``.

    Each layout entry must expose ``count``, ``fan_in`` and ``kind``.  Dense
    weights are N(0, 1/fan_in) drawn from ``numpy.random.default_rng(seed)`` in
    layout order; biases are 0; envelope weights and exponents are 1.
    """
    rng = np.random.default_rng(seed)
    chunks = []
    for e in layout:
        cnt = int(e.count)
        if e.kind == INIT_NORMAL:
            chunks.append(rng.standard_normal(cnt) / math.sqrt(max(int(e.fan_in), 1)))
        elif e.kind == INIT_ZERO:
            chunks.append(np.zeros(cnt))
        elif e.kind == INIT_ONE:
            chunks.append(np.ones(cnt))
        elif e.kind == INIT_EYE3:
            if cnt % 9:
                raise ValueError("a block of 3x3 identities needs a multiple of 9 entries")
            chunks.append(np.tile(np.eye(3).reshape(-1), cnt // 9))
        else:
            raise ValueError(f"unknown init kind {e.kind}")
    if not chunks:
        return np.zeros(0, np.float32)
    return np.concatenate(chunks).astype(np.float32)


def atom(Z: int) -> Geometry:
    return Geometry(R=np.zeros((1, 3)), Z=np.array([float(Z)]))


def c4h6_geometry(seed: int = 0) -> Geometry:
    """C4H6-shaped molecule: 4 carbons on a planar zigzag (bond 2.6 bohr, 120
    degrees, xy-plane), hydrogens 2,1,1,2 per carbon at 2.05 bohr along seeded
    uniform directions, each rejected if it lands within 1.5 bohr of a nucleus
    already placed.  Centred on the carbon centroid."""
    bond = 2.6
    ang = math.radians(30.0)
    C = [np.zeros(3)]
    for k in range(3):
        s = 1.0 if k % 2 == 0 else -1.0
        C.append(C[-1] + bond * np.array([math.cos(ang), s * math.sin(ang), 0.0]))
    C = np.array(C)
    C -= C.mean(axis=0)
    rng = np.random.default_rng(seed)
    placed = [c for c in C]
    H = []
    for ci, nh in zip(range(4), (2, 1, 1, 2)):
        for _ in range(nh):
            for _attempt in range(10000):
                u = rng.standard_normal(3)
                u /= np.linalg.norm(u)
                p = C[ci] + 2.05 * u
                if all(np.linalg.norm(p - q) >= 1.5 for q in placed):
                    break
            placed.append(p)
            H.append(p)
    R = np.vstack([C, np.array(H)])
    Z = np.array([6.0] * 4 + [1.0] * 6)
    return Geometry(R=R, Z=Z)


def c4h4_geometries(n_geom: int = 8) -> List[Geometry]:
    """Rectangular C4H4 shapes: carbons at (+-a/2, +-b/2, 0) with (a, b) stepping
    linearly from (2.7, 2.7) to (2.55, 2.95) bohr; each hydrogen 2.05 bohr
    outward from its carbon along the carbon's direction from the centre."""
    out = []
    for s in range(n_geom):
        t = s / max(n_geom - 1, 1)
        a = 2.7 + (2.55 - 2.7) * t
        b = 2.7 + (2.95 - 2.7) * t
        C = np.array([[sx * a / 2, sy * b / 2, 0.0] for sx in (1, -1) for sy in (1, -1)])
        H = np.array([c + 2.05 * c / np.linalg.norm(c) for c in C])
        out.append(Geometry(R=np.vstack([C, H]), Z=np.array([6.0] * 4 + [1.0] * 4)))
    return out


def electron_centres(geom: Geometry, n_up: int, n_down: int) -> np.ndarray:
    """Nucleus assigned to each electron (up electrons first).

    Electrons are handed out by nuclear charge (nucleus I gets Z_I of them, in
    nucleus order), spins alternate over that global list, and the list is then
    stably split into up and down electrons.  Requires sum(Z) == n_up + n_down
    and an alternation that reaches the requested counts; otherwise electrons
    are assigned round-robin to the nuclei.
    """
    n = n_up + n_down
    owners = []
    for I, z in enumerate(geom.Z):
        owners += [I] * int(round(z))
    if len(owners) != n:
        owners = [k % len(geom.Z) for k in range(n)]
    spins = [k % 2 for k in range(n)]  # 0 up, 1 down
    if spins.count(0) != n_up:
        spins = [0] * n_up + [1] * n_down
    up = [owners[k] for k in range(n) if spins[k] == 0]
    dn = [owners[k] for k in range(n) if spins[k] == 1]
    return np.array(up + dn, dtype=np.int64)


def init_walkers(wl: Workload, seed: int = SEED_WALKERS, counts: Sequence[int] | None = None) -> np.ndarray:
    """Walker positions, float32 [B, n, 3]: electron e of a walker on geometry g
    is N(R_g[owner(e)], walker_var * I)."""
    counts = list(wl.counts if counts is None else counts)
    rng = np.random.default_rng(seed)
    n = wl.net.n_elec
    std = math.sqrt(wl.walker_var)
    blocks = []
    for g, cnt in enumerate(counts):
        geom = wl.geoms[g if len(wl.geoms) > 1 else 0]
        cen = geom.R[electron_centres(geom, wl.net.n_up, wl.net.n_down)]  # [n,3]
        blocks.append(cen[None] + std * rng.standard_normal((cnt, n, 3)))
    return np.concatenate(blocks).astype(np.float32)


def geometry_of_walkers(counts: Sequence[int]) -> np.ndarray:
    return np.concatenate([np.full(c, g, np.int32) for g, c in enumerate(counts)])


def workload(name: str) -> Workload:
    """The standard workloads (by system): li, ne, ar, c4h6, c4h4x8, and kr (36
    electrons at the Ar widths).  "name@B" sets the batch of a one-geometry
    workload to B walkers."""
    if "@" in name:
        base, b = name.split("@", 1)
        wl = workload(base)
        if len(wl.geoms) != 1:
            raise KeyError(name)
        return dataclasses.replace(wl, name=name, counts=[int(b)])
    if name == "li":
        return Workload("li", Net(2, 32, 8, 1, 2, 1, 1), [atom(3)], [256], 1.0, 1, 0.02, "fp32", True)
    if name == "ne":
        return Workload("ne", Net(4, 256, 32, 16, 5, 5, 1), [atom(10)], [4096], 1.0, 10, 0.02, "fp32", True)
    if name == "ar":
        return Workload("ar", Net(4, 512, 32, 32, 9, 9, 1), [atom(18)], [4096], 1.5, 10, 0.02, "mixed", True)
    if name == "c4h6":
        return Workload("c4h6", Net(4, 256, 32, 16, 15, 15, 10), [c4h6_geometry(0)], [4096], 1.0, 10, 0.02,
                        "mixed", True)
    if name == "kr":  # a larger electron count at the second-row widths: 36 electrons, 18 per spin
        return Workload("kr", Net(4, 512, 32, 32, 18, 18, 1), [atom(36)], [4096], 1.5, 10, 0.02, "mixed", True)
    if name == "c4h4x8":
        return Workload("c4h4x8", Net(4, 256, 32, 16, 14, 14, 8), c4h4_geometries(8),
                        [256, 512, 768, 1024, 1536, 2048, 3072, 4096], 1.0, 10, 0.02, "mixed", True)
    raise KeyError(name)


WORKLOADS = ("li", "ne", "ar", "c4h6", "c4h4x8", "kr")


def subset(wl: Workload, per_geom: int) -> Workload:
    """Same workload with at most ``per_geom`` walkers per geometry."""
    return dataclasses.replace(wl, counts=[min(c, per_geom) for c in wl.counts])

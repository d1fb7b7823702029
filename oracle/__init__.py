"""FP64 CPU oracle for the FermiNet VMC hot path — TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline / reference legs of
``bench.py`` may import this package.  The product path (``paper_2011_07125_gb300``)
never imports it, and this package never imports the product path.

The C source ``ferminet_oracle.c`` is compiled with the system C compiler into
``oracle/_build/liboracle.so`` on first use (or by ``build()``) and loaded with ctypes.
Every function below is a thin marshalling wrapper; all arithmetic is in the C file.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass
from typing import List, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ferminet_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None


class ONet(C.Structure):
    _fields_ = [("n_layers", C.c_int), ("d1", C.c_int), ("d2", C.c_int), ("n_det", C.c_int),
                ("n_up", C.c_int), ("n_down", C.c_int), ("n_nuc", C.c_int), ("envelope", C.c_int)]


class OEntry(C.Structure):
    _fields_ = [("name", C.c_char * 32), ("offset", C.c_long), ("count", C.c_long),
                ("fan_in", C.c_long), ("kind", C.c_int), ("pad", C.c_int)]


@dataclass
class Entry:
    name: str
    offset: int
    count: int
    fan_in: int
    kind: int


def build(force: bool = False) -> str:
    """Compile the oracle (gcc, -O2, OpenMP) if it is missing or stale."""
    with _lock:
        if (not force and os.path.exists(_LIB_PATH)
                and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
            return _LIB_PATH
        os.makedirs(_OUT_DIR, exist_ok=True)
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fopenmp", "-fPIC", "-shared",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
        return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = C.CDLL(build())
    dp = C.POINTER(C.c_double)
    ip = C.POINTER(C.c_int)
    np_ = C.POINTER(ONet)
    lib.oracle_param_layout.argtypes = [np_, C.POINTER(OEntry), C.c_int, C.POINTER(C.c_long)]
    lib.oracle_param_layout.restype = C.c_int
    lib.oracle_slogdet.argtypes = [C.c_int, dp, dp, dp]
    lib.oracle_det_leibniz.argtypes = [C.c_int, dp]
    lib.oracle_det_leibniz.restype = C.c_double
    lib.oracle_nuclear_repulsion.argtypes = [C.c_int, dp, dp]
    lib.oracle_nuclear_repulsion.restype = C.c_double
    lib.oracle_potential.argtypes = [C.c_int, C.c_int, dp, dp, dp]
    lib.oracle_potential.restype = C.c_double
    lib.oracle_logpsi.argtypes = [np_, dp, dp, dp, ip, C.c_long, dp, dp, dp]
    lib.oracle_local_energy.argtypes = [np_, dp, dp, dp, ip, C.c_long, dp, dp, dp, dp, dp, dp, dp, dp]
    lib.oracle_logpsi_vjp.argtypes = [np_, dp, dp, dp, ip, C.c_long, dp, dp, dp]
    lib.oracle_energy_grad.argtypes = [np_, dp, dp, dp, ip, C.c_int, C.c_long, dp, dp, dp, dp]
    lib.oracle_philox4x32_10.argtypes = [C.POINTER(C.c_uint32), C.POINTER(C.c_uint32), C.POINTER(C.c_uint32)]
    lib.oracle_mcmc_randoms.argtypes = [C.c_int, C.c_ulonglong, C.c_ulonglong, C.c_ulonglong, dp, dp]
    lib.oracle_mcmc.argtypes = [np_, dp, dp, dp, ip, C.c_long, dp, dp, C.c_int, C.c_double,
                                C.c_ulonglong, C.c_ulonglong, ip, dp]
    lib.oracle_logpsi_jet.argtypes = [np_, dp, dp, dp, C.c_int, dp, dp]
    lib.oracle_clip_seeds.argtypes = [C.c_int, C.c_long, ip, dp, C.c_double, dp, dp]
    lib.oracle_energy_grad_clipped.argtypes = [np_, dp, dp, dp, ip, C.c_int, C.c_long, dp, dp, C.c_double, dp,
                                               dp]
    lib.oracle_kfac_size.argtypes = [np_]
    lib.oracle_kfac_size.restype = C.c_long
    lib.oracle_kfac_factors.argtypes = [np_, dp, dp, dp, ip, C.c_long, dp, dp]
    lib.oracle_kfac_precondition.argtypes = [np_, dp, dp, C.c_double, dp]
    lib.oracle_adapt_width.argtypes = [C.c_double] * 6
    lib.oracle_adapt_width.restype = C.c_double
    _lib = lib
    return lib


def _d(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _dp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _net(net) -> ONet:
    return ONet(net.n_layers, net.d1, net.d2, net.n_det, net.n_up, net.n_down, net.n_nuc,
                int(getattr(net, "envelope", 0)))


def _geo_arrays(geoms, n_nuc):
    R = _d(np.stack([np.asarray(g.R, np.float64).reshape(n_nuc, 3) for g in geoms]))
    Z = _d(np.stack([np.asarray(g.Z, np.float64).reshape(n_nuc) for g in geoms]))
    return R, Z


def _geo_idx(geo, B):
    if geo is None:
        return np.zeros(max(B, 1), np.int32)
    g = np.ascontiguousarray(geo, dtype=np.int32)
    assert g.shape[0] == B
    return g


def layout(net) -> List[Entry]:
    lib = _load()
    onet = _net(net)
    n_params = C.c_long(0)
    ne = lib.oracle_param_layout(C.byref(onet), None, 0, C.byref(n_params))
    if ne < 0:
        raise ValueError("invalid network shape")
    arr = (OEntry * ne)()
    lib.oracle_param_layout(C.byref(onet), arr, ne, C.byref(n_params))
    return [Entry(e.name.decode(), e.offset, e.count, e.fan_in, e.kind) for e in arr]


def n_params(net) -> int:
    ents = layout(net)
    return int(sum(e.count for e in ents))


def logpsi(net, params, geoms, x, geo=None):
    lib = _load()
    x = _d(x)
    B = x.shape[0]
    R, Z = _geo_arrays(geoms, net.n_nuc)
    P = _d(params)
    lp = np.zeros(B)
    sg = np.zeros(B)
    g = _geo_idx(geo, B)
    rc = lib.oracle_logpsi(C.byref(_net(net)), _dp(P), _dp(R), _dp(Z), g.ctypes.data_as(C.POINTER(C.c_int)),
                           B, _dp(x), _dp(lp), _dp(sg))
    if rc:
        raise ValueError("oracle_logpsi failed")
    return lp, sg


def local_energy(net, params, geoms, x, geo=None):
    """Dict with logpsi, sign, grad [B,3n], d2 [B,3n], kinetic, potential, eloc."""
    lib = _load()
    x = _d(x)
    B = x.shape[0]
    n3 = 3 * (net.n_up + net.n_down)
    R, Z = _geo_arrays(geoms, net.n_nuc)
    P = _d(params)
    out = {k: np.zeros(B) for k in ("logpsi", "sign", "kinetic", "potential", "eloc")}
    out["grad"] = np.zeros((B, n3))
    out["d2"] = np.zeros((B, n3))
    g = _geo_idx(geo, B)
    rc = lib.oracle_local_energy(C.byref(_net(net)), _dp(P), _dp(R), _dp(Z),
                                 g.ctypes.data_as(C.POINTER(C.c_int)), B, _dp(x),
                                 _dp(out["logpsi"]), _dp(out["sign"]), _dp(out["grad"]), _dp(out["d2"]),
                                 _dp(out["kinetic"]), _dp(out["potential"]), _dp(out["eloc"]))
    if rc:
        raise ValueError("oracle_local_energy failed")
    return out


def logpsi_vjp(net, params, geoms, x, seeds, geo=None):
    lib = _load()
    x = _d(x)
    B = x.shape[0]
    R, Z = _geo_arrays(geoms, net.n_nuc)
    P = _d(params)
    s = _d(seeds)
    grad = np.zeros(P.shape[0])
    g = _geo_idx(geo, B)
    rc = lib.oracle_logpsi_vjp(C.byref(_net(net)), _dp(P), _dp(R), _dp(Z), g.ctypes.data_as(C.POINTER(C.c_int)),
                               B, _dp(x), _dp(s), _dp(grad))
    if rc:
        raise ValueError("oracle_logpsi_vjp failed")
    return grad


def energy_grad(net, params, geoms, x, eloc, geo=None):
    """(emean [G], grad [P]) of the VMC energy gradient."""
    lib = _load()
    x = _d(x)
    B = x.shape[0]
    R, Z = _geo_arrays(geoms, net.n_nuc)
    P = _d(params)
    e = _d(eloc)
    grad = np.zeros(P.shape[0])
    em = np.zeros(len(geoms))
    g = _geo_idx(geo, B)
    rc = lib.oracle_energy_grad(C.byref(_net(net)), _dp(P), _dp(R), _dp(Z), g.ctypes.data_as(C.POINTER(C.c_int)),
                                len(geoms), B, _dp(x), _dp(e), _dp(em), _dp(grad))
    if rc:
        raise ValueError("oracle_energy_grad failed")
    return em, grad


def clip_seeds(eloc, scale, geo=None, n_geo=None):
    """(seeds [B], stats [G,3] = median, mean |E_L - median|, clipped mean) of
    the clipped VMC gradient."""
    lib = _load()
    e = _d(eloc)
    B = e.shape[0]
    g = _geo_idx(geo, B)
    G = int(n_geo if n_geo is not None else (int(g[:B].max()) + 1 if B else 1))
    seeds = np.zeros(max(B, 1))
    stats = np.zeros((G, 3))
    rc = lib.oracle_clip_seeds(G, B, g.ctypes.data_as(C.POINTER(C.c_int)), _dp(e) if B else None, float(scale),
                               _dp(seeds), _dp(stats))
    if rc:
        raise ValueError("oracle_clip_seeds failed")
    return seeds[:B], stats


def energy_grad_clipped(net, params, geoms, x, eloc, scale, geo=None):
    """(emean [G], grad [P]) of the VMC gradient with clipped local energies."""
    lib = _load()
    x = _d(x)
    B = x.shape[0]
    R, Z = _geo_arrays(geoms, net.n_nuc)
    P = _d(params)
    e = _d(eloc)
    grad = np.zeros(P.shape[0])
    em = np.zeros(len(geoms))
    g = _geo_idx(geo, B)
    rc = lib.oracle_energy_grad_clipped(C.byref(_net(net)), _dp(P), _dp(R), _dp(Z),
                                        g.ctypes.data_as(C.POINTER(C.c_int)), len(geoms), B, _dp(x), _dp(e),
                                        float(scale), _dp(em), _dp(grad))
    if rc:
        raise ValueError("oracle_energy_grad_clipped failed")
    return em, grad


def kfac_factors(net, params, geoms, x, geo=None):
    """Flat FP64 buffer of the KFAC factors (layout in ferminet_oracle.c)."""
    lib = _load()
    x = _d(x)
    B = x.shape[0]
    R, Z = _geo_arrays(geoms, net.n_nuc)
    P = _d(params)
    F = np.zeros(lib.oracle_kfac_size(C.byref(_net(net))))
    g = _geo_idx(geo, B)
    rc = lib.oracle_kfac_factors(C.byref(_net(net)), _dp(P), _dp(R), _dp(Z), g.ctypes.data_as(C.POINTER(C.c_int)),
                                 B, _dp(x), _dp(F))
    if rc:
        raise ValueError("oracle_kfac_factors failed")
    return F


def kfac_precondition(net, factors, grad, lam):
    lib = _load()
    F = _d(factors)
    gr = _d(grad)
    out = np.zeros_like(gr)
    if lib.oracle_kfac_precondition(C.byref(_net(net)), _dp(F), _dp(gr), float(lam), _dp(out)):
        raise ValueError("oracle_kfac_precondition failed")
    return out


def kfac_blocks(net):
    """Names, offsets and shapes of the factor blocks, in buffer order."""
    L, d1, d2, K = net.n_layers, net.d1, net.d2, net.n_det
    din1 = [4 * net.n_nuc if l == 0 else d1 for l in range(L)]
    din2 = [4 if l == 0 else d2 for l in range(L)]
    out, off = [], 0
    for l in range(L):
        a = 3 * din1[l] + 2 * din2[l] + 1
        out.append((f"A1_{l}", off, a)); off += a * a
        out.append((f"G1_{l}", off, d1)); off += d1 * d1
    for l in range(L - 1):
        a = din2[l] + 1
        out.append((f"A2_{l}", off, a)); off += a * a
        out.append((f"G2_{l}", off, d2)); off += d2 * d2
    for s, ns in enumerate((net.n_up, net.n_down)):
        out.append((f"Ao_{s}", off, d1 + 1)); off += (d1 + 1) ** 2
        out.append((f"Go_{s}", off, K * ns)); off += (K * ns) ** 2
    return out, off


def adapt_width(width, accepted, moves, lo, hi, factor):
    return _load().oracle_adapt_width(float(width), float(accepted), float(moves), float(lo), float(hi),
                                      float(factor))


def mcmc(net, params, geoms, x, logpsi0, n_steps, width, seed, counter, geo=None):
    """Returns (x_new [B,n,3], logpsi_new [B], accepted [B], margin [B])."""
    lib = _load()
    x = _d(x).copy()
    B = x.shape[0]
    lp = _d(logpsi0).copy()
    R, Z = _geo_arrays(geoms, net.n_nuc)
    P = _d(params)
    acc = np.zeros(max(B, 1), np.int32)
    mg = np.zeros(max(B, 1))
    g = _geo_idx(geo, B)
    rc = lib.oracle_mcmc(C.byref(_net(net)), _dp(P), _dp(R), _dp(Z), g.ctypes.data_as(C.POINTER(C.c_int)),
                         B, _dp(x), _dp(lp), int(n_steps), float(width), int(seed), int(counter),
                         acc.ctypes.data_as(C.POINTER(C.c_int)), _dp(mg))
    if rc:
        raise ValueError("oracle_mcmc failed")
    return x, lp, acc[:B], mg[:B]


def philox4x32_10(ctr: Sequence[int], key: Sequence[int]):
    lib = _load()
    c = (C.c_uint32 * 4)(*ctr)
    k = (C.c_uint32 * 2)(*key)
    o = (C.c_uint32 * 4)()
    lib.oracle_philox4x32_10(c, k, o)
    return [int(v) for v in o]


def mcmc_randoms(n3, walker, seed, counter):
    lib = _load()
    z = np.zeros(n3)
    u = C.c_double(0)
    lib.oracle_mcmc_randoms(int(n3), int(walker), int(seed), int(counter), _dp(z), C.byref(u))
    return z, u.value


def slogdet(A):
    lib = _load()
    A = _d(A)
    n = A.shape[0]
    s = C.c_double(0)
    la = C.c_double(0)
    lib.oracle_slogdet(n, _dp(A) if n else None, C.byref(s), C.byref(la))
    return s.value, la.value


def det_leibniz(A):
    lib = _load()
    A = _d(A)
    return lib.oracle_det_leibniz(A.shape[0], _dp(A))


def potential(R, Z, x):
    lib = _load()
    R, Z, x = _d(R), _d(Z), _d(x)
    return lib.oracle_potential(x.shape[0], R.shape[0], _dp(R), _dp(Z), _dp(x))


def nuclear_repulsion(R, Z):
    lib = _load()
    R, Z = _d(R), _d(Z)
    return lib.oracle_nuclear_repulsion(R.shape[0], _dp(R), _dp(Z))


def logpsi_jet(net, params, geom, x, coord):
    """(value, d/dx_coord, d^2/dx_coord^2) of log|psi| for one walker."""
    lib = _load()
    P = _d(params)
    R = _d(np.asarray(geom.R).reshape(-1, 3))
    x = _d(x).reshape(-1)
    out = np.zeros(3)
    s = C.c_double(0)
    lib.oracle_logpsi_jet(C.byref(_net(net)), _dp(P), _dp(R), _dp(x), int(coord), _dp(out), C.byref(s))
    return out, s.value

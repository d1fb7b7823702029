"""Python binding of libferminet (the C ABI declared in include/ferminet.h).

Argument marshalling only: every step of the hot path runs in the library's
CUDA kernels.  PyTorch supplies device memory and the stream.  There is no CPU
fallback: if the library is missing or no CUDA device is present, the calls
raise.
"""
from __future__ import annotations

import ctypes as C
import os
import threading
from dataclasses import dataclass
from typing import List, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libferminet.so")
_lock = threading.Lock()
_lib = None

STATUS = {0: "FN_OK", 1: "FN_EINVAL", 2: "FN_ECUDA", 3: "FN_ENOMEM", 4: "FN_ENONFINITE", 5: "FN_ETIMEOUT",
          6: "FN_ESINGULAR"}
PREC = {"fp32": 0, "mixed": 1}


class FnNet(C.Structure):
    _fields_ = [("n_layers", C.c_int), ("d1", C.c_int), ("d2", C.c_int), ("n_det", C.c_int),
                ("n_up", C.c_int), ("n_down", C.c_int), ("n_nuc", C.c_int), ("envelope", C.c_int)]


class FnGeometry(C.Structure):
    _fields_ = [("R", C.POINTER(C.c_double)), ("Z", C.POINTER(C.c_double)),
                ("walker_offset", C.c_long), ("walker_count", C.c_long)]


class FnTuning(C.Structure):
    _fields_ = [("layer_groups", C.c_int), ("feature_tile", C.c_int), ("tangent_chunk", C.c_long),
                ("residual_smem", C.c_int), ("pair_unfused", C.c_int), ("adjoint_simt", C.c_int),
                ("orbital_joint", C.c_int)]


class FnTrainOpts(C.Structure):
    _fields_ = [("clip_scale", C.c_float), ("d_width", C.c_void_p), ("accept_lo", C.c_float),
                ("accept_hi", C.c_float), ("width_factor", C.c_float)]


class FnParamEntry(C.Structure):
    _fields_ = [("name", C.c_char * 32), ("offset", C.c_long), ("count", C.c_long),
                ("fan_in", C.c_long), ("kind", C.c_int), ("pad", C.c_int)]


@dataclass
class Entry:
    name: str
    offset: int
    count: int
    fan_in: int
    kind: int


class FermiNetError(RuntimeError):
    pass


EXPORTS = ("ferminet_init", "ferminet_param_layout", "ferminet_net_layout", "ferminet_set_params",
           "ferminet_logpsi", "ferminet_local_energy", "ferminet_logpsi_vjp", "ferminet_energy_grad",
           "ferminet_energy_sums", "ferminet_energy_grad_partial", "ferminet_mcmc_step", "ferminet_step", "ferminet_sync", "ferminet_flagged_matrices", "ferminet_profile",
           "ferminet_profile_read", "ferminet_launch_count", "ferminet_get_tuning", "ferminet_set_tuning",
           "ferminet_autotune", "ferminet_set_train_opts", "ferminet_kfac_size", "ferminet_kfac_factors",
           "ferminet_kfac_precondition", "ferminet_last_error", "ferminet_destroy")
KERNEL_CLASSES = {"tangent_gemm": 0, "det_tangent": 1, "two_layer": 2, "means": 3, "tanh": 4, "value_pass": 5,
                  "adjoint": 6}


def load(path: Optional[str] = None):
    """Loads libferminet.so (building it first if it is absent)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if path is None:
            # incremental: recompiles only translation units newer than their objects
            from . import build as _build
            _build.build()
        lib = C.CDLL(p)
        vp = C.c_void_p
        lib.ferminet_init.argtypes = [C.POINTER(FnNet), C.POINTER(FnGeometry), C.c_int, C.c_int, vp,
                                      C.POINTER(vp)]
        lib.ferminet_param_layout.argtypes = [vp, C.POINTER(FnParamEntry), C.c_int, C.POINTER(C.c_int),
                                              C.POINTER(C.c_long)]
        lib.ferminet_net_layout.argtypes = [C.POINTER(FnNet), C.POINTER(FnParamEntry), C.c_int,
                                            C.POINTER(C.c_int), C.POINTER(C.c_long)]
        lib.ferminet_set_params.argtypes = [vp, vp]
        lib.ferminet_logpsi.argtypes = [vp, vp, C.c_long, vp, vp]
        lib.ferminet_local_energy.argtypes = [vp, vp, C.c_long, vp, vp, vp, vp]
        lib.ferminet_logpsi_vjp.argtypes = [vp, vp, C.c_long, vp, vp]
        lib.ferminet_energy_grad.argtypes = [vp, vp, C.c_long, vp, vp, vp]
        lib.ferminet_energy_sums.argtypes = [vp, vp, C.c_long, vp]
        lib.ferminet_energy_grad_partial.argtypes = [vp, vp, C.c_long, vp, vp, vp, vp, vp]
        lib.ferminet_mcmc_step.argtypes = [vp, vp, vp, C.c_long, C.c_int, C.c_float, C.c_uint64, C.c_uint64, vp]
        lib.ferminet_step.argtypes = [vp, vp, vp, C.c_long, C.c_int, C.c_float, C.c_uint64, C.c_uint64, vp, vp, vp,
                                      vp, C.c_int]
        lib.ferminet_sync.argtypes = [vp]
        lib.ferminet_flagged_matrices.argtypes = [vp]
        lib.ferminet_flagged_matrices.restype = C.c_long
        lib.ferminet_last_error.argtypes = [vp]
        lib.ferminet_last_error.restype = C.c_char_p
        lib.ferminet_destroy.argtypes = [vp]
        lib.ferminet_destroy.restype = None
        lib.ferminet_profile.argtypes = [vp, C.c_int]
        lib.ferminet_profile_read.argtypes = [vp, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_long),
                                              C.POINTER(C.c_double)]
        lib.ferminet_get_tuning.argtypes = [vp, C.POINTER(FnTuning)]
        lib.ferminet_set_tuning.argtypes = [vp, C.POINTER(FnTuning)]
        lib.ferminet_autotune.argtypes = [vp, vp, C.c_long, C.c_int, C.POINTER(FnTuning)]
        lib.ferminet_set_train_opts.argtypes = [vp, C.POINTER(FnTrainOpts)]
        lib.ferminet_kfac_size.argtypes = [C.POINTER(FnNet), C.POINTER(C.c_long)]
        lib.ferminet_kfac_factors.argtypes = [vp, vp, C.c_long, vp]
        lib.ferminet_kfac_precondition.argtypes = [vp, vp, vp, C.c_float, vp]
        lib.ferminet_launch_count.argtypes = []
        lib.ferminet_launch_count.restype = C.c_longlong
        for f in EXPORTS:
            if f not in ("ferminet_flagged_matrices", "ferminet_last_error", "ferminet_destroy",
                         "ferminet_launch_count"):
                getattr(lib, f).restype = C.c_int
        _lib = lib
        return lib


def _net(net) -> FnNet:
    return FnNet(net.n_layers, net.d1, net.d2, net.n_det, net.n_up, net.n_down, net.n_nuc,
                 int(getattr(net, "envelope", 0)))


def net_layout(net) -> List[Entry]:
    """Parameter layout for a network shape (no device needed)."""
    lib = load()
    ne = C.c_int(0)
    npar = C.c_long(0)
    fnet = _net(net)
    rc = lib.ferminet_net_layout(C.byref(fnet), None, 0, C.byref(ne), C.byref(npar))
    if rc != 0:
        raise FermiNetError(f"ferminet_net_layout: {STATUS.get(rc, rc)}")
    arr = (FnParamEntry * ne.value)()
    lib.ferminet_net_layout(C.byref(fnet), arr, ne.value, C.byref(ne), C.byref(npar))
    return [Entry(e.name.decode(), e.offset, e.count, e.fan_in, e.kind) for e in arr]


def _ptr(t) -> Optional[int]:
    return None if t is None else t.data_ptr()


class FermiNet:
    """One library context: network shape, geometries, precision, stream."""

    def __init__(self, net, geoms, counts: Optional[Sequence[int]] = None, precision: str = "fp32",
                 stream=None):
        import torch
        if not torch.cuda.is_available():
            raise FermiNetError("no CUDA device: the FermiNet hot path runs only on the GPU")
        self.torch = torch
        self.lib = load()
        self.net = net
        self.n = net.n_up + net.n_down
        self.G = len(geoms)
        counts = list(counts) if counts is not None else [0] * self.G
        self._R = [np.ascontiguousarray(np.asarray(g.R, np.float64).reshape(-1, 3)) for g in geoms]
        self._Z = [np.ascontiguousarray(np.asarray(g.Z, np.float64).reshape(-1)) for g in geoms]
        garr = (FnGeometry * self.G)()
        off = 0
        for i in range(self.G):
            garr[i].R = self._R[i].ctypes.data_as(C.POINTER(C.c_double))
            garr[i].Z = self._Z[i].ctypes.data_as(C.POINTER(C.c_double))
            garr[i].walker_offset = off
            garr[i].walker_count = int(counts[i])
            off += int(counts[i])
        self.total = off
        self.counts = [int(c) for c in counts]
        self.precision = precision
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        ctx = C.c_void_p()
        fnet = _net(net)
        rc = self.lib.ferminet_init(C.byref(fnet), garr, self.G, PREC[precision],
                                    C.c_void_p(self.stream.cuda_stream), C.byref(ctx))
        if rc != 0:
            raise FermiNetError(f"ferminet_init: {STATUS.get(rc, rc)}")
        self.ctx = ctx
        ne = C.c_int(0)
        npar = C.c_long(0)
        self.lib.ferminet_param_layout(self.ctx, None, 0, C.byref(ne), C.byref(npar))
        arr = (FnParamEntry * ne.value)()
        self.lib.ferminet_param_layout(self.ctx, arr, ne.value, C.byref(ne), C.byref(npar))
        self.layout = [Entry(e.name.decode(), e.offset, e.count, e.fan_in, e.kind) for e in arr]
        self.n_params = int(npar.value)

    # -- helpers ---------------------------------------------------------
    def _check(self, rc, what):
        if rc != 0:
            msg = self.lib.ferminet_last_error(self.ctx).decode()
            raise FermiNetError(f"{what}: {STATUS.get(rc, rc)} {msg}")

    def _f32(self, t, shape=None):
        torch = self.torch
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
            raise FermiNetError("expected a contiguous float32 CUDA tensor")
        if shape is not None and tuple(t.shape) != tuple(shape):
            raise FermiNetError(f"expected shape {shape}, got {tuple(t.shape)}")
        return t

    def _empty(self, *shape, dtype=None):
        return self.torch.empty(*shape, dtype=dtype or self.torch.float32, device="cuda")

    # -- API -------------------------------------------------------------
    def set_params(self, params):
        self._f32(params, (self.n_params,))
        self._check(self.lib.ferminet_set_params(self.ctx, _ptr(params)), "ferminet_set_params")
        self._params_ref = params

    def logpsi(self, x, with_sign=True):
        B = x.shape[0]
        self._f32(x, (B, self.n, 3))
        lp = self._empty(B)
        sg = self._empty(B) if with_sign else None
        self._check(self.lib.ferminet_logpsi(self.ctx, _ptr(x), B, _ptr(lp), _ptr(sg)), "ferminet_logpsi")
        return (lp, sg) if with_sign else lp

    def local_energy(self, x):
        B = x.shape[0]
        self._f32(x, (B, self.n, 3))
        out = {k: self._empty(B) for k in ("eloc", "logpsi", "sign", "kinetic")}
        self._check(self.lib.ferminet_local_energy(self.ctx, _ptr(x), B, _ptr(out["eloc"]), _ptr(out["logpsi"]),
                                                   _ptr(out["sign"]), _ptr(out["kinetic"])),
                    "ferminet_local_energy")
        return out

    def logpsi_vjp(self, x, seeds):
        B = x.shape[0]
        self._f32(x, (B, self.n, 3))
        self._f32(seeds, (B,))
        g = self._empty(self.n_params)
        self._check(self.lib.ferminet_logpsi_vjp(self.ctx, _ptr(x), B, _ptr(seeds), _ptr(g)), "ferminet_logpsi_vjp")
        return g

    def energy_grad(self, x, eloc):
        B = x.shape[0]
        self._f32(x, (B, self.n, 3))
        self._f32(eloc, (B,))
        em = self._empty(self.G, dtype=self.torch.float64)
        g = self._empty(self.n_params)
        self._check(self.lib.ferminet_energy_grad(self.ctx, _ptr(x), B, _ptr(eloc), _ptr(em), _ptr(g)),
                    "ferminet_energy_grad")
        return em, g

    def walker_counts(self, B):
        """Walkers of each geometry in a batch of B (float64 [G], on the GPU)."""
        c = [B] if self.G == 1 else self.counts
        return self.torch.tensor(c, dtype=self.torch.float64, device="cuda")

    def energy_sums(self, eloc):
        """FP64 sum of eloc over each geometry's walkers (float64 [G])."""
        B = eloc.shape[0]
        self._f32(eloc, (B,))
        s = self._empty(self.G, dtype=self.torch.float64)
        self._check(self.lib.ferminet_energy_sums(self.ctx, _ptr(eloc), B, _ptr(s)), "ferminet_energy_sums")
        return s

    def energy_grad_partial(self, x, eloc, esum, count):
        """This process's share of the VMC gradient given the energy sum and
        walker count of every geometry over the whole batch.  The library
        divides them (FP64, on the GPU).  Returns (emean [G], grad [P]), both
        float64."""
        B = x.shape[0]
        self._f32(x, (B, self.n, 3))
        self._f32(eloc, (B,))
        for t in (esum, count):
            if not (t.is_cuda and t.dtype == self.torch.float64 and t.is_contiguous() and t.numel() == self.G):
                raise FermiNetError(f"expected a contiguous float64 CUDA tensor of {self.G} elements")
        em = self._empty(self.G, dtype=self.torch.float64)
        g = self._empty(self.n_params, dtype=self.torch.float64)
        self._check(self.lib.ferminet_energy_grad_partial(self.ctx, _ptr(x), B, _ptr(eloc), _ptr(esum), _ptr(count),
                                                          _ptr(em), _ptr(g)), "ferminet_energy_grad_partial")
        return em, g

    def mcmc_step(self, x, logpsi, n_steps, width, seed, counter, accepted=None):
        """Advances x and logpsi in place; returns the accepted-move counts."""
        B = x.shape[0]
        self._f32(x, (B, self.n, 3))
        self._f32(logpsi, (B,))
        if accepted is None:
            accepted = self._empty(B, dtype=self.torch.int32)
        self._check(self.lib.ferminet_mcmc_step(self.ctx, _ptr(x), _ptr(logpsi), B, int(n_steps), float(width),
                                                int(seed), int(counter), _ptr(accepted)), "ferminet_mcmc_step")
        return accepted

    def step(self, x, logpsi, n_steps, width, seed, counter, use_graph=True, out=None):
        """One VMC step (Metropolis moves, local energy, VMC gradient); x and
        logpsi are advanced in place.  Returns dict(eloc, emean, grad, accepted)."""
        B = x.shape[0]
        self._f32(x, (B, self.n, 3))
        self._f32(logpsi, (B,))
        if out is None:
            out = {"eloc": self._empty(B), "emean": self._empty(self.G, dtype=self.torch.float64),
                   "grad": self._empty(self.n_params), "accepted": self._empty(B, dtype=self.torch.int32)}
        self._check(self.lib.ferminet_step(self.ctx, _ptr(x), _ptr(logpsi), B, int(n_steps), float(width), int(seed),
                                           int(counter), _ptr(out["eloc"]), _ptr(out["emean"]), _ptr(out["grad"]),
                                           _ptr(out["accepted"]), 1 if use_graph else 0), "ferminet_step")
        return out

    def sync(self):
        rc = self.lib.ferminet_sync(self.ctx)
        return STATUS.get(rc, rc)

    def profile(self, enable=True):
        self._check(self.lib.ferminet_profile(self.ctx, 1 if enable else 0), "ferminet_profile")

    def profile_read(self, name):
        ms = C.c_double(0)
        n = C.c_long(0)
        fl = C.c_double(0)
        self._check(self.lib.ferminet_profile_read(self.ctx, KERNEL_CLASSES[name], C.byref(ms), C.byref(n),
                                                   C.byref(fl)), "ferminet_profile_read")
        return {"ms": ms.value, "launches": n.value, "alg_flops": fl.value}

    @staticmethod
    def _tdict(t):
        return {"layer_groups": t.layer_groups, "feature_tile": t.feature_tile, "tangent_chunk": t.tangent_chunk,
                "residual_smem": t.residual_smem, "pair_unfused": t.pair_unfused, "adjoint_simt": t.adjoint_simt,
                "orbital_joint": t.orbital_joint}

    def get_tuning(self):
        t = FnTuning()
        self._check(self.lib.ferminet_get_tuning(self.ctx, C.byref(t)), "ferminet_get_tuning")
        return self._tdict(t)

    def set_tuning(self, layer_groups=0, feature_tile=0, tangent_chunk=0, residual_smem=0, pair_unfused=0,
                   adjoint_simt=0, orbital_joint=0):
        t = FnTuning(int(layer_groups), int(feature_tile), int(tangent_chunk), int(residual_smem), int(pair_unfused),
                     int(adjoint_simt), int(orbital_joint))
        self._check(self.lib.ferminet_set_tuning(self.ctx, C.byref(t)), "ferminet_set_tuning")

    def autotune(self, x, repeats=2):
        """Times the candidate tile shapes on these walkers and installs the fastest."""
        B = x.shape[0]
        self._f32(x, (B, self.n, 3))
        t = FnTuning()
        self._check(self.lib.ferminet_autotune(self.ctx, _ptr(x), B, int(repeats), C.byref(t)), "ferminet_autotune")
        return self._tdict(t)

    def autotune_cached(self, x, cache_path=None, repeats=2):
        """Tuning from a JSON cache keyed by network shape, batch, precision and
        GPU; runs the autotuner and records the result on a miss."""
        import json
        torch = self.torch
        path = cache_path or os.path.join(_HERE, "_build", "autotune.json")
        key = "|".join(str(v) for v in (self.net.n_layers, self.net.d1, self.net.d2, self.net.n_det, self.net.n_up,
                                         self.net.n_down, self.net.n_nuc, self.G, x.shape[0], self.precision,
                                         torch.cuda.get_device_name()))
        cache = {}
        if os.path.exists(path):
            try:
                cache = json.load(open(path))
            except Exception:
                cache = {}
        if key in cache:
            self.set_tuning(**cache[key])
            return cache[key], True
        best = self.autotune(x, repeats)
        cache[key] = best
        try:
            os.makedirs(os.path.dirname(path), exist_ok=True)
            with open(path + ".tmp", "w") as fh:
                json.dump(cache, fh, indent=1)
            os.replace(path + ".tmp", path)
        except OSError:
            pass
        return best, False

    def set_train_opts(self, clip_scale=0.0, width=None, accept_lo=0.5, accept_hi=0.55, width_factor=1.1):
        """Training-loop options: local-energy clipping in the gradient
        (clip_scale > 0) and proposal-width adaptation (width: a float32 CUDA
        tensor of one element that the moves read and the library updates;
        None = off)."""
        if width is not None:
            self._f32(width, (1,))
        self._width_ref = width
        o = FnTrainOpts(float(clip_scale), None if width is None else width.data_ptr(), float(accept_lo),
                        float(accept_hi), float(width_factor))
        self._check(self.lib.ferminet_set_train_opts(self.ctx, C.byref(o)), "ferminet_set_train_opts")

    def kfac_size(self):
        n = C.c_long(0)
        fnet = _net(self.net)
        self._check(self.lib.ferminet_kfac_size(C.byref(fnet), C.byref(n)), "ferminet_kfac_size")
        return int(n.value)

    def kfac_factors(self, x):
        """KFAC factors of the batch (float64 CUDA tensor; layout in ferminet.h)."""
        B = x.shape[0]
        self._f32(x, (B, self.n, 3))
        F = self._empty(self.kfac_size(), dtype=self.torch.float64)
        self._check(self.lib.ferminet_kfac_factors(self.ctx, _ptr(x), B, _ptr(F)), "ferminet_kfac_factors")
        return F

    def kfac_precondition(self, factors, grad, lam):
        """KFAC update for a gradient (float32 [n_params])."""
        torch = self.torch
        if not (factors.is_cuda and factors.dtype == torch.float64 and factors.is_contiguous()):
            raise FermiNetError("expected a contiguous float64 CUDA factor buffer")
        self._f32(grad, (self.n_params,))
        out = self._empty(self.n_params)
        self._check(self.lib.ferminet_kfac_precondition(self.ctx, _ptr(factors), _ptr(grad), float(lam), _ptr(out)),
                    "ferminet_kfac_precondition")
        return out

    def flagged_matrices(self):
        return int(self.lib.ferminet_flagged_matrices(self.ctx))

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.ferminet_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def launch_count() -> int:
    """Kernels launched by libferminet in this process."""
    return int(load().ferminet_launch_count())


def logpsi_autograd(fn: FermiNet, params, x):
    """log|psi|(x) as a differentiable function of the flat parameter vector:
    forward runs ferminet_logpsi, backward the hand-written adjoint
    (ferminet_logpsi_vjp) seeded with the incoming per-walker cotangent."""
    import torch

    class _LogPsi(torch.autograd.Function):
        @staticmethod
        def forward(ctx, p, xx):
            fn.set_params(p)
            ctx.save_for_backward(xx)
            return fn.logpsi(xx, with_sign=False)

        @staticmethod
        def backward(ctx, gout):
            (xx,) = ctx.saved_tensors
            return fn.logpsi_vjp(xx, gout.contiguous().float()), None

    return _LogPsi.apply(params, x)

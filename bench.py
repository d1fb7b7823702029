#!/usr/bin/env python
"""Benchmark of the FermiNet VMC step on GB300.

One step = the whole hot path over one batch of walkers: the workload's
Metropolis moves (value passes), log|psi| and the local energy (tangent pass),
and the VMC energy gradient (adjoint) -- all through the C ABI of libferminet.

Prints ONE JSON line (rank 0).  --impl reference times the FP64 CPU oracle on
bounded samples of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "VMC walker-steps/sec (psi, E_L, grad) vs plain FP32 path at stated error"
UNIT = "walker-steps/s"
DEFAULT_WORKLOAD = "c4h4x8"
L2_FLUSH_BYTES = 256 << 20  # twice the 129 MB L2


def describe(wl) -> str:
    t = wl.net
    geo = f"{len(wl.geoms)} geometries" if len(wl.geoms) > 1 else f"{t.n_nuc} nuclei"
    return (f"{wl.name}: {geo}, {t.n_elec} electrons ({t.n_up}/{t.n_down}), L={t.n_layers}, d1={t.d1}, "
            f"d2={t.d2}, K={t.n_det} determinants, {wl.batch} walkers; step = {wl.mcmc_steps} Metropolis moves "
            f"(width {wl.mcmc_width}) + log|psi| + E_L + VMC energy gradient")


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            d = json.load(open(p))
            return d, "measured"
        except Exception:
            pass
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def _num(d, *keys):
    for k in keys:
        v = d.get(k)
        if isinstance(v, (int, float)):
            return float(v)
        if isinstance(v, dict):
            for kk in ("value", "gbs", "tflops"):
                if isinstance(v.get(kk), (int, float)):
                    return float(v[kk])
    return None


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sm.append(float(f[1]))
                    smax.append(float(f[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, f[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        except Exception:
            pass
        finally:
            try:
                os.unlink(self.path)
            except Exception:
                pass
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# CPU oracle (baseline / reference arm)
# ---------------------------------------------------------------------------

def oracle_step_sample(wl, P, x, counter):
    """One step of the oracle on walkers x (a bounded sample, all on the first
    geometry): Metropolis moves, local energy and VMC gradient.
    Returns (seconds, E_L, positions after the moves)."""
    import oracle
    from paper_2011_07125_gb300 import synth
    geoms = wl.geoms[:1]
    t0 = time.perf_counter()
    lp, _ = oracle.logpsi(wl.net, P, geoms, x)
    x2, lp2, _, _ = oracle.mcmc(wl.net, P, geoms, x, lp, wl.mcmc_steps, wl.mcmc_width, synth.SEED_MCMC, counter)
    out = oracle.local_energy(wl.net, P, geoms, x2)
    oracle.energy_grad(wl.net, P, geoms, x2, out["eloc"])
    return time.perf_counter() - t0, out["eloc"], x2


def cpu_sample_size(wl, P, x, target_s: float) -> int:
    """Walkers per oracle sample so that one sample takes about target_s on
    all host cores (calibrated on one walker)."""
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    t1, _, _ = oracle_step_sample(wl, P, x[:1], 0)
    n = int(cores * target_s / max(t1, 1e-3))
    n = max(1, min(n, wl.batch, 64 * cores))
    return n


def run_reference(args, wl):
    """--impl reference: the FP64 oracle as it stands, on the host cores."""
    import numpy as np
    import oracle
    from paper_2011_07125_gb300 import synth
    if int(os.environ.get("WORLD_SIZE", "1")) > 1:
        # under a rank launcher (which sets one thread per rank) rank 0 runs alone
        os.environ["OMP_NUM_THREADS"] = str(os.cpu_count() or 1)
    os.environ.setdefault("OMP_NUM_THREADS", str(os.cpu_count() or 1))
    cores = int(os.environ["OMP_NUM_THREADS"])
    lay = oracle.layout(wl.net)
    P = synth.init_params(lay)
    xall = synth.init_walkers(wl)
    per_step_s = max(2.0, 150.0 / max(args.steps + args.warmup, 1))
    S = cpu_sample_size(wl, P, xall, per_step_s)
    times = []
    for k in range(args.warmup + args.steps):
        xs = xall[(k * S) % max(wl.batch - S, 1):][:S] if wl.batch > S else xall
        dt, _, _ = oracle_step_sample(wl, P, xs, k * wl.mcmc_steps)
        if k >= args.warmup:
            times.append(dt)
    tot = sum(times)
    value = S * len(times) / tot
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(times) * wl.batch / S,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded walkers, N(0,1/fan_in) weights)",
            "config": {"workload": describe(wl), "walkers": wl.batch, "precision": "fp64 oracle"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{S} walkers per step of the {wl.batch}-walker batch; ms_per_step scaled "
                                       f"to the full batch"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def code_only(src: bytes) -> bytes:
    """C++ source without its comments, whitespace runs collapsed: two sources
    that differ only in comments or layout compile to the same kernels (none of
    the hashed sources holds a comment marker inside a string literal)."""
    import re
    src = re.sub(rb"/\*.*?\*/", b" ", src, flags=re.S)
    src = re.sub(rb"//[^\n]*", b" ", src)
    return b" ".join(src.split())


def kernel_source_hash() -> str:
    """Hash of what the timed GEMM class's traffic depends on: the code (not the
    comments) of the tensor-core GEMM sources and of the network pass
    (forward() in ferminet.cu) that sizes and tiles its launches."""
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2011_07125_gb300", "csrc")
    for f in ("k_tc_gemm.cu", "tc_gemm.cuh"):
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(code_only(fh.read()))
    with open(os.path.join(csrc, "ferminet.cu"), "rb") as fh:
        src = fh.read()
    start = src.find(b"\nvoid forward(fn_ctx* c")
    end = src.find(b"\n}\n", start)
    h.update(code_only(src[start:end] if start >= 0 and end > start else src))
    return h.hexdigest()[:16]


TRAFFIC_TUNING = ("layer_groups", "residual_smem")  # tuning fields a traffic record is keyed by


def layer_groups_used(groups: int, C: int) -> int:
    """(walker, electron) groups per tile of the layer GEMM for the tuning
    field layer_groups and C tangent columns per group: the field when it
    gives a valid tile, else the library's default (the most groups whose tile
    is at most 256 rows and a multiple of 16)."""
    if groups > 0 and groups * C <= 256 and (groups * C) % 16 == 0:
        return groups
    for g in range(256 // C, 0, -1):
        if (g * C) % 16 == 0:
            return g
    return 0


def recorded_traffic(workload: str, prec: str, tuning=None, net=None):
    """DRAM bytes per walker of the timed GEMM class from the committed ncu
    summary (profiles/roofline_traffic.md), or None if the kernel sources have
    changed since the capture or the record's tuning (layer_groups,
    residual_smem) differs from the timed one.  With the network shape given,
    layer_groups compares as the tile it selects (0 and the default's group
    count are the same tile)."""
    path = os.path.join(ROOT, "profiles", "roofline_traffic.md")
    if not os.path.exists(path):
        return None
    src = kernel_source_hash()
    C = None if net is None else ((3 * net.n_elec + 2 + 7) // 8) * 8

    def field(t, k):
        v = int(t.get(k, 0))
        return layer_groups_used(v, C) if (k == "layer_groups" and C) else v

    for line in open(path):
        if not line.startswith("traffic:"):
            continue
        kv = dict(t.split("=", 1) for t in line.split()[1:] if "=" in t)
        if kv.get("workload") != workload or kv.get("precision") != prec or kv.get("source") != src:
            continue
        if "tuning" in kv:
            rec = dict(t.split(":", 1) for t in kv["tuning"].split(",") if ":" in t)
            cur = tuning or {}
            if any(field(rec, k) != field(cur, k) for k in TRAFFIC_TUNING):
                continue
        return float(kv["bytes_per_walker"])
    return None


def gemm_class_alg_bytes(net) -> float:
    """Algorithmic HBM bytes per walker of the layer + orbital GEMMs of one
    local-energy pass: every operand and result crossing HBM once, with the
    real tangent columns (C = 3n + 2) and features only.  Activations, spin
    means and U count 4 bytes an element (BF16 hi + lo, or FP32); orbitals
    count the same-spin blocks only (FP32)."""
    n, N, d1, d2, K, L = net.n_elec, net.n_nuc, net.d1, net.d2, net.n_det, net.n_layers
    C = 3 * n + 2
    R = n * C  # rows of one walker
    tot = 0.0
    for l in range(L):
        a1 = 4 * N if l == 0 else d1
        a2 = 4 if l == 0 else d2
        tot += 4.0 * (C * 2 * a1 + C * d1)                    # U GEMM: spin means in, U out
        tot += 4.0 * (R * a1 + R * 2 * a2 + C * d1 + R * d1)  # layer: h, pair means, U in; h' out
    tot += 4.0 * (R * d1 + (net.n_up ** 2 + net.n_down ** 2) * K * C)  # orbitals
    return tot


def tangent_roofline(fn, prec, clocks, pk, pk_kind, workload=None, walkers_per_launch=None, net=None, tuning=None):
    r = fn.profile_read("tangent_gemm")
    if r["launches"] == 0 or r["ms"] <= 0:
        return None
    achieved = r["alg_flops"] / (r["ms"] * 1e-3) / 1e12
    if prec == "fp32":
        import torch
        mhz = clocks.get("sm_max_mhz") or 2070.0
        sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
        peak = sms * 128 * 2 * mhz * 1e6 / 1e12
        bound, note = "alu", (f"FP32 FMA peak: {sms} SMs (from the device) x 128 FP32 lanes x 2 flops x "
                              f"{mhz:.0f} MHz (maximum SM clock seen)")
    else:
        peak = _num(pk, "bf16_tflops_sustained", "bf16_tflops") or 1700.0
        bound, note = "tensor", f"bf16 sustained, {pk_kind}"
    bpw = recorded_traffic(workload, prec, tuning, net) if workload else None
    traffic = bpw * walkers_per_launch if (bpw is not None and walkers_per_launch) else None
    hbm = None
    if net is not None and walkers_per_launch:
        hpk = _num(pk, "hbm_gbs") or 6800.0
        gbs = gemm_class_alg_bytes(net) * walkers_per_launch / (r["ms"] / r["launches"] * 1e-3) / 1e9
        hbm = {"achieved": gbs, "peak": hpk, "unit": "GB/s", "frac": gbs / hpk,
               "bytes_per_walker": gemm_class_alg_bytes(net),
               "note": "algorithmic bytes (real columns and features, once) over the same launches; "
                       f"copy peak, {pk_kind}"}
    return {"bound": bound, "kernel": "layer + orbital GEMMs of the local-energy pass", "achieved": achieved,
            "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak, "traffic": traffic,
            "traffic_unit": "bytes per launch (DRAM read + write, ncu)",
            "launches": r["launches"], "avg_launch_ms": r["ms"] / r["launches"], "peak_note": note,
            "hbm_view": hbm}


def geometry_sample(wl, per_geom: int):
    """Indices of `per_geom` walkers of every geometry, spread over its range."""
    import numpy as np
    idx, off = [], 0
    for c in wl.counts:
        k = min(per_geom, c)
        idx.extend(off + np.linspace(0, c - 1, k).astype(int))
        off += c
    return np.array(idx, np.int64)


def error_report(wl, P, xs, geo, eloc, logpsi, prec, grad_fn=None):
    """Errors of the GPU results on sampled walkers against the FP64 oracle:
    per-geometry batch-mean E_L error, per-walker E_L and log|psi| errors with
    the fraction inside the FP32 bars (1e-4 Ha, 1e-5 relative), and, when
    grad_fn is given, the VMC gradient's relative L2 error (grad_fn(ref_eloc)
    returns the GPU gradient on the same walkers)."""
    import numpy as np
    import oracle
    ref = oracle.local_energy(wl.net, P, wl.geoms, xs, geo=geo)
    de = eloc.astype(np.float64) - ref["eloc"]
    dl = np.abs(logpsi.astype(np.float64) - ref["logpsi"]) / np.maximum(np.abs(ref["logpsi"]), 1.0)
    gs = [g for g in range(len(wl.geoms)) if np.any(geo == g)]
    per_geo = [float(de[geo == g].mean()) for g in gs]
    # standard error of each geometry's sample mean (pooled spread): the
    # sample estimates the mean error over the geometry's whole batch
    rms = float(np.sqrt(np.mean(de ** 2)))
    stderr = [rms / np.sqrt(int((geo == g).sum())) for g in gs]
    rep = {"walkers": int(len(xs)), "eloc_mean_err_per_geometry": per_geo,
           "eloc_mean_err_stderr_per_geometry": stderr,
           "eloc_mean_err_max_abs": float(np.max(np.abs(per_geo))),
           "eloc_mean_err_all_sampled": float(de.mean()),
           "eloc_mean_err_all_sampled_stderr": rms / np.sqrt(len(de)),
           "eloc_max_abs": float(np.abs(de).max()), "eloc_median_abs": float(np.median(np.abs(de))),
           "frac_eloc_within_1e-4": float(np.mean(np.abs(de) <= 1e-4)),
           "logpsi_max_rel": float(dl.max()), "frac_logpsi_within_1e-5": float(np.mean(dl <= 1e-5)),
           "bar": ("batch-mean E_L within 1e-3 Ha" if prec == "mixed" else
                   "1e-5 relative log|psi|, 1e-4 Ha per walker, 1e-5 Ha batch mean")}
    if grad_fn is not None:
        _, g_o = oracle.energy_grad(wl.net, P, wl.geoms, xs, ref["eloc"], geo=geo)
        g = grad_fn()
        rep["grad_rel_l2"] = float(np.linalg.norm(g - g_o) / np.linalg.norm(g_o))
    return rep


def sample_context_grad(wl, prec, params, xs_np, counts):
    """VMC gradient of the GPU path on the sampled walkers alone (a context
    whose geometry table holds the sample's counts)."""
    import numpy as np
    import torch
    from paper_2011_07125_gb300.binding import FermiNet
    f = FermiNet(wl.net, wl.geoms, counts=counts, precision=prec)
    f.set_params(params)
    xx = torch.from_numpy(np.ascontiguousarray(xs_np)).cuda()
    e = f.local_energy(xx)["eloc"]
    _, g = f.energy_grad(xx, e)
    out = g.cpu().numpy().astype(np.float64)
    f.close()
    return out


def timed_steps(fn, wl, x, lp, steps, warmup, flush, grad_of, counter0=0):
    """Runs `warmup` then `steps` VMC steps (moves, E_L, gradient) on the
    context stream; returns (per-step ms list, last local-energy output)."""
    import torch
    from paper_2011_07125_gb300 import synth
    counter = [counter0]
    s = torch.cuda.current_stream()

    def step():
        fn.mcmc_step(x, lp, wl.mcmc_steps, wl.mcmc_width, synth.SEED_MCMC, counter[0])
        counter[0] += wl.mcmc_steps
        out = fn.local_energy(x)
        grad_of(fn, x, out["eloc"])
        return out

    out = None
    for _ in range(warmup):
        out = step()
    torch.cuda.synchronize()
    ms = []
    for k in range(steps):
        flush.fill_(float(k))  # L2 flush outside the timed events
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(s)
        out = step()
        b.record(s)
        ms.append((a, b))
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in ms], out


def side_workload(name, flush, args):
    """A shorter measurement of another workload in the same run: its own
    precision (and the other one for comparison), and its error against the
    oracle on sampled walkers."""
    import numpy as np
    import torch
    from paper_2011_07125_gb300 import synth
    from paper_2011_07125_gb300.binding import FermiNet
    wl = synth.workload(name)
    res = {"workload": describe(wl), "precision": wl.precision}
    x0 = synth.init_walkers(wl)
    P = None
    for prec in (wl.precision, "fp32" if wl.precision == "mixed" else "mixed"):
        fn = FermiNet(wl.net, wl.geoms, counts=wl.counts, precision=prec)
        if P is None:
            P = synth.init_params(fn.layout)
            params = torch.from_numpy(P).cuda()
        fn.set_params(params)
        x = torch.from_numpy(x0).cuda()
        lp = fn.logpsi(x, with_sign=False)
        if prec == "mixed" and not args.no_autotune:
            fn.autotune_cached(x, repeats=1)
        main = prec == wl.precision
        ms, out = timed_steps(fn, wl, x, lp, 3 if main else 2, 2 if main else 1, flush,
                              lambda f, xx, e: f.energy_grad(xx, e))
        st = fn.sync()
        v = wl.batch * len(ms) / (sum(ms) * 1e-3)
        res[prec] = {"value": v, "unit": UNIT, "ms_per_step": sum(ms) / len(ms), "status": st}
        if prec == wl.precision and not args.no_cpu_baseline:
            idx = geometry_sample(wl, 32 if prec == "fp32" else 16)
            xs = np.ascontiguousarray(x.cpu().numpy()[idx])
            geo = synth.geometry_of_walkers(wl.counts)[idx]
            res["error_vs_oracle"] = error_report(
                wl, P, xs, geo, out["eloc"].cpu().numpy()[idx], out["logpsi"].cpu().numpy()[idx], prec,
                grad_fn=lambda: sample_context_grad(wl, prec, params, xs, [len(xs)]))
        fn.close()
    if "fp32" in res and "mixed" in res:
        res["mixed_over_fp32"] = res["mixed"]["value"] / res["fp32"]["value"]
    return res


def envelope_overhead(flush, args):
    """The full-covariance envelope (Eq. 4) against the isotropic one (Sec. 3)
    on the C4H6 workload (the bicyclobutane stand-in of the paper's 40%
    comparison): whole-step time of each, mixed precision."""
    import dataclasses
    import torch
    from paper_2011_07125_gb300 import synth
    from paper_2011_07125_gb300.binding import FermiNet
    wl0 = synth.workload("c4h6")
    x0 = synth.init_walkers(wl0)
    res = {"workload": describe(wl0)}
    for env in (0, 1):
        wl = dataclasses.replace(wl0, net=dataclasses.replace(wl0.net, envelope=env))
        fn = FermiNet(wl.net, wl.geoms, counts=wl.counts, precision="mixed")
        fn.set_params(torch.from_numpy(synth.init_params(fn.layout)).cuda())
        x = torch.from_numpy(x0).cuda()
        lp = fn.logpsi(x, with_sign=False)
        if not args.no_autotune:
            fn.autotune_cached(x, repeats=1)
        fn.profile(True)
        ms, _ = timed_steps(fn, wl, x, lp, 3, 2, flush, lambda f, xx, e: f.energy_grad(xx, e))
        det = fn.profile_read("det_tangent")["ms"]
        fn.profile(False)
        res["full_covariance" if env else "isotropic"] = {
            "ms_per_step": sum(ms) / len(ms), "value": wl.batch * len(ms) / (sum(ms) * 1e-3), "unit": UNIT,
            "det_tangent_ms_per_step": det / len(ms), "status": fn.sync()}
        fn.close()
    res["full_over_isotropic_step_time"] = res["full_covariance"]["ms_per_step"] / res["isotropic"]["ms_per_step"]
    return res


def run_eloc_pass(args, wl):
    """One local-energy pass (with --pass-kind value one log|psi| pass, with
    --pass-kind grad a local-energy pass and the VMC gradient) of
    the workload with every geometry's walker count divided by --eloc-pass (at
    least one walker each), after --warmup passes: the small case on which ncu
    captures the DRAM traffic of the tensor-core GEMM class (only k_tc_gemm
    launches of local-energy passes run after the context is set up) or a
    pass's launch list.  Prints the walkers and tuning as one JSON line."""
    import dataclasses
    import torch
    from paper_2011_07125_gb300 import synth
    from paper_2011_07125_gb300.binding import FermiNet
    div = args.eloc_pass
    wl = dataclasses.replace(wl, counts=[max(1, c // div) for c in wl.counts])
    prec = args.precision or wl.precision
    fn = FermiNet(wl.net, wl.geoms, counts=wl.counts, precision=prec)
    fn.set_params(torch.from_numpy(synth.init_params(fn.layout)).cuda())
    x = torch.from_numpy(synth.init_walkers(wl)).cuda()
    tuning = dict(t.split("=", 1) for t in args.pass_tuning.split(",") if "=" in t)
    tuning = {k: int(v) for k, v in tuning.items()}
    if prec == "mixed":
        fn.set_tuning(**tuning)
    def run():
        if args.pass_kind == "value":
            fn.logpsi(x)
        elif args.pass_kind == "grad":
            fn.energy_grad(x, fn.local_energy(x)["eloc"])
        else:
            fn.local_energy(x)
    for _ in range(args.warmup):
        run()
    torch.cuda.synchronize()
    fn.profile(True)
    run()
    torch.cuda.synchronize()
    r = fn.profile_read("tangent_gemm")
    st = fn.sync()
    print(json.dumps({"pass": args.pass_kind, "workload": wl.name, "walkers": wl.batch, "counts": wl.counts, "precision": prec,
                      "tuning": tuning, "gemm_class_launches": r["launches"], "gemm_class_ms": r["ms"],
                      "status": st}), flush=True)
    fn.close()
    if st != "FN_OK":
        sys.exit(1)


def run_gpu(args, wl):
    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_2011_07125_gb300 import synth
    from paper_2011_07125_gb300 import replicas
    from paper_2011_07125_gb300.binding import FermiNet, launch_count

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    prec = args.precision or wl.precision
    fn = FermiNet(wl.net, wl.geoms, counts=wl.counts, precision=prec)
    P = synth.init_params(fn.layout)
    x0 = synth.init_walkers(wl, synth.SEED_WALKERS + rank)
    params = torch.from_numpy(P).to(dev)
    fn.set_params(params)
    x = torch.from_numpy(x0).to(dev)
    lp = fn.logpsi(x, with_sign=False)
    tuning = None
    if prec == "mixed" and not args.no_autotune:
        tuning, cached = fn.autotune_cached(x, repeats=3)
        tuning = dict(tuning, cached=cached)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    counter = [0]

    def grad_of(xx, eloc):
        # several processes: the batch-wide mean energy and gradient (two all-reduces)
        return replicas.energy_grad(fn, xx, eloc) if world > 1 else fn.energy_grad(xx, eloc)

    def step():
        fn.mcmc_step(x, lp, wl.mcmc_steps, wl.mcmc_width, synth.SEED_MCMC, counter[0])
        counter[0] += wl.mcmc_steps
        out = fn.local_energy(x)
        em, g = grad_of(x, out["eloc"])
        return out, em, g

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    s = torch.cuda.current_stream()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    fn.profile(True)
    l0 = launch_count()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    # the timed steps form the profiler range: `ncu --profile-from-start off`
    # lists exactly these launches (a no-op without a profiler)
    torch.cuda.profiler.start()
    with ClockSampler(local) as cs:
        for k in range(args.steps):
            flush.fill_(float(k))  # L2 flush outside the timed events
            evs[k][0].record(s)
            out, em, g = step()
            evs[k][1].record(s)
        torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    if world > 1:
        dist.barrier()
    launches = launch_count() - l0
    ms = sum(a.elapsed_time(b) for a, b in evs)
    if world > 1:
        t = torch.tensor([ms], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    clocks = cs.summary()
    st = fn.sync()
    pk, pk_kind = peaks()
    r_tg = fn.profile_read("tangent_gemm")
    passes = args.steps  # one local-energy pass per step
    roof = tangent_roofline(fn, prec, clocks, pk, pk_kind, wl.name,
                            wl.batch * passes / max(r_tg["launches"], 1), net=wl.net, tuning=tuning)
    classes = {k: fn.profile_read(k) for k in ("tangent_gemm", "det_tangent", "two_layer", "means", "tanh",
                                                 "value_pass", "adjoint")}
    fn.profile(False)
    ms_per_step = ms / args.steps
    value = world * wl.batch * args.steps / (ms * 1e-3)
    # positions and local energies of the last timed step, for the error report
    x_last = x.clone()
    eloc_last = out["eloc"].cpu().numpy()
    logpsi_last = out["logpsi"].cpu().numpy()

    # plain FP32 path on the same workload (the metric's comparison), when the timed path is mixed
    fp32 = None
    if prec != "fp32" and not args.no_fp32_compare:
        f32 = FermiNet(wl.net, wl.geoms, counts=wl.counts, precision="fp32")
        f32.set_params(params)
        xs = torch.from_numpy(x0).to(dev)
        lps = f32.logpsi(xs, with_sign=False)
        n32 = max(2, min(args.steps // 2, 4))
        t32, _ = timed_steps(f32, wl, xs, lps, n32, max(1, min(args.warmup // 2, 2)), flush,
                             lambda f, xx, e: f.energy_grad(xx, e))
        fp32 = {"value": wl.batch * n32 / (sum(t32) * 1e-3), "unit": UNIT, "ms_per_step": sum(t32) / n32,
                "status": f32.sync()}
        f32.close()

    # end to end through the public API (ferminet_step, replayed from its CUDA
    # graph): walker state in from pinned host memory and walker state, local
    # energies, energy means and gradient back to pinned host memory, every step
    xh = torch.from_numpy(x0).pin_memory()
    lph = fn.logpsi(torch.from_numpy(x0).to(dev), with_sign=False).cpu().pin_memory()
    eh = torch.empty(wl.batch, dtype=torch.float32).pin_memory()
    gh = torch.empty(fn.n_params, dtype=torch.float32).pin_memory()
    mh = torch.empty(len(wl.geoms), dtype=torch.float64).pin_memory()
    xd = torch.empty_like(x)
    lpd = torch.empty_like(lp)
    outb = {"eloc": torch.empty(wl.batch, device=dev), "emean": torch.empty(len(wl.geoms), dtype=torch.float64,
                                                                            device=dev),
            "grad": torch.empty(fn.n_params, device=dev), "accepted": torch.empty(wl.batch, dtype=torch.int32,
                                                                                  device=dev)}
    n_e2e = max(2, min(args.steps, 5))

    def e2e_step(k):
        xd.copy_(xh, non_blocking=True)
        lpd.copy_(lph, non_blocking=True)
        if world == 1:
            fn.step(xd, lpd, wl.mcmc_steps, wl.mcmc_width, synth.SEED_MCMC, 10 ** 6 + k * wl.mcmc_steps,
                    use_graph=True, out=outb)
        else:
            fn.mcmc_step(xd, lpd, wl.mcmc_steps, wl.mcmc_width, synth.SEED_MCMC, 10 ** 6 + k * wl.mcmc_steps)
            outb["eloc"] = fn.local_energy(xd)["eloc"]
            em, g = replicas.energy_grad(fn, xd, outb["eloc"])
            outb["emean"], outb["grad"] = em, g.float()
        xh.copy_(xd, non_blocking=True)
        lph.copy_(lpd, non_blocking=True)
        eh.copy_(outb["eloc"], non_blocking=True)
        gh.copy_(outb["grad"], non_blocking=True)
        mh.copy_(outb["emean"], non_blocking=True)

    e2e_step(-1)  # capture
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(s)
    for k in range(n_e2e):
        e2e_step(k)
    t1.record(s)
    torch.cuda.synchronize()
    e2e_ms = t0.elapsed_time(t1) / n_e2e
    if world > 1:
        t = torch.tensor([e2e_ms], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_ms = float(t.item())
    e2e = {"value": world * wl.batch / (e2e_ms * 1e-3), "unit": UNIT, "ms_per_step": e2e_ms,
           "h2d_bytes_per_step": int(xh.numel() * 4 + lph.numel() * 4),
           "d2h_bytes_per_step": int(xh.numel() * 4 + lph.numel() * 4 + eh.numel() * 4 + gh.numel() * 4 +
                                     mh.numel() * 8),
           "api": "ferminet_step (CUDA graph replay)" if world == 1 else
                  "ferminet_mcmc_step + ferminet_local_energy + two-phase gradient all-reduce"}
    e2e_status = fn.sync()
    fn.close()

    cpu = None
    err = None
    side = {}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        os.environ.setdefault("OMP_NUM_THREADS", str(os.cpu_count() or 1))
        xs_np = x_last.cpu().numpy().astype(np.float32)
        S = cpu_sample_size(wl, P, xs_np, 15.0)
        dt, _, _ = oracle_step_sample(wl, P, xs_np[:S], 0)
        cpu = {"value": S / dt, "unit": UNIT, "cores": int(os.environ["OMP_NUM_THREADS"]), "kind": "oracle",
               "sample": f"{S} walkers of the {wl.batch}-walker batch ({wl.mcmc_steps} moves + E_L + gradient), "
                         f"{dt:.1f} s"}
        # error of the timed path on walkers sampled from every geometry (the
        # positions and local energies of the last timed step)
        idx = geometry_sample(wl, args.err_per_geom)
        geo = synth.geometry_of_walkers(wl.counts)[idx]
        xs = np.ascontiguousarray(xs_np[idx])
        cnt = [int((geo == g).sum()) for g in range(len(wl.geoms))]
        err = error_report(wl, P, xs, geo, eloc_last[idx], logpsi_last[idx], prec,
                           grad_fn=lambda: sample_context_grad(wl, prec, params, xs, cnt))
    if rank == 0 and world == 1 and args.side:
        for name in args.side.split(","):
            if name == "envelope":
                side[name] = envelope_overhead(flush, args)
            elif name and name != wl.name:
                side[name] = side_workload(name, flush, args)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32" if prec == "fp32" else "bf16/f32",
                "data": "synthetic (seeded walkers, N(0,1/fan_in) weights; the paper ships no data)",
                "config": {"workload": describe(wl), "walkers": wl.batch, "walkers_per_geometry": wl.counts,
                           "precision": prec,
                           "l2": "256 MiB buffer written between timed steps, outside the timed events",
                           "parallelism": f"data parallel over walkers x{world} (all-reduce of energy sums and "
                                          f"FP64 gradient shares)" if world > 1 else "single GPU",
                           "tuning": tuning},
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches),
                "clocks": clocks, "status": st, "e2e_status": e2e_status, "fp32_path": fp32,
                "mixed_over_fp32": (value / fp32["value"]) if fp32 else None,
                "error_vs_oracle": err,
                "kernel_classes_ms_per_step": {k: v["ms"] / args.steps for k, v in classes.items()},
                "other_workloads": side or None}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def check_launch(args):
    """Host-only check of the rank launch (gloo): every rank joins, rank 0
    prints the world size and the ranks that answered."""
    import torch
    import torch.distributed as dist
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1:
        dist.init_process_group("gloo")
    t = torch.zeros(max(world, 1), dtype=torch.int64)
    t[rank] = rank + 1
    if world > 1:
        dist.all_reduce(t)
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps({"check_launch": True, "n_gpus": world, "ranks": [int(v) - 1 for v in t.tolist()]}),
              flush=True)


def _free_port() -> int:
    import socket
    sk = socket.socket()
    sk.bind(("127.0.0.1", 0))
    port = sk.getsockname()[1]
    sk.close()
    return port


def launch_ranks(args) -> None:
    """--gpus N > 1 without a launcher: start N ranks on this node through
    torch.distributed.run (one process per GPU) and exit with its status."""
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={args.gpus}",
           "--master-addr", "127.0.0.1", f"--master-port={_free_port()}", os.path.abspath(__file__),
           *sys.argv[1:]]
    sys.stdout.flush()
    os.execv(sys.executable, cmd)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--precision", default=None, choices=[None, "fp32", "mixed"])
    ap.add_argument("--side", default=None,
                    help="comma-separated workloads measured briefly after the main one, 'envelope' for the "
                         "full-covariance against the isotropic envelope, name@B for another batch size "
                         "(default: ne,ar,ar@16384,kr,envelope with the default workload, none otherwise)")
    ap.add_argument("--err-per-geom", type=int, default=16, help="walkers per geometry in the oracle error check")
    ap.add_argument("--no-fp32-compare", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--check-launch", action="store_true", help="host-only check of the rank launch, then exit")
    ap.add_argument("--eloc-pass", type=int, default=0, metavar="DIV",
                    help="run one local-energy pass on the workload's walker counts divided by DIV (after --warmup "
                         "passes) and exit: the small case for ncu captures of the GEMM class")
    ap.add_argument("--pass-kind", default="eloc", choices=["eloc", "value", "grad"],
                    help="with --eloc-pass: the pass to run (local energy, log|psi| alone, or local energy and "
                         "the VMC gradient)")
    ap.add_argument("--pass-tuning", default="residual_smem=1",
                    help="tuning fields for --eloc-pass, e.g. residual_smem=1,layer_groups=2")
    args = ap.parse_args()
    if args.side is None:
        args.side = ("ne,ar,ar@16384,kr,envelope" if args.workload == DEFAULT_WORKLOAD and args.impl == "ours"
                     else "")
    if args.side == "none":
        args.side = ""
    if args.gpus < 1:
        sys.exit("--gpus must be at least 1")
    world = os.environ.get("WORLD_SIZE")
    if world is None and args.gpus > 1 and args.impl == "ours":
        launch_ranks(args)
        return
    if world is not None and int(world) != args.gpus:
        sys.exit(f"--gpus {args.gpus} but the launcher started {world} ranks")
    if args.check_launch:
        check_launch(args)
        return
    from paper_2011_07125_gb300 import synth
    wl = synth.workload(args.workload)
    if args.impl == "reference":
        if int(os.environ.get("RANK", "0")) != 0:
            return
        run_reference(args, wl)
        return
    if args.eloc_pass > 0:
        run_eloc_pass(args, wl)
        return
    run_gpu(args, wl)


if __name__ == "__main__":
    main()

#!/usr/bin/env python
"""Benchmark of the SORF + FCHL19 hot path on GB300.

One step = one pass of the whole path over the QM9-shaped workload
(100 000 synthetic molecules, 3-29 atoms, ~1.77 M atoms, N_F = 16384):
training (FCHL19 -> per-element projection -> SORF + segment sum -> split
BF16 Gram on the tensor cores -> FP64 Cholesky + PCG on the exact operator)
followed by energy + force prediction of the same molecules with the trained
weights. The metric is microseconds per atom of that step (lower is better),
with train seconds, prediction us/atom and the plain-FP32 comparison reported
beside it.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun (N > 1) every rank runs an independent replica (the path is
not sharded across GPUs here); rank 0 prints the line with max-over-ranks time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "µs/atom E+F predict, train s at 16k feats, p50/p99 latency vs plain FP32 form"
# Gram form of the training step (the preconditioner input): a qmlr precision
# (1 = 2-way BF16 split, three tensor-core products; 2 = 3-way split, six
# products; 3 = one BF16 part; 4 = e4m3 with per-feature scales), the K blocks
# summed in the tensor cores' accumulator between promotions (0 = the whole
# K range) and the tile width; set by --gram-form / --gram-promote / --gram-tile.
GRAM = {"precision": 1, "promote": 1, "tile": 128}
GRAM_FORMS = {"x3": 1, "x6": 2, "x1": 3, "fp8": 4}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--scale", type=float, default=1.0,
                    help="fraction of the 100k-molecule workload (1.0 for the reported line)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-ef", action="store_true")
    ap.add_argument("--no-periodic", action="store_true")
    ap.add_argument("--z-kernel", default="fwht", choices=["tc", "fwht"],
                    help="SORF segment sums Z of training: the in-register fast Walsh-Hadamard kernel (fwht) or "
                         "the forward chains as tensor-core FP16 products (tc)")
    ap.add_argument("--sorf-kernel", default="tc", choices=["tc", "fwht"],
                    help="SORF energies + gradients of the prediction: both Hadamard chains as tensor-core "
                         "FP16 products (tc) or the in-register fast Walsh-Hadamard kernel (fwht)")
    ap.add_argument("--serve-seconds", type=float, default=10.0)
    ap.add_argument("--pcg-iters", type=int, default=30)
    ap.add_argument("--pcg-tol", type=float, default=1e-8)
    ap.add_argument("--gram-form", default="x3", choices=sorted(GRAM_FORMS),
                    help="tensor-core Gram: x3 (2-way BF16 split), x6 (3-way), x1 (one BF16 part), "
                         "fp8 (e4m3, per-feature scales)")
    ap.add_argument("--gram-promote", type=int, default=None,
                    help="K blocks per tensor-core accumulation (0: whole K); default 1")
    ap.add_argument("--gram-tile", type=int, default=None, choices=[128, 256],
                    help="tile width; default 128 for x6, 256 otherwise")
    ap.add_argument("--shift", type=float, default=None,
                    help="relative diagonal shift of the preconditioner factor (default: the form's)")
    ap.add_argument("--nf-sweep", action="store_true",
                    help="instead of the step: train time and held-out MAE at N_F = 4096 ... 32768")
    ap.add_argument("--rff-sweep", action="store_true",
                    help="instead of the step: SORF vs dense RFF time and held-out MAE on MD17-shaped data")
    ap.add_argument("--gram-sweep", action="store_true",
                    help="instead of the step: train with each Gram form and shift on the workload and "
                         "report Gram, factor and PCG times, iterations and training MAE")
    ap.add_argument("--factor", default="mixed", choices=["mixed", "fp64"],
                    help="preconditioner factor: tensor-core trailing updates (mixed) or FP64 throughout")
    ap.add_argument("--kernel-times", action="store_true",
                    help="instead of the step: time the FCHL19 forward and adjoints on the workload and the "
                         "mixed-precision factor of a random SPD matrix of order --factor-n")
    ap.add_argument("--factor-n", type=int, default=16384)
    ap.add_argument("--feature-sweep", action="store_true",
                    help="instead of the step: time the SORF segment sum over N_transform and N_F, and "
                         "the dense RFF map beside it, on the workload's projected features")
    return ap.parse_args()


# ----------------------------------------------------------------------------
# clocks sampled during the timed region

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------
# oracle (CPU) timing on a bounded sample: the reported CPU baseline

ORACLE_SAMPLE = 20   # molecules of the workload per oracle step


def oracle_step_times(w, n_mol_sample: int, threads: int):
    """Time the FP64 oracle's training + E+F prediction on a bounded sample of the
    workload and extrapolate to the full workload: features and prediction scale
    with atoms, the Gram with rows, the Cholesky solve is fixed (N_F^3)."""
    import torch
    torch.set_num_threads(threads)
    from oracle import fchl19 as o_fchl19
    from oracle import model as o_model
    from oracle import regression as o_reg
    mols = w.mols.subset(range(n_mol_sample))
    p = o_fchl19.params(w.params_column, n2=w.n2, n3=w.n3)
    t0 = time.perf_counter()
    reps = o_fchl19.representation_batch(mols.coords, mols.elem, mols.mol_ptr, p)
    U = o_reg.pca_bases(reps, mols.elem, 5, w.d)
    m = o_model.sorf_model(p, U, w.signs, w.b, w.sigma)
    t1 = time.perf_counter()
    Z = o_model.feature_matrix(mols.coords, mols.elem, mols.mol_ptr, m)
    t2 = time.perf_counter()
    A, c = o_reg.normal_equations(Z, w.energies[:n_mol_sample], w.lam)
    t3 = time.perf_counter()
    alpha, _ = o_reg.cholesky_solve(A, c, refine=1)
    t4 = time.perf_counter()
    m.alpha = alpha
    o_model.energies_forces(mols.coords, mols.elem, mols.mol_ptr, m)
    t5 = time.perf_counter()
    n_atoms_s = mols.n_atoms
    full_atoms, full_rows = w.mols.n_atoms, w.mols.n_mol
    feat = (t2 - t1) * full_atoms / n_atoms_s
    gram = (t3 - t2) * full_rows / n_mol_sample
    chol = t4 - t3
    pred = (t5 - t4) * full_atoms / n_atoms_s
    total = feat + gram + chol + pred
    return {"total_s": total, "features_s": feat, "gram_s": gram, "solve_s": chol, "predict_s": pred,
            "sample_molecules": n_mol_sample, "sample_atoms": n_atoms_s, "sample_wall_s": t5 - t0,
            "train_s": feat + gram + chol, "predict_us_per_atom": pred / full_atoms * 1e6}


def oracle_per_atom_one_core(w, n_mol_sample: int):
    """The oracle's per-atom parts (SORF features of the molecules, then energies
    and forces) on one thread, us per atom of the sample."""
    import torch
    from oracle import fchl19 as o_fchl19
    from oracle import model as o_model
    from oracle import regression as o_reg
    prev = torch.get_num_threads()
    torch.set_num_threads(1)
    try:
        mols = w.mols.subset(range(n_mol_sample))
        p = o_fchl19.params(w.params_column, n2=w.n2, n3=w.n3)
        reps = o_fchl19.representation_batch(mols.coords, mols.elem, mols.mol_ptr, p)
        U = o_reg.pca_bases(reps, mols.elem, 5, w.d)
        rng = np.random.default_rng(0)
        m = o_model.sorf_model(p, U, w.signs, w.b, w.sigma, rng.normal(size=w.n_features))
        t0 = time.perf_counter()
        o_model.feature_matrix(mols.coords, mols.elem, mols.mol_ptr, m)
        t1 = time.perf_counter()
        o_model.energies_forces(mols.coords, mols.elem, mols.mol_ptr, m)
        t2 = time.perf_counter()
    finally:
        torch.set_num_threads(prev)
    n = mols.n_atoms
    return {"cores": 1, "sample_molecules": n_mol_sample, "sample_atoms": n,
            "features_us_per_atom": (t1 - t0) / n * 1e6, "predict_ef_us_per_atom": (t2 - t1) / n * 1e6}


def oracle_parity_workload_full():
    """The oracle on the whole parity workload (64 molecules x 9 atoms, N_F = 512):
    training (features, normal equations, Cholesky + one refinement) and E+F
    prediction, all host cores."""
    from oracle import fchl19 as o_fchl19
    from oracle import model as o_model
    from oracle import regression as o_reg
    from paper_2206_01580_gb300 import synth
    w = synth.workload(0)
    mols = w.mols
    p = o_fchl19.params(w.params_column, n2=w.n2, n3=w.n3)
    t0 = time.perf_counter()
    reps = o_fchl19.representation_batch(mols.coords, mols.elem, mols.mol_ptr, p)
    U = o_reg.pca_bases(reps, mols.elem, 5, w.d)
    m = o_model.sorf_model(p, U, w.signs, w.b, w.sigma)
    alpha, _ = o_model.train(mols.coords, mols.elem, mols.mol_ptr, w.energies, m, w.lam)
    t1 = time.perf_counter()
    m.alpha = alpha
    o_model.energies_forces(mols.coords, mols.elem, mols.mol_ptr, m)
    t2 = time.perf_counter()
    return {"workload": "parity-64x9 (64 molecules x 9 atoms, N_F = 512), in full", "train_s": t1 - t0,
            "predict_ef_us_per_atom": (t2 - t1) / mols.n_atoms * 1e6, "cores": os.cpu_count() or 1}


def fchl19_exps_per_atom(w, frac: float = 0.02) -> float:
    """Radial-grid exponentials per atom of FCHL19 on the workload: n2 per
    neighbour within r_cut and n3 per pair of neighbours whose distance is also
    within r_cut (counted on the first `frac` of the molecules)."""
    mols = w.mols
    rc = 6.0
    n_mol = max(1, int(frac * mols.n_mol))
    tot = 0
    n_at = 0
    for k in range(n_mol):
        a, b = int(mols.mol_ptr[k]), int(mols.mol_ptr[k + 1])
        x = mols.coords[a:b]
        d = np.sqrt(((x[:, None, :] - x[None, :, :]) ** 2).sum(-1))
        inside = d < rc
        np.fill_diagonal(inside, False)
        for i in range(b - a):
            nb = np.nonzero(inside[i])[0]
            tot += len(nb) * w.n2 + int(np.triu(inside[np.ix_(nb, nb)], 1).sum()) * w.n3
        n_at += b - a
    return tot / max(n_at, 1)


def workload_config(args, w, world, gram_text, solve_text):
    """The config object of the bench line (the same keys in both arms)."""
    return {"workload": "qm9-shaped-100k" if args.scale == 1.0 else f"qm9-shaped x{args.scale}",
            "n_molecules": w.mols.n_mol, "n_atoms": w.mols.n_atoms, "n_features": w.n_features, "d": w.d,
            "n_transform": w.n_transform, "gram": gram_text, "solve": solve_text,
            "sorf_prediction": ("both Hadamard chains as tcgen05 FP16 products (exact FP16 chain tables, "
                                "two-part operands)" if args.sorf_kernel == "tc"
                                else "in-register fast Walsh-Hadamard transform (FP32)"),
            "sorf_training": ("forward chains as tcgen05 FP16 products, ordered molecule sums"
                              if getattr(args, "z_kernel", "fwht") == "tc"
                              else "in-register fast Walsh-Hadamard transform (FP32), ordered molecule sums"),
            "parallelism": "replicas" if world > 1 else "single",
            "l2": "inputs larger than L2 (rep 5.5 GB, Z 6.6 GB)",
            "step": "one training (FCHL19 -> projection -> SORF -> Z -> Gram -> factor + PCG) plus E+F "
                    "prediction of the same molecules; value = us per atom of that step"}


# ----------------------------------------------------------------------------
# serving: Poisson request streams through the continuous-batching server

SIZE_BINS = ((5, 25), (26, 50), (51, 100), (101, 200))


def latency_bins(lat_us, atoms):
    """p50 / p99 latency (ms) and request count per molecule-size bin."""
    out = []
    for lo, hi in SIZE_BINS:
        sel = (atoms >= lo) & (atoms <= hi)
        if sel.any():
            v = np.sort(lat_us[sel])
            out.append({"atoms": f"{lo}-{hi}", "requests": int(sel.sum()),
                        "p50_ms": float(v[int(0.50 * (len(v) - 1) + 0.5)]) / 1e3,
                        "p99_ms": float(v[int(0.99 * (len(v) - 1) + 0.5)]) / 1e3})
    return out


def serving_phase(model_args, rates, seconds):
    """p50/p99 latency, throughput and us/atom of the server under Poisson
    arrivals of 5-200-atom molecules, and of one request at a time; latencies
    also per molecule-size bin."""
    from paper_2206_01580_gb300 import qmlr, synth
    p, U, signs, T, b, sigma, alpha = model_args
    pool = synth.serving_molecules(synth.rng_for(4), 2000)
    mols = [(np.ascontiguousarray(c, dtype=np.float32), np.ascontiguousarray(e, dtype=np.int32))
            for c, e in (pool.molecule(i) for i in range(pool.n_mol))]
    model = qmlr.Model(p, 200, U, signs, T, b, sigma, alpha)
    rng = np.random.default_rng(4)

    def run_stream(srv, rate):
        arrivals = synth.poisson_arrivals(rng, rate, seconds)
        picks = rng.integers(0, pool.n_mol, size=len(arrivals))
        st = srv.replay(pool.coords, pool.elem, pool.mol_ptr, arrivals, picks)
        lat, at = srv.latencies()
        return {"rate_rps": rate, "requests": len(arrivals), "rejected": st["rejected"],
                "p50_ms": st["p50_us"] / 1e3, "p99_ms": st["p99_us"] / 1e3,
                "throughput_rps": st["throughput_rps"], "us_per_atom": st["us_per_atom"],
                "mean_batch_atoms": st["mean_batch_atoms"], "by_size": latency_bins(lat, at)}

    srv = qmlr.Server(model, n_lanes=2, max_batch_atoms=16384, max_batch_mols=4096, use_graphs=True)
    # warm-up: every batch-size bucket once outside capture and once captured
    for burst in (1, 2, 4, 8, 16, 32, 64, 128, 256, 320):
        for _ in range(2):
            ts = [(srv.submit(*mols[i % len(mols)]), len(mols[i % len(mols)][1])) for i in range(burst)]
            for t, n in ts:
                srv.poll(t, n)
    out = {"streams": [run_stream(srv, r) for r in rates]}
    srv.close()
    # one request at a time, no batching, no graphs (the plain form)
    one = qmlr.Server(model, n_lanes=1, max_batch_atoms=256, max_batch_mols=128, use_graphs=False)
    for i in range(20):
        t = one.submit(*mols[i])
        one.poll(t, len(mols[i][1]))
    # one request at a time: each arrives after the previous result (closed loop, 600 requests)
    one.reset_stats()
    for i in range(600):
        c, e = mols[(7 * i) % len(mols)]
        t = one.submit(c, e)
        one.poll(t, len(e))
    st = one.stats()
    lat, at = one.latencies()
    out["one_at_a_time"] = {"p50_ms": st["p50_us"] / 1e3, "p99_ms": st["p99_us"] / 1e3,
                            "throughput_rps": st["throughput_rps"], "us_per_atom": st["us_per_atom"],
                            "by_size": latency_bins(lat, at)}
    one.close()
    model.close()
    out["molecules"] = "5-200 atoms, log-uniform (mean %.1f)" % pool.sizes().mean()
    out["duration_s_per_rate"] = seconds
    return out


# ----------------------------------------------------------------------------
# energy + force training on the 3BPA-shaped workload

def ef_training_phase(config, pcg_iters, pcg_tol, factor):
    """Energy + force training on the MD17-shaped (config 2: 1000 conformations,
    64 000 x 8192 rows) or 3BPA-shaped workload (config 3: 500 conformations,
    41 000 x 16384 rows), then prediction of the held-out conformations (3BPA)
    or of the training set (MD17, which has no test split); stage times by CUDA
    events."""
    import torch
    from paper_2206_01580_gb300 import pipeline, qmlr, synth
    from paper_2206_01580_gb300.params import from_table
    w = synth.workload(config)
    p = from_table(w.params_column, n2=w.n2, n3=w.n3)
    spec = pipeline.spec_from(p, w.d, w.signs, w.b, w.sigma)
    tr = pipeline.Batch.from_host(w.mols.coords, w.mols.elem, w.mols.mol_ptr)
    rep, perm, offs = pipeline.representations(tr, spec)
    U = pipeline.fit_pca(rep, perm, offs, spec)
    del rep
    y = torch.cat([torch.as_tensor(w.energies), torch.as_tensor(w.forces).reshape(-1)]).cuda()

    def once():
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        s = torch.cuda.current_stream()
        ev[0].record(s)
        rows = pipeline.energy_force_rows(tr, spec, U)
        ev[1].record(s)
        G = pipeline.gram(rows, GRAM["precision"], GRAM["promote"], GRAM["tile"])
        ev[2].record(s)
        alpha, it, rel = qmlr.gram_solve(G, rows, y, w.lam, max_iter=pcg_iters, tol=pcg_tol, factor=factor,
                                         shift=GRAM["shift"])
        ev[3].record(s)
        torch.cuda.synchronize()
        so = qmlr.last_solve
        n_rows = rows.shape[0]
        del rows, G
        return alpha, {"rows_ms": ev[0].elapsed_time(ev[1]), "gram_ms": ev[1].elapsed_time(ev[2]),
                       "solve_ms": ev[2].elapsed_time(ev[3]), "factor_ms": so.factor_ms,
                       "refine_ms": so.refine_ms, "train_s": ev[0].elapsed_time(ev[3]) / 1e3,
                       "pcg_iters": it, "rel_resid": rel, "n_rows": n_rows, "n_features": w.n_features}

    once()                     # warm-up
    alpha, st = once()
    model = qmlr.Model(p, int(w.mols.sizes().max()), U, w.signs, w.n_transform, w.b, w.sigma,
                       alpha.float().cpu().numpy())
    if w.test is not None:
        E, F = model.predict(w.test.coords, w.test.elem, w.test.mol_ptr)
        mae_e = float(np.mean(np.abs(E.cpu().numpy() - w.test_energies)))
        mae_f = float(np.mean(np.abs(F.cpu().numpy() - w.test_forces)))
        split = "test"
    else:
        E, F = model.predict(w.mols.coords, w.mols.elem, w.mols.mol_ptr)
        mae_e = float(np.mean(np.abs(E.cpu().numpy() - w.energies)))
        mae_f = float(np.mean(np.abs(F.cpu().numpy() - w.forces)))
        split = "train"
    model.close()
    name = ("md17-shaped-1k (1000 conformations of a 21-atom C9H8O4-like molecule, N_F = 8192)" if config == 2
            else "3bpa-shaped-500 (500 train / 2000 test conformations, 27 atoms, N_F = 16384)")
    st.update({"workload": name, f"{split}_mae_E_eV": mae_e, f"{split}_mae_F_eV_per_A": mae_f})
    return st


def periodic_phase():
    """E+F prediction of the periodic stand-ins for the paper's liquid water
    (4000 waters, 12 000 atoms) and MOF (16 848 atoms) rows: random-weight model
    (N_F = 16384, d = 128, T = 3, E+F parameters, per-system PCA basis); device
    time (CUDA events, median of 5 after a warm-up) and the same with the
    host->device copy of the coordinates and the device->host copy of E and F
    inside the timed region; the host cell list (a per-geometry setup) timed apart."""
    import torch
    from paper_2206_01580_gb300 import pipeline, qmlr, synth
    from paper_2206_01580_gb300.params import from_table
    p = from_table("EF", n2=24, n3=22)
    out = []
    for name, gen in (("water-shaped (4000 rigid waters, 12 000 atoms, 1 g/cm^3, cubic cell)",
                       lambda: synth.water_box(synth.rng_for(5, 10), 4000)),
                      ("mof-shaped (16 848 atoms, framework density 0.075 atoms/A^3, orthorhombic cell)",
                       lambda: synth.framework_crystal(synth.rng_for(5, 11), 16848))):
        ps = gen()
        rng = np.random.default_rng(12)
        signs, b = synth.sorf_draw(rng, 16384, 128, 3)
        alpha = torch.as_tensor(rng.normal(size=16384).astype(np.float32)).cuda()
        spec = pipeline.spec_from(p, 128, signs, b.astype(np.float32), 2.0)
        t0 = time.perf_counter()
        system = qmlr.PeriodicSystem(ps.coords, ps.elem, ps.cell, p.rcut)
        env_s = time.perf_counter() - t0
        rep = qmlr.fchl19_periodic(system, p)
        perm, offs = qmlr.group_by_element(system.elem, p.n_el)
        U = qmlr.pca_fit(rep, p.rep_dim, perm, offs, p.n_el, 128)
        del rep
        host_x = torch.as_tensor(ps.coords.astype(np.float32)).pin_memory()
        host_E = torch.empty(1, dtype=torch.float64).pin_memory()
        host_F = torch.empty((ps.n_atoms, 3), dtype=torch.float32).pin_memory()

        def run(e2e):
            if e2e:
                system.coords.copy_(host_x, non_blocking=True)
            E, F = pipeline.predict_periodic(system, spec, U, alpha)
            if e2e:
                host_E.copy_(E, non_blocking=True)
                host_F.copy_(F, non_blocking=True)

        res = {}
        for e2e in (False, True):
            run(e2e)
            ts = []
            for _ in range(5):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                e0.record()
                run(e2e)
                e1.record()
                torch.cuda.synchronize()
                ts.append(e0.elapsed_time(e1))
            res["e2e_ms" if e2e else "device_ms"] = statistics.median(ts)
        n_env = np.diff(system.env_ptr.cpu().numpy())
        out.append({"workload": name, "n_atoms": ps.n_atoms, "env_mean": float(n_env.mean()),
                    "env_max": int(n_env.max()), "cell_list_s": env_s,
                    "device_ms": res["device_ms"], "device_us_per_atom": res["device_ms"] * 1e3 / ps.n_atoms,
                    "e2e_ms": res["e2e_ms"], "e2e_us_per_atom": res["e2e_ms"] * 1e3 / ps.n_atoms})
        del system, U
        torch.cuda.empty_cache()
    return out


def max_over_ranks(x: float, dist, device: str) -> float:
    """The largest value over the ranks (every rank gets it); x itself without a
    process group."""
    if not dist:
        return x
    import torch
    t = torch.tensor([x], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def us_per_atom(ms_max: float, atoms_per_rank: int, world: int) -> float:
    """Whole-job time per atom: every rank (a replica) processed atoms_per_rank
    atoms within the slowest rank's time ms_max."""
    return ms_max * 1e3 / (atoms_per_rank * world)


def measured_traffic(kind, kernel):
    """DRAM bytes per launch of the dominant kernel from the committed ncu
    summary, or None when it was taken for another kernel or the kernel's
    source changed since the capture."""
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "dram_traffic.json")))[kind]
    except (OSError, ValueError, KeyError):
        return None
    if not kernel.startswith(rec["kernel"]):
        return None
    src = os.path.join(ROOT, rec["source"])
    try:
        digest = hashlib.sha256(open(src, "rb").read()).hexdigest()
    except OSError:
        return None
    if digest != rec["sha256"]:
        return None
    return rec


def build_workload(scale):
    from paper_2206_01580_gb300 import synth
    t = time.perf_counter()
    w = synth.workload(1, scale=scale)
    return w, time.perf_counter() - t


def run_reference(args, rank, world):
    """The oracle as it stands, on the host cores: each step is a bounded sample
    (20 molecules) of the same workload, extrapolated to the whole workload."""
    if rank != 0:
        return
    w, _ = build_workload(args.scale)
    threads = os.cpu_count() or 1
    times = []
    for k in range(args.warmup + args.steps):
        r = oracle_step_times(w, ORACLE_SAMPLE, threads)
        if k >= args.warmup:
            times.append(r)
    total = statistics.mean(t["total_s"] for t in times)
    val = total / w.mols.n_atoms * 1e6
    sample = (f"{ORACLE_SAMPLE} molecules per step ({times[0]['sample_atoms']} atoms); features, Gram rows and "
              "prediction extrapolated linearly to the workload (values extrapolated, not a full run); "
              "full N_F^3 Cholesky")
    line = {"metric": METRIC, "impl": "reference", "value": val, "unit": "us/atom",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": total * 1e3, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(args, w, world, "fp64 dense Z^T Z (numpy)",
                                      "fp64 dense Cholesky + one refinement step (numpy/scipy)"),
            "train_s": statistics.mean(t["train_s"] for t in times),
            "predict_us_per_atom": statistics.mean(t["predict_us_per_atom"] for t in times),
            "cpu_baseline": {"value": val, "unit": "us/atom", "cores": threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": val, "unit": "us/atom", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args, rank, world):
    import torch
    from paper_2206_01580_gb300 import pipeline, qmlr
    from paper_2206_01580_gb300.params import from_table

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    # the step runs on a high-priority stream (the library launches on the current stream)
    torch.cuda.set_stream(torch.cuda.Stream(priority=-100))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")

    w, gen_s = build_workload(args.scale)
    mols = w.mols
    n_atoms, n_mol = mols.n_atoms, mols.n_mol
    p = from_table(w.params_column, n2=w.n2, n3=w.n3)
    spec = pipeline.spec_from(p, w.d, w.signs, w.b, w.sigma)
    batch = pipeline.Batch.from_host(mols.coords, mols.elem, mols.mol_ptr)
    y = torch.as_tensor(w.energies).cuda()

    # setup (untimed): PCA basis on the device, model handle for prediction
    rep, perm, offs = pipeline.representations(batch, spec)
    U = pipeline.fit_pca(rep, perm, offs, spec)
    model = qmlr.Model(p, batch.max_atoms, U, w.signs, w.n_transform, w.b, w.sigma,
                       np.zeros(w.n_features, np.float32))
    model.reserve(n_atoms)
    model.set_timing(True)          # CUDA events around the prediction's kernels (read per timed step)
    if args.sorf_kernel == "fwht" and model.sorf_tc:
        model.set_sorf_tc(False)
    pipeline.SORF_TC = args.z_kernel == "tc"
    sorf_tc = model.sorf_tc
    del rep, perm, offs
    torch.cuda.synchronize()

    stream = torch.cuda.current_stream()
    factor = qmlr.FACTOR_MIXED if args.factor == "mixed" else qmlr.FACTOR_FP64

    # the side stream (prediction features) at the lowest priority, so that the
    # solve's kernels on the main stream are scheduled first whenever they wait
    side = torch.cuda.Stream(priority=0)

    def step(b: pipeline.Batch, yv, precision=None, timing=None):
        precision = GRAM["precision"] if precision is None else precision
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(8)]
        sev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record(stream)
        rep, perm, offs = pipeline.representations(b, spec)
        ev[1].record(stream)
        x = qmlr.project(rep, p.rep_dim, perm, offs, p.n_el, U)
        ev[2].record(stream)
        Z = pipeline.segment_features(x, b.mol_ptr, spec)
        ev[3].record(stream)
        zt = pipeline.gram_operand(Z, precision)
        ev[7].record(stream)
        if precision == GRAM["precision"]:
            G = pipeline.gram(Z, precision, GRAM["promote"], GRAM["tile"], operand=zt)
        else:
            G = pipeline.gram(Z, precision, operand=zt)
        del zt
        ev[4].record(stream)
        # the prediction's weight-independent half (representations, grouping,
        # projection) runs on a second stream beside the solve
        side.wait_stream(stream)
        with torch.cuda.stream(side):
            sev[0].record(side)
            model.predict_features(b.coords, b.elem, b.mol_ptr)
            sev[1].record(side)
        alpha, it, rel = qmlr.gram_solve(G, Z, yv, w.lam, method=qmlr.SOLVE_PCG,
                                         max_iter=args.pcg_iters if precision != qmlr.GRAM_FP32 else 4 * args.pcg_iters,
                                         tol=args.pcg_tol, factor=factor,
                                         shift=GRAM["shift"] if precision == GRAM["precision"]
                                         else pipeline.DEFAULT_SHIFT[precision])
        ev[5].record(stream)
        model.set_alpha_device(alpha)
        stream.wait_stream(side)
        E, F = model.predict_from_features(b.coords, b.elem, b.mol_ptr)
        ev[6].record(stream)
        if timing is not None:
            torch.cuda.synchronize()
            so = qmlr.last_solve
            mt = model.timings()
            timing.append({"sorf_atom": mt["sorf_energy_grad"], "fchl19_vjp": mt["fchl19_vjp"],
                           "project_t": mt["project_t"],
                           "fchl19": ev[0].elapsed_time(ev[1]), "project": ev[1].elapsed_time(ev[2]),
                           "sorf_Z": ev[2].elapsed_time(ev[3]), "gram_operand": ev[3].elapsed_time(ev[7]),
                           "gram": ev[7].elapsed_time(ev[4]),
                           "solve": ev[4].elapsed_time(ev[5]), "factor": so.factor_ms,
                           "refine": so.refine_ms, "predict_ef": ev[5].elapsed_time(ev[6]),
                           "predict_features_beside_solve": sev[0].elapsed_time(sev[1]),
                           "total": ev[0].elapsed_time(ev[6]), "pcg_iters": it, "rel_resid": rel})
        return alpha, E, F

    for _ in range(args.warmup):
        step(batch, y)
    torch.cuda.synchronize()

    # ---------------- timed region: device-resident inputs
    sampler = ClockSampler(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    launches0 = qmlr.launch_count()
    t_ev0 = torch.cuda.Event(enable_timing=True)
    t_ev1 = torch.cuda.Event(enable_timing=True)
    timing = []
    t_ev0.record(stream)
    for _ in range(args.steps):
        alpha, E, F = step(batch, y, timing=timing)
    t_ev1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    launches = qmlr.launch_count() - launches0
    clocks = sampler.stop()
    ms = max_over_ranks(t_ev0.elapsed_time(t_ev1) / args.steps, dist, "cuda")
    st = {k: statistics.median(t[k] for t in timing) for k in timing[0]}
    mae = float(torch.mean(torch.abs(E - y)).item())

    # ---------------- end to end: host buffers in, results out, copies timed
    h_coords = torch.as_tensor(mols.coords.astype(np.float32)).pin_memory()
    h_elem = torch.as_tensor(mols.elem.astype(np.int32)).pin_memory()
    h_ptr = torch.as_tensor(mols.mol_ptr.astype(np.int32)).pin_memory()
    h_y = torch.as_tensor(w.energies.astype(np.float64)).pin_memory()
    out_alpha = torch.empty(w.n_features, dtype=torch.float64).pin_memory()
    out_E = torch.empty(n_mol, dtype=torch.float64).pin_memory()
    out_F = torch.empty((n_atoms, 3), dtype=torch.float32).pin_memory()
    h2d = (h_coords.numel() * 4 + h_elem.numel() * 4 + h_ptr.numel() * 4 + h_y.numel() * 8)
    d2h = out_alpha.numel() * 8 + out_E.numel() * 8 + out_F.numel() * 4
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        b2 = pipeline.Batch(h_coords.cuda(non_blocking=True), h_elem.cuda(non_blocking=True),
                            h_ptr.cuda(non_blocking=True), batch.max_atoms)
        y2 = h_y.cuda(non_blocking=True)
        a2, E2, F2 = step(b2, y2)
        out_alpha.copy_(a2, non_blocking=True)
        out_E.copy_(E2, non_blocking=True)
        out_F.copy_(F2, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, dist, "cuda")

    # ---------------- plain FP32 form (FP32 SIMT Gram, same solve), one step
    plain = None
    if not args.no_plain:
        pt = []
        _, Ep, _ = step(batch, y, precision=qmlr.GRAM_FP32, timing=pt)
        plain = {"gram_ms": pt[0]["gram"], "train_s": (pt[0]["total"] - pt[0]["predict_ef"]) / 1e3,
                 "step_ms": pt[0]["total"], "pcg_iters": pt[0]["pcg_iters"],
                 "rel_resid": pt[0]["rel_resid"],
                 "train_mae_eV": float(torch.mean(torch.abs(Ep - y)).item())}

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    # ---------------- roofline of the dominant kernel
    # Candidates are the single kernels the step times on its own stream: the
    # tensor-core Gram (split kernel) and the SORF segment sum. The Cholesky
    # factor, the PCG and the prediction are sequences of kernels; their shares
    # are in the committed launch list.
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    nf = w.n_features
    rows = n_mol
    bf16_sust = peaks.get("bf16_tflops_sustained", 1707.8)
    gdesc = gram_description()
    # ALU peak of the SORF kernels (adds dominate): SMs x 128 FP32 lanes x max SM clock
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    sm_max_mhz = peaks.get("sm_max_mhz", 2070.0)
    fp32_add_peak = props.multi_processor_count * 128 * sm_max_mhz * 1e6 / 1e12
    try:
        fadd_measured = qmlr.unit_rates()["fadd"] / 1e12
    except Exception:   # diagnostics only
        fadd_measured = None
    n_stack = nf // w.d
    sorf_ops_atom = n_stack * w.n_transform * w.d * int(math.log2(w.d)) + 6 * nf
    butterflies = n_stack * w.n_transform * w.d * int(math.log2(w.d))
    sorf_atom_ops = 2 * butterflies + 4 * nf
    try:
        exp_rate = qmlr.unit_rates()["expf"] / 1e12
    except Exception:   # diagnostics only
        exp_rate = None
    exps_atom = fchl19_exps_per_atom(w)
    cands = {
        "gram": {"kernel": gdesc["kernel"],
                 "bound": "tensor",
                 "achieved": rows * nf * nf / (st["gram"] * 1e-3) / 1e12,
                 "peak": bf16_sust * gdesc["rate"] / gdesc["products"],
                 "unit": "TFLOP/s",
                 "work": f"N_rows*N_F^2 = {rows * nf * nf:.3e} flop (symmetric half, 2 flop/MAC)",
                 "peak_source": f"MEASURED_PEAKS.json bf16_tflops_sustained x {gdesc['rate']} / "
                                f"{gdesc['products']} ({gdesc['products']} tensor-core products per Gram "
                                f"product; {gdesc['rate']} x the BF16 rate for its operand type, the nominal "
                                "dense ratio)"},
        "sorf_Z": ({"kernel": "qmlr::stc::sorf_z_tc_kernel (SORF forward chains as tcgen05 FP16 products, cos, "
                               "ordered molecule sums into Z)",
                    "bound": "tensor",
                    "achieved": 2 * w.d * nf * n_atoms / (st["sorf_Z"] * 1e-3) / 1e12, "peak": bf16_sust / 2,
                    "unit": "TFLOP/s",
                    "work": f"2*d*N_F = {2 * w.d * nf} flop/atom (dense chain product x M_s^T)",
                    "peak_source": "MEASURED_PEAKS.json bf16_tflops_sustained / 2 (two FP16 products per dense "
                                   "product; FP16 at the BF16 rate)",
                    "mufu": {"achieved": nf * n_atoms / (st["sorf_Z"] * 1e-3) / 1e12, "peak": exp_rate,
                             "unit": "T op/s", "work": "cos per feature (N_F per atom)",
                             "peak_source": "measured __expf rate (MUFU), qmlr_unit_rates"}}
                   if pipeline.SORF_TC else
                   {"kernel": "qmlr::sorf_mol_kernel<128> (SORF + segment sum into Z)", "bound": "alu",
                    "achieved": sorf_ops_atom * n_atoms / (st["sorf_Z"] * 1e-3) / 1e12, "peak": fp32_add_peak,
                    "unit": "TFLOP/s",
                    "work": f"{sorf_ops_atom} FP32 ops/atom (n_stack*T*d*log2 d butterflies + 6*N_F "
                            "for phase, cos, sum)",
                    "peak_source": f"{props.multi_processor_count} SMs x 128 FP32 lanes x {sm_max_mhz:.0f} MHz "
                                   f"(measured FP32 add rate {fadd_measured} T/s, qmlr_unit_rates)"}),
        "sorf_atom": ({"kernel": "qmlr::stc::sorf_tc_kernel (SORF energies + gradient, both Hadamard chains "
                                 "as tcgen05 FP16 products, prediction)",
                       "bound": "tensor",
                       "achieved": 4 * w.d * nf * n_atoms / (st["sorf_atom"] * 1e-3) / 1e12,
                       "peak": bf16_sust / 2,
                       "unit": "TFLOP/s",
                       "work": f"2 directions x 2*d*N_F = {4 * w.d * nf} flop/atom (dense chain products "
                               "x M_s^T and y M_s)",
                       "peak_source": "MEASURED_PEAKS.json bf16_tflops_sustained / 2 (two FP16 products per "
                                      "dense product: two-part operands, exact FP16 chain tables; FP16 at the "
                                      "BF16 rate)",
                       "mufu": {"achieved": 2 * nf * n_atoms / (st["sorf_atom"] * 1e-3) / 1e12,
                                "peak": exp_rate, "unit": "T op/s",
                                "work": "sin and cos per feature (2*N_F per atom)",
                                "peak_source": "measured __expf rate (MUFU), qmlr_unit_rates"},
                       "timing": "CUDA events of the model's prediction in every timed step (x split, "
                                 "tensor-core kernel, molecule sums)"}
                      if sorf_tc else
                      {"kernel": "qmlr::sorf_atom_kernel<128, 1> (SORF energies + gradient, prediction)",
                       "bound": "alu",
                       "achieved": sorf_atom_ops * n_atoms / (st["sorf_atom"] * 1e-3) / 1e12,
                       "peak": fp32_add_peak,
                       "unit": "TFLOP/s",
                       "work": f"{sorf_atom_ops} FP32 ops/atom (forward and transposed butterflies "
                               f"2*n_stack*T*d*log2 d = {2 * butterflies}, plus 4*N_F for phase, energy and "
                               "gradient scaling; sign flips and sin/cos not counted)",
                       "peak_source": f"{props.multi_processor_count} SMs x 128 FP32 lanes x {sm_max_mhz:.0f} MHz",
                       "timing": "CUDA events of the model's prediction in every timed step"}),
        "fchl19_fwd": {"kernel": "qmlr::fchl19_forward_reg_kernel (FCHL19 forward, training pass)",
                       "bound": "alu",
                       "achieved": exps_atom * n_atoms / (st["fchl19"] * 1e-3) / 1e12,
                       "peak": exp_rate, "unit": "T exp/s",
                       "work": f"{exps_atom:.0f} radial-grid exponentials per atom (n*n2 two-body + in-cutoff "
                               "triplets*n3, counted on a 2 % sample of the workload)",
                       "peak_source": "measured __expf rate (MUFU), qmlr_unit_rates"},
        "fchl19_vjp": {"kernel": "qmlr::fchl19_vjp_centre_kernel + vjp_reduce_kernel (FCHL19 adjoint, prediction)",
                       "bound": "alu",
                       "achieved": exps_atom * n_atoms / (st["fchl19_vjp"] * 1e-3) / 1e12,
                       "peak": exp_rate, "unit": "T exp/s",
                       "work": f"{exps_atom:.0f} radial-grid exponentials per atom (as the forward; the "
                               "derivative arithmetic not counted)",
                       "peak_source": "measured __expf rate (MUFU), qmlr_unit_rates",
                       "timing": "CUDA events of the model's prediction in every timed step"},
    }
    for c in cands.values():
        c["frac"] = c["achieved"] / c["peak"] if c["peak"] else None
        c["traffic"] = None
    stage_of = {"gram": "gram", "sorf_Z": "sorf_Z", "sorf_atom": "sorf_atom", "fchl19_fwd": "fchl19",
                "fchl19_vjp": "fchl19_vjp"}
    for k, c in cands.items():
        c["ms"] = st[stage_of[k]]
    dom = max(cands, key=lambda k: st[stage_of[k]])
    roof = dict(cands[dom])
    tr = measured_traffic(dom, roof["kernel"])
    if tr is not None:
        roof["traffic"] = tr["bytes_per_launch"]
        roof["traffic_source"] = tr["summary"]
    line = {
        "metric": METRIC, "value": us_per_atom(ms, n_atoms, world), "unit": "us/atom", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": f"f32 features, {gdesc['dtype']} gram, f64 solve",
        "data": "synthetic",
        "config": workload_config(args, w, world, gdesc["text"] + f", shift {GRAM['shift']:.3g} x max G_ii "
                                  "(preconditioner input)",
                                  ("mixed-precision cholesky (double-float panels, tcgen05 trailing updates)"
                                   if args.factor == "mixed" else "fp64 cholesky") + " + pcg (exact fp64 operator)"),
        "train_s": (st["total"] - st["predict_ef"]) / 1e3,
        # prediction cost: its feature half (timed on the side stream, beside the
        # solve) plus the weight-dependent half
        "predict_us_per_atom": (st["predict_ef"] + st["predict_features_beside_solve"]) * 1e3 / n_atoms,
        "stages_ms": {k: round(v, 3) for k, v in st.items() if k not in ("pcg_iters", "rel_resid")},
        "pcg": {"iters": st["pcg_iters"], "rel_resid": st["rel_resid"]},
        "train_mae_eV": mae,
        "roofline": roof,
        "kernel_rooflines": cands,
        "plain_fp32": plain,
        "clocks": clocks,
        "gpu_launches": launches,
        "e2e": {"value": us_per_atom(e2e_ms, n_atoms, world), "unit": "us/atom", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "workload_gen_s": gen_s,
    }
    if not args.no_ef and world == 1:
        line["ef_training"] = ef_training_phase(3, args.pcg_iters, args.pcg_tol, factor)
        line["ef_training_md17"] = ef_training_phase(2, args.pcg_iters, args.pcg_tol, factor)
    if not args.no_periodic and world == 1:
        line["periodic"] = periodic_phase()
    if not args.no_serve and world == 1:
        alpha_host = alpha.float().cpu().numpy()
        line["serving"] = serving_phase((p, U, w.signs, w.n_transform, w.b, w.sigma, alpha_host),
                                        (1000, 5000, 10000, 20000), args.serve_seconds)
    if not args.no_cpu_baseline and world == 1:
        threads = os.cpu_count() or 1
        cb = oracle_step_times(w, ORACLE_SAMPLE, threads)
        line["cpu_baseline"] = {"value": cb["total_s"] / n_atoms * 1e6, "unit": "us/atom", "cores": threads,
                                "kind": "oracle",
                                "sample": f"{cb['sample_molecules']} molecules ({cb['sample_atoms']} atoms); "
                                          "features, Gram rows and prediction extrapolated linearly to the "
                                          "workload (values extrapolated, not a full run); full N_F^3 Cholesky",
                                "train_s": cb["train_s"], "predict_us_per_atom": cb["predict_us_per_atom"],
                                "one_core": oracle_per_atom_one_core(w, 4),
                                "parity_workload_full": oracle_parity_workload_full()}
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def run_kernel_times(args):
    """FCHL19 forward, per-molecule adjoint and per-centre adjoint on the QM9-shaped
    workload (at --scale), and the mixed-precision factor of A = X^T X + I (X
    Gaussian, order --factor-n); each: one warm-up call, then the median of three
    CUDA-event-timed calls. Prints one JSON line (a fixed small command for
    kernel counter captures)."""
    import torch
    from paper_2206_01580_gb300 import qmlr
    from paper_2206_01580_gb300.params import from_table

    torch.cuda.set_device(0)
    w, _ = build_workload(args.scale)
    mols = w.mols
    p = from_table(w.params_column, n2=w.n2, n3=w.n3)
    coords = torch.as_tensor(mols.coords, dtype=torch.float32).cuda()
    elem = torch.as_tensor(mols.elem, dtype=torch.int32).cuda()
    mp = torch.as_tensor(mols.mol_ptr, dtype=torch.int32).cuda()
    mx = int(np.max(np.diff(mols.mol_ptr)))
    rep = qmlr.fchl19(coords, elem, mp, mx, p)
    g = torch.randn_like(rep)

    def timed(fn):
        fn()
        ts = []
        for _ in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.median(ts)

    out = {"workload": w.name, "n_atoms": int(mols.n_atoms),
           "fchl19_fwd_ms": timed(lambda: qmlr.fchl19(coords, elem, mp, mx, p, out=rep)),
           "fchl19_vjp_ms": timed(lambda: qmlr.fchl19_vjp(coords, elem, mp, mx, p, g)),
           "fchl19_vjp_atoms_ms": timed(lambda: qmlr.fchl19_vjp_atoms(coords, elem, mp, mx, p, g))}
    del rep, g
    n = args.factor_n
    gen = torch.Generator(device="cuda").manual_seed(0)
    X = torch.randn(n + 64, n, device="cuda", generator=gen)
    A = (X.T @ X).double() + torch.eye(n, device="cuda", dtype=torch.float64)
    del X
    out.update({"factor_n": n, "factor_ms": timed(lambda: qmlr.cholesky_mixed(A))})
    assert qmlr.device_status() == 0
    print(json.dumps(out))


def run_feature_sweep(args):
    """SORF -> Z for N_transform in {1, 2, 3} and N_F in {8192, 16384, 32768}, and the
    dense RFF map (W = G / sigma) at N_F in {8192, 16384}, on the projected features of
    the QM9-shaped workload (setup untimed; each point: one warm-up call, then the
    median of three CUDA-event-timed calls). Prints one JSON line."""
    import torch
    from paper_2206_01580_gb300 import pipeline, qmlr, synth
    from paper_2206_01580_gb300.params import from_table

    torch.cuda.set_device(0)
    w, _ = build_workload(args.scale)
    mols = w.mols
    p = from_table(w.params_column, n2=w.n2, n3=w.n3)
    spec = pipeline.spec_from(p, w.d, w.signs, w.b, w.sigma)
    batch = pipeline.Batch.from_host(mols.coords, mols.elem, mols.mol_ptr)
    rep, perm, offs = pipeline.representations(batch, spec)
    U = pipeline.fit_pca(rep, perm, offs, spec)
    x = qmlr.project(rep, p.rep_dim, perm, offs, p.n_el, U)
    del rep
    n_atoms, d = mols.n_atoms, w.d
    props = torch.cuda.get_device_properties(0)
    alu_peak = props.multi_processor_count * 128 * 2070e6 / 1e12   # FP32 lanes x max SM clock, T op/s

    def timed(fn):
        fn()
        ts = []
        for _ in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            out = fn()
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
            del out
        return statistics.median(ts)

    rng = np.random.default_rng(220601580 + 41)
    sorf_pts, rff_pts = [], []
    for nf in (8192, 16384, 32768):
        for T in (1, 2, 3):
            signs, b = synth.sorf_draw(rng, nf, d, T)
            bits = qmlr.pack_signs(signs)
            bt = torch.as_tensor(b.astype(np.float32)).cuda()
            ms = timed(lambda: qmlr.sorf(x, batch.mol_ptr, bits, T, bt, w.sigma, qmlr.SORF_PER_MOL))
            ops = (nf // d) * T * d * int(math.log2(d)) + 6 * nf
            sorf_pts.append({"n_features": nf, "n_transform": T, "ms": ms, "us_per_atom": ms * 1e3 / n_atoms,
                             "t_op_s": ops * n_atoms / (ms * 1e-3) / 1e12,
                             "alu_frac": ops * n_atoms / (ms * 1e-3) / 1e12 / alu_peak})
    for nf in (8192, 16384):
        G, b = synth.rff_draw(rng, nf, d)
        Gt = torch.as_tensor(G.astype(np.float32)).cuda()
        bt = torch.as_tensor(b.astype(np.float32)).cuda()
        ms = timed(lambda: qmlr.rff(x, batch.mol_ptr, Gt, bt, w.sigma, qmlr.SORF_PER_MOL))
        ms_tc = timed(lambda: qmlr.rff_tc(x, batch.mol_ptr, Gt, bt, w.sigma, qmlr.SORF_PER_MOL))
        flop = 2 * nf * d
        rff_pts.append({"n_features": nf, "simt_ms": ms, "simt_us_per_atom": ms * 1e3 / n_atoms,
                        "simt_tflop_s": flop * n_atoms / (ms * 1e-3) / 1e12,
                        "simt_fma_frac": flop * n_atoms / (ms * 1e-3) / 1e12 / (2 * alu_peak),
                        "tc_ms": ms_tc, "tc_us_per_atom": ms_tc * 1e3 / n_atoms,
                        "tc_tflop_s": flop * n_atoms / (ms_tc * 1e-3) / 1e12})
    print(json.dumps({"feature_sweep": {
        "workload": "qm9-shaped-100k" if args.scale == 1.0 else f"qm9-shaped x{args.scale}",
        "n_atoms": n_atoms, "n_molecules": mols.n_mol, "d": d, "sigma": w.sigma,
        "alu_peak_t_op_s": alu_peak, "sorf_Z": sorf_pts, "rff_Z": rff_pts}}), flush=True)


def run_gram_sweep(args):
    """Training on the workload with each preconditioner Gram form and shift:
    Gram (operand + product) time, factor and PCG times, iterations, final
    residual and training MAE (|Z alpha - y|), all by CUDA events. Setup
    (features, Z) untimed. Prints one JSON line."""
    import torch
    from paper_2206_01580_gb300 import pipeline, qmlr
    from paper_2206_01580_gb300.params import from_table

    torch.cuda.set_device(0)
    torch.cuda.set_stream(torch.cuda.Stream(priority=-100))
    w, _ = build_workload(args.scale)
    mols = w.mols
    p = from_table(w.params_column, n2=w.n2, n3=w.n3)
    spec = pipeline.spec_from(p, w.d, w.signs, w.b, w.sigma)
    batch = pipeline.Batch.from_host(mols.coords, mols.elem, mols.mol_ptr)
    y = torch.as_tensor(w.energies).cuda()
    rep, perm, offs = pipeline.representations(batch, spec)
    U = pipeline.fit_pca(rep, perm, offs, spec)
    Z = pipeline.feature_matrix(batch, spec, U, rep, perm, offs)
    del rep, perm, offs
    factor = qmlr.FACTOR_MIXED if args.factor == "mixed" else qmlr.FACTOR_FP64
    s = torch.cuda.current_stream()
    configs = [(1, 1, 128, -2.0 ** -15), (1, 2, 128, -2.0 ** -15), (1, 2, 128, -2.0 ** -14),
               (1, 4, 128, -2.0 ** -14),
               (1, 1, 256, -2.0 ** -15), (1, 1, 256, -2.0 ** -14), (1, 2, 256, -2.0 ** -14),
               (1, 2, 256, -2.0 ** -13),
               (3, 1, 256, -2.0 ** -12), (3, 1, 256, -2.0 ** -11), (3, 1, 256, -2.0 ** -10),
               (3, 1, 256, -2.0 ** -9), (3, 1, 256, -2.0 ** -8), (3, 2, 256, -2.0 ** -10),
               (4, 1, 256, -2.0 ** -8), (4, 1, 256, -2.0 ** -7), (4, 1, 256, -2.0 ** -6),
               (4, 1, 256, -2.0 ** -5), (4, 1, 256, -2.0 ** -4),
               (0, 0, 0, -2.0 ** -11), (0, 0, 0, -2.0 ** -10), (0, 0, 0, -2.0 ** -9), (0, 0, 0, -2.0 ** -8)]
    pts = []
    for prec, promote, tile, shift in configs:
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        for rep_i in range(2):            # the first pass warms up kernels and the allocator
            ev[0].record(s)
            zt = pipeline.gram_operand(Z, prec)
            ev[1].record(s)
            G = pipeline.gram(Z, prec, promote if prec else None, tile if prec else None, operand=zt)
            ev[2].record(s)
            del zt
            try:
                alpha, it, rel = qmlr.gram_solve(G, Z, y, w.lam, max_iter=args.pcg_iters, tol=args.pcg_tol,
                                                 factor=factor, shift=shift)
                ok = True
            except qmlr.QMLRError as e:
                ok, it, rel, alpha = False, -1, float("nan"), None
                err = str(e)
            ev[3].record(s)
            torch.cuda.synchronize()
            del G
        so = qmlr.last_solve
        pt = {"precision": prec, "promote": promote, "tile": tile, "shift": shift,
              "operand_ms": ev[0].elapsed_time(ev[1]), "gram_ms": ev[1].elapsed_time(ev[2]),
              "solve_ms": ev[2].elapsed_time(ev[3]), "train_tail_ms": ev[0].elapsed_time(ev[3]),
              "pcg_iters": it, "rel_resid": rel}
        if ok:
            pt.update({"factor_ms": so.factor_ms, "refine_ms": so.refine_ms, "shift_used": so.shift_used,
                       "train_mae_eV": float(torch.mean(torch.abs(Z.double() @ alpha - y)).item())})
        else:
            pt["error"] = err
        pts.append(pt)
        print(json.dumps(pt), flush=True)
    print(json.dumps({"gram_sweep": {
        "workload": "qm9-shaped-100k" if args.scale == 1.0 else f"qm9-shaped x{args.scale}",
        "n_rows": mols.n_mol, "n_features": w.n_features, "pcg_max_iter": args.pcg_iters, "pcg_tol": args.pcg_tol,
        "points": pts}}), flush=True)


def run_nf_sweep(args):
    """Training time and held-out MAE against the feature count: QM9-shaped
    workload, the first 90 % of the molecules for training and the last 10 %
    held out, N_F in {4096, 8192, 16384, 32768} (T = 3, d = 128); train time =
    FCHL19 -> projection -> SORF -> Z -> Gram -> factor + PCG by CUDA events.
    Prints one JSON line."""
    import torch
    from paper_2206_01580_gb300 import pipeline, qmlr, synth
    from paper_2206_01580_gb300.params import from_table

    torch.cuda.set_device(0)
    torch.cuda.set_stream(torch.cuda.Stream(priority=-100))
    w, _ = build_workload(args.scale)
    n_tr = int(0.9 * w.mols.n_mol)
    tr, te = w.mols.subset(range(n_tr)), w.mols.subset(range(n_tr, w.mols.n_mol))
    y = torch.as_tensor(w.energies[:n_tr]).cuda()
    y_te = w.energies[n_tr:]
    p = from_table(w.params_column, n2=w.n2, n3=w.n3)
    btr = pipeline.Batch.from_host(tr.coords, tr.elem, tr.mol_ptr)
    factor = qmlr.FACTOR_MIXED if args.factor == "mixed" else qmlr.FACTOR_FP64
    s = torch.cuda.current_stream()
    pts = []
    U = None
    for nf in (4096, 8192, 16384, 32768):
        signs, b = synth.sorf_draw(synth.rng_for(1, 60 + nf // 4096), nf, w.d, w.n_transform)
        spec = pipeline.spec_from(p, w.d, signs, b, w.sigma)
        if U is None:
            rep, perm, offs = pipeline.representations(btr, spec)
            U = pipeline.fit_pca(rep, perm, offs, spec)
            del rep, perm, offs
        for rep_i in range(2):           # the first pass warms up
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            ev[0].record(s)
            Z = pipeline.feature_matrix(btr, spec, U)
            ev[1].record(s)
            alpha, it, rel = pipeline.solve(Z, y, w.lam, GRAM["precision"], max_iter=args.pcg_iters,
                                            tol=args.pcg_tol, shift=GRAM["shift"], factor=factor,
                                            promote=GRAM["promote"], tile=GRAM["tile"])
            ev[2].record(s)
            torch.cuda.synchronize()
            del Z
        so = qmlr.last_solve
        model = qmlr.Model(p, int(te.sizes().max()), U, signs, w.n_transform, b, w.sigma,
                           alpha.float().cpu().numpy())
        E, _ = model.predict(te.coords, te.elem, te.mol_ptr, forces=False)
        mae = float(np.mean(np.abs(E.cpu().numpy() - y_te)))
        model.close()
        pt = {"n_features": nf, "features_ms": ev[0].elapsed_time(ev[1]), "solve_ms": ev[1].elapsed_time(ev[2]),
              "train_s": ev[0].elapsed_time(ev[2]) / 1e3, "factor_ms": so.factor_ms, "refine_ms": so.refine_ms,
              "pcg_iters": it, "rel_resid": rel, "test_mae_eV": mae}
        print(json.dumps(pt), flush=True)
        pts.append(pt)
        del alpha
        torch.cuda.empty_cache()
    print(json.dumps({"nf_sweep": {
        "workload": f"qm9-shaped ({n_tr} training / {te.n_mol} held-out molecules)",
        "gram": gram_description()["text"], "shift": GRAM["shift"], "points": pts}}), flush=True)


def run_rff_sweep(args):
    """SORF against dense RFF (W = G / sigma) at equal feature counts on the
    MD17-shaped conformations (energies only: 800 for training, 200 held out):
    feature-map time and held-out MAE for N_F in {512, ..., 8192}. Prints one
    JSON line."""
    import torch
    from paper_2206_01580_gb300 import pipeline, qmlr, synth
    from paper_2206_01580_gb300.params import from_table

    torch.cuda.set_device(0)
    w = synth.workload(2)
    tr, te = w.mols.subset(range(800)), w.mols.subset(range(800, 1000))
    y = torch.as_tensor(w.energies[:800]).cuda()
    y_te = torch.as_tensor(w.energies[800:]).cuda()
    p = from_table(w.params_column, n2=w.n2, n3=w.n3)
    spec0 = pipeline.spec_from(p, w.d, w.signs, w.b, w.sigma)
    btr = pipeline.Batch.from_host(tr.coords, tr.elem, tr.mol_ptr)
    bte = pipeline.Batch.from_host(te.coords, te.elem, te.mol_ptr)
    rep, perm, offs = pipeline.representations(btr, spec0)
    U = pipeline.fit_pca(rep, perm, offs, spec0)
    x_tr = qmlr.project(rep, p.rep_dim, perm, offs, p.n_el, U)
    rep, perm, offs = pipeline.representations(bte, spec0)
    x_te = qmlr.project(rep, p.rep_dim, perm, offs, p.n_el, U)
    del rep
    factor = qmlr.FACTOR_MIXED if args.factor == "mixed" else qmlr.FACTOR_FP64

    def timed(fn):
        fn()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        out = fn()
        e1.record()
        torch.cuda.synchronize()
        return out, e0.elapsed_time(e1)

    def fit_mae(Z_tr, Z_te):
        alpha, it, rel = pipeline.solve(Z_tr, y, w.lam, GRAM["precision"], max_iter=args.pcg_iters,
                                        tol=args.pcg_tol, shift=GRAM["shift"], factor=factor,
                                        promote=GRAM["promote"], tile=GRAM["tile"])
        E = Z_te.double() @ alpha
        return float(torch.mean(torch.abs(E - y_te)).item()), it, rel

    pts = []
    for nf in (512, 1024, 2048, 4096, 8192):
        rng = synth.rng_for(2, 70 + nf // 512)
        signs, b = synth.sorf_draw(rng, nf, w.d, w.n_transform)
        bits = qmlr.pack_signs(signs)
        bt = torch.as_tensor(b.astype(np.float32)).cuda()
        Zs, ms_s = timed(lambda: qmlr.sorf(x_tr, btr.mol_ptr, bits, w.n_transform, bt, w.sigma, qmlr.SORF_PER_MOL))
        Zs_te = qmlr.sorf(x_te, bte.mol_ptr, bits, w.n_transform, bt, w.sigma, qmlr.SORF_PER_MOL)
        mae_s, it_s, _ = fit_mae(Zs, Zs_te)
        G, b2 = synth.rff_draw(rng, nf, w.d)
        Gt = torch.as_tensor(G.astype(np.float32)).cuda()
        bt2 = torch.as_tensor(b2.astype(np.float32)).cuda()
        Zr, ms_r = timed(lambda: qmlr.rff(x_tr, btr.mol_ptr, Gt, bt2, w.sigma, qmlr.SORF_PER_MOL))
        Zr_te = qmlr.rff(x_te, bte.mol_ptr, Gt, bt2, w.sigma, qmlr.SORF_PER_MOL)
        mae_r, it_r, _ = fit_mae(Zr, Zr_te)
        Zt, ms_t = timed(lambda: qmlr.rff_tc(x_tr, btr.mol_ptr, Gt, bt2, w.sigma, qmlr.SORF_PER_MOL))
        Zt_te = qmlr.rff_tc(x_te, bte.mol_ptr, Gt, bt2, w.sigma, qmlr.SORF_PER_MOL)
        mae_t, _, _ = fit_mae(Zt, Zt_te)
        pt = {"n_features": nf, "sorf_ms": ms_s, "rff_simt_ms": ms_r, "rff_tc_ms": ms_t,
              "sorf_test_mae_eV": mae_s, "rff_test_mae_eV": mae_r, "rff_tc_test_mae_eV": mae_t,
              "sorf_pcg_iters": it_s, "rff_pcg_iters": it_r}
        print(json.dumps(pt), flush=True)
        pts.append(pt)
    print(json.dumps({"rff_sweep": {
        "workload": "md17-shaped (800 training / 200 held-out conformations, energies only)",
        "sigma": w.sigma, "d": w.d, "n_transform": w.n_transform, "points": pts}}), flush=True)


def gram_description():
    """Kernel name, tensor-core products per Gram product, rate relative to BF16
    and a text description of the training step's Gram form."""
    prec, promote, tile = GRAM["precision"], GRAM["promote"], GRAM["tile"]
    S = {1: 2, 2: 3, 3: 1, 4: 1}[prec]
    f8 = prec == 4
    kahan = prec in (1, 2) and tile == 128
    acc = "whole K in TMEM" if promote == 0 else f"{promote} K block(s) per TMEM accumulation"
    sums = "FP32 Kahan register sums" if kahan else "FP32 register sums"
    kind = "e4m3 (per-feature scales)" if f8 else (f"{S}-way bf16 split" if S > 1 else "one-part bf16")
    products = {1: 3, 2: 6, 3: 1, 4: 1}[prec]
    return {"kernel": f"tc::gram_persist_kernel<{S}, {str(f8).lower()}, {tile}, {str(kahan).lower()}> "
                      f"({kind}, tcgen05, 128x{tile} tiles, one CTA per SM, wave-aligned loads)",
            "products": products, "rate": 2 if f8 else 1,
            "dtype": "e4m3" if f8 else (f"bf16 {S}-way split" if S > 1 else "bf16"),
            "text": f"{kind}, {products} tcgen05 product(s), {acc}, {sums}, 128x{tile} tiles"}


def main():
    args = parse()
    prec = GRAM_FORMS[args.gram_form]
    from paper_2206_01580_gb300 import pipeline
    p0, t0 = pipeline.DEFAULT_TC[prec]
    GRAM.update({"precision": prec, "promote": p0 if args.gram_promote is None else args.gram_promote,
                 "tile": t0 if args.gram_tile is None else args.gram_tile,
                 "shift": pipeline.DEFAULT_SHIFT[prec] if args.shift is None else -abs(args.shift)})
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.kernel_times:
        if rank == 0:
            run_kernel_times(args)
    elif args.feature_sweep:
        if rank == 0:
            run_feature_sweep(args)
    elif args.gram_sweep:
        if rank == 0:
            run_gram_sweep(args)
    elif args.nf_sweep:
        if rank == 0:
            run_nf_sweep(args)
    elif args.rff_sweep:
        if rank == 0:
            run_rff_sweep(args)
    else:
        run_ours(args, rank, world)


if __name__ == "__main__":
    main()

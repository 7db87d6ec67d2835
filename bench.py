#!/usr/bin/env python3
"""Throughput of the MC 2->2 collision term with symmetrical sampling + drift.

One step = one pass of the whole hot path on the workload: thermal masses,
drift (+ f for the lookups), collision sampling and deposition (FP32
integrand with float-float re-evaluation of ill-conditioned terms), moments.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl bz|reference]
                  [--workload gluon_bump|qgp|gluon_step|batch|tts|stability]

Default workload: the largest single-GPU configuration, pure gluons on a
16^3 periodic spatial grid (dx = 0.2 fm) times a 20^3 momentum grid on
[-2, 2) GeV, 256 samples per cell, 32.8 M phase-space cells.

Prints one JSON line (rank 0).  Metric: collision samples/s, a sample being
one (species, x cell, p cell, sample) anchor evaluated over all terms of its
species' equation, with cell-updates/s beside it.  The reference arm (--impl
reference) is the FP64 CPU oracle on a bounded sample of anchors of the same
workload.
"""
import argparse
import hashlib
import re
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "collision samples/s and cell-updates/s vs plain FP64 GPU path at equal MC error"
L2_FLUSH_BYTES = 256 << 20     # > 129 MB L2
# algorithmic FP32 operations (add, sub, mul, div, sqrt each 1) of the formula:
FLOP_PER_SAMPLE = 60           # jitter, k1_perp, k3, |p|^2, |k3|^2, P, a^2, b^2, bin of k3
FLOP_PER_TERM = 29             # Ep, E3, D, kappa, H, sqrt(H), Q, two root candidates
FLOP_PER_ROOT = 81             # validity, E1, E2, J, s, t, u, |M|^2, three bins, W, c~, weight


def workloads():
    from paper_1912_04457_gb300 import inputs as I
    return {"qgp": I.qgp_box, "gluon_step": I.gluon_step_box, "gluon_bump": I.gluon_bump_xp}


def describe(w):
    return {"workload": w.name, "species": w.nslots, "x_cells": w.nxc, "p_grid": list(w.np_),
            "L_GeV": w.L, "samples_per_cell": w.nsamples, "dt_fm": w.dt, "alpha_s": w.alpha_s,
            "anchors_per_step": w.nslots * w.nxc * w.npc, "l2": "flushed between timed steps",
            "initial_state": "synthetic closed form (seeded)"}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.lines = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
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
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for name, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        loaded = [s for s in sm if smax and s > 0.5 * max(smax)] or sm
        return {"sm_mhz": statistics.median(loaded) if loaded else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def source_hash():
    """Hash of the collision kernel's sources without comments and blank
    space, so that the committed ncu traffic is tied to the code it measured."""
    h = hashlib.sha256()
    for f in ("collide.cuh", "k_collide_f32.cu", "bz_internal.h"):
        src = open(os.path.join(ROOT, "paper_1912_04457_gb300", "csrc", f)).read()
        src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
        src = re.sub(r"//[^\n]*", " ", src)
        h.update(" ".join(src.split()).encode())
    return h.hexdigest()[:16]


def ncu_summary(workload):
    """The committed ncu counters of the collision kernel on this workload
    (DRAM bytes and executed FP32 flops per full launch), if they were taken
    on the current kernel source; else None."""
    path = os.path.join(ROOT, "profiles", "collide_%s_traffic.json" % workload)
    try:
        d = json.load(open(path))
    except (OSError, ValueError):
        return None
    if d.get("source_hash") != source_hash():
        return None
    return d


def term_counts(w):
    """Term evaluations of one step: every sample of every anchor times its equation's terms."""
    from paper_1912_04457_gb300 import inputs as I
    per_species = []
    for s in I.slots(w.species_mask):
        per_species.append(_nterms(s, w.species_mask))
    anchors_per_slot = w.nxc * w.npc
    return sum(per_species) * anchors_per_slot * w.nsamples


def _nterms(d, mask):
    """Number of terms of species d's equation whose four species are all active."""
    def active(*ss):
        return all(mask & (1 << s) for s in ss)
    n = 0
    if d == 0:
        n += active(0)
        for f in range(3):
            q, qb = 1 + f, 4 + f
            n += active(q, 0) + active(qb, 0) + active(q, qb)
    else:
        anti = d >= 4
        fa = (d - 1) % 3
        me, bar = (4 + fa, 1 + fa) if anti else (1 + fa, 4 + fa)
        n += active(me) + active(bar, me) + active(0, bar, me) + active(0, me)
        for fb in range(3):
            if fb == fa:
                continue
            Qb, QBb = (4 + fb, 1 + fb) if anti else (1 + fb, 4 + fb)
            n += active(Qb, me) + active(QBb, me) + active(Qb, QBb, bar, me)
    return n


def oracle_sample(w, target_s, step=0):
    """Times the oracle's step pieces on an anchor subset sized to ~target_s.
    Returns (samples/s, anchors, cores, seconds, accepted roots per term-eval)."""
    import numpy as np
    import oracle as O
    cfg = O.make_config(nx=w.nx, dx=w.dx, np_=w.np_, L=w.L, seed=w.seed,
                        species_mask=w.species_mask, alpha_s=w.alpha_s)
    st = w.state()
    total = st.size
    m2 = O.masses(cfg, st)
    stride = max(1, total // 64)
    t0 = time.perf_counter()
    r = O.collision(cfg, st, m2, w.nsamples, step=step, dt=w.dt, anchor_stride=stride,
                    want_audit=True)
    dt0 = time.perf_counter() - t0
    n0 = (total + stride - 1) // stride
    rate = n0 / max(dt0, 1e-6)
    n_target = max(n0, int(rate * target_s))
    stride = max(1, total // n_target)
    t0 = time.perf_counter()
    m2 = O.masses(cfg, st)
    r = O.collision(cfg, st, m2, w.nsamples, step=step, dt=w.dt, anchor_stride=stride,
                    want_audit=True)
    if w.nxc > 1:
        O.drift(cfg, st, m2, w.dt)
    O.moments(cfg, st, m2)
    secs = time.perf_counter() - t0
    anchors = (total + stride - 1) // stride
    terms = term_counts(w) * anchors / total
    roots_per_term = float(r["audit"][5]) / max(terms, 1)
    return anchors * w.nsamples / secs, anchors, O.num_threads(), secs, roots_per_term, stride


# ---------------------------------------------------------------------------
# Weak scaling over ranks (one GPU each): every rank runs its own box (the
# path shards into independent problems, so there is no data-path
# collective); only the timing is reduced.
# ---------------------------------------------------------------------------
def rank_seed(base_seed, rank):
    """Seed of a rank's own box: rank 0 keeps the workload's seed."""
    return base_seed + 1000 * rank


def max_over_ranks(t_local, world, device=None):
    """The slowest rank's time (seconds) of the timed region; the job is as
    fast as its slowest rank."""
    if world <= 1:
        return float(t_local)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(t_local)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank_step, steps, world, t_max):
    """Units all ranks processed per second of the slowest rank."""
    return units_per_rank_step * steps * world / t_max


def run_reference(args):
    """FP64 CPU oracle as the reference arm, on a bounded sample of anchors."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from oracle.build import build_oracle
    build_oracle()
    w = workloads()[args.workload]()
    per_step = []
    info = None
    for k in range(args.warmup + args.steps):
        rate, anchors, cores, secs, _, stride = oracle_sample(w, 2.0, step=k)
        if k >= args.warmup:
            per_step.append((anchors * w.nsamples, secs))
            info = (anchors, cores, stride)
    samples = sum(s for s, _ in per_step)
    secs = sum(t for _, t in per_step)
    value = samples / secs
    anchors, cores, stride = info
    line = {"metric": METRIC, "value": value, "unit": "samples/s", "impl": "reference",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * secs / len(per_step), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": describe(w),
            "cpu_baseline": {"value": value, "unit": "samples/s", "cores": cores, "kind": "oracle",
                             "sample": "every %d-th anchor (%d of %d) of one step per timed step, "
                                       "plus full-grid masses and moments" %
                                       (stride, anchors, w.nslots * w.nxc * w.npc)},
            "e2e": {"value": value, "unit": "samples/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_bz(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)

    from paper_1912_04457_gb300 import build as B
    B.build()
    from paper_1912_04457_gb300 import bz
    from paper_1912_04457_gb300 import inputs as I

    mk = workloads()[args.workload]
    kw = {"nsamples": args.nsamples} if args.nsamples else {}
    if args.nxs:
        kw["nxs"] = args.nxs
    w = mk(seed=rank_seed(mk().seed, rank), **kw) if world > 1 else mk(**kw)
    prec = bz.PREC_F32 if args.prec == "f32" else bz.PREC_F64
    h = bz.Handle(nx=w.nx, dx=w.dx, np_=w.np_, L=w.L, seed=w.seed, species_mask=w.species_mask,
                  alpha_s=w.alpha_s)
    host_state = torch.from_numpy(w.state().reshape(-1)).pin_memory()
    state = host_state.cuda()
    mom = torch.empty(w.nxc * w.nslots * 5, dtype=torch.float64, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()

    for k in range(args.warmup):
        h.step(state, w.dt, 1, w.nsamples, prec, step0=k, moments_out=mom)
    barrier()

    clocks = ClockSampler(local)
    clocks.start()
    h.profile(True)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    wall0 = time.perf_counter()
    for k in range(args.steps):
        flush.zero_()
        ev[k][0].record(stream)
        h.step(state, w.dt, 1, w.nsamples, prec, step0=args.warmup + k, moments_out=mom)
        ev[k][1].record(stream)
    barrier()
    wall = time.perf_counter() - wall0
    mom_last = mom.cpu().numpy().reshape(w.nxc, w.nslots, 5).copy()
    number_conserved = int(state.sum().item()) == int(host_state.sum().item())
    prof = h.profile_read()
    h.profile(False)
    clk = clocks.stop()
    t_steps = sum(a.elapsed_time(b) for a, b in ev) / 1e3
    t_max = max_over_ranks(t_steps, world, "cuda")

    anchors = w.nslots * w.nxc * w.npc
    samples_step = anchors * w.nsamples
    value = whole_job_rate(samples_step, args.steps, world, t_max)
    cell_updates = whole_job_rate(anchors, args.steps, world, t_max)

    # e2e through the public API with host buffers
    n_e2e = min(args.steps, 5)
    out_host = torch.empty_like(host_state).pin_memory()
    mom_host = torch.empty(mom.numel(), dtype=torch.float64).pin_memory()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k in range(n_e2e):
        state.copy_(host_state, non_blocking=True)
        h.step(state, w.dt, 1, w.nsamples, prec, step0=1000 + k, moments_out=mom)
        out_host.copy_(state, non_blocking=True)
        mom_host.copy_(mom, non_blocking=True)
    e1.record(stream)
    barrier()
    t_e2e = e0.elapsed_time(e1) / 1e3
    e2e_value = samples_step * n_e2e * world / t_e2e

    # energy balance of one more step (outside the timed region), Eq. (current
    # conservation): d_0 T^00 against S_ex^0 = (1/2) sum_a (dm_a^2/dt) int N_a f_a/E_a
    energy = None
    if rank == 0:
        mom_a = torch.empty_like(mom)
        h.step(state, w.dt, 1, w.nsamples, prec, step0=3000, moments_out=mom_a)
        m_prev = h.get_masses()
        f_n = state.clone()
        mom_b = torch.empty_like(mom)
        h.step(state, w.dt, 1, w.nsamples, prec, step0=3001, moments_out=mom_b)
        src = h.energy_source(f_n, w.dt, m_prev).view(w.nxc, w.nslots, 3)
        t_a = mom_a.view(w.nxc, w.nslots, 5)[:, :, 1].sum(1).mean().item()
        t_b = mom_b.view(w.nxc, w.nslots, 5)[:, :, 1].sum(1).mean().item()
        energy = {"dT00_dt": (t_b - t_a) / w.dt, "S_ex0": src[:, :, 1].sum(1).mean().item(),
                  "T00": t_b, "T_total_term": src[:, :, 2].sum(1).mean().item(),
                  "unit": "GeV^4 per fm/c (T00 and T_total_term: GeV^4), averaged over x cells",
                  "note": "one step of the FP32 path after the timed loop: the change of the kinetic energy "
                          "density against the mass-variation source; the collisions conserve energy up to "
                          "the binning of the legs, so the two agree up to that error"}
        del f_n, mom_a, mom_b, src

    # step loop of several steps per call: replayed step graphs against direct
    # launches (outside the timed region; launch-bound small boxes gain)
    step_loop = None
    if rank == 0 and 1e3 * t_max / args.steps < 5.0:
        loop = {}
        nloop = 10
        for mode in ("graph", "direct"):
            if mode == "direct":
                os.environ["BZ_STEP_GRAPH"] = "0"
            s_loop = state.clone()
            h.step(s_loop, w.dt, nloop, w.nsamples, prec, step0=4000)   # warm (captures the graph)
            barrier()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            h.step(s_loop, w.dt, nloop, w.nsamples, prec, step0=4000 + nloop)
            b.record(stream)
            barrier()
            loop[mode] = {"ms_per_step": a.elapsed_time(b) / nloop, "checksum": int(s_loop.sum().item())}
            os.environ.pop("BZ_STEP_GRAPH", None)
            del s_loop
        step_loop = {"steps_per_call": nloop, "graph": loop["graph"], "direct": loop["direct"],
                     "same_state": loop["graph"]["checksum"] == loop["direct"]["checksum"],
                     "note": "one bz_step call of 10 steps: the first step launched directly, then 2-step CUDA "
                             "graphs replayed (device-side step index), against every step launched directly "
                             "(BZ_STEP_GRAPH=0); not part of the timed loop, which calls one step at a time"}

    # streaming kernels of inhomogeneous grids against the HBM roofline, and the
    # cost of the optional force term (outside the timed region)
    transport = None
    if w.nxc > 1 and rank == 0:
        transport = transport_rooflines(h, w, state, mom, prof, args.steps, stream, barrier)

    result = None
    if rank == 0:
        coll_ms, coll_n = prof["collide"]
        drift_kernels = 2 if w.nxc > 1 else 1   # k_mass_table + the drift kernel on inhomogeneous grids
        nsm_ = torch.cuda.get_device_properties(local).multi_processor_count
        # k_moments + k_moments_finish when few (x cell, slot) rows are split into p-cell chunks
        mom_kernels = 2 if (w.nxc * w.nslots < 2 * nsm_ and w.npc // 1024 > 1) else 1
        launches = (2 * prof["masses"][1] + drift_kernels * prof["drift"][1] + prof["collide"][1]
                    + prof["fixup"][1] + mom_kernels * prof["moments"][1] + prof["convert"][1])
        # algorithmic work of one collision launch
        cpu_rate, cpu_anchors, cores, cpu_secs, roots_per_term, cpu_stride = (None,) * 6
        if not args.no_cpu_baseline and world == 1:
            cpu_rate, cpu_anchors, cores, cpu_secs, roots_per_term, cpu_stride = oracle_sample(w, 15.0)
        terms = term_counts(w)
        rpt = roots_per_term if roots_per_term is not None else 0.36
        flops = FLOP_PER_SAMPLE * samples_step + FLOP_PER_TERM * terms + FLOP_PER_ROOT * rpt * terms
        coll_s = coll_ms / 1e3 / max(coll_n, 1)
        achieved = flops / coll_s / 1e12
        nsm = torch.cuda.get_device_properties(local).multi_processor_count
        mhz = clk.get("sm_mhz") or 1447.0
        peak = nsm * 128 * 2 * mhz * 1e6 / 1e12
        summ = ncu_summary(args.workload) if not (args.nsamples or args.nxs) else None
        traffic = summ.get("dram_bytes_per_launch") if summ else None
        executed = None
        if summ and summ.get("fp32_flop_executed_per_launch"):
            ex = summ["fp32_flop_executed_per_launch"] / coll_s / 1e12
            executed = {"achieved": ex, "frac": ex / peak, "unit": "TFLOP/s",
                        "basis": "FP32 add + mul + 2 x FMA executed per launch (ncu instruction counters, "
                                 "committed summary) over the same event-timed launch duration"}
        issue = None
        if summ and summ.get("warp_inst_executed_per_launch"):
            # the kernel is bound by instruction issue: warp instructions per second against one
            # instruction per scheduler per clock (4 schedulers per SM)
            ia = summ["warp_inst_executed_per_launch"] / coll_s / 1e9
            ip = nsm * 4 * mhz * 1e6 / 1e9
            issue = {"achieved": ia, "peak": ip, "unit": "G warp instructions/s", "frac": ia / ip,
                     "basis": "warp instructions executed per launch (ncu, committed summary) over the "
                              "event-timed launch duration; peak = SMs x 4 schedulers x sampled SM clock"}

        # the plain FP64 GPU path on the same workload (one step, same samples)
        fp64 = None
        if not args.no_fp64:
            # one step of the FP64 path (bit-identical to the oracle) and one of the FP32 path from
            # the same state, masses and step index: time and deviation of the increments
            s0 = state.clone()
            m_saved = h.get_masses()
            warm = s0.clone()
            h.step(warm, w.dt, 1, w.nsamples, bz.PREC_F64, step0=2000)
            h.set_masses(m_saved)
            s64 = s0.clone()
            barrier()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            h.step(s64, w.dt, 1, w.nsamples, bz.PREC_F64, step0=2001, moments_out=mom)
            b.record(stream)
            barrier()
            t64 = a.elapsed_time(b) / 1e3
            # deviation of the FP32 step from the FP64 step on the same (23-bit) sample points
            h.set_masses(m_saved)
            h.set_uniform_bits(23)
            s64 = s0.clone()
            h.step(s64, w.dt, 1, w.nsamples, bz.PREC_F64, step0=2001)
            h.set_uniform_bits(32)
            h.set_masses(m_saved)
            s32 = s0.clone()
            h.step(s32, w.dt, 1, w.nsamples, bz.PREC_F32, step0=2001)
            d64 = (s64 - s0).double()
            d32 = (s32 - s0).double()
            err = float((d32 - d64).norm() / d64.norm())
            fp64 = {"samples_per_s": samples_step / t64, "ms_per_step": 1e3 * t64,
                    "speedup_at_equal_samples": (samples_step / t64) and value / (samples_step / t64),
                    "f32_step_rel_l2_vs_f64": err,
                    "note": "the FP64 path is bit-identical to the CPU oracle; on the same (23-bit) sample "
                            "points the FP32 step increment deviates from the FP64 one by "
                            "f32_step_rel_l2_vs_f64 (relative L2); both paths draw the same distribution of "
                            "samples, so equal samples means equal MC error"}
            del s0, warm, s64, s32, d64, d32

        result = {
            "metric": METRIC, "value": value, "unit": "samples/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if prec == bz.PREC_F32 else "f64", "data": "synthetic",
            "config": describe(w),
            "cell_updates_per_s": cell_updates,
            "term_evaluations_per_s": whole_job_rate(terms, args.steps, world, t_max),
            "accepted_roots_per_s": whole_job_rate(terms * rpt, args.steps, world, t_max),
            "wall_s_timed_loop": wall,
            "kernel_ms_per_step": {k: v[0] / max(args.steps, 1) for k, v in prof.items()},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "kernel": "k_collide_f32 (FP32 pipe)",
                         "executed": executed, "issue": issue,
                         "peak_basis": "%d SMs x 128 FP32 lanes x 2 flop (FMA) x %.0f MHz sampled "
                                       "median SM clock" % (nsm, mhz),
                         "work_basis": "%d flop/sample + %d flop/term + %d flop/accepted root, "
                                       "%.3f accepted roots per term evaluation (oracle audit)" %
                                       (FLOP_PER_SAMPLE, FLOP_PER_TERM, FLOP_PER_ROOT, rpt)},
            "cpu_baseline": None if cpu_rate is None else {
                "value": cpu_rate, "unit": "samples/s", "cores": cores, "kind": "oracle",
                "sample": "one step of the same workload on every %d-th anchor (%d anchors x %d "
                          "samples, %.1f s)" % (cpu_stride, cpu_anchors, w.nsamples, cpu_secs)},
            "e2e": {"value": e2e_value, "unit": "samples/s",
                    "h2d_bytes_per_step": host_state.numel() * 8,
                    "d2h_bytes_per_step": host_state.numel() * 8 + mom.numel() * 8},
            "gpu_launches": launches,
            "clocks": clk,
            "fp64_gpu_path": fp64,
            "transport": transport,
            "step_loop": step_loop,
            "physics": {
                "number_conserved_exactly": number_conserved,
                "species": {I.SPECIES[sp]: {"number_density_GeV3": float(mom_last[:, k, 0].mean()),
                                            "energy_density_GeV4": float(mom_last[:, k, 1].mean()),
                                            "momentum_density_GeV4": [float(mom_last[:, k, 2 + i].mean())
                                                                      for i in range(3)]}
                            for k, sp in enumerate(I.slots(w.species_mask))},
                "after_steps": args.warmup + args.steps, "dt_fm": w.dt,
                "energy_balance": energy,
            },
        }
        print(json.dumps(result), flush=True)
    h.close()
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def measured_hbm_gbs():
    """The machine's measured copy bandwidth, else the recipe's fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def transport_rooflines(h, w, state, mom, prof, steps, stream, barrier):
    """Drift (k_mass_table + drift kernel; algorithmic bytes 8 B read + 8 B
    write + 4 B f per cell), moments and thermal masses (8 B read per cell
    each) of the timed steps against the HBM peak, and the drift with the
    force term switched on, timed over separate calls."""
    import torch
    ncell = w.nslots * w.nxc * w.npc
    peak, basis = measured_hbm_gbs()
    out = {"hbm_peak_GBs": peak, "peak_basis": basis}
    for name, nbytes in (("drift", 20 * ncell), ("moments", 8 * ncell), ("masses", 8 * ncell)):
        ms = prof[name][0] / max(prof[name][1], 1)
        gbs = nbytes / (ms * 1e-3) / 1e9
        out[name] = {"ms": ms, "algorithmic_bytes": nbytes, "achieved_GBs": gbs, "frac": gbs / peak}
    nxt = torch.empty_like(state)
    reps = 10
    for force in (False, True):
        h.set_force_term(force)
        h.drift(state, nxt, w.dt)
        barrier()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            h.drift(state, nxt, w.dt)
        b.record(stream)
        barrier()
        out["drift_force_on_ms" if force else "drift_force_off_ms"] = a.elapsed_time(b) / reps
    h.set_force_term(False)
    out["force_note"] = ("bz_drift over the same state with the force term -div_p[(grad_x E) f] off and on "
                         "(not part of the timed step)")
    del nxt
    return out


def run_batch(args):
    """64 independent homogeneous boxes of ragged size in one persistent,
    graph-replayed launch per step (FP32 integrand, int64 deposits)."""
    import numpy as np
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_1912_04457_gb300 import build as B
    B.build()
    from paper_1912_04457_gb300 import bz
    from paper_1912_04457_gb300 import inputs as I

    boxes, states, dt, nsteps = I.batched_boxes(seed=rank_seed(5, rank))
    batch = bz.Batch(boxes)
    host = torch.from_numpy(np.concatenate([s.reshape(-1) for s in states])).pin_memory()
    state = host.cuda()
    mom = torch.empty(batch.nslots_total * 5, dtype=torch.float64, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    samples_step = sum(int(np.prod(b["np_"])) * bin(b["species_mask"]).count("1") * b["nsamples"]
                       for b in boxes)
    cells_step = batch.ncell

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()

    for k in range(args.warmup):
        batch.step(state, dt, 1, step0=k, moments_out=mom)
    barrier()
    clocks = ClockSampler(local)
    clocks.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    for k in range(args.steps):
        flush.zero_()
        ev[k][0].record(stream)
        batch.step(state, dt, 1, step0=args.warmup + k, moments_out=mom)
        ev[k][1].record(stream)
    barrier()
    clk = clocks.stop()
    t = max_over_ranks(sum(a.elapsed_time(b) for a, b in ev) / 1e3, world, "cuda")
    tun = batch.tuning()
    value = whole_job_rate(samples_step, args.steps, world, t)
    # e2e: host state in, state and moments out, every step
    out_host = torch.empty_like(host).pin_memory()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n_e2e = min(args.steps, 5)
    e0.record(stream)
    for k in range(n_e2e):
        state.copy_(host, non_blocking=True)
        batch.step(state, dt, 1, step0=500 + k, moments_out=mom)
        out_host.copy_(state, non_blocking=True)
    e1.record(stream)
    barrier()
    e2e = samples_step * n_e2e * world / (e0.elapsed_time(e1) / 1e3)
    if rank == 0:
        nsm = torch.cuda.get_device_properties(local).multi_processor_count
        mhz = clk.get("sm_mhz") or 1447.0
        peak = nsm * 128 * 2 * mhz * 1e6 / 1e12
        terms = sum(sum(_nterms(s, b["species_mask"]) for s in I.slots(b["species_mask"])) * int(np.prod(b["np_"]))
                    * b["nsamples"] for b in boxes)
        flops = FLOP_PER_SAMPLE * samples_step + FLOP_PER_TERM * terms + FLOP_PER_ROOT * 0.357 * terms
        achieved = flops / (tun["collide_ms"] / 1e3) / 1e12
        line = {
            "metric": METRIC, "value": value, "unit": "samples/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "batched_64_boxes_ragged", "boxes": len(boxes), "cells": cells_step,
                       "samples_per_step": samples_step, "l2": "flushed between timed steps",
                       "grids": sorted({b["np_"][0] for b in boxes}), "dt_fm": dt},
            "cell_updates_per_s": cells_step * args.steps * world / t,
            "tuning": tun,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "traffic": None,
                         "kernel": "k_collide_f32_batch (persistent, autotuned chunk/occupancy)",
                         "work_basis": "as the single-box line; collision time from the autotuner's events"},
            "cpu_baseline": None,
            "e2e": {"value": e2e, "unit": "samples/s", "h2d_bytes_per_step": host.numel() * 8,
                    "d2h_bytes_per_step": host.numel() * 8},
            "gpu_launches": None, "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    batch.close()
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def run_stability(args):
    """The stability comparison of Sec. III.A (Fig. 2): 40^3 gluons on
    [-2, 2) GeV, f uniform in [0, 1] (seeded), alpha_s = 0.3, 100 samples per
    cell, dt = 0.01 fm/c, the plain (own-cell) estimator on the FP64 path;
    the gluon number after one step over independent evaluations, with k2
    (the paper's choice) or k3 eliminated.  Prints one JSON report."""
    import numpy as np
    import torch
    torch.cuda.set_device(0)
    from paper_1912_04457_gb300 import build as B
    B.build()
    from paper_1912_04457_gb300 import bz
    from paper_1912_04457_gb300 import inputs as I
    n, L, N, dt, evals = 40, 2.0, 100, 0.01, 20
    st = I.encode(I.random_f((n, n, n), 1, 1, 11, 0.0, 1.0), 0x01)
    dev = torch.from_numpy(st.reshape(-1)).cuda()
    number0 = float(dev.double().sum().item())
    out = {"workload": "stability_gluon_40cube_N100", "evaluations": evals, "sampler": "plain (own cell)",
           "precision": "f64", "data": "synthetic: f uniform in [0, 1], seed 11"}
    for param, name in ((0, "k2_eliminated"), (1, "k3_eliminated")):
        numbers, ms = [], []
        for e in range(evals):
            h = bz.Handle(np_=(n, n, n), L=L, seed=500 + e, species_mask=0x01, alpha_s=0.3)
            h.set_parameterisation(param)
            A = torch.empty_like(dev)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            h.collision_term(dev, A, N, 0, dt, bz.PREC_F64, bz.SAMPLER_PLAIN)
            b.record()
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
            numbers.append((number0 + float(A.double().sum().item())) / number0)
            h.close()
        v = np.array(numbers)
        out[name] = {"relative_number_mean": float(v.mean()), "relative_number_std": float(v.std(ddof=1)),
                     "ms_per_evaluation_median": float(np.median(ms))}
    out["std_ratio_k3_over_k2"] = out["k3_eliminated"]["relative_number_std"] / out["k2_eliminated"]["relative_number_std"]
    print(json.dumps(out), flush=True)
    return 0


def run_tts(args):
    """Time to solution of the collision term at equal MC error on the 7-species
    32^3 box: FP64 uniform (symmetric and plain deposition) against FP32
    uniform and FP32 with the learned proposal, trained on records of the
    uniform sampler at t = 0, 0.25 and 0.5 fm/c.

    The MC error of an unbiased estimator A_N is its spread: eps(N)^2 =
    E|A_a - A_b|^2 / (2 |C|^2) over independent sample streams a, b, with |C|
    from the mean of 64 uniform estimates at N = 4096.  eps sqrt(N) is constant, so the
    samples needed for a target eps are N(eps) = (eps(N) sqrt(N) / eps)^2 and
    the time to solution is N(eps) times the measured time per sample.  The
    FP64 and FP32 kernels evaluate the same samples (deviation <= 2e-5 relative
    L2), so the FP64 paths take the FP32 error curves of the same sampler,
    checked at one N."""
    import numpy as np
    import torch
    torch.cuda.set_device(0)
    from paper_1912_04457_gb300 import build as B
    B.build()
    from paper_1912_04457_gb300 import bz
    from paper_1912_04457_gb300 import inputs as I

    w = I.qgp_box()
    anchors = w.nslots * w.nxc * w.npc
    h = bz.Handle(np_=w.np_, L=w.L, seed=w.seed, species_mask=w.species_mask, alpha_s=w.alpha_s)
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    st0 = torch.from_numpy(w.state().reshape(-1)).cuda()
    # states at t = 0, 0.25, 0.5 fm/c (50 steps of 0.005 fm/c each, FP32 symmetric)
    states, s = [st0.clone()], st0.clone()
    for k in range(2):
        h.step(s, w.dt, 50, w.nsamples, bz.PREC_F32, step0=50 * k)
        states.append(s.clone())
    torch.cuda.synchronize()

    # training records: 16 uniform samples per anchor at each time, w > 0 kept
    t0 = time.perf_counter()
    recs = []
    for i, st in enumerate(states):
        h.reset_masses()
        rec, n = h.record(st, args.rec_samples, step=1 << 20 | i, dt=w.dt, max_records=1 << 23)
        recs.append(rec[: n * bz.RECORD_BYTES].view(n, bz.RECORD_BYTES))
    rec = torch.cat(recs)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(17)
    rec = rec[torch.randperm(rec.shape[0], device="cuda", generator=gen)].contiguous().view(-1)
    nrec = rec.numel() // bz.RECORD_BYTES
    torch.cuda.synchronize()
    t_rec = time.perf_counter() - t0
    h.proposal_init(1)
    t0 = time.perf_counter()
    losses = h.proposal_train(rec, nrec, args.train_steps, batch=16384, lr=2e-3)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0

    def timed(fn, reps=3):
        fn()
        ts = []
        for _ in range(reps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b) / 1e3)
        return statistics.median(ts)

    t_infer = timed(h.proposal_infer)
    A = torch.empty_like(st0)

    def call(st, N, step, prec, sampler):
        h.reset_masses()
        h.collision_term(st, A, N, step=step, dt=w.dt, prec=prec, sampler=sampler)

    def estimates(st, N, prec, sampler, seeds, base):
        out = []
        for sd in range(seeds):
            call(st, N, base + sd, prec, sampler)
            out.append(A.to(torch.float64))
        return out

    def spread(outs):
        d2 = [float(((outs[i] - outs[j]) ** 2).sum()) for i in range(len(outs)) for j in range(i + 1, len(outs))]
        return (sum(d2) / len(d2) / 2.0) ** 0.5

    result = {"metric": "time to solution of the collision term at equal MC error (relative L2)",
              "workload": describe(w), "targets": [1e-2, 3e-3],
              "training": {"records": nrec, "record_samples_per_anchor": args.rec_samples,
                           "record_times_fm": [0.0, 0.25, 0.5], "record_s": t_rec,
                           "train_steps": args.train_steps, "batch": 16384, "train_s": t_train,
                           "loss_first": float(losses[:50].mean()), "loss_last": float(losses[-50:].mean()),
                           "infer_ms": 1e3 * t_infer}, "times": {}}
    Ns = [64, 128, 256, 512, 1024, 2048, 4096]
    seeds = 8
    for ti, st in ((0, states[0]), (2, states[2])):
        ref = torch.zeros_like(st0, dtype=torch.float64)
        for r in range(64):   # 64 independent N = 4096 estimates = one at N = 262144
            call(st, 4096, 1 << 16 | r, bz.PREC_F32, bz.SAMPLER_SYMMETRIC)
            ref += A.to(torch.float64)
        ref /= 64.0
        cnorm = float(ref.norm())
        paths, means = {}, {}
        samplers = (("f32_symmetric", bz.SAMPLER_SYMMETRIC), ("f32_learned", bz.SAMPLER_LEARNED),
                    ("f32_plain", bz.SAMPLER_PLAIN))
        for name, smp in samplers:
            eps = {}
            for N in (Ns if ti == 0 else [1024]):
                outs = estimates(st, N, bz.PREC_F32, smp, seeds, 100 + 10 * N)
                eps[N] = spread(outs) / cnorm
                if N == max(eps):
                    means[name] = sum(outs) / len(outs)
            tN = timed(lambda: call(st, 1024, 3, bz.PREC_F32, smp))
            if smp == bz.SAMPLER_LEARNED:
                tN += t_infer
            paths[name] = {"eps": eps, "eps_sqrtN": statistics.median(e * N ** 0.5 for N, e in eps.items()),
                           "s_per_sample": tN / (anchors * 1024)}
        for name, smp, src in (("f64_symmetric", bz.SAMPLER_SYMMETRIC, "f32_symmetric"),
                               ("f64_plain", bz.SAMPLER_PLAIN, "f32_plain")):
            e64 = spread(estimates(st, 64, bz.PREC_F64, smp, 4, 5000)) / cnorm
            t64 = timed(lambda: call(st, 64, 3, bz.PREC_F64, smp), reps=2)
            paths[name] = {"eps_check_N64": e64, "eps": paths[src]["eps"], "eps_sqrtN": paths[src]["eps_sqrtN"],
                           "s_per_sample": t64 / (anchors * 64)}
        for p in paths.values():
            p["tts_s"] = {str(e): p["s_per_sample"] * anchors * (p["eps_sqrtN"] / e) ** 2
                          for e in result["targets"]}
        # speedup at equal error, N by N: (eps_base / eps_path)^2 x (t_base / t_path)
        base = paths["f64_symmetric"]
        for p in paths.values():
            r = [(base["eps"][N] / p["eps"][N]) ** 2 * base["s_per_sample"] / p["s_per_sample"] for N in p["eps"]]
            p["speedup_vs_f64_symmetric"] = {"min_over_N": min(r), "median_over_N": statistics.median(r)}
        # unbiasedness of the learned estimator against the reference
        nl = max(paths["f32_learned"]["eps"])
        dev = float((means["f32_learned"] - ref).norm()) / cnorm
        expect = (paths["f32_learned"]["eps"][nl] ** 2 / seeds
                  + paths["f32_symmetric"]["eps"][max(paths["f32_symmetric"]["eps"])] ** 2
                  * max(paths["f32_symmetric"]["eps"]) / (64 * 4096)) ** 0.5
        result["times"]["t=%.2f fm" % (0.25 * ti)] = {
            "C_norm": cnorm, "paths": paths,
            "learned_mean_vs_reference": {"rel_l2": dev, "expected_from_spread": expect, "N": nl, "seeds": seeds}}
    print(json.dumps(result), flush=True)
    h.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="bz", choices=["bz", "reference"])
    ap.add_argument("--workload", default="gluon_bump",
                    choices=["qgp", "gluon_step", "gluon_bump", "batch", "tts", "stability"])
    ap.add_argument("--prec", default="f32", choices=["f32", "f64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--nsamples", type=int, default=0, help="override samples per cell (small profiling cases)")
    ap.add_argument("--nxs", type=int, default=0,
                    help="gluon_bump: spatial cells per axis (small profiling cases of the same box)")
    ap.add_argument("--rec-samples", type=int, default=16, help="tts: uniform samples per anchor recorded")
    ap.add_argument("--train-steps", type=int, default=3000, help="tts: Adam steps")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch":
        return run_batch(args)
    if args.workload == "tts":
        return run_tts(args)
    if args.workload == "stability":
        return run_stability(args)
    return run_bz(args)


if __name__ == "__main__":
    sys.exit(main())

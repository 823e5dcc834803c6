"""Benchmark of the single-pulse search hot path on one GB300 (or N replicas).

Workload (the full-band plain search): 4096 channels 1000-1500 MHz, tsamp
49.152 us, 2^18 uint8 samples of N(128,12) noise with 20 injected dispersed
pulses (DM 50-1000, width 0.2-10 ms, S/N 6-30), DM trials 0..1000 step 1,
boxcar widths 1..256 (powers of two), threshold S/N 8.

A step is one pass of the device path: dedispersion -> row sums -> boxcar S/N
-> candidate compaction, on inputs already resident in HBM (`value`).  The
e2e figure runs the same search through the host-buffer entry point af_search
(pinned host input copied in, candidates copied out and clustered on the host).

metric: DM-trial x channel x output-sample additions per second (the brute-force
work ndm*nchan*nout), plus the real-time factor R = nout*tsamp / kernel time.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
For N > 1 launch with torch.distributed.run; every rank searches its own beam
(same workload shape, different seed): weak scaling, no data-path collective.
"""
import argparse
import gc
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "DM-trial·chan·samples/s, realtime factor, p99 chunk latency at equal recall"
UNIT = "DM-trial·chan·samples/s"
WORKLOAD = ("plain search, full band: 4096 ch 1000-1500 MHz, tsamp 49.152 us, 2^18 samples uint8 "
            "N(128,12) + 20 injected pulses DM 50-1000 width 0.2-10 ms S/N 6-30; DMs 0-1000 step 1; "
            "boxcar 1..256 (powers of two); threshold 8")
NCHAN, F_LO, F_HI, TSAMP, NSAMP = 4096, 1000.0, 1500.0, 49.152e-6, 1 << 18
DMS = np.arange(0.0, 1001.0, 1.0)
WIDTHS = [1, 2, 4, 8, 16, 32, 64, 128, 256]
THRESH = 8.0
CAP = 1 << 20
SM_MAX_MHZ_FALLBACK = 2070.0


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def make_input(seed, delays_fn):
    """Noise + 20 pulses; the pulses' per-channel start samples come from
    delays_fn(dm_list) -> int [n][nchan] (the library's plan on the GPU arm)."""
    from paper_2511_02328_gb300 import synth
    pp = synth.pulse_params(20, seed + 1000, (50.0, 1000.0), (0.2e-3, 10e-3), (6.0, 30.0),
                            (0.5, (NSAMP - 50000) * TSAMP - 0.5), 0.45, TSAMP)
    D = delays_fn([p["dm"] for p in pp])
    pulses = [synth.Pulse(p["t0"] + D[i].astype(np.int64), p["width"],
                          synth.pulse_amplitude(p["snr"], NCHAN, p["width"])) for i, p in enumerate(pp)]
    return synth.filterbank(NCHAN, NSAMP, seed=seed, pulses=pulses), pp


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.rows = []
        self.proc = None
        self.active = False
        self.lock = threading.Lock()

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu_id), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.th = threading.Thread(target=self._read, daemon=True)
        self.th.start()

    def _read(self):
        for line in self.proc.stdout:
            with self.lock:
                if self.active:
                    self.rows.append([x.strip() for x in line.split(",")])

    def mark(self, on):
        with self.lock:
            self.active = on

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[0]))
                mx.append(float(r[1]))
            except Exception:
                continue
            for n, v in zip(names, r[4:8]):
                if v.strip().lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup(n):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world != n:
        raise SystemExit("--gpus %d but WORLD_SIZE=%d" % (n, world))
    return rank, world, local


def beam_seed(rank):
    """Input seed of a replica: every rank searches its own beam."""
    return 1 + 7919 * rank


def max_over_ranks(v, dist, dev):
    """The slowest rank's time (replicas: the job ends when the last one does)."""
    if dist is None:
        return float(v)
    import torch
    t = torch.tensor([float(v)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(world, work_per_rank, seconds):
    """Whole-job rate of N replicas: the units all ranks processed over the slowest time."""
    return world * work_per_rank / seconds


def oracle_cflags():
    from oracle.build import CFLAGS
    return [f for f in CFLAGS if f not in ("-fPIC", "-shared")]


def cpu_oracle_sample(x, D, rows, nout):
    """Time the oracle (as it stands) on a bounded sample: the listed DM rows of
    the same workload, dedispersion + S/N + candidates."""
    import oracle
    t0 = time.perf_counter()
    Y = oracle.dedisperse(x, D[rows], nout=nout)
    snr, bw = oracle.boxcar_snr(Y, WIDTHS)
    oracle.peaks(snr, bw, WIDTHS, THRESH)
    dt = time.perf_counter() - t0
    work = len(rows) * NCHAN * int(nout)
    return work / dt, dt


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    cores = oracle.threads()
    x, _ = make_input(12345, lambda dms: oracle.delay_table(NCHAN, F_LO, F_HI, TSAMP, dms))
    D = oracle.delay_table(NCHAN, F_LO, F_HI, TSAMP, DMS)
    nout = NSAMP - int(D.max())
    rows_per_step = 4 * cores          # the oracle runs one DM row per thread at a time
    rng = np.random.default_rng(5)
    for _ in range(args.warmup):
        cpu_oracle_sample(x, D, rng.choice(len(DMS), 2, replace=False), nout)
    times = []
    for _ in range(args.steps):
        rows = np.sort(rng.choice(len(DMS), rows_per_step, replace=False))
        _, dt = cpu_oracle_sample(x, D, rows, nout)
        times.append(dt)
    total = sum(times)
    value = args.steps * rows_per_step * NCHAN * nout / total
    sample = ("%d random DM rows of 1001 per step (full nout=%d, all 4096 channels): dedispersion + S/N + peaks; "
              "%d OpenMP threads, gcc %s" % (rows_per_step, nout, cores, " ".join(oracle_cflags())))
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic", "config": {"workload": WORKLOAD, "sample": sample},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


STREAM_WORKLOAD = ("streaming: 19 beams, 4096 ch x 49.152 us uint8, windows of 2^18 samples overlapping by the "
                   "DM-2000 delay, DMs 0-2000 step 1, boxcar 1..256, candidates at S/N 6; independent synthetic data per "
                   "beam with two dispersed pulses per hop (DM 50-1950, 0.2-10 ms, S/N 6-30) and RFI (two narrowband "
                   "channels, zero-DM bursts, drifting tones); every cluster classified inline by the trained CNN")
STREAM_CKPT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "paper_2511_02328_gb300", "data",
                           "stream_cnn_4096ch.ckpt")
STREAM_THRESH = 6.0


SB_N0, SB_NSUB = 8, 64
# DRAM read + write bytes of one stage-2 group-row tile launch (k_pair_tile) on this workload, from an ncu
# capture of the same kernel (dram__bytes_read.sum + dram__bytes_write.sum); None until captured, and reset
# to None whenever the kernel changes
PAIR_TILE_TRAFFIC = {   # keyed by channels per row: (bytes per launch, basis), from a capture of the current kernel
    3: (3.64e10, "ncu dram__bytes read+write of k_pair_tile<15,3> on rows of 3 channels at 2^16 samples (3.26 GB, "
                 "19 output tiles), scaled by the output tiles to this 2^18-sample launch (212 tiles)"),
}


def match_pulses(cands, pulses, dms):
    """Best S/N of a candidate within |dDM| < 20 and |dTOA| < 0.2 s of each
    injected pulse (the paper's matching rule, Sec. 4.2); NaN if none."""
    out = []
    for p in pulses:
        ok = (np.abs(dms[cands["dm_idx"]] - p["dm"]) < 20.0) & \
             (np.abs(cands["abs_sample"].astype(np.float64) - p["t0"]) * TSAMP < 0.2)
        out.append(float(cands["snr"][ok].max()) if ok.any() else float("nan"))
    return np.array(out)


def run_subband(args, dev, x, x_host, pulses, brute, ms_brute, stream, n0=None, nsub=None):
    """Two-stage subband dedispersion (Sec. 2.3) of the same input: device time
    of af_dedisperse, the equivalent brute-force rate, and the S/N kept on the
    injected pulses against the brute-force plane (same boxcar and threshold)."""
    import torch
    from paper_2511_02328_gb300 import _lib
    from paper_2511_02328_gb300.search import Plan
    n0 = SB_N0 if n0 is None else n0
    nsub = SB_NSUB if nsub is None else nsub
    sbp = Plan(NCHAN, F_LO, F_HI, TSAMP, DMS, subband=dict(n0=n0, nsub=nsub, fs_mode=_lib.AF_FS_INVSQ,
                                                           block_len=NSAMP))
    info = sbp.subband_info()
    nout = sbp.nout(NSAMP)
    sp = stream.cuda_stream
    plane = torch.empty((sbp.ndm, nout), dtype=torch.int32, device=dev)
    stats = torch.empty((sbp.ndm, 2), dtype=torch.int64, device=dev)
    for _ in range(args.warmup):
        _lib.af_dedisperse(sbp.handle, x.data_ptr(), NSAMP, plane.data_ptr(), stats.data_ptr(), sp)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for i in range(args.steps):
        ev[i][0].record(stream)
        _lib.af_dedisperse(sbp.handle, x.data_ptr(), NSAMP, plane.data_ptr(), stats.data_ptr(), sp)
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    _lib.af_plan_check(sbp.handle)
    ms = float(np.mean([a.elapsed_time(b) for a, b in ev]))
    launches = 2 * ((nout + info["block_len"] - 1) // info["block_len"])

    # S/N on the injected pulses, subband vs brute force
    found = {}
    for name, pl in (("subband", sbp), ("brute", brute)):
        _lib.af_search_reserve(pl.handle, NSAMP, CAP)
        c, _ = _lib.af_search(pl.handle, x_host, NSAMP, WIDTHS, THRESH, CAP, sp)
        found[name] = match_pulses(c, pulses, DMS)
    both = np.isfinite(found["subband"]) & np.isfinite(found["brute"])
    ratio = found["subband"][both] / found["brute"][both]
    work = float(sbp.ndm) * NCHAN * nout
    stage1 = float(info["ncoarse"]) * NCHAN * (nout + int(info["R"].max()))
    stage2 = float(sbp.ndm) * nsub * nout
    res = {
        "workload": "the same input, two-stage subband dedispersion: n0=%d fine DMs per coarse DM, %d subbands of "
                    "%d channels, 1/f^2-weighted centres, one time block" % (n0, nsub, NCHAN // nsub),
        "n0": n0, "nsub": nsub,
        "ms": ms, "effective_rate": work / (ms * 1e-3), "unit": UNIT, "speedup_vs_brute": ms_brute / ms,
        "block_len": info["block_len"],
        "realtime_factor": nout * TSAMP / (ms * 1e-3), "launches": launches,
        "adds_stage1": stage1, "adds_stage2": stage2, "adds_vs_brute": (stage1 + stage2) / work,
        "pulses_found": {"subband": int(np.isfinite(found["subband"]).sum()),
                         "brute": int(np.isfinite(found["brute"]).sum()), "injected": len(pulses)},
        "snr_ratio_vs_brute": {"mean": float(ratio.mean()) if ratio.size else None,
                               "min": float(ratio.min()) if ratio.size else None},
    }
    sbp.close()
    return res


def run_prep(args, dev, x, plane, snr, bw, ms_brute, stream):
    """Preprocessing and normalisation steps around the dedispersion on the same
    input and plane: zero-DM filter, square-law downsampling by 8, median/MAD
    row statistics and the robust S/N, and the L / H halves of the multi-band
    search (Sec. 2.1, 2.2).  Device times (CUDA events, mean of --steps) and
    HBM rates of algorithmic bytes."""
    import torch
    from paper_2511_02328_gb300 import _lib
    from paper_2511_02328_gb300.search import Plan
    sp = stream.cuda_stream
    hbm_peak = float(peaks().get("hbm_gbs", 6800.0))
    nout = plane.shape[1]
    ndm = plane.shape[0]
    y = torch.empty_like(x)
    ds = torch.empty((NCHAN, (NSAMP + 7) // 8), dtype=torch.uint8, device=dev)
    rob = torch.empty((ndm, 2), dtype=torch.int64, device=dev)
    ns_grid = int(np.ceil(0.5 / TSAMP))                 # 0.5 s slices (the paper's T_grid)
    S_grid = -(-nout // ns_grid)
    gimg = torch.empty((S_grid, 512, 512), dtype=torch.uint8, device=dev)
    gwork = torch.empty((S_grid, 2), dtype=torch.int64, device=dev)
    halves = {name: Plan(NCHAN, F_LO, F_HI, TSAMP, DMS, channels=rng)
              for name, rng in (("L", (0, NCHAN // 2)), ("H", (NCHAN // 2, NCHAN)))}
    hplanes = {k: torch.empty((ndm, v.nout(NSAMP)), dtype=torch.int32, device=dev) for k, v in halves.items()}
    for v in halves.values():
        _lib.af_dedisperse_reserve(v.handle, NSAMP)
    jobs = {
        "zerodm": (lambda: _lib.af_zerodm(x.data_ptr(), NCHAN, NSAMP, y.data_ptr(), sp), 2.0 * NCHAN * NSAMP),
        "downsample_8": (lambda: _lib.af_downsample(x.data_ptr(), NCHAN, NSAMP, 8, ds.data_ptr(), sp),
                         NCHAN * NSAMP * (1 + 1 / 8)),
        "rowstats_robust": (lambda: _lib.af_rowstats_robust(halves["L"].handle, plane.data_ptr(), nout,
                                                            rob.data_ptr(), sp), 4.0 * ndm * nout),
        "boxcar_robust": (lambda: _lib.af_boxcar_snr_robust(halves["L"].handle, plane.data_ptr(), nout,
                                                            rob.data_ptr(), WIDTHS, snr.data_ptr(), bw.data_ptr(),
                                                            sp), 9.0 * ndm * nout),
        "grid_512": (lambda: _lib.af_grid(plane.data_ptr(), ndm, nout, ns_grid, 512, gimg.data_ptr(),
                                          gwork.data_ptr(), sp), 4.0 * ndm * nout + S_grid * 512 * 512),
        "dedisperse_L": (lambda: _lib.af_dedisperse(halves["L"].handle, x.data_ptr(), NSAMP, hplanes["L"].data_ptr(),
                                                    0, sp), None),
        "dedisperse_H": (lambda: _lib.af_dedisperse(halves["H"].handle, x[NCHAN // 2:].data_ptr(), NSAMP,
                                                    hplanes["H"].data_ptr(), 0, sp), None),
    }
    res = {}
    for name, (fn, nbytes) in jobs.items():
        for _ in range(3):
            fn()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        for a, b in ev:
            a.record(stream)
            fn()
            b.record(stream)
        torch.cuda.synchronize()
        ms = float(np.mean([a.elapsed_time(b) for a, b in ev]))
        r = {"ms": ms}
        if nbytes is not None:
            gbs = nbytes / (ms * 1e-3) / 1e9
            r.update({"hbm_gbs": gbs, "hbm_frac": gbs / hbm_peak})
        res[name] = r
    res["multiband_FLH_vs_F"] = (ms_brute + res["dedisperse_L"]["ms"] + res["dedisperse_H"]["ms"]) / ms_brute
    res["note"] = ("algorithmic bytes: zero-DM reads and writes the input once; downsampling reads it once and "
                   "writes 1/8; median/MAD reads the plane once (the kernel makes 3 passes on noise-like rows); "
                   "the robust boxcar reads the plane and writes S/N + width (4 + 4 + 1 bytes per output); gridding "
                   "reads the plane "
                   "once (the kernel makes 2 passes) into 0.5 s slices of 512 x 512 (area path); HBM peak of "
                   "measured")
    for v in halves.values():
        v.close()
    return res


def run_batch(args, dev, stream):
    """The multi-beam batch (pattern 2): 19 beams of uneven channel count, DM
    range and length (workloads.multibeam: 10.7 GB of input, 1.07e13
    DM-trial·chan·samples), each with 5 injected pulses, searched in one
    persistent dedispersion launch + per-beam S/N and candidates, replayed as
    a CUDA graph with the autotuned tile shape; compared with the same beams
    searched one plan after another on the same stream (per-beam launches)."""
    import torch
    from paper_2511_02328_gb300 import _lib, synth, workloads
    from paper_2511_02328_gb300.search import Plan

    def dmax_of(nchan, f_lo, f_hi, tsamp, dm):
        q = Plan(nchan, f_lo, f_hi, tsamp, [dm])
        d = q.dmax
        q.close()
        return d

    beams = workloads.multibeam(19, dmax_of)
    xs, descs, work = [], [], 0.0
    for b, bm in enumerate(beams):
        q = Plan(bm["nchan"], bm["f_lo"], bm["f_hi"], bm["tsamp"], bm["dm_list"])
        nout = q.nout(bm["nsamp"])
        work += float(q.ndm) * bm["nchan"] * nout
        pp = synth.pulse_params(5, 5000 + b, (0.1 * bm["dm_list"][-1], 0.9 * bm["dm_list"][-1]), (0.5e-3, 5e-3),
                                (8.0, 20.0), (0.2, nout * bm["tsamp"] - 0.2), 0.1, bm["tsamp"])
        D = Plan(bm["nchan"], bm["f_lo"], bm["f_hi"], bm["tsamp"], [p_["dm"] for p_ in pp]).delays()
        pulses = [synth.Pulse(p_["t0"] + D[i].astype(np.int64), p_["width"],
                              synth.pulse_amplitude(p_["snr"], bm["nchan"], p_["width"])) for i, p_ in enumerate(pp)]
        x = synth.filterbank_torch(bm["nchan"], bm["nsamp"], seed=6000 + b, pulses=pulses, device=dev)
        xs.append(x)
        descs.append(dict(nchan=bm["nchan"], f_lo=bm["f_lo"], f_hi=bm["f_hi"], tsamp=bm["tsamp"],
                          dm_list=bm["dm_list"], d_in=x.data_ptr(), nsamp=bm["nsamp"], widths=bm["widths"],
                          thresh=bm["thresh"], cap=1 << 16))
        q.close()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    batch = _lib.af_batch_build(descs)
    build_s = time.perf_counter() - t0
    nw, m, tuned_ms, cached = _lib.af_batch_shape(batch)
    tuning = _lib.af_batch_tuning(batch)
    sp = stream.cuda_stream
    steps = max(1, min(args.steps, 5))

    def timed(fn, n):
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        a, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(n):
            fn()
        b_.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b_) / n

    ms_batch = timed(lambda: _lib.af_batch_run(batch, sp), steps)
    ncand = sum(_lib.af_batch_candidates(batch, i, 1 << 16)[1] for i in range(len(beams)))

    # the same searches one plan at a time, writing into the batch's buffers (the channel tile kernel, the
    # batch's own kernel family: 19 group-row buffers would not fit the device)
    plans, bufs = [], []
    for i, bm in enumerate(beams):
        plans.append(Plan(bm["nchan"], bm["f_lo"], bm["f_hi"], bm["tsamp"], bm["dm_list"]))
        bufs.append(_lib.af_batch_buffers(batch, i))
    cnt = torch.empty(1, dtype=torch.int32, device=dev)
    cands = torch.empty((1 << 16, 24), dtype=torch.uint8, device=dev)

    def one_by_one():
        for q, bm, (pl, sn, bw_, nout), x in zip(plans, beams, bufs, xs):
            _lib.af_dedisperse(q.handle, x.data_ptr(), bm["nsamp"], pl, 0, sp)
            _lib.af_boxcar_snr(q.handle, pl, nout, 0, bm["widths"], sn, bw_, sp)
            _lib.af_candidates(q.handle, sn, bw_, nout, bm["widths"], bm["thresh"], 0, cands.data_ptr(), 1 << 16,
                               cnt.data_ptr(), sp)

    ms_sep = timed(one_by_one, steps)
    for q in plans:
        q.close()
    _lib.af_batch_destroy(batch)
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_max = float(peaks().get("sm_max_mhz", SM_MAX_MHZ_FALLBACK))
    alu_peak = nsm * 128 * sm_max * 1e6
    kinds = {0: "persistent channel tiles", 1: "beam after beam (group rows, no graph)",
             2: "persistent group rows"}
    beam_by_beam = [t["ms"] for t in tuning if t["kind"] == 1]
    strategy = "persistent group rows" if m < 0 else "beam after beam" if m == 0 else "persistent channel tiles"
    return {
        "workload": "19 beams: nchan 1024/2048/4096, tsamp 49.152 us x 4096/nchan, DM max 500-2000 step 0.5-2, "
                    "2^16-2^19 samples (>= 2 Dmax), widths 1..256, threshold 8, 5 pulses per beam",
        "input_gb": sum(x.numel() for x in xs) / 1e9, "work": work, "ms_per_batch": ms_batch,
        "rate": work / (ms_batch * 1e-3), "unit": UNIT, "strategy": strategy, "shape": [nw, m],
        "autotune_ms": tuned_ms, "autotune_cached": bool(cached),
        "candidates_timed": [dict(t, name=kinds[t["kind"]]) for t in tuning],
        "speedup_vs_beam_by_beam": (beam_by_beam[0] / tuned_ms) if beam_by_beam and tuned_ms > 0 else None,
        "ms_one_plan_at_a_time_tile_kernel": ms_sep, "speedup_vs_one_plan_at_a_time_tile_kernel": ms_sep / ms_batch,
        "build_s": build_s, "candidates": int(ncand), "steps": steps,
        "note": "ms_per_batch = one CUDA graph replay: the dedispersion of all beams by the autotuned strategy plus "
                "every beam's S/N and candidates; candidates_timed = the autotuner's dedispersion-only times (ms) of "
                "each strategy on this batch (kind 1, beam after beam on group rows without a graph, is the fair "
                "baseline: speedup_vs_beam_by_beam = its time / the winner's); one_plan_at_a_time runs the channel "
                "tile kernel per beam with its S/N and candidates",
    }


CNN_FWD_FLOP = 2 * (64 * 64 * 16 * 2 * 9 + 32 * 32 * 32 * 16 * 9 + 16 * 16 * 64 * 32 * 9 + 64 * 2)


def run_classifier(args, dev, x, plan, stream):
    """The candidate classifier (pattern 4) on the benchmark input: cut-outs of
    256 candidates + CNN forward (af_classify), forward alone, and one training
    step (forward + backward + Adam) on a batch of 256; achieved TFLOP/s of the
    convolutions against the measured bf16 peak."""
    import torch
    from paper_2511_02328_gb300 import _lib
    sp = stream.cuda_stream
    n = 256
    nout = plan.nout(NSAMP)
    plane = torch.empty((plan.ndm, nout), dtype=torch.int32, device=dev)
    plan.dedisperse(x, plane=plane, stream=stream)
    rng = np.random.default_rng(4)
    c = np.zeros(n, dtype=_lib.CAND_DTYPE)
    c["dm_idx"] = rng.integers(0, plan.ndm, n)
    c["t"] = rng.integers(0, nout, n)
    c["width"] = 2 ** rng.integers(0, 9, n)
    c["abs_sample"] = c["t"]
    cands = torch.from_numpy(c.view(np.uint8).reshape(n, 24)).to(dev)
    xin = torch.empty((n, 64, 64, 2), dtype=torch.bfloat16, device=dev)
    y = torch.from_numpy(rng.integers(0, 2, n).astype(np.int32)).to(dev)
    prob = torch.empty(n, dtype=torch.float32, device=dev)
    loss = torch.empty(1, dtype=torch.float32, device=dev)
    model = _lib.af_model_create(n, 7)
    _lib.af_cutouts(plan.handle, x.data_ptr(), NSAMP, plane.data_ptr(), nout, cands.data_ptr(), n, xin.data_ptr(), sp)

    def timed(fn, k):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(k):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / k

    k = max(3, args.steps)
    ms_classify = timed(lambda: _lib.af_classify(model, plan.handle, x.data_ptr(), NSAMP, plane.data_ptr(), nout,
                                                 cands.data_ptr(), n, prob.data_ptr(), sp), k)
    ms_fwd = timed(lambda: _lib.af_model_forward(model, xin.data_ptr(), n, 0, prob.data_ptr(), sp), k)
    ms_train = timed(lambda: _lib.af_train_step(model, xin.data_ptr(), y.data_ptr(), n, 1e-3, loss.data_ptr(), sp), k)
    _lib.af_model_destroy(model)
    # the fused one-kernel network on the same batch (the library takes it below 256 images), forced
    os.environ["AFGB_CNN_UMMA_MIN"] = str(1 << 30)
    mfu = _lib.af_model_create(n, 7)
    ms_fwd_fused = timed(lambda: _lib.af_model_forward(mfu, xin.data_ptr(), n, 0, prob.data_ptr(), sp), k)
    _lib.af_model_destroy(mfu)
    # the tcgen05 layers for inference, forced, and a large batch
    os.environ["AFGB_CNN_UMMA_MIN"] = "1"
    big = 4096
    mtc = _lib.af_model_create(big, 7)
    os.environ.pop("AFGB_CNN_UMMA_MIN", None)
    ms_fwd_tc = timed(lambda: _lib.af_model_forward(mtc, xin.data_ptr(), n, 0, prob.data_ptr(), sp), k)
    xbig = xin.repeat(big // n, 1, 1, 1).contiguous()
    ybig = y.repeat(big // n).contiguous()
    pbig = torch.empty(big, dtype=torch.float32, device=dev)
    ms_fwd_big = timed(lambda: _lib.af_model_forward(mtc, xbig.data_ptr(), big, 0, pbig.data_ptr(), sp), 20)
    ms_train_big = timed(lambda: _lib.af_train_step(mtc, xbig.data_ptr(), ybig.data_ptr(), big, 1e-4, loss.data_ptr(),
                                                    sp), 10)
    _lib.af_model_get_params(mtc)   # reports a bounded wait that ran out
    _lib.af_model_destroy(mtc)
    del xbig
    pk = peaks()
    peak = float(pk.get("bf16_tflops_sustained", 1700.0))

    def tf(batch, ms, mult=1):
        return mult * batch * CNN_FWD_FLOP / (ms * 1e-3) / 1e12
    return {
        "batch": n, "flop_per_sample_forward": CNN_FWD_FLOP,
        "ms_classify": ms_classify, "candidates_per_s": n / (ms_classify * 1e-3),
        "ms_forward": ms_fwd, "forward_tflops": tf(n, ms_fwd), "ms_forward_tcgen05": ms_fwd_tc,
        "ms_forward_fused": ms_fwd_fused,
        "ms_train_step": ms_train, "train_tflops": tf(n, ms_train, 3),
        "large_batch": {"batch": big, "ms_forward_tcgen05": ms_fwd_big, "forward_tflops": tf(big, ms_fwd_big),
                        "ms_train_step": ms_train_big, "train_tflops": tf(big, ms_train_big, 3)},
        "peak_tflops": peak, "forward_frac": tf(n, ms_fwd) / peak, "train_frac": tf(n, ms_train, 3) / peak,
        "train_frac_large_batch": tf(big, ms_train_big, 3) / peak,
        "forward_frac_large_batch": tf(big, ms_fwd_big) / peak,
        "note": "training: the convolutions as implicit GEMMs on the tcgen05 tensor cores (bf16 operands, fp32 "
                "accumulators in tensor memory; forward with bias, ReLU and max pool fused, data and weight "
                "gradients); inference of this batch: the library's choice (the tcgen05 layers from 256 images "
                "up, the fused one-kernel mma.sync network below), ms_forward_tcgen05 / ms_forward_fused each "
                "forced on the same batch; a training step counts 3x the "
                "forward FLOP; peak = measured bf16 sustained (cuBLAS); af_classify includes the cut-out kernel",
    }


# The paper's GPU benchmarks (Sec. 3): 8-bit synthetic data, 40 us, 1000-1500 MHz, DM 0-1024; the kernel times
# it prints for an RTX 4090 at the ends of each sweep (dedisp = the brute-force comparison code, ASTROFLOW = its
# approximate subband kernel), in seconds.
PAPER_SEC3 = {
    "channels": {"span_s": 22.0, "ndm": 1500, "sweep": [512, 1024, 2048, 4096, 8192],
                 "rtx4090_dedisp_s": {512: 1.03, 8192: 8.72}, "rtx4090_astroflow_s": {512: 0.11, 8192: 0.96}},
    "dm_trials": {"span_s": 20.0, "nchan": 2048, "sweep": [512, 1024, 2048, 4096, 8192],
                  "rtx4090_dedisp_s": {543: 1.21, 8298: 9.21}, "rtx4090_astroflow_s": {512: 0.091, 8192: 1.295}},
}


def run_paper_sec3(args, dev, stream):
    """Our exact brute-force dedispersion and our two-stage subband dedispersion (n0 = 8, 64 subbands of 7.8 MHz) on
    the configurations of the paper's Sec. 3 benchmarks; kernel time (CUDA events, mean of 3 after a warm-up)
    and R = span / time."""
    import torch
    from paper_2511_02328_gb300 import _lib, synth
    from paper_2511_02328_gb300.search import Plan
    sp = stream.cuda_stream
    tsamp = 40e-6

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(3):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / 3

    def one(nchan, ndm, span_s, seed):
        dms = np.linspace(0.0, 1024.0, ndm)
        bp = Plan(nchan, F_LO, F_HI, tsamp, dms)
        nout = int(round(span_s / tsamp))
        nsamp = nout + bp.dmax
        sb = Plan(nchan, F_LO, F_HI, tsamp, dms, subband=dict(n0=8, nsub=min(64, nchan),
                                                               fs_mode=_lib.AF_FS_INVSQ, block_len=1 << 17))
        x = synth.filterbank_torch(nchan, nsamp, seed=seed, device=dev)
        plane = torch.empty((ndm, nout), dtype=torch.int32, device=dev)
        _lib.af_dedisperse_reserve(bp.handle, nsamp)
        ms_b = timed(lambda: _lib.af_dedisperse(bp.handle, x.data_ptr(), nsamp, plane.data_ptr(), 0, sp))
        nout_s = sb.nout(nsamp)
        ms_s = timed(lambda: _lib.af_dedisperse(sb.handle, x.data_ptr(), nsamp, plane.data_ptr(), 0, sp))
        _lib.af_plan_check(bp.handle)
        _lib.af_plan_check(sb.handle)
        kb = bp.kernel()
        out = {"nchan": nchan, "ndm": ndm, "nout": nout,
               "brute_kernel": f'{kb["path"]}/ring {kb["ring"]}/group {kb["group"]}',
               "brute_ms": ms_b, "brute_R": span_s / (ms_b * 1e-3),
               "brute_rate": float(ndm) * nchan * nout / (ms_b * 1e-3), "subband_ms": ms_s,
               "subband_R": nout_s * tsamp / (ms_s * 1e-3)}
        del x, plane
        bp.close()
        sb.close()
        torch.cuda.empty_cache()
        return out

    res = {}
    c = PAPER_SEC3["channels"]
    res["channels"] = [one(n, c["ndm"], c["span_s"], 900 + i) for i, n in enumerate(c["sweep"])]
    d = PAPER_SEC3["dm_trials"]
    res["dm_trials"] = [one(d["nchan"], n, d["span_s"], 950 + i) for i, n in enumerate(d["sweep"])]
    res["paper_rtx4090_s"] = {k: {"dedisp": v["rtx4090_dedisp_s"], "astroflow": v["rtx4090_astroflow_s"]}
                              for k, v in PAPER_SEC3.items()}
    res["note"] = ("brute = the exact plane; subband = n0 8, 64 subbands, 1/f^2 centres (approximate, like the "
                   "paper's own kernel); kernel time only, inputs resident, as the paper's R")
    return res


def run_stream(args, dev, clocks):
    """The streaming engine (pattern 5) with the classified search inline, at
    equal recall against the plain threshold (Sec. 4.2 matching).

    19 beams of independent data, generated on the GPU chunk by chunk (seeded
    torch RNG, the synth recipe) and copied to pinned host memory before each
    push: window 0 of each beam, then one hop per push.  Per beam two pulses
    per hop on average, in distinct 0.5 s slots, DM U(50, 1950), width
    log-U(0.2, 10) ms, S/N U(6, 30), per-channel starts from the library's
    delay table; two persistent narrowband channels per beam, and per chunk
    two zero-DM bursts (1-20 samples, S/N 10-50) and one drifting tone.
    Arrivals come at `--stream-speed` times the real-time rate, beams staggered
    over one hop.  The engine searches at S/N 6; each window's candidates are
    clustered (Sec. 4.2) and every cluster is classified (cut-outs + CNN) by
    the checkpoint trained on oracle-injected data.  Afterwards every cluster
    is matched to the injections; the plain method keeps clusters with S/N >=
    8, the classified one those with S/N >= 6 and P(pulse) >= p at equal
    recall (within 1 %).  Latency = push call to classified clusters in host
    memory."""
    import threading
    import torch
    from paper_2511_02328_gb300 import _lib, classifier, synth
    from paper_2511_02328_gb300.search import Plan
    nbeams, window = 19, 1 << 18
    dms = np.arange(0.0, 2001.0, 1.0)
    s = _lib.af_stream_open(nbeams, NCHAN, F_LO, F_HI, TSAMP, dms, window, WIDTHS, STREAM_THRESH, 1 << 16,
                            hbm_budget=64 << 30, max_slots=19, timeout_ms=120000)
    model = _lib.af_model_create(256, 1)
    _lib.af_model_load(model, STREAM_CKPT)
    hop, dmax, nslots = _lib.af_stream_info(s)
    rounds, speed = max(2, args.stream_rounds), float(args.stream_speed)
    hop_s = hop * TSAMP
    rng = np.random.default_rng(2025)
    slot = int(round(0.5 / TSAMP))
    inj = []
    for b in range(nbeams):
        npl = 2 * rounds
        pick = np.sort(rng.choice(rounds * hop // slot, npl, replace=False))
        d = dict(t0=pick * slot + rng.integers(0, slot // 4, npl), dm=rng.uniform(50.0, 1950.0, npl),
                 w=np.maximum(1, np.round(np.exp(rng.uniform(np.log(0.2e-3), np.log(10e-3), npl)) / TSAMP)).astype(
                     np.int64), snr=rng.uniform(6.0, 30.0, npl), narrow=rng.choice(NCHAN, 2, replace=False))
        p = Plan(NCHAN, F_LO, F_HI, TSAMP, d["dm"])
        d["D"] = p.delays().astype(np.int64)
        p.close()
        d["lo"], d["hi"] = d["t0"] + d["D"].min(1), d["t0"] + d["D"].max(1) + d["w"]
        inj.append(d)
    pinned = torch.empty(NCHAN * window, dtype=torch.uint8).pin_memory()
    gstream = torch.cuda.Stream(device=dev)

    def make_chunk(b, k):
        a0, n = (0, window) if k == 0 else (window + (k - 1) * hop, hop)
        d = inj[b]
        sel = np.nonzero((d["hi"] > a0) & (d["lo"] < a0 + n))[0]
        pulses = [synth.Pulse(d["t0"][j] + d["D"][j] - a0, int(d["w"][j]),
                              synth.pulse_amplitude(d["snr"][j], NCHAN, int(d["w"][j]))) for j in sel]
        cr = np.random.default_rng(1000003 * b + k)
        bursts = []
        for _ in range(2):
            ln = int(cr.integers(1, 21))
            bursts.append((int(cr.integers(0, n)), ln, synth.pulse_amplitude(cr.uniform(10, 50), NCHAN, ln)))
        tones = [(float(cr.integers(0, NCHAN)), int(cr.integers(0, n - 3000)), 2000,
                  float(cr.choice([-1, 1]) * 0.005), float(cr.uniform(2, 5)) * synth.NOISE_SIGMA)]
        rfi = synth.RFI(narrow_channels=list(d["narrow"]), bursts=bursts, tones=tones)
        with torch.cuda.stream(gstream):
            xg = synth.filterbank_torch(NCHAN, n, 7919 * b + 104729 * k + 1, pulses=pulses, rfi=rfi, device=dev)
            host = pinned[: NCHAN * n].view(NCHAN, n)
            host.copy_(xg)
        gstream.synchronize()
        return host.numpy()

    results, pushed = [], {}
    done = threading.Event()
    lock = threading.Lock()

    def poller():
        n = 0
        while n < nbeams * rounds:
            r = _lib.af_stream_poll(s, 1000)
            if r is None:
                continue
            reps = _lib.af_stream_cluster(s, r["cands"])
            prob = _lib.af_stream_classify(s, r["slot"], model, reps)
            t_cls = time.perf_counter()
            _lib.af_stream_release(s, r["slot"])
            with lock:
                t_push = pushed[(r["beam"], r["seq"])]
            r["latency_cls_ms"] = 1e3 * (t_cls - t_push)
            r["reps"], r["prob"] = reps, prob
            results.append(r)
            n += 1
        done.set()

    th = threading.Thread(target=poller, daemon=True)
    th.start()
    events = sorted(((k * hop_s + b * hop_s / nbeams) / speed, b, k) for k in range(rounds) for b in range(nbeams))
    t0 = time.perf_counter()
    late = 0.0
    for at, b, k in events:
        chunk = make_chunk(b, k)
        delay = t0 + at - time.perf_counter()
        if delay > 0:
            time.sleep(delay)
        else:
            late = max(late, -delay)
        with lock:
            pushed[(b, k)] = time.perf_counter()
        _lib.af_stream_push(s, b, chunk, k)
    t_fed = time.perf_counter() - t0
    done.wait(900)
    st = _lib.af_stream_stats(s)
    _lib.af_stream_close(s)
    _lib.af_model_destroy(model)
    del pinned
    # ---- match every cluster to its beam's injections; equal-recall comparison
    snr, prob, match, inj_snr = [], [], [], []
    for b in range(nbeams):
        d = inj[b]
        lst = [(float(d["dm"][j]), float(d["t0"][j]) * TSAMP, int(d["w"][j]), float(d["snr"][j]))
               for j in range(len(d["t0"]))]
        reps = [r for r in results if r["beam"] == b]
        if reps:
            rp = np.concatenate([r["reps"] for r in reps])
            pr = np.concatenate([r["prob"] for r in reps])
            m = classifier.match(rp, lst, dms, TSAMP)
            snr.append(rp["snr"].astype(np.float64))
            prob.append(pr.astype(np.float64))
            match.append(np.where(m >= 0, m + len(inj_snr), -1))
        inj_snr.extend(d["snr"].tolist())
    hours = len(results) * hop_s / 3600.0
    ev = classifier.equal_recall(np.concatenate(snr), np.concatenate(prob), np.concatenate(match), inj_snr, hours)
    lat = np.array([r["latency_ms"] for r in results])
    lat_cls = np.array([r["latency_cls_ms"] for r in results])
    return {"workload": STREAM_WORKLOAD, "beams": nbeams, "windows": int(st["windows"]), "slots": int(st["slots"]),
            "launches": int(st["launches"]), "max_inflight": int(st["max_inflight"]),
            "arrival_speed_vs_realtime": speed, "fed_s": t_fed, "max_late_s": late,
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "max_ms": float(lat.max()), "hop_s": hop_s, "chunk_s": window * TSAMP,
            "p50_ms_with_classifier": float(np.percentile(lat_cls, 50)),
            "p99_ms_with_classifier": float(np.percentile(lat_cls, 99)),
            "clusters_classified": int(sum(len(r["reps"]) for r in results)),
            "pulses_injected": len(inj_snr), "equal_recall": ev, "rate": st["rate"], "unit": UNIT,
            "note": ("latency = push call to candidates in host memory; with_classifier adds host clustering and "
                     "cut-outs + CNN of every cluster; arrivals at %g x the real-time rate; data generated on the "
                     "same GPU between pushes" % speed)}


def _g5(v):
    """A secondary scalar of the bench line at 5 significant digits (the line stays short)."""
    return None if v is None else float("%.5g" % v)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="afgb", choices=["afgb", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-stream", action="store_true")
    ap.add_argument("--no-subband", action="store_true")
    ap.add_argument("--no-prep", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-classifier", action="store_true")
    ap.add_argument("--subband-sweep", default="", help="extra subband settings, e.g. 4x64,16x64,8x32 (n0 x nsub)")
    ap.add_argument("--paper-sec3", action="store_true", help="also time the paper's Sec. 3 benchmark configurations")
    ap.add_argument("--stream-rounds", type=int, default=53, help="windows per beam in the streaming block")
    ap.add_argument("--stream-speed", type=float, default=8.0, help="arrival rate in units of the real-time rate")
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)

    import torch
    rank, world, local = dist_setup(args.gpus)
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    import __graft_entry__
    __graft_entry__.build()
    from paper_2511_02328_gb300 import _lib
    from paper_2511_02328_gb300.search import Plan

    plan = Plan(NCHAN, F_LO, F_HI, TSAMP, DMS)
    nout = plan.nout(NSAMP)
    x_host, pulses = make_input(beam_seed(rank), lambda dms: Plan(NCHAN, F_LO, F_HI, TSAMP, dms).delays())
    dev = torch.device("cuda", local)
    x = torch.from_numpy(x_host).to(dev)
    plane = torch.empty((plan.ndm, nout), dtype=torch.int32, device=dev)
    stats = torch.empty((plan.ndm, 2), dtype=torch.int64, device=dev)
    snr = torch.empty((plan.ndm, nout), dtype=torch.float32, device=dev)
    bw = torch.empty((plan.ndm, nout), dtype=torch.uint8, device=dev)
    cands = torch.empty((CAP, 24), dtype=torch.uint8, device=dev)
    count = torch.empty(1, dtype=torch.int32, device=dev)
    stream = torch.cuda.Stream(device=dev)
    sp = stream.cuda_stream
    H = plan.handle
    _lib.af_dedisperse_reserve(H, NSAMP)   # the group-row buffer (setup, outside the timed region)
    kern = plan.kernel()
    # dedispersion (group rows: stage 1 + stage 2; else one tile launch), rowconst, boxcar, candidates
    launches_per_step = (5 if kern["path"] == "pairs" else 4)

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]

    def step(i=None):
        if i is not None:
            ev[i][0].record(stream)
        _lib.af_dedisperse(H, x.data_ptr(), NSAMP, plane.data_ptr(), stats.data_ptr(), sp)
        if i is not None:
            ev[i][1].record(stream)
        _lib.af_boxcar_snr(H, plane.data_ptr(), nout, stats.data_ptr(), WIDTHS, snr.data_ptr(), bw.data_ptr(), sp)
        _lib.af_candidates(H, snr.data_ptr(), bw.data_ptr(), nout, WIDTHS, THRESH, 0, cands.data_ptr(), CAP,
                           count.data_ptr(), sp)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    if kern["path"] == "pairs":
        _lib.af_dedisperse_timing(H, args.steps)   # per-stage events of the timed calls
    gpu_id = local
    clocks = ClockSampler(gpu_id)
    clocks.start()
    time.sleep(0.3)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    clocks.mark(True)
    t_start.record(stream)
    for i in range(args.steps):
        step(i)
    t_end.record(stream)
    torch.cuda.synchronize()
    clocks.mark(False)
    clocks.stop()         # the sampler covers the timed device region; nvidia-smi stays out of the host-path timing
    if dist is not None:
        dist.barrier()
    ms_total = t_start.elapsed_time(t_end)
    ms_dedisp = float(np.mean([a.elapsed_time(b) for a, b in ev]))
    stage = None
    if kern["path"] == "pairs":
        st = [_lib.af_dedisperse_times(H, i) for i in range(args.steps)]
        stage = {"rows_ms": float(np.mean([x[0] for x in st])), "tiles_ms": float(np.mean([x[1] for x in st])),
                 "row_bytes": int(st[-1][2]), "copy_bytes": int(st[-1][3])}
        _lib.af_dedisperse_timing(H, 0)
    ncand = int(count.item())
    ms_total = max_over_ranks(ms_total, dist, dev)

    # ---- e2e through the host-buffer entry point (pinned input, copies timed)
    x_pin = torch.from_numpy(x_host).pin_memory()
    _lib.af_search_reserve(H, NSAMP, CAP)
    out = np.empty(CAP, dtype=_lib.CAND_DTYPE)
    for _ in range(2):
        _lib.af_search(H, x_pin.data_ptr(), NSAMP, WIDTHS, THRESH, CAP, sp, out=out)
    if dist is not None:
        dist.barrier()
    gc_was = gc.isenabled()
    gc.disable()          # no collector pause inside the timed calls
    _lib.af_search_timing(H, 1)   # four events per call: where each call's time goes
    t0 = time.perf_counter()
    nc = 0
    walls, phases = [], []
    for _ in range(args.e2e_steps):
        ta = time.perf_counter()
        c, nc = _lib.af_search(H, x_pin.data_ptr(), NSAMP, WIDTHS, THRESH, CAP, sp, out=out)
        plan.cluster(c)
        walls.append((time.perf_counter() - ta) * 1e3)
        phases.append(_lib.af_search_times(H))
    e2e_s = (time.perf_counter() - t0) / args.e2e_steps
    _lib.af_search_timing(H, 0)
    if gc_was:
        gc.enable()
    ph = np.median(np.asarray(phases), axis=0)
    e2e_phases = {"copy_wait_ms": float(ph[0]), "dedisp_ms": float(ph[1]), "snr_candidates_ms": float(ph[2]),
                  "call_ms": {"min": min(walls), "median": float(np.median(walls)), "max": max(walls),
                              "each": [round(v, 2) for v in walls]},
                  "each_phase_ms": [[round(float(v), 2) for v in p] for p in phases],
                  "note": "medians over the timed calls of: first time block's input copy (its outputs + Dmax), "
                          "dedispersion with the rest of the copy overlapped, S/N + candidate kernels (device "
                          "events); the remainder of a call's wall time is host work and the candidate copy back; "
                          "call_ms = each timed call's wall time (search + clustering)"}
    # the input copy alone (pinned host -> device), for the e2e breakdown
    h2d = torch.empty_like(x)
    for _ in range(2):
        h2d.copy_(x_pin, non_blocking=True)
    torch.cuda.synchronize()
    ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ea.record()
    for _ in range(5):
        h2d.copy_(x_pin, non_blocking=True)
    eb.record()
    torch.cuda.synchronize()
    h2d_ms = ea.elapsed_time(eb) / 5
    del h2d
    e2e_s = max_over_ranks(e2e_s, dist, dev)

    sec3_res = None
    if args.paper_sec3:
        del snr, bw
        torch.cuda.empty_cache()
        sec3_res = run_paper_sec3(args, dev, stream)
        snr = torch.empty((plan.ndm, nout), dtype=torch.float32, device=dev)
        bw = torch.empty((plan.ndm, nout), dtype=torch.uint8, device=dev)

    cls_res = None
    if not args.no_classifier:
        cls_res = run_classifier(args, dev, x, plan, stream)

    batch_res = None
    if not args.no_batch:
        batch_res = run_batch(args, dev, stream)
        torch.cuda.empty_cache()

    prep_res = None
    if not args.no_prep:
        prep_res = run_prep(args, dev, x, plane, snr, bw, ms_dedisp, stream)

    sub_res = None
    if not args.no_subband:
        del snr, bw
        torch.cuda.empty_cache()
        sub_res = run_subband(args, dev, x, x_host, pulses, plan, ms_dedisp, stream)
        if args.subband_sweep:
            sweep = []
            for item in args.subband_sweep.split(","):
                a_, b_ = item.split("x")
                r_ = run_subband(args, dev, x, x_host, pulses, plan, ms_dedisp, stream, int(a_), int(b_))
                sweep.append({k: r_[k] for k in ("n0", "nsub", "ms", "speedup_vs_brute", "snr_ratio_vs_brute",
                                                  "pulses_found")})
            sub_res["sweep"] = sweep

    stream_res = None
    if not args.no_stream:
        del plane
        torch.cuda.empty_cache()
        stream_res = run_stream(args, dev, clocks)

    work = float(plan.ndm) * NCHAN * nout
    ms_step = ms_total / args.steps
    value = aggregate_rate(world, work, ms_step * 1e-3)
    pk = peaks()
    sm_max = float(pk.get("sm_max_mhz", SM_MAX_MHZ_FALLBACK))
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    alu_peak = nsm * 128 * sm_max * 1e6 / 1e12          # T int32 lane-ops/s
    smem_derived = nsm * 128 * sm_max * 1e6 / 1e12      # TB/s: 128 B of shared loads per clock per SM
    smem_peak = _lib.af_diag_smem_rate() / 1e12         # TB/s, measured on this device (probe kernel)
    add_rate, pattern_rate = _lib.af_diag_int_rates()  # measured on this device (probe kernels)
    achieved = work / (ms_dedisp * 1e-3) / 1e12        # T adds/s, both stages
    hbm_peak = float(pk.get("hbm_gbs", 6800.0))
    alg_bytes = NCHAN * NSAMP + plan.ndm * nout * 4
    hbm_ach = alg_bytes / (ms_dedisp * 1e-3) / 1e9
    if stage is not None:
        # stage 2: every (DM, channel group, output) is one 2-byte shared load and one 16-bit lane add
        G = kern["group"]
        ngroups = (NCHAN + G - 1) // G
        lds_bytes = 2.0 * plan.ndm * ngroups * nout
        traffic, traffic_basis = PAIR_TILE_TRAFFIC.get(G, (None, None))
        s2_ach = lds_bytes / (stage["tiles_ms"] * 1e-3) / 1e12
        s1_bytes = stage["row_bytes"] + NCHAN * NSAMP
        performed = stage["row_bytes"] / 2 * (G - 1) + plan.ndm * ngroups * nout
        s1_ach = s1_bytes / (stage["rows_ms"] * 1e-3) / 1e9
        roofline = {
            "bound": "smem", "kernel": "k_pair_tile<15,%d> (stage 2 of the group-row dedispersion, %d channels "
                                       "per row)" % (kern["ring"], G),
            "achieved": s2_ach, "peak": smem_peak, "unit": "TB/s", "frac": s2_ach / smem_peak,
            "traffic": traffic, "traffic_basis": traffic_basis,
            "work": "2 B shared load per (DM, channel group, output): %.3g B per launch" % lds_bytes,
            "ms": stage["tiles_ms"],
            "with_copies": {"achieved": (lds_bytes + stage["copy_bytes"]) / (stage["tiles_ms"] * 1e-3) / 1e12,
                            "frac": (lds_bytes + stage["copy_bytes"]) / (stage["tiles_ms"] * 1e-3) / 1e12 / smem_peak,
                            "copy_bytes": stage["copy_bytes"],
                            "note": "shared-memory bytes including the row windows the producer copies in (the "
                                    "kernel's whole shared-memory traffic but its small tables)"},
            "peak_basis": "of measured: shared-load bandwidth of a conflict-free 32-bit load probe on this "
                          "device (af_diag_smem_rate)",
            "derived_peak": {"value": smem_derived, "frac": s2_ach / smem_derived,
                             "basis": "%d SMs x 128 B per clock x %.0f MHz (max clock)" % (nsm, sm_max)},
            "stage1": {"kernel": "k_group_rows<%d>" % G, "bound": "hbm", "ms": stage["rows_ms"], "achieved": s1_ach,
                       "peak": hbm_peak, "unit": "GB/s", "frac": s1_ach / hbm_peak, "basis": "of measured",
                       "work": "row writes %.3g B + input read %.3g B" % (stage["row_bytes"], NCHAN * NSAMP)},
            "dedispersion": {"ms": ms_dedisp, "effective_adds_per_s": achieved * 1e12,
                             "performed_adds_per_s": performed / (ms_dedisp * 1e-3),
                             "performed_frac_of_measured_int32_add_rate": performed / (ms_dedisp * 1e-3) / add_rate,
                             "measured_int32_add_rate": add_rate,
                             "note": "effective = the brute-force sum's ndm x nchan x nout additions per second "
                                     "(the metric); performed = the additions the two stages execute: (G - 1) per "
                                     "row sample in stage 1 + one per (DM, channel group, output) in stage 2",
                             "hbm": {"achieved": hbm_ach, "peak": hbm_peak, "unit": "GB/s",
                                     "frac": hbm_ach / hbm_peak, "basis": "of measured"}},
        }
    else:
        roofline = {"bound": "alu", "kernel": "k_tile<11,8>", "achieved": achieved, "peak": alu_peak,
                    "unit": "Tops/s", "frac": achieved / alu_peak, "traffic": None,
                    "peak_basis": "%d SMs x 128 int32 lanes x %.0f MHz (derived, of max clock)" % (nsm, sm_max),
                    "measured_int32_add_peak": add_rate / 1e12,
                    "frac_of_measured_add_peak": achieved * 1e12 / add_rate,
                    "measured_inner_pattern_peak": pattern_rate / 1e12,
                    "frac_of_measured_pattern_peak": achieved * 1e12 / pattern_rate,
                    "hbm": {"achieved": hbm_ach, "peak": hbm_peak, "unit": "GB/s", "frac": hbm_ach / hbm_peak,
                            "basis": "of measured"}}
    clk = clocks.summary()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        D = plan.delays()
        nthr = oracle.threads()
        rows = np.unique(np.linspace(0, len(DMS) - 1, 4 * nthr).round().astype(np.int64))
        v, dt = cpu_oracle_sample(x_host, D, rows, nout)
        cpu = {"value": v, "unit": UNIT, "cores": nthr, "kind": "oracle",
               "sample": "%d evenly spaced DM rows of 1001 (full nout=%d, 4096 channels): dedispersion + S/N + "
                         "peaks, %.2f s on %d OpenMP threads; gcc %s"
                         % (len(rows), nout, dt, nthr, " ".join(oracle_cflags()))}

    if rank == 0:
        # one compact line: the contract's keys, then the secondary results as
        # top-level scalars (the detail of every block goes to stderr first)
        sres = stream_res or {}
        er = sres.get("equal_recall", {})
        detail = {"stream": stream_res, "subband": sub_res, "prep": prep_res, "batch": batch_res,
                  "classifier": cls_res, "paper_sec3": sec3_res, "e2e_phases": e2e_phases, "dedisp_kernel": kern,
                  "candidates": ncand, "roofline_detail": roofline}
        sys.stderr.write("bench-detail " + json.dumps(detail) + "\n")
        sys.stderr.flush()
        rl = {k: roofline[k] for k in ("bound", "kernel", "achieved", "peak", "unit", "frac", "traffic")}
        rl["basis"] = roofline.get("peak_basis", "")
        if "stage1" in roofline:
            rl["stage1_frac_of_hbm"] = roofline["stage1"]["frac"]
            rl["dedisp_effective_adds_per_s"] = roofline["dedispersion"]["effective_adds_per_s"]
            rl["dedisp_performed_frac_of_measured_int32"] = \
                roofline["dedispersion"]["performed_frac_of_measured_int32_add_rate"]
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "nchan": NCHAN, "nsamp": NSAMP, "ndm": plan.ndm, "nout": nout,
                       "widths": WIDTHS, "threshold": THRESH, "parallelism": "replicas (one beam per GPU)",
                       "l2": "inputs larger than L2 (1.07 GB input, 0.86 GB plane per step)"},
            "roofline": rl,
            "cpu_baseline": cpu,
            "e2e": {"value": aggregate_rate(world, work, e2e_s), "unit": UNIT, "ms": e2e_s * 1e3,
                    "ms_median": e2e_phases["call_ms"]["median"], "h2d_ms": h2d_ms,
                    "h2d_bytes_per_step": NCHAN * NSAMP, "d2h_bytes_per_step": 4 + 24 * min(nc, CAP)},
            "gpu_launches": launches_per_step * args.steps,
            "clocks": clk,
            "realtime_factor": _g5(nout * TSAMP / (ms_dedisp * 1e-3)),
            "dedisp_ms": _g5(ms_dedisp),
            "stage1_ms": _g5(stage["rows_ms"] if stage else None),
            "stage2_ms": _g5(stage["tiles_ms"] if stage else None),
            "batch_ms": _g5(batch_res["ms_per_batch"] if batch_res else None),
            "batch_strategy": batch_res["strategy"] if batch_res else None,
            "batch_speedup_vs_beam_by_beam": _g5(batch_res.get("speedup_vs_beam_by_beam") if batch_res else None),
            "subband_ms": _g5(sub_res["ms"] if sub_res else None),
            "cnn_train_ms": _g5(cls_res["ms_train_step"] if cls_res else None),
            "cnn_train_frac": _g5(cls_res["train_frac"] if cls_res else None),
            "cnn_forward_frac": _g5(cls_res["forward_frac"] if cls_res else None),
            "cnn_train_frac_4096": _g5(cls_res["train_frac_large_batch"] if cls_res else None),
            "cnn_forward_frac_4096": _g5(cls_res["forward_frac_large_batch"] if cls_res else None),
            "stream_windows": sres.get("windows"),
            "stream_speed_vs_realtime": sres.get("arrival_speed_vs_realtime"),
            "p50_chunk_latency_ms": _g5(sres.get("p50_ms_with_classifier")),
            "p99_chunk_latency_ms": _g5(sres.get("p99_ms_with_classifier")),
            "hop_ms": _g5(sres.get("hop_s", 0) * 1e3 if sres else None),
            "pulses_snr8": er.get("injected"),
            "recall_threshold": _g5(er.get("recall_threshold")),
            "recall_cnn": _g5(er.get("recall_cnn")),
            "fp_per_hour_threshold": _g5(er.get("fp_per_hour_threshold")),
            "fp_per_hour_cnn": _g5(er.get("fp_per_hour_cnn")),
        }
        print(json.dumps(line))
    plan.close()
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

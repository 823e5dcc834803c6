"""Shapes of the synthetic workloads (no search arithmetic here).

The paper's data sets (FAST_FREX, FAST / QUEST observations) are not
available; these shapes follow its benchmark set-ups (Sec. 3: 1000-1500 MHz,
8-bit, 512-8192 channels, DM 0-1024) and the multi-beam survey (Sec. 4.3).
"""
import numpy as np


def plain_full_band():
    """The 4096-channel plain search: 1000-1500 MHz, 49.152 us, 2^18 samples,
    DMs 0..1000 step 1, boxcar widths 1..256 (powers of two)."""
    return dict(nchan=4096, f_lo=1000.0, f_hi=1500.0, tsamp=49.152e-6, nsamp=1 << 18,
                dm_list=np.arange(0.0, 1001.0, 1.0), widths=[1, 2, 4, 8, 16, 32, 64, 128, 256])


def multibeam(nbeams=19, max_delay_fn=None):
    """The uneven multi-beam batch: beam b has
        nchan  = [1024, 2048, 4096][b % 3], tsamp = 49.152 us * 4096 / nchan,
        DMmax  = [500, 1000, 1500, 2000][(b // 3) % 4],
        step   = [0.5, 1, 2][(b // 4) % 3],
        nsamp  = 2^(16 + b % 4), doubled until it is at least 2 * Dmax
    where Dmax comes from max_delay_fn(nchan, f_lo, f_hi, tsamp, dm_max) (the
    caller's delay table).  Widths 1..256 (powers of two), threshold 8."""
    beams = []
    for b in range(nbeams):
        nchan = [1024, 2048, 4096][b % 3]
        tsamp = 49.152e-6 * 4096 / nchan
        dm_max = [500.0, 1000.0, 1500.0, 2000.0][(b // 3) % 4]
        step = [0.5, 1.0, 2.0][(b // 4) % 3]
        dms = np.arange(0.0, dm_max + step / 2, step)
        nsamp = 1 << (16 + b % 4)
        if max_delay_fn is not None:
            dmax = int(max_delay_fn(nchan, 1000.0, 1500.0, tsamp, dm_max))
            while nsamp < 2 * dmax:
                nsamp *= 2
        beams.append(dict(nchan=nchan, f_lo=1000.0, f_hi=1500.0, tsamp=tsamp, dm_list=dms, nsamp=nsamp,
                          widths=[1, 2, 4, 8, 16, 32, 64, 128, 256], thresh=8.0))
    return beams


def _run(argv=None):
    """Runs one step of a workload `repeat` times on cuda:0 (inputs resident on
    the device) -- the command the kernel profiles are taken with:
        python -m paper_2511_02328_gb300.workloads search|subband|prep|train|infer [--nsamp N] [--repeat R] [--batch B]
    search:  brute-force dedispersion (row sums fused) + boxcar S/N + candidates
    subband: two-stage subband dedispersion (n0 = 8, 64 subbands)
    prep:    zero-DM filter, square-law downsampling by 8, median/MAD + robust S/N
    on the 4096-channel full-band shape with nsamp samples (default 2^18);
    train:   classifier training steps (forward, backward, Adam) on a batch of
             B random 64 x 64 x 2 bf16 cut-outs (default 1024);
    infer:   classifier forward passes on such a batch (the library's choice of
             kernels for that batch size)."""
    import argparse
    import torch
    from . import _lib, synth
    from .search import Plan
    ap = argparse.ArgumentParser(prog="python -m paper_2511_02328_gb300.workloads")
    ap.add_argument("step", choices=["search", "subband", "prep", "train", "infer"])
    ap.add_argument("--nsamp", type=int, default=1 << 18)
    ap.add_argument("--repeat", type=int, default=3)
    ap.add_argument("--batch", type=int, default=1024)
    a = ap.parse_args(argv)
    if a.step in ("train", "infer"):
        g = torch.Generator(device="cuda")
        g.manual_seed(1)
        x = torch.rand((a.batch, 64, 64, 2), device="cuda", generator=g).to(torch.bfloat16)
        y = torch.randint(0, 2, (a.batch,), device="cuda", dtype=torch.int32, generator=g)
        loss = torch.empty(1, device="cuda")
        m = _lib.af_model_create(a.batch, 3)
        prob = torch.empty(a.batch, device="cuda")
        for _ in range(a.repeat):
            if a.step == "train":
                _lib.af_train_step(m, x.data_ptr(), y.data_ptr(), a.batch, 1e-4, loss.data_ptr())
            else:
                _lib.af_model_forward(m, x.data_ptr(), a.batch, 0, prob.data_ptr())
        torch.cuda.synchronize()
        _lib.af_model_get_params(m)      # reports a bounded wait that ran out
        _lib.af_model_destroy(m)
        print("ok", a.step, a.batch, a.repeat)
        return
    w = plain_full_band()
    nch, nsamp = w["nchan"], a.nsamp
    x = synth.filterbank_torch(nch, nsamp, seed=1, device="cuda")
    sub = dict(n0=8, nsub=64, fs_mode=_lib.AF_FS_INVSQ, block_len=nsamp) if a.step == "subband" else None
    p = Plan(nch, w["f_lo"], w["f_hi"], w["tsamp"], w["dm_list"], subband=sub)
    nout = p.nout(nsamp)
    plane = torch.empty((p.ndm, nout), dtype=torch.int32, device="cuda")
    stats = torch.empty((p.ndm, 2), dtype=torch.int64, device="cuda")
    if a.step != "subband":
        snr = torch.empty((p.ndm, nout), dtype=torch.float32, device="cuda")
        bw = torch.empty((p.ndm, nout), dtype=torch.uint8, device="cuda")
    if a.step == "prep":
        y = torch.empty_like(x)
        ds = torch.empty((nch, (nsamp + 7) // 8), dtype=torch.uint8, device="cuda")
        p.dedisperse(x, plane=plane, stats=stats)
    for _ in range(a.repeat):
        if a.step == "search":
            p.dedisperse(x, plane=plane, stats=stats)
            p.boxcar_snr(plane, w["widths"], stats=stats, snr=snr, bw=bw)
            p.candidates(snr, bw, w["widths"], 8.0)
        elif a.step == "subband":
            p.dedisperse(x, plane=plane, stats=stats)
        else:
            _lib.af_zerodm(x.data_ptr(), nch, nsamp, y.data_ptr())
            _lib.af_downsample(x.data_ptr(), nch, nsamp, 8, ds.data_ptr())
            _lib.af_boxcar_snr_robust(p.handle, plane.data_ptr(), nout, 0, w["widths"], snr.data_ptr(), bw.data_ptr())
    torch.cuda.synchronize()
    _lib.af_plan_check(p.handle)
    print("ok", a.step, nsamp, a.repeat)
    p.close()


if __name__ == "__main__":
    _run()

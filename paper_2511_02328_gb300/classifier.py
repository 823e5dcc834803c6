"""Training and evaluation of the candidate classifier on synthetic data.

The paper trains its detector on pulses injected into real spectrograms
(Sec. 4.1) and names the RFI that triggers its search (Sec. 4.4): impulsive
broadband (zero-DM) bursts, narrowband interference and burst-like
fluctuations.  Here every chunk is synthetic noise of one workload's band and
sampling (CHUNK: the 256-channel search; STREAM_CHUNK: the streaming
workload's 4096 channels and DM 0-2000 grid, in chunks of 2^15 outputs) with
injected dispersed pulses and the three RFI shapes; the search runs on the
GPU, its candidates are clustered with the true-positive rule of Sec. 4.2,
and each cluster's strongest candidate becomes one sample (two 64 x 64
cut-outs), labelled 1 when it matches an injected pulse.

Where a pulse lands in each channel comes from the caller's `offsets_fn(dm,
t0)` (per-channel start samples of a pulse arriving at the top of the band at
sample t0): the test-suite and the checkpoint script pass the CPU oracle's
injector; without one, the library's own delay table is used.

equal_recall() compares the plain boxcar-S/N threshold (the method without
the network) with threshold-then-network at equal recall of injected pulses
with S/N >= 8, and reports both false-positive rates.
"""
import numpy as np
import torch

from . import _lib, synth
from .search import Plan

WIDTHS = [1, 2, 4, 8, 16, 32, 64, 128, 256]
CHUNK = dict(nchan=256, f_lo=1000.0, f_hi=1500.0, tsamp=98.304e-6, nsamp=1 << 15,
             dm_list=np.arange(0.0, 501.0, 1.0), widths=[1, 2, 4, 8, 16, 32], inj_dm=(20.0, 480.0), n_pulses=4)
# 4096 channels, 49.152 us, DMs 0..2000: the DM-2000 delay (93,766 samples) + 2^15 outputs
STREAM_CHUNK = dict(nchan=4096, f_lo=1000.0, f_hi=1500.0, tsamp=49.152e-6, nsamp=93766 + (1 << 15),
                    dm_list=np.arange(0.0, 2001.0, 1.0), widths=WIDTHS, inj_dm=(50.0, 1950.0), n_pulses=3)
DM_TOL, TOA_TOL = 20.0, 0.2


def library_offsets(cfg, pool=4096, seed=0):
    """offsets_fn from the library's delay table: a plan over `pool` random
    DMs in cfg's injection range, each pulse snapped to the nearest of them."""
    rng = np.random.default_rng(seed)
    dms = np.sort(rng.uniform(cfg["inj_dm"][0], cfg["inj_dm"][1], pool))
    p = Plan(cfg["nchan"], cfg["f_lo"], cfg["f_hi"], cfg["tsamp"], dms)
    D = p.delays().astype(np.int64)
    p.close()

    def fn(dm, t0):
        j = int(np.clip(np.searchsorted(dms, dm), 0, pool - 1))
        return int(t0) + D[j], float(dms[j])
    return fn


class Generator:
    """Chunks of cfg's shape with n_pulses injected pulses and RFI."""

    def __init__(self, cfg=CHUNK, nout=None, offsets_fn=None, seed=0, device="cuda"):
        self.cfg, self.device, self.seed = cfg, device, seed
        self.n_pulses = cfg.get("n_pulses", 4)
        self.rng = np.random.default_rng(seed)
        self.nout = nout if nout is not None else cfg["nsamp"] - 11682
        self.offsets_fn = offsets_fn or library_offsets(cfg, seed=seed)
        self.count = 0

    def chunk(self, rfi=True):
        cfg, rng = self.cfg, self.rng
        nchan, nsamp, tsamp = cfg["nchan"], cfg["nsamp"], cfg["tsamp"]
        span = self.nout // (self.n_pulses + 1)
        pulses, inj = [], []
        for s in range(1, self.n_pulses + 1):
            dm = float(rng.uniform(*cfg["inj_dm"]))
            w = max(1, int(round(np.exp(rng.uniform(np.log(0.2e-3), np.log(10e-3))) / tsamp)))
            snr = float(rng.uniform(6.0, 30.0))
            t0 = int(s * span + rng.integers(-span // 4, span // 4))
            offs = self.offsets_fn(dm, t0)
            if isinstance(offs, tuple):      # (offsets, the DM actually injected)
                offs, dm = offs
            pulses.append(synth.Pulse(np.asarray(offs, dtype=np.int64), w, synth.pulse_amplitude(snr, nchan, w)))
            inj.append((dm, t0 * tsamp, w, snr))
        r = None
        if rfi:
            narrow = list(rng.choice(nchan, size=2, replace=False))
            bursts = []
            for _ in range(2):
                ln = int(rng.integers(1, 21))
                bursts.append((int(rng.integers(0, self.nout)), ln,
                               synth.pulse_amplitude(rng.uniform(10, 50), nchan, ln)))
            tones = [(float(rng.integers(0, nchan)), int(rng.integers(0, nsamp - 3000)), 2000,
                      float(rng.choice([-1, 1]) * 0.005), float(rng.uniform(2, 5)) * synth.NOISE_SIGMA)]
            r = synth.RFI(narrow_channels=narrow, bursts=bursts, tones=tones)
        x = synth.filterbank_torch(nchan, nsamp, self.seed * 1000003 + self.count, pulses=pulses, rfi=r,
                                   device=self.device)
        self.count += 1
        return x, inj


class Searcher:
    """Plain search of one chunk on the GPU, clustering on the host."""

    def __init__(self, cfg=CHUNK, thresh=6.0, cap=1 << 16):
        self.cfg, self.thresh, self.cap = cfg, thresh, cap
        self.plan = Plan(cfg["nchan"], cfg["f_lo"], cfg["f_hi"], cfg["tsamp"], cfg["dm_list"])
        self.nout = self.plan.nout(cfg["nsamp"])
        dev = "cuda"
        self.plane = torch.empty((self.plan.ndm, self.nout), dtype=torch.int32, device=dev)
        self.stats = torch.empty((self.plan.ndm, 2), dtype=torch.int64, device=dev)
        self.snr = torch.empty((self.plan.ndm, self.nout), dtype=torch.float32, device=dev)
        self.bw = torch.empty((self.plan.ndm, self.nout), dtype=torch.uint8, device=dev)
        self.cands = torch.empty((cap, 24), dtype=torch.uint8, device=dev)
        self.count = torch.empty(1, dtype=torch.int32, device=dev)

    def run(self, x):
        p, cfg = self.plan, self.cfg
        p.dedisperse(x, plane=self.plane, stats=self.stats)
        p.boxcar_snr(self.plane, cfg["widths"], stats=self.stats, snr=self.snr, bw=self.bw)
        p.candidates(self.snr, self.bw, cfg["widths"], self.thresh, cap=self.cap, out=self.cands, count=self.count)
        cands, n = Plan.cands_to_numpy(self.cands, self.count)
        clusters = p.cluster(cands, DM_TOL, TOA_TOL) if len(cands) else cands
        return clusters

    def cutouts(self, x, reps):
        n = len(reps)
        out = torch.empty((max(n, 1), 64, 64, 2), dtype=torch.bfloat16, device="cuda")
        if n:
            cd = torch.from_numpy(np.ascontiguousarray(reps).view(np.uint8).reshape(n, 24)).cuda()
            _lib.af_cutouts(self.plan.handle, x.data_ptr(), self.cfg["nsamp"], self.plane.data_ptr(), self.nout,
                            cd.data_ptr(), n, out.data_ptr())
        return out[:n]

    def close(self):
        self.plan.close()


def match(reps, inj, dm_list, tsamp):
    """For each cluster: index of the first injection it matches (Sec. 4.2
    rule: |dDM| < 20 and |dTOA| < 0.2 s) or -1."""
    res = np.full(len(reps), -1, dtype=np.int64)
    if len(reps) == 0 or len(inj) == 0:
        return res
    dm = np.asarray(dm_list, dtype=np.float64)[np.asarray(reps["dm_idx"], dtype=np.int64)]
    toa = np.asarray(reps["abs_sample"], dtype=np.int64) * tsamp
    idm = np.array([v[0] for v in inj], dtype=np.float64)
    itoa = np.array([v[1] for v in inj], dtype=np.float64)
    for i0 in range(0, len(dm), 4096):      # blocks of clusters x all injections
        ok = (np.abs(dm[i0:i0 + 4096, None] - idm[None, :]) < DM_TOL) & \
             (np.abs(toa[i0:i0 + 4096, None] - itoa[None, :]) < TOA_TOL)
        hit = ok.any(axis=1)
        res[i0:i0 + 4096][hit] = ok.argmax(axis=1)[hit]
    return res


def build_dataset(n_chunks, seed, searcher=None, gen=None, offsets_fn=None):
    """Returns (cut-outs bf16 [N][64][64][2] on the GPU, labels int32 [N] on the
    GPU, per-sample cluster S/N, per-chunk records for evaluation)."""
    own = searcher is None
    searcher = searcher or Searcher()
    gen = gen or Generator(searcher.cfg, nout=searcher.nout, offsets_fn=offsets_fn, seed=seed)
    xs, ys, snrs, records = [], [], [], []
    for _ in range(n_chunks):
        x, inj = gen.chunk()
        reps = searcher.run(x)
        m = match(reps, inj, searcher.cfg["dm_list"], searcher.cfg["tsamp"])
        if len(reps):
            xs.append(searcher.cutouts(x, reps))
            ys.append(torch.from_numpy((m >= 0).astype(np.int32)))
            snrs.append(reps["snr"].astype(np.float64))
        records.append(dict(snr=reps["snr"].astype(np.float64) if len(reps) else np.zeros(0), match=m, inj=inj,
                            start=sum(len(s) for s in snrs) - (len(reps) if len(reps) else 0), n=len(reps)))
    X = torch.cat(xs) if xs else torch.empty((0, 64, 64, 2), dtype=torch.bfloat16, device="cuda")
    Y = torch.cat(ys).cuda() if ys else torch.empty(0, dtype=torch.int32, device="cuda")
    if own:
        searcher.close()
    return X, Y, np.concatenate(snrs) if snrs else np.zeros(0), records


def train(model, X, Y, epochs=3, batch=256, lr=1e-3, seed=0):
    """Adam on the GPU with the library's kernels; returns the mean loss per epoch."""
    n = X.shape[0]
    g = torch.Generator(device="cpu")
    g.manual_seed(seed)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    hist = []
    for _ in range(epochs):
        perm = torch.randperm(n, generator=g).cuda()
        tot, k = 0.0, 0
        for i0 in range(0, n - batch + 1, batch):
            idx = perm[i0:i0 + batch]
            xb = X[idx].contiguous()
            yb = Y[idx].contiguous()
            _lib.af_train_step(model, xb.data_ptr(), yb.data_ptr(), batch, lr, loss.data_ptr())
            tot += float(loss.item())
            k += 1
        hist.append(tot / max(k, 1))
    return hist


def predict(model, X, batch=256):
    n = X.shape[0]
    prob = torch.empty(max(n, 1), dtype=torch.float32, device="cuda")
    for i0 in range(0, n, batch):
        k = min(batch, n - i0)
        xb = X[i0:i0 + k].contiguous()
        _lib.af_model_forward(model, xb.data_ptr(), k, 0, prob[i0:].data_ptr())
    torch.cuda.synchronize()
    return prob[:n].cpu().numpy()


def equal_recall(snr, prob, match, inj_snr, hours, thresh=8.0, min_inj_snr=8.0, low=6.0):
    """The plain threshold against threshold-then-network at equal recall.

    snr, prob: per cluster representative; match: index of the injection it
    matches (Sec. 4.2 rule) or -1; inj_snr: per injection.  Recall = the
    fraction of injections with S/N >= min_inj_snr matched by a selected
    cluster; false positives = selected clusters matching none.  The network
    keeps clusters with S/N >= low and P(pulse) >= p, p the largest cut whose
    recall is within 1 % of the plain threshold's."""
    snr, prob, match = np.asarray(snr), np.asarray(prob), np.asarray(match, dtype=np.int64)
    inj_snr = np.asarray(inj_snr, dtype=np.float64)
    want = inj_snr >= min_inj_snr
    tot = int(want.sum())

    def score(sel):
        m = match[sel]
        found = np.zeros(len(inj_snr), dtype=bool)
        found[m[m >= 0]] = True
        return float((found & want).sum()) / max(tot, 1), int((m < 0).sum())

    base_rec, base_fp = score(snr >= thresh)
    cand = snr >= low
    best = None
    for p in np.unique(np.concatenate([[0.0], prob[cand]]))[::-1]:
        rec, fp = score(cand & (prob >= p))
        if rec >= base_rec - 0.01:
            best = (float(p), rec, fp)
            break
    if best is None:
        best = (0.0,) + score(cand)
    return dict(injected=tot, threshold=thresh, recall_threshold=base_rec, fp_threshold=base_fp,
                p_cut=best[0], recall_cnn=best[1], fp_cnn=best[2], hours=hours,
                fp_per_hour_threshold=base_fp / hours, fp_per_hour_cnn=best[2] / hours)


def evaluate(snr, prob, records, thresh=8.0, min_inj_snr=8.0, tsamp=CHUNK["tsamp"], nout=None):
    """equal_recall() over build_dataset()'s per-chunk records."""
    match, inj_snr = [], []
    for r in records:
        idx = np.arange(r["start"], r["start"] + r["n"])
        off = len(inj_snr)
        m = r["match"] if r["n"] else np.zeros(0, dtype=np.int64)
        match.append(np.where(m >= 0, m + off, -1) if len(idx) else np.zeros(0, dtype=np.int64))
        inj_snr.extend(s for (_, _, _, s) in r["inj"])
    match = np.concatenate(match) if match else np.zeros(0, dtype=np.int64)
    span_s = len(records) * (nout or (CHUNK["nsamp"] - 11682)) * tsamp
    return equal_recall(snr, prob, match, inj_snr, span_s / 3600.0, thresh=thresh, min_inj_snr=min_inj_snr)


def main(argv=None):
    """Train on `--chunks` generated chunks, evaluate on `--eval-chunks` held-out
    ones, print one JSON line, optionally save the checkpoint."""
    import argparse
    import json
    import time
    ap = argparse.ArgumentParser()
    ap.add_argument("--chunks", type=int, default=40000)
    ap.add_argument("--eval-chunks", type=int, default=2000)
    ap.add_argument("--epochs", type=int, default=3)
    ap.add_argument("--batch", type=int, default=256)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--out", default="")
    a = ap.parse_args(argv)
    t0 = time.time()
    searcher = Searcher()
    X, Y, _, _ = build_dataset(a.chunks, a.seed, searcher=searcher)
    t1 = time.time()
    model = _lib.af_model_create(a.batch, a.seed)
    hist = train(model, X, Y, epochs=a.epochs, batch=a.batch, lr=a.lr, seed=a.seed)
    torch.cuda.synchronize()
    t2 = time.time()
    Xe, Ye, snr_e, rec_e = build_dataset(a.eval_chunks, a.seed + 7919, searcher=searcher)
    prob = predict(model, Xe, batch=a.batch)
    res = evaluate(snr_e, prob, rec_e, nout=searcher.nout)
    res.update(samples=int(X.shape[0]), positives=int(Y.sum().item()), eval_samples=int(Xe.shape[0]),
               loss_per_epoch=hist, data_s=t1 - t0, train_s=t2 - t1)
    if a.out:
        _lib.af_model_save(model, a.out)
    print(json.dumps(res))
    _lib.af_model_destroy(model)
    searcher.close()


if __name__ == "__main__":
    main()

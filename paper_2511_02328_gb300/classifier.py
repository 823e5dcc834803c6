"""Training and evaluation of the candidate classifier on synthetic data.

The paper trains its detector on pulses injected into real spectrograms
(Sec. 4.1) and names the RFI that triggers its search (Sec. 4.4): impulsive
broadband (zero-DM) bursts, narrowband interference and burst-like
fluctuations.  Here every chunk is the 256-channel workload (1000-1500 MHz,
98.304 us, 2^15 samples of N(128,12)) with injected dispersed pulses and the
three RFI shapes; the search runs on the GPU, its candidates are clustered
with the true-positive rule of Sec. 4.2, and each cluster's strongest
candidate becomes one sample (two 64 x 64 cut-outs), labelled 1 when it
matches an injected pulse.  The per-channel start samples of the pulses come
from the library's own delay table (a plan over the pulses' DMs).

evaluate() compares, on held-out chunks, the plain boxcar-S/N threshold (the
method without the network) with threshold-then-network at equal recall of
injected pulses with S/N >= 8, and reports both false-positive rates.
"""
import numpy as np
import torch

from . import _lib, synth
from .search import Plan

CHUNK = dict(nchan=256, f_lo=1000.0, f_hi=1500.0, tsamp=98.304e-6, nsamp=1 << 15,
             dm_list=np.arange(0.0, 501.0, 1.0), widths=[1, 2, 4, 8, 16, 32])
DM_TOL, TOA_TOL = 20.0, 0.2


class Generator:
    """Chunks with injected pulses and RFI; pulse delays from the library."""

    def __init__(self, cfg=CHUNK, n_pulses=4, seed=0, device="cuda"):
        self.cfg, self.n_pulses, self.device = cfg, n_pulses, device
        self.rng = np.random.default_rng(seed)
        self.seed = seed
        # one plan over a pool of random injection DMs
        self.pool_dm = self.rng.uniform(20.0, 480.0, 4096)
        p = Plan(cfg["nchan"], cfg["f_lo"], cfg["f_hi"], cfg["tsamp"], self.pool_dm)
        self.pool_delays = p.delays().astype(np.int64)
        self.dmax_search = None
        p.close()
        self.count = 0

    def chunk(self, rfi=True):
        cfg, rng = self.cfg, self.rng
        nchan, nsamp, tsamp = cfg["nchan"], cfg["nsamp"], cfg["tsamp"]
        nout_guess = nsamp - 11682            # output span of the 0..500 DM search at this sampling
        slots = rng.choice(np.arange(1, 5), size=self.n_pulses, replace=False) if self.n_pulses <= 4 else \
            np.arange(1, self.n_pulses + 1)
        pulses, inj = [], []
        span = nout_guess // 5
        for k, s in enumerate(slots):
            j = int(rng.integers(len(self.pool_dm)))
            dm = float(self.pool_dm[j])
            w = max(1, int(round(np.exp(rng.uniform(np.log(0.2e-3), np.log(10e-3))) / tsamp)))
            snr = float(rng.uniform(6.0, 30.0))
            t0 = int(s * span + rng.integers(-span // 4, span // 4))
            pulses.append(synth.Pulse(t0 + self.pool_delays[j], w, synth.pulse_amplitude(snr, nchan, w)))
            inj.append((dm, t0 * tsamp, w, snr))
        r = None
        if rfi:
            narrow = list(rng.choice(nchan, size=2, replace=False))
            bursts = []
            for _ in range(2):
                ln = int(rng.integers(1, 21))
                bursts.append((int(rng.integers(0, nout_guess)), ln, synth.pulse_amplitude(rng.uniform(10, 50), nchan, ln)))
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
    """For each cluster: index of the injection it matches (Sec. 4.2 rule) or -1."""
    res = np.full(len(reps), -1, dtype=np.int64)
    for i, c in enumerate(reps):
        dm, toa = dm_list[int(c["dm_idx"])], int(c["abs_sample"]) * tsamp
        for j, (idm, itoa, _, _) in enumerate(inj):
            if abs(dm - idm) < DM_TOL and abs(toa - itoa) < TOA_TOL:
                res[i] = j
                break
    return res


def build_dataset(n_chunks, seed, searcher=None, gen=None):
    """Returns (cut-outs bf16 [N][64][64][2] on the GPU, labels int32 [N] on the
    GPU, per-sample cluster S/N, per-chunk records for evaluation)."""
    own = searcher is None
    searcher = searcher or Searcher()
    gen = gen or Generator(seed=seed)
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


def evaluate(snr, prob, records, thresh=8.0, min_inj_snr=8.0, tsamp=CHUNK["tsamp"], nout=None):
    """Recall of injected pulses with S/N >= min_inj_snr and false positives
    (clusters matching no injection), for the plain threshold and for the
    network at the probability cut that gives equal recall (within 1 %)."""
    def score(sel):
        hit, tot, fp = 0, 0, 0
        for r in records:
            idx = np.arange(r["start"], r["start"] + r["n"])
            chosen = idx[sel[idx]] if r["n"] else idx
            m = r["match"][chosen - r["start"]] if r["n"] else np.zeros(0, dtype=np.int64)
            fp += int((m < 0).sum())
            found = set(int(j) for j in m if j >= 0)
            for j, (_, _, _, s) in enumerate(r["inj"]):
                if s >= min_inj_snr:
                    tot += 1
                    hit += j in found
        return hit / max(tot, 1), fp, tot
    base_rec, base_fp, tot = score(snr >= thresh)
    best = None
    for p in np.unique(np.concatenate([[0.0], prob]))[::-1]:
        rec, fp, _ = score((snr >= 6.0) & (prob >= p))
        if rec >= base_rec - 0.01:
            best = (float(p), rec, fp)
            break
    if best is None:
        best = (0.0,) + score(snr >= 6.0)[:2]
    span_s = len(records) * (nout or (CHUNK["nsamp"] - 11682)) * tsamp
    return dict(injected=tot, threshold=thresh, recall_threshold=base_rec, fp_threshold=base_fp,
                p_cut=best[0], recall_cnn=best[1], fp_cnn=best[2], hours=span_s / 3600.0,
                fp_per_hour_threshold=base_fp / (span_s / 3600.0), fp_per_hour_cnn=best[2] / (span_s / 3600.0))


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

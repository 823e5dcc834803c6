"""Seeded synthetic filterbank inputs (uint8 [nchan][nsamp], channel-major).

This module only draws and places numbers: Gaussian noise quantised to 8 bits,
boxcar pulses at per-channel start samples that the CALLER supplies, and RFI
shapes.  It contains none of the search's arithmetic (no delay law, no
dedispersion, no S/N), so both the CUDA path and the CPU oracle can be fed the
same inputs from it.  The caller computes the per-channel start samples of a
dispersed pulse with whichever delay table it trusts.

Recipe (stands in for the paper's FAST / QUEST / FAST_FREX data, which are not
available): noise N(128, 12) per sample, rounded half-to-even and clipped to
[0, 255]; a pulse of integrated S/N `snr` and width W samples adds
a = snr * sigma / sqrt(nchan * W) to W samples of every channel before
quantisation.  Random draws use numpy's PCG64 with explicit seeds.
"""
import numpy as np

NOISE_MEAN = 128.0
NOISE_SIGMA = 12.0


def pulse_amplitude(snr, nchan, width, sigma=NOISE_SIGMA):
    """Per-channel amplitude of a boxcar pulse whose matched-filter S/N summed
    over nchan channels and `width` samples is `snr`."""
    return float(snr) * sigma / np.sqrt(float(nchan) * float(width))


class Pulse:
    """A boxcar pulse: starts at offsets[c] in channel c, lasts `width` samples,
    adds `amp` (scalar or per-channel array) before quantisation."""

    def __init__(self, offsets, width, amp):
        self.offsets = np.asarray(offsets, dtype=np.int64)
        self.width = int(width)
        self.amp = amp


class RFI:
    """RFI shapes of the paper's trigger taxonomy (Sec. 4.4): persistent
    narrowband channels, zero-DM broadband bursts and drifting tones."""

    def __init__(self, narrow_channels=(), narrow_mean=3.0, narrow_var=2.0,
                 bursts=(), tones=()):
        # narrow_mean in units of sigma added to the mean; narrow_var scales the variance
        self.narrow_channels = list(narrow_channels)
        self.narrow_mean = narrow_mean
        self.narrow_var = narrow_var
        self.bursts = list(bursts)      # (t_start, length, amplitude)
        self.tones = list(tones)        # (channel0, t_start, length, drift_ch_per_sample, amplitude)


def filterbank(nchan, nsamp, seed, pulses=(), rfi=None, rows_per_chunk=64,
               mean=NOISE_MEAN, sigma=NOISE_SIGMA):
    """uint8 [nchan][nsamp] noise + pulses + RFI, generated channel block by
    channel block from one PCG64 stream (identical for any chunking)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = np.empty((nchan, nsamp), dtype=np.uint8)
    narrow = set(rfi.narrow_channels) if rfi is not None else set()
    for c0 in range(0, nchan, rows_per_chunk):
        c1 = min(nchan, c0 + rows_per_chunk)
        blk = rng.standard_normal((c1 - c0, nsamp), dtype=np.float32)
        blk *= np.float32(sigma)
        blk += np.float32(mean)
        if narrow:
            for c in range(c0, c1):
                if c in narrow:
                    s = np.float32(np.sqrt(rfi.narrow_var))
                    blk[c - c0] = (blk[c - c0] - np.float32(mean)) * s + np.float32(mean + rfi.narrow_mean * sigma)
        for p in pulses:
            amp = np.broadcast_to(np.asarray(p.amp, dtype=np.float32), (nchan,))
            for c in range(c0, c1):
                a = int(p.offsets[c])
                lo, hi = max(0, a), min(nsamp, a + p.width)
                if lo < hi:
                    blk[c - c0, lo:hi] += amp[c]
        if rfi is not None:
            for (t0, ln, amp) in rfi.bursts:
                lo, hi = max(0, int(t0)), min(nsamp, int(t0) + int(ln))
                if lo < hi:
                    blk[:, lo:hi] += np.float32(amp)
            for (ch0, t0, ln, drift, amp) in rfi.tones:
                for k in range(int(ln)):
                    t = int(t0) + k
                    c = int(round(ch0 + drift * k))
                    if c0 <= c < c1 and 0 <= t < nsamp:
                        blk[c - c0, t] += np.float32(amp)
        np.rint(blk, out=blk)
        np.clip(blk, 0, 255, out=blk)
        out[c0:c1] = blk.astype(np.uint8)
    return out


def pulse_params(n, seed, dm_range, width_range_s, snr_range, t_range_s, min_sep_s, tsamp):
    """Draw n pulses: DM ~ U(dm_range), width ~ log-U(width_range_s) rounded to
    >= 1 sample, S/N ~ U(snr_range), arrival times in distinct slots of
    min_sep_s within t_range_s, each jittered by up to a quarter slot (so
    neighbours are at least 0.75 * min_sep_s apart).  Returns a list of dicts
    (dm, width_samples, snr, t0_sample)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t_lo, t_hi = t_range_s
    slots = int((t_hi - t_lo) // min_sep_s)
    if slots < n:
        raise ValueError("not enough room for %d pulses" % n)
    pick = np.sort(rng.choice(slots, size=n, replace=False))
    res = []
    for k in range(n):
        dm = float(rng.uniform(*dm_range))
        w_s = float(np.exp(rng.uniform(np.log(width_range_s[0]), np.log(width_range_s[1]))))
        snr = float(rng.uniform(*snr_range))
        jitter = float(rng.uniform(0.0, 0.25 * min_sep_s))
        t0 = t_lo + pick[k] * min_sep_s + jitter
        res.append(dict(dm=dm, width=max(1, int(round(w_s / tsamp))), snr=snr,
                        t0=int(round(t0 / tsamp))))
    return res


def filterbank_torch(nchan, nsamp, seed, pulses=(), rfi=None, device="cuda", mean=NOISE_MEAN, sigma=NOISE_SIGMA):
    """The same recipe as filterbank(), drawn with a seeded torch generator on
    the GPU (for large training sets); returns a uint8 tensor [nchan][nsamp]."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    x = torch.randn((nchan, nsamp), generator=g, device=device, dtype=torch.float32)
    x.mul_(sigma).add_(mean)
    if rfi is not None:
        for c in rfi.narrow_channels:
            x[c] = (x[c] - mean) * float(np.sqrt(rfi.narrow_var)) + mean + rfi.narrow_mean * sigma
    rows = torch.arange(nchan, device=device)
    for p in pulses:
        offs = torch.as_tensor(np.asarray(p.offsets, dtype=np.int64), device=device)
        cols = offs[:, None] + torch.arange(p.width, device=device)[None, :]
        ok = (cols >= 0) & (cols < nsamp)
        r = rows[:, None].expand_as(cols)[ok]
        amp = torch.as_tensor(np.broadcast_to(np.asarray(p.amp, dtype=np.float32), (nchan,)).copy(), device=device)
        x.index_put_((r, cols[ok]), amp[r], accumulate=True)
    if rfi is not None:
        for (t0, ln, amp) in rfi.bursts:
            lo, hi = max(0, int(t0)), min(nsamp, int(t0) + int(ln))
            if lo < hi:
                x[:, lo:hi] += float(amp)
        for (ch0, t0, ln, drift, amp) in rfi.tones:
            k = torch.arange(int(ln), device=device, dtype=torch.float32)
            c = torch.round(ch0 + drift * k).long()
            t = int(t0) + k.long()
            ok = (c >= 0) & (c < nchan) & (t >= 0) & (t < nsamp)
            x.index_put_((c[ok], t[ok]), torch.full((int(ok.sum()),), float(amp), device=device), accumulate=True)
    x.round_().clamp_(0, 255)
    return x.to(torch.uint8)

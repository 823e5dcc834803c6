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

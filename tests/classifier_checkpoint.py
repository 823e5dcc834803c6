"""Trains a candidate classifier on oracle-injected pulses and writes its
checkpoint; by default the streaming workload's, which the benchmark's
streaming block classifies with.

    python tests/classifier_checkpoint.py --chunks 12000 \
        --out paper_2511_02328_gb300/data/stream_cnn_4096ch.ckpt
    python tests/classifier_checkpoint.py --workload 256ch --chunks 28000 --eval-chunks 3000 --out cnn_256ch.ckpt

The 256ch workload is the learned-classifier configuration: the 256-channel
search's data (1000-1500 MHz, 98.304 us, 2^15 samples, DMs 0..500) with four
pulses per chunk (DM U(20, 480)) and the same RFI classes.

Training data: chunks of the streaming workload's band and DM grid (4096
channels, 1000-1500 MHz, 49.152 us, DMs 0..2000, 2^15 outputs each) of
N(128, 12) noise with three dispersed pulses each (DM U(50, 1950), width
log-U(0.2, 10) ms, S/N U(6, 30)) placed by the CPU oracle's injector
(oracle.injection_offsets, the delay law of Eq. (coarse_delay) applied to
the pulse's DM), plus the RFI of Sec. 4.4 (two narrowband channels, two
zero-DM bursts, one drifting tone).  Each chunk is searched on the GPU at
S/N 6 and clustered (Sec. 4.2); every cluster's strongest candidate becomes
one sample, labelled by whether it matches an injection.  The network trains
with the library's own tcgen05 forward and backward kernels and Adam, then
is scored on held-out chunks against the plain S/N >= 8 threshold at equal
recall.  One JSON line is printed.

This script lives with the tests because it calls the oracle; the library
and the benchmark only read the checkpoint it writes.
"""
import argparse
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--chunks", type=int, default=8000)
    ap.add_argument("--eval-chunks", type=int, default=600)
    ap.add_argument("--epochs", type=int, default=4)
    ap.add_argument("--batch", type=int, default=256)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--seed", type=int, default=11)
    ap.add_argument("--workload", choices=["stream", "256ch"], default="stream")
    ap.add_argument("--out", default=os.path.join(ROOT, "paper_2511_02328_gb300", "data", "stream_cnn_4096ch.ckpt"))
    a = ap.parse_args(argv)
    import __graft_entry__
    __graft_entry__.build()
    import torch
    import oracle
    from paper_2511_02328_gb300 import _lib, classifier

    c = classifier.STREAM_CHUNK if a.workload == "stream" else classifier.CHUNK

    def offsets(dm, t0):
        return oracle.injection_offsets(c["nchan"], c["f_lo"], c["f_hi"], c["tsamp"], dm, t0)

    t0 = time.time()
    searcher = classifier.Searcher(c)
    X, Y, _, _ = classifier.build_dataset(a.chunks, a.seed, searcher=searcher, offsets_fn=offsets)
    t1 = time.time()
    model = _lib.af_model_create(a.batch, a.seed)
    hist = classifier.train(model, X, Y, epochs=a.epochs, batch=a.batch, lr=a.lr, seed=a.seed)
    torch.cuda.synchronize()
    t2 = time.time()
    Xe, Ye, snr_e, rec_e = classifier.build_dataset(a.eval_chunks, a.seed + 7919, searcher=searcher,
                                                    offsets_fn=offsets)
    prob = classifier.predict(model, Xe, batch=a.batch)
    res = classifier.evaluate(snr_e, prob, rec_e, tsamp=c["tsamp"], nout=searcher.nout)
    res.update(samples=int(X.shape[0]), positives=int(Y.sum().item()), eval_samples=int(Xe.shape[0]),
               loss_per_epoch=hist, data_s=t1 - t0, train_s=t2 - t1, chunks=a.chunks, eval_chunks=a.eval_chunks,
               injector="oracle.injection_offsets", workload=a.workload)
    os.makedirs(os.path.dirname(os.path.abspath(a.out)), exist_ok=True)
    _lib.af_model_save(model, a.out)
    print(json.dumps(res))
    _lib.af_model_destroy(model)
    searcher.close()


if __name__ == "__main__":
    main()

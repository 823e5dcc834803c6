"""Torch-facing convenience layer over the C ABI (device memory from torch,
streams from torch.cuda).  Every step runs in the library's CUDA kernels;
this module only allocates tensors and forwards pointers."""
import numpy as np
import torch

from . import _lib


def _stream(stream):
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


class _CudaArray:
    def __init__(self, ptr, shape, typestr):
        self.__cuda_array_interface__ = {"data": (int(ptr), False), "shape": tuple(int(v) for v in shape),
                                         "typestr": typestr, "version": 3, "strides": None}


def device_view(ptr, shape, dtype):
    """A torch tensor viewing library-owned device memory (no copy)."""
    typestr = {torch.int32: "<i4", torch.float32: "<f4", torch.uint8: "|u1", torch.int64: "<i8"}[dtype]
    return torch.as_tensor(_CudaArray(ptr, shape, typestr), device="cuda")


class Plan:
    """Delay-table plan (Eq. coarse_delay, Sec. 2.3) on the current device."""

    def __init__(self, nchan, f_lo, f_hi, tsamp, dm_list, subband=None, channels=None):
        """subband=None: brute-force plan; subband=dict(n0=, nsub=, fs_mode=, block_len=):
        two-stage subband plan (Sec. 2.3, af_plan_subband); channels=(c0, c1): plan for
        that channel range of the band (af_plan_channels, the multi-band search)."""
        self.dm_list = np.ascontiguousarray(dm_list, dtype=np.float64)
        self.c0 = 0
        if channels is not None:
            self.c0 = int(channels[0])
            self.handle = _lib.af_plan_channels(nchan, f_lo, f_hi, tsamp, self.dm_list, channels[0], channels[1])
        elif subband is None:
            self.handle = _lib.af_plan(nchan, f_lo, f_hi, tsamp, self.dm_list)
        else:
            self.handle = _lib.af_plan_subband(nchan, f_lo, f_hi, tsamp, self.dm_list, subband["n0"],
                                               subband["nsub"], subband.get("fs_mode", _lib.AF_FS_INVSQ),
                                               subband.get("block_len", 0))
        self.nchan, self.ndm, self.dmax, self.tsamp = _lib.af_plan_info(self.handle)

    def subband_info(self):
        return _lib.af_plan_subband_info(self.handle)

    def kernel(self):
        """dict(path='simple'|'tile'|'subband'|'pairs', ring, spread, group) of the dedispersion kernel."""
        path, ring, spread, group = _lib.af_plan_kernel(self.handle)
        return dict(path=("simple", "tile", "subband", "pairs")[path], ring=ring, spread=spread, group=group)

    def close(self):
        if self.handle:
            _lib.af_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def delays(self):
        return _lib.af_plan_delays(self.handle)[0]

    def nout(self, nsamp):
        return _lib.af_plan_nout(self.handle, nsamp)

    def reserve(self, nsamp):
        """Reserve the group-row buffer for inputs of up to nsamp samples (no-op for
        plans that cannot use group rows, or when already reserved that far)."""
        if nsamp > getattr(self, "_reserved", 0):
            _lib.af_dedisperse_reserve(self.handle, nsamp)
            self._reserved = nsamp

    def dedisperse(self, x, plane=None, stats=None, stream=None):
        """x: uint8 cuda tensor [nchan][nsamp] -> int32 plane [ndm][nout].  Reserves
        the group-row buffer first when nsamp exceeds the reservation (a
        synchronous allocation; the C call itself never allocates)."""
        assert x.dtype == torch.uint8 and x.is_cuda and x.is_contiguous() and x.shape[0] == self.nchan
        nsamp = x.shape[1]
        self.reserve(nsamp)
        nout = self.nout(nsamp)
        if plane is None:
            plane = torch.empty((self.ndm, nout), dtype=torch.int32, device=x.device)
        _lib.af_dedisperse(self.handle, x.data_ptr(), nsamp, plane.data_ptr(),
                           stats.data_ptr() if stats is not None else 0, _stream(stream))
        return plane

    def rowstats(self, plane, stats=None, stream=None):
        if stats is None:
            stats = torch.empty((self.ndm, 2), dtype=torch.int64, device=plane.device)
        _lib.af_rowstats(self.handle, plane.data_ptr(), plane.shape[1], stats.data_ptr(), _stream(stream))
        return stats

    def boxcar_snr(self, plane, widths, stats=None, snr=None, bw=None, stream=None):
        nout = plane.shape[1]
        if snr is None:
            snr = torch.empty((self.ndm, nout), dtype=torch.float32, device=plane.device)
        if bw is None:
            bw = torch.empty((self.ndm, nout), dtype=torch.uint8, device=plane.device)
        _lib.af_boxcar_snr(self.handle, plane.data_ptr(), nout, stats.data_ptr() if stats is not None else 0,
                           widths, snr.data_ptr(), bw.data_ptr(), _stream(stream))
        return snr, bw

    def candidates(self, snr, bw, widths, thresh, cap=1 << 20, sample0=0, out=None, count=None, stream=None):
        """Returns (candidate tensor [cap, 24 bytes] as uint8, count tensor [1])."""
        dev = snr.device
        if out is None:
            out = torch.empty((cap, _lib.CAND_DTYPE.itemsize), dtype=torch.uint8, device=dev)
        if count is None:
            count = torch.empty(1, dtype=torch.int32, device=dev)
        _lib.af_candidates(self.handle, snr.data_ptr(), bw.data_ptr(), snr.shape[1], widths, thresh, sample0,
                           out.data_ptr(), cap, count.data_ptr(), _stream(stream))
        return out, count

    @staticmethod
    def cands_to_numpy(out, count):
        n = int(count.item())
        m = min(n, out.shape[0])
        arr = out[:m].cpu().numpy().view(_lib.CAND_DTYPE).reshape(-1)
        arr = np.sort(arr, order=["dm_idx", "t"])
        return arr, n

    def search_host(self, h_in, widths, thresh, cap=1 << 20):
        """Whole search from a host uint8 array through af_search."""
        _lib.af_search_reserve(self.handle, h_in.shape[1], cap)
        return _lib.af_search(self.handle, h_in, h_in.shape[1], widths, thresh, cap)

    def cluster(self, cands, dm_tol=20.0, toa_tol=0.2):
        return _lib.af_cluster(self.handle, cands, dm_tol, toa_tol)

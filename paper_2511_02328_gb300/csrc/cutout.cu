// cutout.cu -- the classifier's input: two 64 x 64 cut-outs around each
// candidate (DM-time from the plane, frequency-time from the input
// dedispersed at the candidate's DM), min-max normalised and rounded to
// bfloat16.  This replaces the paper's gridding of DM-time slices into
// 512 x 512 images (Sec. 2.4) and keeps its per-image min-max normalisation
// (without the 8-bit quantisation).  Definitions, per candidate (d, t, w):
//   bins       b = max(1, w / 2); bin j covers output samples
//              [t - 32 b + j b, t - 32 b + (j + 1) b), samples outside [0, nout) count 0
//   DM-time    [i][j] = sum over the bin of plane row d - 32 + i (0 outside [0, ndm))
//   freq-time  [g][j] = sum over channels c of group g (nchan / 64 each) and the
//              bin's samples s of X[c][s + D[d][c]]
//   normalise  v' = float(v - min) / (float(max - min) + 1e-6f), then bf16 (rn)
// Output NHWC bf16 [n][64][64][2]: channel 0 DM-time, 1 freq-time.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <limits.h>
#include <stdint.h>

#include "internal.h"
#include "nn.h"

namespace {

constexpr int S = 64, T = 256;

__device__ __forceinline__ void block_minmax(long long& lo, long long& hi)
{
    __shared__ long long slo[T / 32], shi[T / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        slo[w] = lo;
        shi[w] = hi;
    }
    __syncthreads();
    lo = slo[0];
    hi = shi[0];
    for (int i = 1; i < T / 32; i++) {
        lo = min(lo, slo[i]);
        hi = max(hi, shi[i]);
    }
    __syncthreads();
}

__global__ void __launch_bounds__(T) k_cutout(const uint8_t* __restrict__ X, int64_t nsamp, int nchan,
                                              const int32_t* __restrict__ D, int ndm,
                                              const int32_t* __restrict__ plane, int64_t nout,
                                              const af_cand_t* __restrict__ cands, __nv_bfloat16* __restrict__ out)
{
    constexpr int PER = S * S / T;  // 16 cells per thread and cut-out
    const af_cand_t cd = cands[blockIdx.x];
    const int d = cd.dm_idx;
    if (d < 0 || d >= ndm) {  // not a row of this plan: zero cut-outs
        for (int e = threadIdx.x; e < S * S * 2; e += T) out[(int64_t)blockIdx.x * S * S * 2 + e] = __float2bfloat16(0.f);
        return;
    }
    const int64_t b = cd.width / 2 > 1 ? cd.width / 2 : 1;
    const int64_t start = (int64_t)cd.t - 32 * b;
    const int gsz = nchan / S;
    long long va[PER], vf[PER];
    long long alo = LLONG_MAX, ahi = LLONG_MIN, flo = LLONG_MAX, fhi = LLONG_MIN;
#pragma unroll
    for (int q = 0; q < PER; q++) {
        const int e = threadIdx.x + q * T;
        const int i = e / S, j = e % S;
        const int64_t s0 = max((int64_t)0, start + j * b), s1 = min(nout, start + (j + 1) * b);
        long long a = 0, f = 0;
        const int r = d - 32 + i;
        if (r >= 0 && r < ndm)
            for (int64_t s = s0; s < s1; s++) a += __ldg(plane + (int64_t)r * nout + s);
        for (int c = i * gsz; c < (i + 1) * gsz; c++) {
            const uint8_t* xc = X + (int64_t)c * nsamp + __ldg(D + (int64_t)d * nchan + c);
            for (int64_t s = s0; s < s1; s++) f += __ldg(xc + s);
        }
        va[q] = a;
        vf[q] = f;
        alo = min(alo, a);
        ahi = max(ahi, a);
        flo = min(flo, f);
        fhi = max(fhi, f);
    }
    block_minmax(alo, ahi);
    block_minmax(flo, fhi);
    const float ad = (float)(ahi - alo) + 1e-6f, fd = (float)(fhi - flo) + 1e-6f;
    __nv_bfloat16* o = out + (int64_t)blockIdx.x * S * S * 2;
#pragma unroll
    for (int q = 0; q < PER; q++) {
        const int e = threadIdx.x + q * T;
        o[2 * e] = __float2bfloat16_rn(__fdiv_rn((float)(va[q] - alo), ad));
        o[2 * e + 1] = __float2bfloat16_rn(__fdiv_rn((float)(vf[q] - flo), fd));
    }
}

}  // namespace

int nn_cutouts(const uint8_t* X, int64_t nsamp, int nchan, const int32_t* D, int ndm, const int32_t* plane,
               int64_t nout, const af_cand_t* cands, int n, __nv_bfloat16* out, cudaStream_t s)
{
    if (n <= 0) return AF_OK;
    k_cutout<<<n, T, 0, s>>>(X, nsamp, nchan, D, ndm, plane, nout, cands, out);
    return af_cuda_check(cudaGetLastError(), "cut-out launch");
}

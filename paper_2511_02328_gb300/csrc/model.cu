// model.cu -- the candidate classifier: parameters, workspace, forward,
// backward and Adam, built from the kernels of conv_umma.cu and nn.cu (the
// paper's detector is YOLOv11n on DM-time images, Sec. 2.5; this small CNN
// replaces it).
//
// The convolutions run on the tcgen05 tensor cores with their operand tiles
// staged by TMA from channel-blocked activations (conv_tma.cu: forward with
// bias, ReLU and max pool fused; data and weight gradients), keeping the
// pooled activations and argmax bytes the backward pass needs.  Inference of
// batches below a measured size runs the one-kernel mma.sync network of
// nn_fused.cu instead, which needs no intermediate activations in memory.
// Network: input NHWC bf16 [n][64][64][2]; three blocks conv3x3 (+bias) ->
// ReLU -> 2x2 max pool with 2 -> 16 -> 32 -> 64 channels; global average pool;
// fully connected 64 -> 2; softmax cross-entropy (label 1 = pulse).
// Parameters, fp32, flat in this order: w0 [16][3][3][2], b0 [16],
// w1 [32][3][3][16], b1 [32], w2 [64][3][3][32], b2 [64], fw [2][64], fb [2].
// Tensor-core operands are bf16 (input, packed weights, pooled activations,
// activation gradients); accumulation, ReLU outputs, biases, weight gradients,
// master weights and Adam state are fp32.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "internal.h"
#include "nn.h"

namespace {

constexpr int NL = 3;
constexpr int CH[NL + 1] = {2, 16, 32, 64};

struct Layer {
    int cin, cout, H, W, k9;
    int64_t woff, boff;
};


// Inference batches of at least this many images run the layered tensor-core
// network; smaller ones the fused one-kernel network (AFGB_CNN_UMMA_MIN
// overrides at model creation).  Measured on GB300, fused / layered: 0.040 /
// 0.058 ms at 128 images, 0.074 / 0.070 ms at 256, 0.141 / 0.087 ms at 512.
constexpr int kUmmaInferMin = 256;

}  // namespace

struct af_model_s {
    int device = 0, max_batch = 0;
    int64_t nparams = 0;
    int step = 0;
    Layer L[NL];
    int64_t fw_off = 0, fb_off = 0;
    float *d_params = nullptr, *d_grads = nullptr, *d_m = nullptr, *d_v = nullptr;
    __nv_bfloat16* d_wt[NL] = {};      // forward weights, packed for the tensor cores (nn_tpack)
    __nv_bfloat16* d_wd[NL] = {};      // data-gradient weights, packed (l >= 1)
    __nv_bfloat16* d_a[NL + 1] = {};   // pooled activations, channel-blocked; d_a[0] unused
    uint8_t* d_idx[NL] = {};           // argmax of each pool window | 4 if its maximum > 0
    __nv_bfloat16* d_da[NL + 1] = {};  // gradients w.r.t. d_a[l] (l >= 1)
    __nv_bfloat16* d_dz[NL] = {};      // gradients w.r.t. the pre-pool ReLU outputs (layers 1, 2)
    float* d_logits = nullptr;
    float* d_loss = nullptr;
    int* d_err = nullptr;              // raised by a bounded tensor-core wait that ran out
    __nv_bfloat16* d_cut = nullptr;    // cut-outs for af_classify
    int umma_min = 0;                  // inference batches of at least this size use the tensor-core layers
    // d_wt holds the packed form of the current d_params (set by a forward pass
    // that packed them, on the stream where packed_ev is recorded; cleared by
    // every call that changes the parameters)
    bool packed = false;
    cudaEvent_t packed_ev = nullptr;
};

static void free_model(af_model_t m)
{
    if (!m) return;
    cudaFree(m->d_params);
    cudaFree(m->d_grads);
    cudaFree(m->d_m);
    cudaFree(m->d_v);
    for (int l = 0; l < NL; l++) {
        cudaFree(m->d_wt[l]);
        cudaFree(m->d_wd[l]);
        cudaFree(m->d_idx[l]);
        cudaFree(m->d_dz[l]);
    }
    for (int l = 0; l <= NL; l++) {
        cudaFree(m->d_a[l]);
        cudaFree(m->d_da[l]);
    }
    cudaFree(m->d_err);
    cudaFree(m->d_logits);
    cudaFree(m->d_loss);
    cudaFree(m->d_cut);
    if (m->packed_ev) cudaEventDestroy(m->packed_ev);
    delete m;
}

// He-normal initial weights from a counter-free PCG32 stream + Box-Muller.
static void init_weights(af_model_t m, uint64_t seed, std::vector<float>& p)
{
    uint64_t state = seed * 6364136223846793005ULL + 1442695040888963407ULL;
    auto next = [&]() {
        const uint64_t old = state;
        state = old * 6364136223846793005ULL + 1442695040888963407ULL;
        const uint32_t xs = (uint32_t)(((old >> 18) ^ old) >> 27), rot = (uint32_t)(old >> 59);
        return (xs >> rot) | (xs << ((32 - rot) & 31));
    };
    auto normal = [&]() {
        const double u1 = ((double)next() + 1.0) / 4294967297.0, u2 = (double)next() / 4294967296.0;
        return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
    };
    p.assign(m->nparams, 0.0f);
    for (int l = 0; l < NL; l++) {
        const double sd = sqrt(2.0 / (9.0 * m->L[l].cin));
        for (int64_t i = 0; i < (int64_t)m->L[l].cout * m->L[l].k9; i++) p[m->L[l].woff + i] = (float)(sd * normal());
    }
    for (int i = 0; i < 128; i++) p[m->fw_off + i] = (float)(normal() / 8.0);
}

extern "C" int af_model_create(af_model_t* out, int max_batch, uint64_t seed)
try {
    if (!out || max_batch < 1 || max_batch > 65536) return af_set_error(AF_EINVAL, "af_model_create: bad arguments");
    *out = nullptr;
    af_model_s* m = new (std::nothrow) af_model_s();
    if (!m) return af_set_error(AF_ENOMEM, "af_model_create: host allocation");
    cudaGetDevice(&m->device);
    m->max_batch = max_batch;
    int64_t off = 0;
    int H = 64;
    for (int l = 0; l < NL; l++) {
        Layer& y = m->L[l];
        y.cin = CH[l];
        y.cout = CH[l + 1];
        y.H = y.W = H;
        y.k9 = 9 * y.cin;
        y.woff = off;
        off += (int64_t)y.cout * y.k9;
        y.boff = off;
        off += y.cout;
        H /= 2;
    }
    m->fw_off = off;
    off += 128;
    m->fb_off = off;
    off += 2;
    m->nparams = off;
    const int64_t n = max_batch;
    cudaError_t e = cudaSuccess;
    auto A = [&](auto** p, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc((void**)p, bytes);
    };
    A(&m->d_params, off * 4);
    A(&m->d_grads, off * 4);
    A(&m->d_m, off * 4);
    A(&m->d_v, off * 4);
    for (int l = 0; l < NL; l++) {
        const Layer& y = m->L[l];
        const int64_t P = n * y.H * y.W;
        A(&m->d_wt[l], nn_tpack_bytes(l, 0));
        if (l > 0) A(&m->d_wd[l], nn_tpack_bytes(l, 1));
        A(&m->d_idx[l], (size_t)P * y.cout / 4);
        if (l > 0) A(&m->d_dz[l], (size_t)P * y.cout * 2);  // layer 0's is never stored
        A(&m->d_a[l + 1], (size_t)P * y.cout / 4 * 2);
        A(&m->d_da[l + 1], (size_t)P * y.cout / 4 * 2);
    }
    A(&m->d_err, 16);
    A(&m->d_logits, (size_t)n * 2 * 4);
    A(&m->d_loss, 16);
    A(&m->d_cut, (size_t)n * 64 * 64 * 2 * 2);
    if (e == cudaSuccess) e = cudaMemset(m->d_err, 0, 16);
    if (e == cudaSuccess) e = cudaMemset(m->d_m, 0, off * 4);
    if (e == cudaSuccess) e = cudaMemset(m->d_v, 0, off * 4);
    if (e != cudaSuccess) {
        int rc = af_cuda_check(e, "af_model_create");
        free_model(m);
        return rc;
    }
    std::vector<float> p;
    init_weights(m, seed, p);
    e = cudaMemcpy(m->d_params, p.data(), off * 4, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        int rc = af_cuda_check(e, "af_model_create: upload");
        free_model(m);
        return rc;
    }
    m->umma_min = kUmmaInferMin;
    if (const char* v = getenv("AFGB_CNN_UMMA_MIN")) m->umma_min = atoi(v);
    *out = m;
    return AF_OK;
} catch (...) {
    return af_host_exception("af_model_create");
}

extern "C" int af_model_destroy(af_model_t m)
try {
    free_model(m);
    return AF_OK;
} catch (...) {
    return af_host_exception("af_model_destroy");
}

extern "C" int af_model_nparams(af_model_t m, int64_t* n)
try {
    if (!m || !n) return af_set_error(AF_EINVAL, "af_model_nparams: NULL argument");
    *n = m->nparams;
    return AF_OK;
} catch (...) {
    return af_host_exception("af_model_nparams");
}

// Reads (and clears) the flag a bounded tensor-core wait raises when it runs
// out; synchronises the device.
static int check_err(af_model_t m, const char* what)
{
    int h = 0;
    AF_CUDA(cudaMemcpy(&h, m->d_err, sizeof h, cudaMemcpyDeviceToHost));
    if (h) {
        AF_CUDA(cudaMemset(m->d_err, 0, sizeof h));
        return af_set_error(AF_ETIMEOUT, "%s: a tensor-core kernel's bounded wait ran out", what);
    }
    return AF_OK;
}

static int copy_params(af_model_t m, float* dst, const float* src, int64_t n, cudaMemcpyKind kind, const char* what)
{
    if (!m || (!dst && !src)) return af_set_error(AF_EINVAL, "%s: NULL argument", what);
    if (int rc = check_err(m, what)) return rc;
    if (n != m->nparams) return af_set_error(AF_EINVAL, "%s: %lld values, the model has %lld", what, (long long)n,
                                             (long long)m->nparams);
    AF_CUDA(cudaMemcpy(dst, src, n * 4, kind));
    return AF_OK;
}

extern "C" int af_model_set_params(af_model_t m, const float* h, int64_t n)
try {
    if (!m || !h) return af_set_error(AF_EINVAL, "af_model_set_params: NULL argument");
    m->packed = false;
    return copy_params(m, m->d_params, h, n, cudaMemcpyHostToDevice, "af_model_set_params");
} catch (...) {
    return af_host_exception("af_model_set_params");
}

extern "C" int af_model_get_params(af_model_t m, float* h, int64_t n)
try {
    if (!m || !h) return af_set_error(AF_EINVAL, "af_model_get_params: NULL argument");
    return copy_params(m, h, m->d_params, n, cudaMemcpyDeviceToHost, "af_model_get_params");
} catch (...) {
    return af_host_exception("af_model_get_params");
}

extern "C" int af_model_get_grads(af_model_t m, float* h, int64_t n)
try {
    if (!m || !h) return af_set_error(AF_EINVAL, "af_model_get_grads: NULL argument");
    return copy_params(m, h, m->d_grads, n, cudaMemcpyDeviceToHost, "af_model_get_grads");
} catch (...) {
    return af_host_exception("af_model_get_grads");
}

static int forward(af_model_t m, const __nv_bfloat16* x, int n, const int32_t* y, float* prob, cudaStream_t s)
{
    const float* P = m->d_params;
    if (!y && n < m->umma_min)  // small inference batch: one fused kernel
        return nn_forward_fused(x, n, P + m->L[0].woff, P + m->L[0].boff, P + m->L[1].woff, P + m->L[1].boff,
                                P + m->L[2].woff, P + m->L[2].boff, P + m->fw_off, P + m->fb_off, m->d_logits, prob,
                                s);
    if (!m->packed) {  // the parameters changed since the last packing
        for (int l = 0; l < NL; l++)
            if (int rc = nn_tpack(l, 0, P + m->L[l].woff, m->d_wt[l], s)) return rc;
        if (!m->packed_ev) AF_CUDA(cudaEventCreateWithFlags(&m->packed_ev, cudaEventDisableTiming));
        AF_CUDA(cudaEventRecord(m->packed_ev, s));
        m->packed = true;
    } else {
        AF_CUDA(cudaStreamWaitEvent(s, m->packed_ev, 0));  // packed on this or another stream
    }
    const __nv_bfloat16* a = x;  // the first layer expands its columns itself
    for (int l = 0; l < NL; l++) {
        const Layer& L = m->L[l];
        if (int rc = nn_tconv_fwd(l, a, n, m->d_wt[l], P + L.boff, m->d_a[l + 1], y ? m->d_idx[l] : nullptr, m->d_err,
                                  s))
            return rc;
        a = m->d_a[l + 1];
    }
    if (y) {
        AF_CUDA(cudaMemsetAsync(m->d_loss, 0, 4, s));
        AF_CUDA(cudaMemsetAsync(m->d_grads, 0, m->nparams * 4, s));
    }
    return nn_head(m->d_a[NL], n, P + m->fw_off, P + m->fb_off, m->d_logits, prob, y, m->d_loss,
                   m->d_grads + m->fw_off, m->d_grads + m->fb_off, m->d_da[NL], s);
}

// After forward() with labels: the channel-blocked input and activations are
// in place.
static int backward(af_model_t m, const __nv_bfloat16* x, int n, cudaStream_t s)
{
    for (int l = NL - 1; l >= 0; l--) {
        const Layer& L = m->L[l];
        if (l == 0)  // the first layer's output gradient feeds only its weight gradient: unpooled inside it
            return nn_tconv_wgrad_unpool(m->d_da[1], m->d_idx[0], x, n, m->d_grads + L.woff,
                                         m->d_grads + L.boff, m->d_err, s);
        if (int rc = nn_pool_back(m->d_da[l + 1], m->d_idx[l], n, L.H, L.W, L.cout, m->d_dz[l], m->d_grads + L.boff, s))
            return rc;
        const __nv_bfloat16* a = l ? m->d_a[l] : x;
        if (int rc = nn_tconv_wgrad(l, m->d_dz[l], a, n, m->d_grads + L.woff, m->d_err, s)) return rc;
        if (l > 0) {
            if (int rc = nn_tpack(l, 1, m->d_params + L.woff, m->d_wd[l], s)) return rc;
            if (int rc = nn_tconv_dgrad(l, m->d_dz[l], n, m->d_wd[l], m->d_da[l], m->d_err, s)) return rc;
        }
    }
    return AF_OK;
}

static int check_batch(af_model_t m, const void* x, int n)
{
    if (!m || !x) return af_set_error(AF_EINVAL, "model: NULL argument");
    if (n < 1 || n > m->max_batch) return af_set_error(AF_EINVAL, "model: batch %d outside 1..%d", n, m->max_batch);
    if ((uintptr_t)x & 15) return af_set_error(AF_EINVAL, "model: input not 16-byte aligned");
    return AF_OK;
}

extern "C" int af_model_forward(af_model_t m, const uint16_t* d_x, int32_t n, float* d_logits, float* d_prob,
                                void* stream)
try {
    if (int rc = check_batch(m, d_x, n)) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    if (int rc = forward(m, (const __nv_bfloat16*)d_x, n, nullptr, d_prob, s)) return rc;
    if (d_logits) AF_CUDA(cudaMemcpyAsync(d_logits, m->d_logits, (size_t)n * 8, cudaMemcpyDeviceToDevice, s));
    return AF_OK;
} catch (...) {
    return af_host_exception("af_model_forward");
}

extern "C" int af_model_backward(af_model_t m, const uint16_t* d_x, const int32_t* d_y, int32_t n, float* d_loss,
                                 void* stream)
try {
    if (int rc = check_batch(m, d_x, n)) return rc;
    if (!d_y) return af_set_error(AF_EINVAL, "af_model_backward: labels NULL");
    cudaStream_t s = (cudaStream_t)stream;
    if (int rc = forward(m, (const __nv_bfloat16*)d_x, n, d_y, nullptr, s)) return rc;
    if (int rc = backward(m, (const __nv_bfloat16*)d_x, n, s)) return rc;
    if (d_loss) AF_CUDA(cudaMemcpyAsync(d_loss, m->d_loss, 4, cudaMemcpyDeviceToDevice, s));
    return AF_OK;
} catch (...) {
    return af_host_exception("af_model_backward");
}

extern "C" int af_train_step(af_model_t m, const uint16_t* d_x, const int32_t* d_y, int32_t n, float lr,
                             float* d_loss, void* stream)
try {
    if (!(lr > 0.0f) || !isfinite(lr)) return af_set_error(AF_EINVAL, "af_train_step: bad learning rate");
    if (int rc = af_model_backward(m, d_x, d_y, n, d_loss, stream)) return rc;
    m->step++;
    m->packed = false;
    return nn_adam(m->d_params, m->d_grads, m->d_m, m->d_v, m->nparams, lr, m->step, (cudaStream_t)stream);
} catch (...) {
    return af_host_exception("af_train_step");
}

extern "C" int af_nn_gemm(int layout, int epi, const uint16_t* d_a, int lda, const uint16_t* d_b, int ldb, int M,
                          int N, int K, int splits, float* d_c, int ldc, const float* d_bias, void* stream)
try {
    if (!d_a || !d_b || !d_c || (epi == NN_EPI_BIAS_RELU && !d_bias) || epi < 0 || epi > 2 || ldc < N)
        return af_set_error(AF_EINVAL, "af_nn_gemm: bad arguments");
    // a test entry point: it allocates its bounded-wait flag, waits for the
    // stream and reports a wait that ran out
    int* d_err = nullptr;
    AF_CUDA(cudaMalloc(&d_err, sizeof(int)));
    cudaStream_t s = (cudaStream_t)stream;
    int rc = af_cuda_check(cudaMemsetAsync(d_err, 0, sizeof(int), s), "af_nn_gemm");
    if (!rc)
        rc = nn_gemm(layout, epi, (const __nv_bfloat16*)d_a, lda, (const __nv_bfloat16*)d_b, ldb, M, N, K, splits, d_c,
                     ldc, d_bias, d_err, s);
    int h = 0;
    if (!rc) rc = af_cuda_check(cudaMemcpyAsync(&h, d_err, sizeof h, cudaMemcpyDeviceToHost, s), "af_nn_gemm");
    if (!rc) rc = af_cuda_check(cudaStreamSynchronize(s), "af_nn_gemm");
    cudaFree(d_err);
    if (!rc && h) rc = af_set_error(AF_ETIMEOUT, "af_nn_gemm: a bounded wait ran out");
    return rc;
} catch (...) {
    return af_host_exception("af_nn_gemm");
}

extern "C" int af_cutouts(af_plan_t p, const uint8_t* d_in, int64_t nsamp, const int32_t* d_plane, int64_t nout,
                          const af_cand_t* d_cands, int32_t n, uint16_t* d_out, void* stream)
try {
    if (int rc = af_check_plan(p)) return rc;
    if (!d_in || !d_plane || (n > 0 && (!d_cands || !d_out)) || n < 0)
        return af_set_error(AF_EINVAL, "af_cutouts: NULL buffer");
    if (p->nchan % 64) return af_set_error(AF_EINVAL, "af_cutouts: nchan %d is not a multiple of 64", p->nchan);
    if (nout != nsamp - p->dmax) return af_set_error(AF_EINVAL, "af_cutouts: nout must be nsamp - Dmax");
    return nn_cutouts(d_in, nsamp, p->nchan, p->d_delays, p->ndm, d_plane, nout, d_cands, n, (__nv_bfloat16*)d_out,
                      (cudaStream_t)stream);
} catch (...) {
    return af_host_exception("af_cutouts");
}

extern "C" int af_classify(af_model_t m, af_plan_t p, const uint8_t* d_in, int64_t nsamp, const int32_t* d_plane,
                           int64_t nout, const af_cand_t* d_cands, int32_t n, float* d_prob, void* stream)
try {
    if (!m || !d_prob) return af_set_error(AF_EINVAL, "af_classify: NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    for (int32_t i0 = 0; i0 < n; i0 += m->max_batch) {
        const int32_t k = std::min(m->max_batch, n - i0);
        if (int rc = af_cutouts(p, d_in, nsamp, d_plane, nout, d_cands + i0, k, (uint16_t*)m->d_cut, stream))
            return rc;
        if (int rc = forward(m, m->d_cut, k, nullptr, d_prob + i0, s)) return rc;
    }
    return AF_OK;
} catch (...) {
    return af_host_exception("af_classify");
}

// Checkpoint: a JSON header line, then raw little-endian fp32 parameters and
// Adam moments.
extern "C" int af_model_save(af_model_t m, const char* path)
try {
    if (!m || !path) return af_set_error(AF_EINVAL, "af_model_save: NULL argument");
    if (int rc = check_err(m, "af_model_save")) return rc;
    std::vector<float> buf(3 * m->nparams);
    AF_CUDA(cudaMemcpy(buf.data(), m->d_params, m->nparams * 4, cudaMemcpyDeviceToHost));
    AF_CUDA(cudaMemcpy(buf.data() + m->nparams, m->d_m, m->nparams * 4, cudaMemcpyDeviceToHost));
    AF_CUDA(cudaMemcpy(buf.data() + 2 * m->nparams, m->d_v, m->nparams * 4, cudaMemcpyDeviceToHost));
    FILE* f = fopen(path, "wb");
    if (!f) return af_set_error(AF_EINVAL, "af_model_save: cannot open %s", path);
    fprintf(f, "{\"format\": \"afgb-cnn-1\", \"nparams\": %lld, \"step\": %d, \"channels\": [2, 16, 32, 64]}\n",
            (long long)m->nparams, m->step);
    const size_t wrote = fwrite(buf.data(), 4, buf.size(), f);
    fclose(f);
    if (wrote != buf.size()) return af_set_error(AF_EINVAL, "af_model_save: short write");
    return AF_OK;
} catch (...) {
    return af_host_exception("af_model_save");
}

extern "C" int af_model_load(af_model_t m, const char* path)
try {
    if (!m || !path) return af_set_error(AF_EINVAL, "af_model_load: NULL argument");
    FILE* f = fopen(path, "rb");
    if (!f) return af_set_error(AF_EINVAL, "af_model_load: cannot open %s", path);
    char line[512];
    if (!fgets(line, sizeof line, f) || !strstr(line, "afgb-cnn-1")) {
        fclose(f);
        return af_set_error(AF_EINVAL, "af_model_load: not a classifier checkpoint");
    }
    long long np = 0;
    int step = 0;
    const char* a = strstr(line, "\"nparams\":");
    const char* b = strstr(line, "\"step\":");
    if (a) np = atoll(a + 10);
    if (b) step = atoi(b + 7);
    if (np != m->nparams) {
        fclose(f);
        return af_set_error(AF_EINVAL, "af_model_load: %lld parameters, the model has %lld", np, (long long)m->nparams);
    }
    std::vector<float> buf(3 * m->nparams);
    const size_t got = fread(buf.data(), 4, buf.size(), f);
    fclose(f);
    if (got != buf.size()) return af_set_error(AF_EINVAL, "af_model_load: truncated checkpoint");
    m->packed = false;
    AF_CUDA(cudaMemcpy(m->d_params, buf.data(), m->nparams * 4, cudaMemcpyHostToDevice));
    AF_CUDA(cudaMemcpy(m->d_m, buf.data() + m->nparams, m->nparams * 4, cudaMemcpyHostToDevice));
    AF_CUDA(cudaMemcpy(m->d_v, buf.data() + 2 * m->nparams, m->nparams * 4, cudaMemcpyHostToDevice));
    m->step = step;
    return AF_OK;
} catch (...) {
    return af_host_exception("af_model_load");
}

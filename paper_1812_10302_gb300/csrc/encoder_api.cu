// encoder_api.cu -- C ABI of the learned proposal encoder that needs no
// search handle: input preparation, forward, loss + gradient, and the Adam
// trainer.  The kernels are in encoder.cu.
#include <cstring>
#include <new>

#include "dtws.h"
#include "dtws_internal.h"

using namespace dtws;

namespace {

#define EK(call)                                                                    \
    do {                                                                            \
        cudaError_t e__ = (call);                                                   \
        if (e__ != cudaSuccess) {                                                   \
            set_error_detail("%s:%d %s: %s", __FILE__, __LINE__, #call,             \
                             cudaGetErrorString(e__));                              \
            return e__ == cudaErrorMemoryAllocation ? DTWS_ENOMEM : DTWS_ECUDA;     \
        }                                                                           \
    } while (0)

// device memory released on scope exit
struct DevMem {
    void *p = nullptr;
    ~DevMem() {
        if (p) cudaFree(p);
    }
    cudaError_t alloc(size_t bytes) { return cudaMalloc(&p, bytes < 256 ? 256 : bytes); }
    template <typename T>
    T *as() const { return reinterpret_cast<T *>(p); }
};

int num_sms() {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    return v > 0 ? v : 1;
}

// Parameters (host or device FP32) -> packed blob in `blob` (device);
// `pbuf` receives the FP32 copy.
cudaError_t pack_params(const float *params, float *pbuf, uint8_t *blob, cudaStream_t s) {
    cudaError_t e = cudaMemcpyAsync(pbuf, params, (size_t)kEncParams * 4, cudaMemcpyDefault, s);
    if (e != cudaSuccess) return e;
    return launch_enc_pack(pbuf, nullptr, nullptr, nullptr, blob, false, 0.f, 0.f, 0.f, 0.f, 1.f, 1.f, s);
}

bool finite_all(const float *v, int64_t n) {
    for (int64_t i = 0; i < n; ++i)
        if (!(v[i] - v[i] == 0.0f)) return false;
    return true;
}

}  // namespace

struct dtws_trainer_ctx {
    int max_batch = 0, sms = 1;
    float *params = nullptr, *grad = nullptr, *m1 = nullptr, *v1 = nullptr, *u = nullptr, *y = nullptr;
    float *loss = nullptr;
    int64_t *off = nullptr;
    uint8_t *blob = nullptr, *ws = nullptr;
    dtws_adam hp{};
    int64_t t = 0;
};

extern "C" {

dtws_status dtws_enc_prep(const float *X, int64_t n, const int64_t *offsets, int32_t rows, int32_t m, float *u,
                          void *stream) {
    if (!X || !offsets || !u || rows < 1 || m < 64 || m > DTWS_M_MAX || n < m) {
        set_error_detail("dtws_enc_prep: null argument, rows < 1 or m out of range [64, min(n, %d)]", DTWS_M_MAX);
        return DTWS_EINVAL;
    }
    for (int32_t i = 0; i < rows; ++i)
        if (offsets[i] < 0 || offsets[i] > n - m) {
            set_error_detail("dtws_enc_prep: offsets[%d] = %lld out of [0, n-m]", i, (long long)offsets[i]);
            return DTWS_EINVAL;
        }
    cudaStream_t s = (cudaStream_t)stream;
    DevMem xd, od, ud;
    EK(xd.alloc((size_t)n * 4));
    EK(od.alloc((size_t)rows * 8));
    EK(ud.alloc((size_t)rows * DTWS_ENC_U * 4));
    EK(cudaMemcpyAsync(xd.p, X, (size_t)n * 4, cudaMemcpyDefault, s));
    EK(cudaMemcpyAsync(od.p, offsets, (size_t)rows * 8, cudaMemcpyHostToDevice, s));
    EK(launch_enc_prep(xd.as<float>(), od.as<int64_t>(), rows, m, ud.as<float>(), s));
    EK(cudaMemcpyAsync(u, ud.p, (size_t)rows * DTWS_ENC_U * 4, cudaMemcpyDefault, s));
    EK(cudaStreamSynchronize(s));
    return DTWS_OK;
}

dtws_status dtws_enc_forward(const float *params, const float *u, int32_t rows, float *e, void *stream) {
    if (!params || !u || !e || rows < 1) {
        set_error_detail("dtws_enc_forward: null argument or rows < 1");
        return DTWS_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    DevMem pb, blob, ud, ed;
    EK(pb.alloc((size_t)kEncParams * 4));
    EK(blob.alloc(kEncBlobBytes));
    EK(ud.alloc((size_t)rows * DTWS_ENC_U * 4));
    EK(ed.alloc((size_t)rows * DTWS_ENC_DIM * 4));
    EK(pack_params(params, pb.as<float>(), blob.as<uint8_t>(), s));
    EK(cudaMemcpyAsync(ud.p, u, (size_t)rows * DTWS_ENC_U * 4, cudaMemcpyDefault, s));
    EK(launch_enc_forward(blob.as<uint8_t>(), ud.as<float>(), rows, ed.as<float>(), nullptr, num_sms(), s));
    EK(cudaMemcpyAsync(e, ed.p, (size_t)rows * DTWS_ENC_DIM * 4, cudaMemcpyDefault, s));
    EK(cudaStreamSynchronize(s));
    return DTWS_OK;
}

dtws_status dtws_enc_loss_grad(const float *params, const float *uq, const float *uc, const float *y,
                               int32_t batch, float *loss, float *grad, void *stream) {
    if (!params || !uq || !uc || !y || !loss || !grad || batch < 1 || batch > 65536) {
        set_error_detail("dtws_enc_loss_grad: null argument or batch out of [1, 65536]");
        return DTWS_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const size_t urow = (size_t)DTWS_ENC_U * 4;
    DevMem pb, blob, ud, yd, ld, gd, ws;
    EK(pb.alloc((size_t)kEncParams * 4));
    EK(blob.alloc(kEncBlobBytes));
    EK(ud.alloc(2 * (size_t)batch * urow));
    EK(yd.alloc((size_t)batch * 4));
    EK(ld.alloc(4));
    EK(gd.alloc((size_t)kEncParams * 4));
    EK(ws.alloc(enc_workspace_bytes(2 * batch)));
    EK(pack_params(params, pb.as<float>(), blob.as<uint8_t>(), s));
    EK(cudaMemcpyAsync(ud.p, uq, (size_t)batch * urow, cudaMemcpyDefault, s));
    EK(cudaMemcpyAsync(ud.as<uint8_t>() + (size_t)batch * urow, uc, (size_t)batch * urow, cudaMemcpyDefault, s));
    EK(cudaMemcpyAsync(yd.p, y, (size_t)batch * 4, cudaMemcpyDefault, s));
    EK(cudaMemsetAsync(ld.p, 0, 4, s));
    const int sms = num_sms();
    EK(launch_enc_forward(blob.as<uint8_t>(), ud.as<float>(), 2 * batch, nullptr, ws.as<uint8_t>(), sms, s));
    EK(launch_enc_backward(blob.as<uint8_t>(), yd.as<float>(), batch, ld.as<float>(), gd.as<float>(),
                           ws.as<uint8_t>(), sms, s));
    EK(cudaMemcpyAsync(grad, gd.p, (size_t)kEncParams * 4, cudaMemcpyDefault, s));
    EK(cudaMemcpyAsync(loss, ld.p, 4, cudaMemcpyDeviceToHost, s));
    EK(cudaStreamSynchronize(s));
    return DTWS_OK;
}

dtws_status dtws_trainer_destroy(dtws_trainer_t t) {
    if (!t) return DTWS_EINVAL;
    cudaDeviceSynchronize();
    void *ptrs[] = {t->params, t->grad, t->m1, t->v1, t->u, t->y, t->loss, t->off, t->blob, t->ws};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    delete t;
    return DTWS_OK;
}

dtws_status dtws_trainer_create(const float *params, int32_t count, int32_t max_batch, const dtws_adam *hp,
                                dtws_trainer_t *out) {
    if (!out) return DTWS_EINVAL;
    *out = nullptr;
    if (!params || count != kEncParams || max_batch < 1 || max_batch > 65536 || !hp || !(hp->lr > 0.0f) ||
        !(hp->beta1 >= 0.0f && hp->beta1 < 1.0f) || !(hp->beta2 >= 0.0f && hp->beta2 < 1.0f) || !(hp->eps > 0.0f)) {
        set_error_detail("dtws_trainer_create: bad arguments");
        return DTWS_EINVAL;
    }
    dtws_trainer_ctx *t = new (std::nothrow) dtws_trainer_ctx();
    if (!t) return DTWS_ENOMEM;
    t->max_batch = max_batch;
    t->hp = *hp;
    t->sms = num_sms();
    auto fail = [&](cudaError_t e) {
        set_error_detail("dtws_trainer_create: %s", cudaGetErrorString(e));
        dtws_trainer_destroy(t);
        return e == cudaErrorMemoryAllocation ? DTWS_ENOMEM : DTWS_ECUDA;
    };
    const size_t P = (size_t)kEncParams * 4;
    cudaError_t e;
    if ((e = cudaMalloc(&t->params, P)) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(&t->grad, P)) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(&t->m1, P)) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(&t->v1, P)) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(&t->u, 2 * (size_t)max_batch * DTWS_ENC_U * 4)) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(&t->y, (size_t)max_batch * 4)) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(&t->loss, 256)) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(&t->off, 2 * (size_t)max_batch * 8)) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(&t->blob, kEncBlobBytes)) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(&t->ws, enc_workspace_bytes(2 * max_batch))) != cudaSuccess) return fail(e);
    if ((e = cudaMemset(t->m1, 0, P)) != cudaSuccess) return fail(e);
    if ((e = cudaMemset(t->v1, 0, P)) != cudaSuccess) return fail(e);
    if ((e = pack_params(params, t->params, t->blob, nullptr)) != cudaSuccess) return fail(e);
    if ((e = cudaDeviceSynchronize()) != cudaSuccess) return fail(e);
    *out = t;
    return DTWS_OK;
}

dtws_status dtws_trainer_step(dtws_trainer_t t, const float *xq, const float *xc, int64_t n, const int64_t *q_off,
                              const int64_t *c_off, int32_t m, const float *y, int32_t batch, float *loss,
                              void *stream) {
    if (!t || !xq || !xc || !q_off || !c_off || !y || batch < 1 || batch > t->max_batch || m < 64 ||
        m > DTWS_M_MAX || n < m) {
        set_error_detail("dtws_trainer_step: null argument, batch out of [1, max_batch] or m out of range");
        return DTWS_EINVAL;
    }
    cudaPointerAttributes aq, ac;
    if (cudaPointerGetAttributes(&aq, xq) != cudaSuccess || cudaPointerGetAttributes(&ac, xc) != cudaSuccess ||
        aq.type != cudaMemoryTypeDevice || ac.type != cudaMemoryTypeDevice) {
        cudaGetLastError();
        set_error_detail("dtws_trainer_step: xq and xc must be device arrays");
        return DTWS_EINVAL;
    }
    for (int32_t i = 0; i < batch; ++i)
        if (q_off[i] < 0 || q_off[i] > n - m || c_off[i] < 0 || c_off[i] > n - m) {
            set_error_detail("dtws_trainer_step: offset %d out of [0, n-m]", i);
            return DTWS_EINVAL;
        }
    if (!finite_all(y, batch)) {
        set_error_detail("dtws_trainer_step: non-finite label");
        return DTWS_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    EK(cudaMemcpyAsync(t->off, q_off, (size_t)batch * 8, cudaMemcpyHostToDevice, s));
    EK(cudaMemcpyAsync(t->off + batch, c_off, (size_t)batch * 8, cudaMemcpyHostToDevice, s));
    EK(cudaMemcpyAsync(t->y, y, (size_t)batch * 4, cudaMemcpyHostToDevice, s));
    EK(launch_enc_prep(xq, t->off, batch, m, t->u, s));
    EK(launch_enc_prep(xc, t->off + batch, batch, m, t->u + (size_t)batch * DTWS_ENC_U, s));
    EK(cudaMemsetAsync(t->loss, 0, 4, s));
    EK(launch_enc_forward(t->blob, t->u, 2 * batch, nullptr, t->ws, t->sms, s));
    EK(launch_enc_backward(t->blob, t->y, batch, t->loss, t->grad, t->ws, t->sms, s));
    ++t->t;
    const double c1 = 1.0 - pow((double)t->hp.beta1, (double)t->t);
    const double c2 = 1.0 - pow((double)t->hp.beta2, (double)t->t);
    EK(launch_enc_pack(t->params, t->grad, t->m1, t->v1, t->blob, true, t->hp.lr, t->hp.beta1, t->hp.beta2,
                       t->hp.eps, (float)c1, (float)c2, s));
    if (loss) {
        EK(cudaMemcpyAsync(loss, t->loss, 4, cudaMemcpyDeviceToHost, s));
        EK(cudaStreamSynchronize(s));
    }
    return DTWS_OK;
}

dtws_status dtws_trainer_params(dtws_trainer_t t, float *params, void *stream) {
    if (!t || !params) return DTWS_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    EK(cudaMemcpyAsync(params, t->params, (size_t)kEncParams * 4, cudaMemcpyDefault, s));
    EK(cudaStreamSynchronize(s));
    return DTWS_OK;
}

}  // extern "C"

// rt_surrogate.cu -- C ABI of the convolutional surrogate's building blocks (raytrax.h).
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdio>
#include <mutex>

#include "raytrax.h"
#include "rt_internal.h"

namespace {

rt_status err(rt_status st, const char* fmt, ...) {
    char buf[384];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    return rt::set_error(st, buf);
}

rt_status cuda_err(cudaError_t e, const char* what) {
    return err(e == cudaErrorMemoryAllocation ? RT_ERR_OOM : RT_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

std::mutex g_mu;
int* g_err[64] = {};

// Device word that kernels with bounded waits set on timeout (one per device, allocated once).
int* error_word() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_err[dev]) {
        int* p = nullptr;
        if (cudaMalloc(&p, sizeof(int)) != cudaSuccess) return nullptr;
        if (cudaMemset(p, 0, sizeof(int)) != cudaSuccess) { cudaFree(p); return nullptr; }
        g_err[dev] = p;
    }
    return g_err[dev];
}

rt_status check_shape(int B, int D, int H, int W) {
    if (B < 1 || D < 1 || H < 2 || W != 64 || H % 2)
        return err(RT_ERR_INVALID_ARG, "conv3d: need B, D >= 1, even H >= 2 and W == 64 (got %d %d %d %d)", B, D,
                   H, W);
    return RT_OK;
}

}  // namespace

extern "C" {

rt_status rt_c32_from_f32(const float* src, int B, int C, int D, int H, int W, void* dst, void* stream) {
    if (!src || !dst || B < 1 || C < 1 || C > 32 || D < 1 || H < 1 || W < 1)
        return err(RT_ERR_INVALID_ARG, "rt_c32_from_f32: bad arguments (1 <= C <= 32)");
    cudaError_t e = rt::launch_to_c32(src, B, C, (long long)D * H * W, dst, (cudaStream_t)stream);
    return e == cudaSuccess ? RT_OK : cuda_err(e, "rt_c32_from_f32");
}

rt_status rt_c32_to_f32(const void* src, int B, int C, int D, int H, int W, float* dst, void* stream) {
    if (!src || !dst || B < 1 || C < 1 || C > 32 || D < 1 || H < 1 || W < 1)
        return err(RT_ERR_INVALID_ARG, "rt_c32_to_f32: bad arguments (1 <= C <= 32)");
    cudaError_t e = rt::launch_from_c32(src, B, C, (long long)D * H * W, dst, (cudaStream_t)stream);
    return e == cudaSuccess ? RT_OK : cuda_err(e, "rt_c32_to_f32");
}

rt_status rt_conv3d_pack_weights(const float* w, int c_in, int c_out, int transpose, void* packed, void* stream) {
    if (!w || !packed || c_in < 1 || c_in > 32 || c_out < 1 || c_out > 32)
        return err(RT_ERR_INVALID_ARG, "rt_conv3d_pack_weights: need 1 <= c_in, c_out <= 32");
    cudaError_t e = rt::launch_pack_weights(w, c_in, c_out, transpose ? 1 : 0, packed, (cudaStream_t)stream);
    return e == cudaSuccess ? RT_OK : cuda_err(e, "rt_conv3d_pack_weights");
}

rt_status rt_conv3d_forward(const void* x, int B, int D, int H, int W, int c_in, const void* w_packed,
                            const float* bias, int c_out, int dilation, int act, float slope, const void* mask,
                            void* y, float* y_f32, void* stream) {
    rt_status s = check_shape(B, D, H, W);
    if (s != RT_OK) return s;
    if (!x || !w_packed || (!y && !y_f32)) return err(RT_ERR_INVALID_ARG, "rt_conv3d_forward: NULL buffer");
    if (c_in < 1 || c_in > 32 || c_out < 1 || c_out > 32 || dilation < 1 || (act != 0 && act != 1))
        return err(RT_ERR_INVALID_ARG, "rt_conv3d_forward: need 1 <= c_in, c_out <= 32, dilation >= 1, act 0/1");
    int* ew = error_word();
    if (!ew) return err(RT_ERR_CUDA, "rt_conv3d_forward: no device error word");
    rt::ConvLaunch c{};
    c.x = x; c.w_packed = w_packed; c.bias = bias; c.mask_src = mask; c.y = y; c.y_f32 = y_f32;
    c.B = B; c.D = D; c.H = H; c.W = W;
    c.c_out = c_out; c.dil = dilation; c.act = act; c.slope = slope; c.err = ew;
    cudaError_t e = rt::launch_conv3d_tc(c, (cudaStream_t)stream);
    return e == cudaSuccess ? RT_OK : cuda_err(e, "rt_conv3d_forward launch");
}

rt_status rt_conv3d_weight_grad(const void* x, const void* dz, int B, int D, int H, int W, int c_in, int c_out,
                                int dilation, float* dw, float* db, void* stream) {
    rt_status s = check_shape(B, D, H, W);
    if (s != RT_OK) return s;
    if (!x || !dz || (!dw && !db)) return err(RT_ERR_INVALID_ARG, "rt_conv3d_weight_grad: NULL buffer");
    if (c_in < 1 || c_in > 32 || c_out < 1 || c_out > 32 || dilation < 1)
        return err(RT_ERR_INVALID_ARG, "rt_conv3d_weight_grad: need 1 <= c_in, c_out <= 32, dilation >= 1");
    int* ew = error_word();
    if (!ew) return err(RT_ERR_CUDA, "rt_conv3d_weight_grad: no device error word");
    cudaStream_t st = (cudaStream_t)stream;
    if (dw) {
        rt::WgradLaunch c{};
        c.x = x; c.dz = dz; c.dw = dw;
        c.B = B; c.D = D; c.H = H; c.W = W;
        c.c_in = c_in; c.c_out = c_out; c.dil = dilation; c.err = ew;
        cudaError_t e = rt::launch_conv3d_wgrad(c, st);
        if (e != cudaSuccess) return cuda_err(e, "rt_conv3d_weight_grad launch");
    }
    if (db) {
        cudaError_t e = rt::launch_bias_grad(dz, B, (long long)D * H * W, c_out, db, st);
        if (e != cudaSuccess) return cuda_err(e, "bias gradient launch");
    }
    return RT_OK;
}

rt_status rt_surrogate_features(const float* kappa, const float* j, int B, int D, int H, int W, void* x,
                                void* stream) {
    if (!kappa || !j || !x || B < 1 || D < 1 || H < 1 || W < 1) return err(RT_ERR_INVALID_ARG, "rt_surrogate_features: bad arguments");
    cudaError_t e = rt::launch_features(kappa, j, B, (long long)D * H * W, x, (cudaStream_t)stream);
    return e == cudaSuccess ? RT_OK : cuda_err(e, "rt_surrogate_features");
}

rt_status rt_field_max(const float* field, int B, long long vox, float* out, void* stream) {
    if (!field || !out || B < 1 || vox < 1) return err(RT_ERR_INVALID_ARG, "rt_field_max: bad arguments");
    cudaError_t e = rt::launch_field_max(field, B, vox, out, (cudaStream_t)stream);
    return e == cudaSuccess ? RT_OK : cuda_err(e, "rt_field_max");
}

rt_status rt_log_field_loss(const float* pred, const float* field, int B, long long vox, const float* fmax,
                            float eps_rel, float mu, float sigma, void* grad, float* loss, void* stream) {
    if (!pred || !field || !fmax || !loss || B < 1 || vox < 1 || !(sigma > 0.0f) || !(eps_rel > 0.0f))
        return err(RT_ERR_INVALID_ARG, "rt_log_field_loss: bad arguments");
    cudaError_t e = rt::launch_log_loss(pred, field, B, vox, fmax, eps_rel, mu, sigma, grad, loss, (cudaStream_t)stream);
    return e == cudaSuccess ? RT_OK : cuda_err(e, "rt_log_field_loss");
}

rt_status rt_field_error(const float* pred, const float* field, int B, long long vox, const float* fmax,
                         float eps_rel, float mu, float sigma, float* out, void* stream) {
    if (!pred || !field || !fmax || !out || B < 1 || vox < 1) return err(RT_ERR_INVALID_ARG, "rt_field_error: bad arguments");
    cudaError_t e = rt::launch_field_error(pred, field, B, vox, fmax, eps_rel, mu, sigma, out, (cudaStream_t)stream);
    return e == cudaSuccess ? RT_OK : cuda_err(e, "rt_field_error");
}

rt_status rt_c32_channel_mean(const void* x, int B, int C, long long vox, float* out, void* stream) {
    if (!x || !out || B < 1 || C < 1 || C > 32 || vox < 1)
        return err(RT_ERR_INVALID_ARG, "rt_c32_channel_mean: bad arguments");
    cudaError_t e = rt::launch_channel_mean(x, B, C, vox, out, (cudaStream_t)stream);
    return e == cudaSuccess ? RT_OK : cuda_err(e, "rt_c32_channel_mean");
}

rt_status rt_adam_step(float* params, const float* grads, float* m, float* v, long long n, float lr, float beta1,
                       float beta2, float eps, int step, void* stream) {
    if (!params || !grads || !m || !v || n < 1 || step < 1) return err(RT_ERR_INVALID_ARG, "rt_adam_step: bad arguments");
    cudaError_t e = rt::launch_adam(params, grads, m, v, n, lr, beta1, beta2, eps, step, (cudaStream_t)stream);
    return e == cudaSuccess ? RT_OK : cuda_err(e, "rt_adam_step");
}

rt_status rt_device_status(int* code) {
    if (!code) return err(RT_ERR_INVALID_ARG, "rt_device_status: NULL");
    int* ew = error_word();
    if (!ew) return err(RT_ERR_CUDA, "rt_device_status: no device error word");
    cudaError_t e = cudaMemcpy(code, ew, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemset(ew, 0, sizeof(int));
    if (e != cudaSuccess) return cuda_err(e, "rt_device_status");
    return *code ? RT_ERR_TIMEOUT : RT_OK;
}

}  // extern "C"

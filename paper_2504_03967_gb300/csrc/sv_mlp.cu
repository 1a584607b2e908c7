// Cost model: a small MLP that predicts the (standardised) log time of a tile
// pass from its feature vector (sv_internal.h pass_features: qubit count,
// dtype, tile width, dense blocks per width, diagonal runs, the paper's
// one-hot gate-type counts of App. D.1 Eq. "onehot" summed over the pass, ...).
//
//   h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2), y = w3 . h2 + b3
//   loss = mean over the batch of (y - t)^2,  t = (log ms - mu) / sigma
//
// Training runs on the GPU with hand-written FP32 kernels: forward (one
// thread per sample), backward deltas (one thread per sample), parameter
// gradients (one thread per parameter, samples summed in order, so results
// are reproducible) and Adam; one epoch is captured once into a CUDA graph
// and replayed.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <mutex>
#include <random>
#include <string>
#include <vector>

#include "sv_internal.h"
#include "sv_selftest.h"

namespace sv {
namespace mlp {

constexpr int F = kFeatures, H1 = 64, H2 = 64;
constexpr int OW1 = 0, OB1 = OW1 + H1 * F, OW2 = OB1 + H1, OB2 = OW2 + H2 * H1, OW3 = OB2 + H2, OB3 = OW3 + H2;
constexpr int P = OB3 + 1;

__global__ void __launch_bounds__(128) k_fwd(const float* __restrict__ p, const float* __restrict__ X, int B,
                                             float* __restrict__ z1, float* __restrict__ z2,
                                             float* __restrict__ y) {
    __shared__ float sp[P];
    for (int i = threadIdx.x; i < P; i += blockDim.x) sp[i] = p[i];
    __syncthreads();
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= B) return;
    float x[F];
#pragma unroll
    for (int j = 0; j < F; ++j) x[j] = X[(size_t)s * F + j];
    float h1[H1];
    for (int i = 0; i < H1; ++i) {
        float a = sp[OB1 + i];
#pragma unroll
        for (int j = 0; j < F; ++j) a = fmaf(sp[OW1 + i * F + j], x[j], a);
        if (z1) z1[(size_t)s * H1 + i] = a;
        h1[i] = a > 0.f ? a : 0.f;
    }
    float out = sp[OB3];
    for (int j = 0; j < H2; ++j) {
        float a = sp[OB2 + j];
#pragma unroll 8
        for (int i = 0; i < H1; ++i) a = fmaf(sp[OW2 + j * H1 + i], h1[i], a);
        if (z2) z2[(size_t)s * H2 + j] = a;
        out = fmaf(sp[OW3 + j], a > 0.f ? a : 0.f, out);
    }
    y[s] = out;
}

__global__ void __launch_bounds__(128) k_delta(const float* __restrict__ p, const float* __restrict__ z1,
                                               const float* __restrict__ z2, const float* __restrict__ y,
                                               const float* __restrict__ t, int B, float* __restrict__ d1,
                                               float* __restrict__ d2, float* __restrict__ err2) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= B) return;
    const float e = y[s] - t[s];
    err2[s] = e * e;
    const float dy = 2.f * e / (float)B;
    float dd2[H2];
    for (int j = 0; j < H2; ++j) {
        dd2[j] = z2[(size_t)s * H2 + j] > 0.f ? dy * p[OW3 + j] : 0.f;
        d2[(size_t)s * H2 + j] = dd2[j];
    }
    for (int i = 0; i < H1; ++i) {
        float a = 0.f;
        for (int j = 0; j < H2; ++j) a = fmaf(p[OW2 + j * H1 + i], dd2[j], a);
        d1[(size_t)s * H1 + i] = z1[(size_t)s * H1 + i] > 0.f ? a : 0.f;
    }
}

// One thread per parameter; every sum runs over samples in ascending order.
__global__ void __launch_bounds__(256) k_grads(const float* __restrict__ X, const float* __restrict__ z1,
                                               const float* __restrict__ z2, const float* __restrict__ d1,
                                               const float* __restrict__ d2, const float* __restrict__ y,
                                               const float* __restrict__ t, int B, float* __restrict__ g) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= P) return;
    float a = 0.f;
    if (q < OB1) {
        const int i = q / F, j = q % F;
        for (int s = 0; s < B; ++s) a = fmaf(d1[(size_t)s * H1 + i], X[(size_t)s * F + j], a);
    } else if (q < OW2) {
        const int i = q - OB1;
        for (int s = 0; s < B; ++s) a += d1[(size_t)s * H1 + i];
    } else if (q < OB2) {
        const int j = (q - OW2) / H1, i = (q - OW2) % H1;
        for (int s = 0; s < B; ++s) {
            const float h = z1[(size_t)s * H1 + i];
            a = fmaf(d2[(size_t)s * H2 + j], h > 0.f ? h : 0.f, a);
        }
    } else if (q < OW3) {
        const int j = q - OB2;
        for (int s = 0; s < B; ++s) a += d2[(size_t)s * H2 + j];
    } else if (q < OB3) {
        const int j = q - OW3;
        for (int s = 0; s < B; ++s) {
            const float h = z2[(size_t)s * H2 + j];
            a = fmaf(2.f * (y[s] - t[s]) / (float)B, h > 0.f ? h : 0.f, a);
        }
    } else {
        for (int s = 0; s < B; ++s) a += 2.f * (y[s] - t[s]) / (float)B;
    }
    g[q] = a;
}

// mean of err2 in FP64, fixed reduction order (one CTA)
__global__ void __launch_bounds__(256) k_loss(const float* __restrict__ err2, int B, double* __restrict__ out) {
    __shared__ double sh[256];
    double a = 0.0;
    for (int s = threadIdx.x; s < B; s += blockDim.x) a += err2[s];
    sh[threadIdx.x] = a;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sh[0] / (double)B;
}

// Adam (Kingma & Ba 2015) with bias correction; the step counter lives on the
// device so that a captured epoch can be replayed.
__global__ void __launch_bounds__(256) k_adam(float* __restrict__ p, const float* __restrict__ g,
                                              float* __restrict__ m, float* __restrict__ v,
                                              int* __restrict__ step, float lr, float b1, float b2, float eps) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    const int st = *step + 1;
    if (q < P) {
        const float mq = b1 * m[q] + (1.f - b1) * g[q];
        const float vq = b2 * v[q] + (1.f - b2) * g[q] * g[q];
        m[q] = mq;
        v[q] = vq;
        const float mh = mq / (1.f - powf(b1, (float)st));
        const float vh = vq / (1.f - powf(b2, (float)st));
        p[q] -= lr * mh / (sqrtf(vh) + eps);
    }
}
__global__ void k_step_inc(int* step) { *step += 1; }

// Device buffers for a batch.
struct Work {
    float *X = nullptr, *t = nullptr, *z1 = nullptr, *z2 = nullptr, *d1 = nullptr, *d2 = nullptr, *y = nullptr,
          *err2 = nullptr, *g = nullptr, *p = nullptr, *m = nullptr, *v = nullptr;
    double* loss = nullptr;
    int* step = nullptr;
    int B = 0;
    cudaError_t alloc(int b) {
        B = b;
        cudaError_t e = cudaSuccess;
        auto A = [&](float** q, size_t n) {
            if (e == cudaSuccess) e = cudaMalloc((void**)q, sizeof(float) * (n ? n : 1));
        };
        A(&X, (size_t)B * F);
        A(&t, B);
        A(&z1, (size_t)B * H1);
        A(&z2, (size_t)B * H2);
        A(&d1, (size_t)B * H1);
        A(&d2, (size_t)B * H2);
        A(&y, B);
        A(&err2, B);
        A(&g, P);
        A(&p, P);
        A(&m, P);
        A(&v, P);
        if (e == cudaSuccess) e = cudaMalloc((void**)&loss, sizeof(double));
        if (e == cudaSuccess) e = cudaMalloc((void**)&step, sizeof(int));
        return e;
    }
    ~Work() {
        for (float* q : {X, t, z1, z2, d1, d2, y, err2, g, p, m, v})
            if (q) cudaFree(q);
        if (loss) cudaFree(loss);
        if (step) cudaFree(step);
    }
};

void launch_fwd(const Work& w, cudaStream_t st) {
    k_fwd<<<(w.B + 127) / 128, 128, 0, st>>>(w.p, w.X, w.B, w.z1, w.z2, w.y);
}
void launch_grad(const Work& w, cudaStream_t st) {
    k_delta<<<(w.B + 127) / 128, 128, 0, st>>>(w.p, w.z1, w.z2, w.y, w.t, w.B, w.d1, w.d2, w.err2);
    k_grads<<<(P + 255) / 256, 256, 0, st>>>(w.X, w.z1, w.z2, w.d1, w.d2, w.y, w.t, w.B, w.g);
}

// ---- process-wide model ------------------------------------------------------
struct Model {
    bool loaded = false;
    std::vector<float> params;
    double mu = 0.0, sigma = 1.0;
    double train_loss = -1.0;
};
std::mutex g_mu;
Model g_model;

void he_init(std::vector<float>* p, uint64_t seed) {
    std::mt19937_64 rng(seed);
    p->assign(P, 0.f);
    auto fill = [&](int off, int rows, int fan_in) {
        const double a = sqrt(6.0 / fan_in);
        std::uniform_real_distribution<double> U(-a, a);
        for (int i = 0; i < rows * fan_in; ++i) (*p)[off + i] = (float)U(rng);
    };
    fill(OW1, H1, F);
    fill(OW2, H2, H1);
    fill(OW3, 1, H2);
}

}  // namespace mlp

// Predicted pass times (ms) for feature rows on the current device; false if
// no model is loaded.
bool cost_model_predict(const std::vector<float>& feat, int count, std::vector<double>* ms) {
    using namespace mlp;
    std::vector<float> params;
    double mu, sigma;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_model.loaded) return false;
        params = g_model.params;
        mu = g_model.mu;
        sigma = g_model.sigma;
    }
    ms->assign(count, 0.0);
    if (count == 0) return true;
    float *dp = nullptr, *dX = nullptr, *dy = nullptr;
    cudaError_t e = cudaMalloc(&dp, sizeof(float) * P);
    if (e == cudaSuccess) e = cudaMalloc(&dX, sizeof(float) * (size_t)count * F);
    if (e == cudaSuccess) e = cudaMalloc(&dy, sizeof(float) * count);
    if (e == cudaSuccess) e = cudaMemcpy(dp, params.data(), sizeof(float) * P, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dX, feat.data(), sizeof(float) * (size_t)count * F, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        count_launch();
        k_fwd<<<(count + 127) / 128, 128>>>(dp, dX, count, nullptr, nullptr, dy);
        e = cudaGetLastError();
    }
    std::vector<float> y(count);
    if (e == cudaSuccess) e = cudaMemcpy(y.data(), dy, sizeof(float) * count, cudaMemcpyDeviceToHost);
    cudaFree(dp);
    cudaFree(dX);
    cudaFree(dy);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    for (int i = 0; i < count; ++i) (*ms)[i] = exp((double)y[i] * sigma + mu);
    return true;
}

}  // namespace sv

using namespace sv;

extern "C" {

int sv_cost_model_train(const float* host_feat, const double* host_ms, int count, int epochs, double lr,
                        uint64_t seed, const char* weights_path, double* final_loss) {
    using namespace sv::mlp;
    if (!host_feat || !host_ms || count < 2 || epochs < 1 || !(lr > 0.0))
        return set_error(SV_EINVAL, "cost model training needs >= 2 samples, >= 1 epoch, lr > 0");
    // standardise the log times
    std::vector<float> t(count);
    double mu = 0.0, var = 0.0;
    for (int i = 0; i < count; ++i) {
        if (!(host_ms[i] > 0.0)) return set_error(SV_EINVAL, "pass times must be positive");
        mu += log(host_ms[i]);
    }
    mu /= count;
    for (int i = 0; i < count; ++i) var += (log(host_ms[i]) - mu) * (log(host_ms[i]) - mu);
    const double sigma = sqrt(var / count) > 1e-6 ? sqrt(var / count) : 1.0;
    for (int i = 0; i < count; ++i) t[i] = (float)((log(host_ms[i]) - mu) / sigma);
    std::vector<float> p0;
    he_init(&p0, seed);
    Work w;
    cudaError_t e = w.alloc(count);
    cudaStream_t st = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMemcpy(w.X, host_feat, sizeof(float) * (size_t)count * F, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(w.t, t.data(), sizeof(float) * count, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(w.p, p0.data(), sizeof(float) * P, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(w.m, 0, sizeof(float) * P);
    if (e == cudaSuccess) e = cudaMemset(w.v, 0, sizeof(float) * P);
    if (e == cudaSuccess) e = cudaMemset(w.step, 0, sizeof(int));
    // one epoch = forward, backward, Adam step; captured once, replayed
    if (e == cudaSuccess) e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        launch_fwd(w, st);
        launch_grad(w, st);
        k_adam<<<(P + 255) / 256, 256, 0, st>>>(w.p, w.g, w.m, w.v, w.step, (float)lr, 0.9f, 0.999f, 1e-8f);
        k_step_inc<<<1, 1, 0, st>>>(w.step);
        e = cudaStreamEndCapture(st, &graph);
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&gexec, graph, 0);
    for (int ep = 0; e == cudaSuccess && ep < epochs; ++ep) {
        count_launch(4);
        e = cudaGraphLaunch(gexec, st);
    }
    double loss = -1.0;
    if (e == cudaSuccess) {
        launch_fwd(w, st);
        k_delta<<<(w.B + 127) / 128, 128, 0, st>>>(w.p, w.z1, w.z2, w.y, w.t, w.B, w.d1, w.d2, w.err2);
        k_loss<<<1, 256, 0, st>>>(w.err2, w.B, w.loss);
        count_launch(3);
        e = cudaGetLastError();
    }
    std::vector<float> pf(P);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = cudaMemcpy(&loss, w.loss, sizeof(double), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(pf.data(), w.p, sizeof(float) * P, cudaMemcpyDeviceToHost);
    if (gexec) cudaGraphExecDestroy(gexec);
    if (graph) cudaGraphDestroy(graph);
    if (st) cudaStreamDestroy(st);
    if (e != cudaSuccess) return cuda_fail(e, "cost model training");
    {
        std::lock_guard<std::mutex> lk(g_mu);
        g_model.params = pf;
        g_model.mu = mu;
        g_model.sigma = sigma;
        g_model.loaded = true;
        g_model.train_loss = loss;
    }
    if (final_loss) *final_loss = loss;
    if (weights_path) {
        return sv_cost_model_save(weights_path);
    }
    return SV_OK;
}

// File: "SVCM", int32 version 1, int32 F, H1, H2, double mu, sigma, P floats.
int sv_cost_model_save(const char* path) {
    using namespace sv::mlp;
    if (!path) return set_error(SV_EINVAL, "NULL path");
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_model.loaded) return set_error(SV_EINVAL, "no cost model loaded");
    FILE* f = fopen(path, "wb");
    if (!f) return set_error(SV_EINVAL, std::string("cannot open ") + path);
    const int32_t hdr[4] = {1, F, H1, H2};
    bool ok = fwrite("SVCM", 1, 4, f) == 4 && fwrite(hdr, 4, 4, f) == 4 && fwrite(&g_model.mu, 8, 1, f) == 1 &&
              fwrite(&g_model.sigma, 8, 1, f) == 1 && fwrite(g_model.params.data(), 4, P, f) == (size_t)P;
    ok = (fclose(f) == 0) && ok;
    return ok ? SV_OK : set_error(SV_EINVAL, "write failed");
}

int sv_cost_model_load(const char* path) {
    using namespace sv::mlp;
    if (!path) return set_error(SV_EINVAL, "NULL path");
    FILE* f = fopen(path, "rb");
    if (!f) return set_error(SV_EINVAL, std::string("cannot open ") + path);
    char magic[4];
    int32_t hdr[4];
    double mu, sigma;
    std::vector<float> p(P);
    bool ok = fread(magic, 1, 4, f) == 4 && memcmp(magic, "SVCM", 4) == 0 && fread(hdr, 4, 4, f) == 4 &&
              hdr[0] == 1 && hdr[1] == F && hdr[2] == H1 && hdr[3] == H2 && fread(&mu, 8, 1, f) == 1 &&
              fread(&sigma, 8, 1, f) == 1 && fread(p.data(), 4, P, f) == (size_t)P;
    fclose(f);
    if (!ok) return set_error(SV_EINVAL, "not a cost-model file of this version");
    std::lock_guard<std::mutex> lk(g_mu);
    g_model.params = p;
    g_model.mu = mu;
    g_model.sigma = sigma;
    g_model.loaded = true;
    return SV_OK;
}

int sv_cost_model_unload(void) {
    std::lock_guard<std::mutex> lk(mlp::g_mu);
    mlp::g_model.loaded = false;
    return SV_OK;
}

int sv_cost_model_loaded(void) {
    std::lock_guard<std::mutex> lk(mlp::g_mu);
    return mlp::g_model.loaded ? 1 : 0;
}

int sv_cost_model_predict(const float* host_feat, int count, double* host_ms) {
    if (count < 0 || (count && (!host_feat || !host_ms))) return set_error(SV_EINVAL, "bad arguments");
    if (!sv_cost_model_loaded()) return set_error(SV_EINVAL, "no cost model loaded");
    std::vector<float> feat(host_feat, host_feat + (size_t)count * mlp::F);
    std::vector<double> ms;
    if (!cost_model_predict(feat, count, &ms)) return set_error(SV_ECUDA, "cost model inference failed");
    for (int i = 0; i < count; ++i) host_ms[i] = ms[i];
    return SV_OK;
}

// Self-test entry: loss and gradient of the network on the GPU for given
// parameters, inputs and (standardised) targets.
int sv_mlp_gradient(const float* params, const float* x, const float* t, int B, double* loss, float* grads) {
    using namespace sv::mlp;
    if (!params || !x || !t || B < 1 || !loss || !grads) return set_error(SV_EINVAL, "bad arguments");
    Work w;
    cudaError_t e = w.alloc(B);
    if (e == cudaSuccess) e = cudaMemcpy(w.p, params, sizeof(float) * P, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(w.X, x, sizeof(float) * (size_t)B * F, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(w.t, t, sizeof(float) * B, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        launch_fwd(w, nullptr);
        launch_grad(w, nullptr);
        k_loss<<<1, 256>>>(w.err2, w.B, w.loss);
        count_launch(4);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(loss, w.loss, sizeof(double), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(grads, w.g, sizeof(float) * P, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "mlp gradient");
    return SV_OK;
}

// Self-test entry: `steps` Adam updates with a fixed gradient, from zero
// moments, on the GPU (params updated in place on the host copy).
int sv_mlp_adam(float* params, const float* grads, int steps, double lr) {
    using namespace sv::mlp;
    if (!params || !grads || steps < 1) return set_error(SV_EINVAL, "bad arguments");
    Work w;
    cudaError_t e = w.alloc(1);
    if (e == cudaSuccess) e = cudaMemcpy(w.p, params, sizeof(float) * P, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(w.g, grads, sizeof(float) * P, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(w.m, 0, sizeof(float) * P);
    if (e == cudaSuccess) e = cudaMemset(w.v, 0, sizeof(float) * P);
    if (e == cudaSuccess) e = cudaMemset(w.step, 0, sizeof(int));
    for (int s = 0; e == cudaSuccess && s < steps; ++s) {
        k_adam<<<(P + 255) / 256, 256>>>(w.p, w.g, w.m, w.v, w.step, (float)lr, 0.9f, 0.999f, 1e-8f);
        k_step_inc<<<1, 1>>>(w.step);
        count_launch(2);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(params, w.p, sizeof(float) * P, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "mlp adam");
    return SV_OK;
}

int sv_mlp_param_count(void) { return mlp::P; }

}  // extern "C"

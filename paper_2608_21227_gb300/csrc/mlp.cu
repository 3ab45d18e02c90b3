// mlp.cu -- the tuner's learned cost model: a 15 -> 128 -> 128 -> 128 -> 1 ReLU
// MLP in FP32 that predicts the log runtime of a configuration, trained and
// evaluated on the GPU by the kernels below (forward, backward, Adam).
//
// Layer l: Z_l = H_{l-1} W_l^T + b_l (W_l: out x in, row-major), H_l = relu(Z_l)
// for the hidden layers; loss = mean squared error.  Backward: G_L = 2/B (p - y),
// dW_l = G_l^T H_{l-1}, db_l = sum_rows G_l, G_{l-1} = (G_l W_l) .* [Z_{l-1} > 0].
// Adam (Kingma & Ba 2015): m <- b1 m + (1-b1) g, v <- b2 v + (1-b2) g^2,
// w <- w - lr (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/kt.h"
#include "common.cuh"
#include "tuned.h"

namespace {

constexpr int kIn = KT_MLP_FEATURES;
constexpr int kH = 128;
constexpr int kLayers = 4;
const int kDims[kLayers + 1] = {kIn, kH, kH, kH, 1};

size_t w_off(int l) {  // offset of W_l (0-based layer) in the packed parameter vector
    size_t o = 0;
    for (int i = 0; i < l; ++i) o += (size_t)kDims[i + 1] * kDims[i] + kDims[i + 1];
    return o;
}
size_t b_off(int l) { return w_off(l) + (size_t)kDims[l + 1] * kDims[l]; }
constexpr size_t kParams = (size_t)kH * kIn + kH + 2 * ((size_t)kH * kH + kH) + kH + 1;

// C(i, j) = sum_k A(i, k) B(k, j) over generic strides; epilogue:
//   mode 0: C = acc                      mode 1: C = acc + bias[j]
//   mode 2: Z = acc + bias[j], H = relu(Z) (C = Z, C2 = H)
//   mode 3: C = acc * [Zmask(i, j) > 0]  (backward through ReLU)
constexpr int kTile = 32;
__global__ void gemm_kernel(int M, int N, int K, const float *__restrict__ A, long sa0, long sa1,
                            const float *__restrict__ B, long sb0, long sb1, float *C, long sc0, long sc1,
                            const float *__restrict__ bias, float *C2, const float *__restrict__ Zmask, int mode) {
    __shared__ float As[kTile][kTile + 1];
    __shared__ float Bs[kTile][kTile + 1];
    const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
    const int i0 = blockIdx.y * kTile, j0 = blockIdx.x * kTile;
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    for (int k0 = 0; k0 < K; k0 += kTile) {
        for (int r = ty; r < kTile; r += 8) {
            int i = i0 + r, k = k0 + tx;
            As[r][tx] = (i < M && k < K) ? A[i * sa0 + k * sa1] : 0.f;
            int kk = k0 + r, j = j0 + tx;
            Bs[r][tx] = (kk < K && j < N) ? B[kk * sb0 + j * sb1] : 0.f;
        }
        __syncthreads();
#pragma unroll 8
        for (int k = 0; k < kTile; ++k) {
            float bv = Bs[k][tx];
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[q] += As[ty + 8 * q][k] * bv;
        }
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        int i = i0 + ty + 8 * q, j = j0 + tx;
        if (i >= M || j >= N) continue;
        float v = acc[q];
        if (mode == 1 || mode == 2) v += bias[j];
        if (mode == 3) v = Zmask[i * sc0 + j * sc1] > 0.f ? v : 0.f;
        C[i * sc0 + j * sc1] = v;
        if (mode == 2) C2[i * sc0 + j * sc1] = fmaxf(v, 0.f);
    }
}

void gemm(cudaStream_t st, int M, int N, int K, const float *A, long sa0, long sa1, const float *B, long sb0, long sb1,
          float *C, long sc0, long sc1, const float *bias, float *C2, const float *Zmask, int mode) {
    dim3 grid((N + kTile - 1) / kTile, (M + kTile - 1) / kTile), block(32, 8);
    gemm_kernel<<<grid, block, 0, st>>>(M, N, K, A, sa0, sa1, B, sb0, sb1, C, sc0, sc1, bias, C2, Zmask, mode);
}

// column sums: out[j] = sum_i G[i*ld + j]
__global__ void colsum_kernel(const float *G, int rows, int cols, long ld, float *out) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= cols) return;
    float s = 0.f;
    for (int i = 0; i < rows; ++i) s += G[i * ld + j];
    out[j] = s;
}

__global__ void loss_grad_kernel(const float *pred, const float *y, int rows, float *G, float *loss_acc) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    float d = 0.f;
    if (i < rows) {
        d = pred[i] - y[i];
        G[i] = 2.f * d / (float)rows;
    }
    float sq = nla::warp_sum(d * d);
    if (loss_acc && (threadIdx.x & 31) == 0) atomicAdd(loss_acc, sq / (float)rows);
}

__global__ void adam_kernel(float *w, const float *g, float *m, float *v, size_t count, float lr, float b1, float b2,
                            float eps, float c1, float c2) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
        float gi = g[i];
        float mi = b1 * m[i] + (1.f - b1) * gi;
        float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

__global__ void gather_rows_kernel(const float *X, const float *y, const int *idx, int rows, float *Xb, float *yb) {
    int i = blockIdx.x;
    if (i >= rows) return;
    int src = idx[i];
    for (int k = threadIdx.x; k < kIn; k += blockDim.x) Xb[i * kIn + k] = X[(long)src * kIn + k];
    if (threadIdx.x == 0) yb[i] = y[src];
}

// Work buffers for a batch of `rows`: Z1..Z3, H1..H3 (rows x 128), pred (rows), G (rows x 128) x 2.
size_t work_floats(int rows) { return (size_t)rows * (6 * kH + 1 + 2 * kH) + 64; }

struct Act {
    float *Z[3], *H[3], *pred, *G0, *G1;
};
Act carve(float *w, int rows) {
    Act a;
    for (int l = 0; l < 3; ++l) {
        a.Z[l] = w + (size_t)l * rows * kH;
        a.H[l] = w + (size_t)(3 + l) * rows * kH;
    }
    a.pred = w + (size_t)6 * rows * kH;
    a.G0 = a.pred + rows + 32;
    a.G1 = a.G0 + (size_t)rows * kH;
    return a;
}

void forward(cudaStream_t st, const float *P, const float *X, int rows, const Act &a) {
    const float *h = X;
    int in = kIn;
    for (int l = 0; l < 3; ++l) {
        gemm(st, rows, kH, in, h, in, 1, P + w_off(l), 1, in, a.Z[l], kH, 1, P + b_off(l), a.H[l], nullptr, 2);
        h = a.H[l];
        in = kH;
    }
    gemm(st, rows, 1, kH, h, kH, 1, P + w_off(3), 1, kH, a.pred, 1, 1, P + b_off(3), nullptr, nullptr, 1);
}

void backward(cudaStream_t st, const float *P, const float *X, const float *y, int rows, const Act &a, float *grads,
              float *loss_acc) {
    float *G = a.G0, *Gn = a.G1;
    loss_grad_kernel<<<(rows + 255) / 256, 256, 0, st>>>(a.pred, y, rows, G, loss_acc);
    int out = 1;
    for (int l = 3; l >= 0; --l) {
        const int in = kDims[l];
        const float *Hprev = l == 0 ? X : a.H[l - 1];
        // dW_l (out x in) = G^T Hprev
        gemm(st, out, in, rows, G, 1, out, Hprev, in, 1, grads + w_off(l), in, 1, nullptr, nullptr, nullptr, 0);
        colsum_kernel<<<(out + 127) / 128, 128, 0, st>>>(G, rows, out, out, grads + b_off(l));
        if (l > 0) {  // G_{l-1} = (G W_l) .* [Z_{l-1} > 0]
            gemm(st, rows, in, out, G, out, 1, P + w_off(l), in, 1, Gn, in, 1, nullptr, nullptr, a.Z[l - 1], 3);
            std::swap(G, Gn);
        }
        out = in;
    }
}

struct Model {
    std::vector<float> mean, sd, params;
    float ymean = 0.f, ysd = 1.f;
};

bool save_model(const char *path, const Model &m) {
    FILE *f = fopen(path, "wb");
    if (!f) return false;
    const char magic[8] = {'K', 'T', 'M', 'L', 'P', '1', 0, 0};
    int hdr[3] = {kIn, kH, (int)kParams};
    bool ok = fwrite(magic, 1, 8, f) == 8 && fwrite(hdr, sizeof(int), 3, f) == 3 &&
              fwrite(m.mean.data(), sizeof(float), kIn, f) == (size_t)kIn &&
              fwrite(m.sd.data(), sizeof(float), kIn, f) == (size_t)kIn && fwrite(&m.ymean, sizeof(float), 1, f) == 1 &&
              fwrite(&m.ysd, sizeof(float), 1, f) == 1 &&
              fwrite(m.params.data(), sizeof(float), kParams, f) == kParams;
    fclose(f);
    return ok;
}

bool load_model(const char *path, Model &m) {
    FILE *f = fopen(path, "rb");
    if (!f) return false;
    char magic[8];
    int hdr[3];
    m.mean.resize(kIn);
    m.sd.resize(kIn);
    m.params.resize(kParams);
    bool ok = fread(magic, 1, 8, f) == 8 && memcmp(magic, "KTMLP1", 6) == 0 && fread(hdr, sizeof(int), 3, f) == 3 &&
              hdr[0] == kIn && hdr[1] == kH && hdr[2] == (int)kParams &&
              fread(m.mean.data(), sizeof(float), kIn, f) == (size_t)kIn &&
              fread(m.sd.data(), sizeof(float), kIn, f) == (size_t)kIn && fread(&m.ymean, sizeof(float), 1, f) == 1 &&
              fread(&m.ysd, sizeof(float), 1, f) == 1 && fread(m.params.data(), sizeof(float), kParams, f) == kParams;
    fclose(f);
    return ok;
}

struct SplitMix {
    unsigned long long s;
    unsigned long long next() {
        s += 0x9E3779B97F4A7C15ull;
        unsigned long long z = s;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    }
    double uniform() { return (double)(next() >> 11) * 0x1p-53; }
};

nla_status merr(nla_status s, const char *msg) {
    nla_set_last_error(msg);
    return s;
}

}  // namespace

namespace nla {

nla_status mlp_predict_host(const char *model_path, const float *X, int rows, float *y) {
    Model m;
    if (!model_path || !load_model(model_path, m)) return merr(NLA_ERR_ARG, "cannot read the MLP model file");
    if (rows <= 0) return NLA_OK;
    std::vector<float> Xs((size_t)rows * kIn);
    for (int i = 0; i < rows; ++i)
        for (int k = 0; k < kIn; ++k) Xs[(size_t)i * kIn + k] = (X[(size_t)i * kIn + k] - m.mean[k]) / m.sd[k];
    float *dP = nullptr, *dX = nullptr, *dW = nullptr;
    cudaStream_t st;
    cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    nla_status s = NLA_OK;
    if (cudaMalloc(&dP, kParams * sizeof(float)) || cudaMalloc(&dX, Xs.size() * sizeof(float)) ||
        cudaMalloc(&dW, work_floats(rows) * sizeof(float))) {
        cudaGetLastError();
        s = merr(NLA_ERR_CUDA, "MLP inference: allocation failed");
    } else {
        cudaMemcpyAsync(dP, m.params.data(), kParams * sizeof(float), cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(dX, Xs.data(), Xs.size() * sizeof(float), cudaMemcpyHostToDevice, st);
        Act a = carve(dW, rows);
        forward(st, dP, dX, rows, a);
        cudaMemcpyAsync(y, a.pred, rows * sizeof(float), cudaMemcpyDeviceToHost, st);
        if (cudaStreamSynchronize(st) != cudaSuccess) s = merr(NLA_ERR_CUDA, "MLP inference failed");
        for (int i = 0; i < rows; ++i) y[i] = y[i] * m.ysd + m.ymean;
    }
    cudaFree(dP);
    cudaFree(dX);
    cudaFree(dW);
    cudaStreamDestroy(st);
    return s;
}

}  // namespace nla

extern "C" {

size_t kt_mlp_param_count(void) { return kParams; }

size_t kt_mlp_work_bytes(int rows) { return work_floats(std::max(rows, 1)) * sizeof(float); }

nla_status kt_mlp_forward_backward(const float *dParams, const float *dX, const float *dY, int rows, float *dPred,
                                   float *dGrads, void *dWork, size_t work_bytes, nla_stream_t stream) {
    if (rows <= 0 || !dParams || !dX || !dY || !dGrads || !dWork) return merr(NLA_ERR_ARG, "bad arguments");
    if (work_bytes < kt_mlp_work_bytes(rows)) return merr(NLA_ERR_WORKSPACE, "MLP workspace too small");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    Act a = carve(reinterpret_cast<float *>(dWork), rows);
    forward(st, dParams, dX, rows, a);
    backward(st, dParams, dX, dY, rows, a, dGrads, nullptr);
    if (dPred) cudaMemcpyAsync(dPred, a.pred, rows * sizeof(float), cudaMemcpyDeviceToDevice, st);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? NLA_OK : merr(NLA_ERR_CUDA, cudaGetErrorString(e));
}

nla_status kt_mlp_adam_step(float *dParams, const float *dGrads, float *dM, float *dV, size_t count, int t, float lr,
                            nla_stream_t stream) {
    if (t < 1 || !dParams || !dGrads || !dM || !dV) return merr(NLA_ERR_ARG, "bad arguments");
    const float b1 = 0.9f, b2 = 0.999f;
    float c1 = 1.f - (float)std::pow(0.9, t), c2 = 1.f - (float)std::pow(0.999, t);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    adam_kernel<<<256, 256, 0, st>>>(dParams, dGrads, dM, dV, count, lr, b1, b2, 1e-8f, c1, c2);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? NLA_OK : merr(NLA_ERR_CUDA, cudaGetErrorString(e));
}

nla_status kt_mlp_train(const float *X, const float *y, int rows, int epochs, int batch, float lr,
                        unsigned long long seed, const char *model_path, float *final_loss) {
    if (!X || !y || rows <= 0 || epochs <= 0 || batch <= 0 || !model_path) return merr(NLA_ERR_ARG, "bad arguments");
    batch = std::min(batch, rows);
    Model m;
    m.mean.assign(kIn, 0.f);
    m.sd.assign(kIn, 1.f);
    // standardisation of inputs and target
    for (int k = 0; k < kIn; ++k) {
        double s = 0, s2 = 0;
        for (int i = 0; i < rows; ++i) {
            double v = X[(size_t)i * kIn + k];
            s += v;
            s2 += v * v;
        }
        double mu = s / rows, var = std::max(0.0, s2 / rows - mu * mu);
        m.mean[k] = (float)mu;
        m.sd[k] = var > 1e-12 ? (float)std::sqrt(var) : 1.f;
    }
    {
        double s = 0, s2 = 0;
        for (int i = 0; i < rows; ++i) {
            s += y[i];
            s2 += (double)y[i] * y[i];
        }
        double mu = s / rows, var = std::max(0.0, s2 / rows - mu * mu);
        m.ymean = (float)mu;
        m.ysd = var > 1e-12 ? (float)std::sqrt(var) : 1.f;
    }
    std::vector<float> Xs((size_t)rows * kIn), ys(rows);
    for (int i = 0; i < rows; ++i) {
        for (int k = 0; k < kIn; ++k) Xs[(size_t)i * kIn + k] = (X[(size_t)i * kIn + k] - m.mean[k]) / m.sd[k];
        ys[i] = (y[i] - m.ymean) / m.ysd;
    }
    // He-uniform initialisation from SplitMix64, zero biases
    SplitMix g{seed};
    m.params.assign(kParams, 0.f);
    for (int l = 0; l < kLayers; ++l) {
        double lim = std::sqrt(6.0 / kDims[l]);
        for (size_t i = 0; i < (size_t)kDims[l + 1] * kDims[l]; ++i)
            m.params[w_off(l) + i] = (float)((2.0 * g.uniform() - 1.0) * lim);
    }
    float *dX = nullptr, *dY = nullptr, *dP = nullptr, *dG = nullptr, *dM = nullptr, *dV = nullptr, *dXb = nullptr,
          *dYb = nullptr, *dW = nullptr, *dLoss = nullptr;
    int *dIdx = nullptr;
    cudaStream_t st;
    cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    nla_status s = NLA_OK;
    if (cudaMalloc(&dX, Xs.size() * 4) || cudaMalloc(&dY, rows * 4) || cudaMalloc(&dP, kParams * 4) ||
        cudaMalloc(&dG, kParams * 4) || cudaMalloc(&dM, kParams * 4) || cudaMalloc(&dV, kParams * 4) ||
        cudaMalloc(&dXb, (size_t)batch * kIn * 4) || cudaMalloc(&dYb, batch * 4) ||
        cudaMalloc(&dW, kt_mlp_work_bytes(batch)) || cudaMalloc(&dLoss, 4) || cudaMalloc(&dIdx, rows * 4)) {
        cudaGetLastError();
        s = merr(NLA_ERR_CUDA, "MLP training: allocation failed");
    }
    float last = NAN;
    if (s == NLA_OK) {
        cudaMemcpyAsync(dX, Xs.data(), Xs.size() * 4, cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(dY, ys.data(), rows * 4, cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(dP, m.params.data(), kParams * 4, cudaMemcpyHostToDevice, st);
        cudaMemsetAsync(dM, 0, kParams * 4, st);
        cudaMemsetAsync(dV, 0, kParams * 4, st);
        std::vector<int> idx(rows);
        int t = 0;
        for (int ep = 0; ep < epochs; ++ep) {
            for (int i = 0; i < rows; ++i) idx[i] = i;
            for (int i = rows - 1; i > 0; --i) std::swap(idx[i], idx[g.next() % (unsigned long long)(i + 1)]);
            cudaMemcpyAsync(dIdx, idx.data(), rows * 4, cudaMemcpyHostToDevice, st);
            cudaMemsetAsync(dLoss, 0, 4, st);
            int nb = 0;
            for (int b0 = 0; b0 + batch <= rows; b0 += batch, ++nb) {
                gather_rows_kernel<<<batch, 32, 0, st>>>(dX, dY, dIdx + b0, batch, dXb, dYb);
                Act a = carve(dW, batch);
                forward(st, dP, dXb, batch, a);
                backward(st, dP, dXb, dYb, batch, a, dG, dLoss);
                kt_mlp_adam_step(dP, dG, dM, dV, kParams, ++t, lr, st);
            }
            float h = 0.f;
            cudaMemcpyAsync(&h, dLoss, 4, cudaMemcpyDeviceToHost, st);
            if (cudaStreamSynchronize(st) != cudaSuccess) {
                s = merr(NLA_ERR_CUDA, "MLP training failed");
                break;
            }
            last = nb ? h / nb : NAN;
        }
        if (s == NLA_OK) {
            cudaMemcpyAsync(m.params.data(), dP, kParams * 4, cudaMemcpyDeviceToHost, st);
            cudaStreamSynchronize(st);
            if (!save_model(model_path, m)) s = merr(NLA_ERR_ARG, "cannot write the MLP model file");
        }
    }
    cudaFree(dX);
    cudaFree(dY);
    cudaFree(dP);
    cudaFree(dG);
    cudaFree(dM);
    cudaFree(dV);
    cudaFree(dXb);
    cudaFree(dYb);
    cudaFree(dW);
    cudaFree(dLoss);
    cudaFree(dIdx);
    cudaStreamDestroy(st);
    if (final_loss) *final_loss = last * m.ysd * m.ysd;  // in units of (log ms)^2
    return s;
}

nla_status kt_mlp_predict(const char *model_path, const float *X, int rows, float *y_out) {
    if (!X || !y_out || rows < 0) return merr(NLA_ERR_ARG, "bad arguments");
    return nla::mlp_predict_host(model_path, X, rows, y_out);
}

}  // extern "C"

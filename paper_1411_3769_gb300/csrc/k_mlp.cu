// Learned warm start: a three-layer ReLU MLP trained and evaluated on the GPU.
// Every matrix product runs on the tcgen05 tensor cores with BF16 operands and
// FP32 accumulation (k_tc_gemm.cu, kind::f16); master weights, biases, Adam
// moments, pre-activations and the loss stay in FP32.
//
// With the GEMM convention D[m][n] = sum_k A[m][k] B[n][k] stored at
// C[n*ldc + m], a layer is D[out][batch] = W[out][in] . H[batch][in], which lands
// row-major as Z[batch][out]; the backward products read the transposed BF16
// copies the forward and elementwise kernels write alongside.
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "psdp_internal.h"

namespace {

constexpr int kT = 256;

int grid1(int64_t n) {
    int64_t b = (n + kT - 1) / kT;
    return (int)(b > 8192 ? 8192 : (b < 1 ? 1 : b));
}

// out[r][c] (bf16) = in[r][c]; outT[c][r] = in[r][c]; rows x cols, leading dims ld_out / ld_t
__global__ void k_to_bf16(int rows, int cols, const float* __restrict__ in, int ld_in, __nv_bfloat16* out, int ld_out,
                          __nv_bfloat16* outT, int ld_t) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (int64_t)rows * cols;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(i / cols), c = (int)(i % cols);
        const __nv_bfloat16 v = __float2bfloat16_rn(in[(int64_t)r * ld_in + c]);
        if (out) out[(int64_t)r * ld_out + c] = v;
        if (outT) outT[(int64_t)c * ld_t + r] = v;
    }
}

// Z[b][j] += bias[j]; H = relu(Z) (or Z for the last layer) as bf16 [b][j] and [j][b]
__global__ void k_bias_act(int B, int n, float* Z, const float* __restrict__ bias, int relu, __nv_bfloat16* H,
                          __nv_bfloat16* HT, int ldT) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (int64_t)B * n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int b = (int)(i / n), j = (int)(i % n);
        const float z = Z[i] + bias[j];
        Z[i] = z;
        const float h = relu ? fmaxf(z, 0.f) : z;
        if (H) H[i] = __float2bfloat16_rn(h);
        if (HT) HT[(int64_t)j * ldT + b] = __float2bfloat16_rn(h);
    }
}

// dY = 2 (Y - T) / (B * n_true) on the true outputs, 0 on the padding; partial loss sums
__global__ void k_mse(int B, int n, int n_true, const float* __restrict__ Y, const float* __restrict__ T, float* dY,
                      double* loss_acc) {
    __shared__ double red[kT / 32];
    double s = 0.0;
    const float scale = 2.f / ((float)B * (float)n_true);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (int64_t)B * n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(i % n);
        float d = 0.f;
        if (j < n_true) {
            d = Y[i] - T[(i / n) * n_true + j];
            s += (double)d * d;
        }
        dY[i] = scale * d;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int q = 0; q < kT / 32; ++q) t += red[q];
        atomicAdd(loss_acc, t);
    }
}

// dZ = dA * (Z > 0) as bf16 [b][k] and [k][b]; dZ kept in FP32 for the bias gradient
__global__ void k_relu_back(int B, int n, float* dA, const float* __restrict__ Z, __nv_bfloat16* D, __nv_bfloat16* DT,
                            int ldT) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (int64_t)B * n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int b = (int)(i / n), k = (int)(i % n);
        const float g = Z[i] > 0.f ? dA[i] : 0.f;
        dA[i] = g;
        const __nv_bfloat16 v = __float2bfloat16_rn(g);
        D[i] = v;
        DT[(int64_t)k * ldT + b] = v;
    }
}

// db[j] = sum_b dZ[b][j]
__global__ void k_colsum(int B, int n, const float* __restrict__ dZ, float* db) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        float s = 0.f;
        for (int b = 0; b < B; ++b) s += dZ[(int64_t)b * n + j];
        db[j] = s;
    }
}

// Adam with bias correction on FP32 masters; refreshes the bf16 weight and its transpose
__global__ void k_adam(int64_t n, float* p, const float* __restrict__ g, float* m, float* v, float lr, float b1, float b2,
                       float eps, float c1, float c2, int cols, __nv_bfloat16* Wb, __nv_bfloat16* WbT, int rows) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float w = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        p[i] = w;
        if (Wb) {
            const int r = (int)(i / cols), c = (int)(i % cols);
            const __nv_bfloat16 bw = __float2bfloat16_rn(w);
            Wb[i] = bw;
            WbT[(int64_t)c * rows + r] = bw;
        }
    }
}

// column mean / std over n rows (std floored at 1e-6)
__global__ void k_colstats(int n, int cols, const float* __restrict__ X, float* mean, float* stdv) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < cols; c += gridDim.x * blockDim.x) {
        double s = 0.0, s2 = 0.0;
        for (int r = 0; r < n; ++r) {
            const double x = X[(int64_t)r * cols + c];
            s += x;
            s2 += x * x;
        }
        const double mu = s / n;
        mean[c] = (float)mu;
        stdv[c] = (float)fmax(sqrt(fmax(s2 / n - mu * mu, 0.0)), 1e-6);
    }
}

// out[i][c] = (in[idx[i]][c] - mean[c]) / std[c]  (gather + standardise)
__global__ void k_gather_std(int rows, int cols, const int32_t* __restrict__ idx, const float* __restrict__ in,
                             const float* __restrict__ mean, const float* __restrict__ stdv, float* out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (int64_t)rows * cols;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(i / cols), c = (int)(i % cols);
        const int src = idx ? idx[r] : r;
        out[i] = (in[(int64_t)src * cols + c] - mean[c]) / stdv[c];
    }
}

// Y[i][c] = Ystd[i][c] * std[c] + mean[c] on the true outputs
__global__ void k_unstd(int rows, int n_pad, int n_true, const float* __restrict__ Ys, const float* __restrict__ mean,
                        const float* __restrict__ stdv, float* Y) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (int64_t)rows * n_true;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(i / n_true), c = (int)(i % n_true);
        Y[i] = Ys[(int64_t)r * n_pad + c] * stdv[c] + mean[c];
    }
}

template <class T>
bool dalloc_n(T** p, size_t n) {
    if (cudaMalloc((void**)p, (n ? n : 1) * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return false;
    }
    return true;
}

}  // namespace

struct psdp_mlp {
    int n_in, width, n_out, n_pad, max_b, device;
    int dims[4];                     // n_in, width, width, n_pad
    cudaStream_t st;
    float *W[3] = {}, *b[3] = {}, *gW[3] = {}, *gb[3] = {}, *mW[3] = {}, *vW[3] = {}, *mb[3] = {}, *vb[3] = {};
    __nv_bfloat16 *Wb[3] = {}, *WbT[3] = {};
    float *Z[3] = {}, *dA = nullptr, *Xf = nullptr, *Tf = nullptr;
    __nv_bfloat16 *H[3] = {}, *HT[3] = {}, *D = nullptr, *DT = nullptr;   // H[0] = input
    float *xmean = nullptr, *xstd = nullptr, *tmean = nullptr, *tstd = nullptr;
    double* loss = nullptr;
    int* flag = nullptr;
    int64_t step = 0;
    bool fitted = false;
};

namespace {

psdp_status mlp_gemm(psdp_mlp* m, const __nv_bfloat16* A, int M, const __nv_bfloat16* B, int N, int K, int lda,
                     int ldb, float* C, int ldc) {
    CUtensorMap ma, mb;
    if (!tc_make_map(&ma, A, true, K, M, 1, lda, 0, 128) || !tc_make_map(&mb, B, true, K, N, 1, ldb, 0, 128))
        return PSDP_ECUDA;
    launch_tc_gemm(m->st, true, 1, ma, mb, nullptr, nullptr, M, N, 1, 0, nullptr, K, C, ldc, 0, 1.f, 0.f, 0, m->flag);
    return PSDP_OK;
}

// forward on H[0] (bf16 [B][n_in]); pre-activations in Z[i], outputs in Z[2]
psdp_status mlp_forward(psdp_mlp* m, int B) {
    for (int i = 0; i < 3; ++i) {
        const int in = m->dims[i], out = m->dims[i + 1];
        psdp_status s = mlp_gemm(m, m->Wb[i], out, m->H[i], B, in, in, in, m->Z[i], out);
        if (s != PSDP_OK) return s;
        const bool last = i == 2;
        k_bias_act<<<grid1((int64_t)B * out), kT, 0, m->st>>>(B, out, m->Z[i], m->b[i], last ? 0 : 1,
                                                              last ? nullptr : m->H[i + 1], last ? nullptr : m->HT[i + 1],
                                                              m->max_b);
    }
    return PSDP_OK;
}

// backward from targets Tf ([B][n_out] FP32); gradients into gW / gb
psdp_status mlp_backward(psdp_mlp* m, int B) {
    cudaMemsetAsync(m->loss, 0, sizeof(double), m->st);
    // dY (FP32 in dA, reusing the widest activation buffer) and its bf16 copies
    k_mse<<<grid1((int64_t)B * m->n_pad), kT, 0, m->st>>>(B, m->n_pad, m->n_out, m->Z[2], m->Tf, m->dA, m->loss);
    k_to_bf16<<<grid1((int64_t)B * m->n_pad), kT, 0, m->st>>>(B, m->n_pad, m->dA, m->n_pad, m->D, m->n_pad, m->DT,
                                                             m->max_b);
    for (int i = 2; i >= 0; --i) {
        const int in = m->dims[i], out = m->dims[i + 1];
        // gW[i][j][k] = sum_b D[b][j] H_i[b][k]:  D[m=k][n=j] over K = B
        psdp_status s = mlp_gemm(m, m->HT[i], in, m->DT, out, B, m->max_b, m->max_b, m->gW[i], in);
        if (s != PSDP_OK) return s;
        k_colsum<<<grid1(out), kT, 0, m->st>>>(B, out, m->dA, m->gb[i]);
        if (i == 0) break;
        // dA_{i}[b][k] = sum_j D[b][j] W_i[j][k]:  D[m=k][n=b] over K = out
        float* dAprev = m->Z[2];   // Y is no longer needed: reuse as FP32 scratch
        s = mlp_gemm(m, m->WbT[i], in, m->D, B, out, out, out, dAprev, in);
        if (s != PSDP_OK) return s;
        k_relu_back<<<grid1((int64_t)B * in), kT, 0, m->st>>>(B, in, dAprev, m->Z[i - 1], m->D, m->DT, m->max_b);
        cudaMemcpyAsync(m->dA, dAprev, (size_t)B * in * sizeof(float), cudaMemcpyDeviceToDevice, m->st);
    }
    return PSDP_OK;
}

void mlp_free(psdp_mlp* m) {
    if (!m) return;
    cudaSetDevice(m->device);
    cudaStreamSynchronize(m->st);
    for (int i = 0; i < 3; ++i) {
        void* ps[] = {m->W[i], m->b[i], m->gW[i], m->gb[i], m->mW[i], m->vW[i], m->mb[i], m->vb[i], m->Wb[i],
                      m->WbT[i], m->Z[i], m->H[i], m->HT[i]};
        for (void* p : ps)
            if (p) cudaFree(p);
    }
    void* ps[] = {m->dA, m->Xf, m->Tf, m->D, m->DT, m->xmean, m->xstd, m->tmean, m->tstd, m->loss, m->flag};
    for (void* p : ps)
        if (p) cudaFree(p);
    cudaStreamDestroy(m->st);
    cudaGetLastError();
    delete m;
}

int64_t nparams(const psdp_mlp* m) {
    int64_t s = 0;
    for (int i = 0; i < 3; ++i) s += (int64_t)m->dims[i + 1] * m->dims[i] + m->dims[i + 1];
    return s;
}

// copy every W_i (true rows only), b_i between the device and a host array
psdp_status params_io(psdp_mlp* m, float* host, bool to_host, bool grads) {
    int64_t off = 0;
    for (int i = 0; i < 3; ++i) {
        const int in = m->dims[i], out = (i == 2) ? m->n_out : m->dims[i + 1];
        float* dW = grads ? m->gW[i] : m->W[i];
        float* db = grads ? m->gb[i] : m->b[i];
        const size_t nw = (size_t)out * in;
        if (to_host) {
            cudaMemcpyAsync(host + off, dW, nw * 4, cudaMemcpyDeviceToHost, m->st);
            cudaMemcpyAsync(host + off + nw, db, out * 4, cudaMemcpyDeviceToHost, m->st);
        } else {
            cudaMemcpyAsync(dW, host + off, nw * 4, cudaMemcpyHostToDevice, m->st);
            cudaMemcpyAsync(db, host + off + nw, out * 4, cudaMemcpyHostToDevice, m->st);
        }
        off += (int64_t)nw + out;
    }
    if (!to_host && !grads) {
        for (int i = 0; i < 3; ++i)
            k_to_bf16<<<grid1((int64_t)m->dims[i + 1] * m->dims[i]), kT, 0, m->st>>>(
                m->dims[i + 1], m->dims[i], m->W[i], m->dims[i], m->Wb[i], m->dims[i], m->WbT[i], m->dims[i + 1]);
    }
    return cudaStreamSynchronize(m->st) == cudaSuccess && cudaGetLastError() == cudaSuccess ? PSDP_OK : PSDP_ECUDA;
}

// put a batch (FP32 host or device rows) into H[0] (bf16) and Tf
void load_batch(psdp_mlp* m, const float* Xd, const float* Td, int B) {
    k_to_bf16<<<grid1((int64_t)B * m->n_in), kT, 0, m->st>>>(B, m->n_in, Xd, m->n_in, m->H[0], m->n_in, m->HT[0],
                                                           m->max_b);
    if (Td && Td != m->Tf) cudaMemcpyAsync(m->Tf, Td, (size_t)B * m->n_out * 4, cudaMemcpyDeviceToDevice, m->st);
}

void adam_step(psdp_mlp* m, float lr) {
    m->step += 1;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float c1 = 1.f - powf(b1, (float)m->step), c2 = 1.f - powf(b2, (float)m->step);
    for (int i = 0; i < 3; ++i) {
        const int in = m->dims[i], out = m->dims[i + 1];
        k_adam<<<grid1((int64_t)out * in), kT, 0, m->st>>>((int64_t)out * in, m->W[i], m->gW[i], m->mW[i], m->vW[i],
                                                          lr, b1, b2, eps, c1, c2, in, m->Wb[i], m->WbT[i], out);
        k_adam<<<grid1(out), kT, 0, m->st>>>(out, m->b[i], m->gb[i], m->mb[i], m->vb[i], lr, b1, b2, eps, c1, c2, 1,
                                            nullptr, nullptr, 0);
    }
}

}  // namespace

extern "C" {

psdp_status psdp_mlp_create(int n_in, int width, int n_out, int max_batch, uint64_t seed, int device, psdp_mlp** out) {
    if (!out || n_in < 8 || width < 8 || n_out < 1 || max_batch < 8 || n_in % 8 || width % 8 || max_batch % 8)
        return PSDP_EINVAL;
    *out = nullptr;
    if (cudaSetDevice(device) != cudaSuccess) { cudaGetLastError(); return PSDP_ECUDA; }
    int optin = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    init_attrs_tc(optin);
    psdp_mlp* m = new (std::nothrow) psdp_mlp();
    if (!m) return PSDP_ENOMEM;
    m->n_in = n_in; m->width = width; m->n_out = n_out; m->n_pad = (n_out + 7) / 8 * 8; m->max_b = max_batch;
    m->device = device;
    m->dims[0] = n_in; m->dims[1] = width; m->dims[2] = width; m->dims[3] = m->n_pad;
    cudaStreamCreateWithFlags(&m->st, cudaStreamNonBlocking);
    const int maxd = std::max(std::max(n_in, width), m->n_pad);
    bool ok = true;
    for (int i = 0; i < 3 && ok; ++i) {
        const size_t nw = (size_t)m->dims[i + 1] * m->dims[i], nb = m->dims[i + 1];
        ok = dalloc_n(&m->W[i], nw) && dalloc_n(&m->b[i], nb) && dalloc_n(&m->gW[i], nw) && dalloc_n(&m->gb[i], nb) &&
             dalloc_n(&m->mW[i], nw) && dalloc_n(&m->vW[i], nw) && dalloc_n(&m->mb[i], nb) && dalloc_n(&m->vb[i], nb) &&
             dalloc_n(&m->Wb[i], nw) && dalloc_n(&m->WbT[i], nw) &&
             dalloc_n(&m->Z[i], (size_t)max_batch * maxd) && dalloc_n(&m->H[i], (size_t)max_batch * m->dims[i]) &&
             dalloc_n(&m->HT[i], (size_t)max_batch * m->dims[i]);
    }
    ok = ok && dalloc_n(&m->dA, (size_t)max_batch * maxd) && dalloc_n(&m->Tf, (size_t)max_batch * n_out) &&
         dalloc_n(&m->Xf, (size_t)max_batch * n_in) && dalloc_n(&m->D, (size_t)max_batch * maxd) &&
         dalloc_n(&m->DT, (size_t)max_batch * maxd) && dalloc_n(&m->xmean, n_in) && dalloc_n(&m->xstd, n_in) &&
         dalloc_n(&m->tmean, n_out) && dalloc_n(&m->tstd, n_out) && dalloc_n(&m->loss, 1) && dalloc_n(&m->flag, 1);
    if (!ok) {
        mlp_free(m);
        return PSDP_ENOMEM;
    }
    // He-normal weights from a seeded host generator (Box-Muller over a 64-bit LCG), zero biases
    std::vector<float> host(nparams(m) + (int64_t)(m->n_pad - n_out) * width, 0.f);
    uint64_t s = seed * 6364136223846793005ull + 1442695040888963407ull;
    auto uni = [&]() {
        s = s * 6364136223846793005ull + 1442695040888963407ull;
        return ((s >> 11) + 0.5) * (1.0 / 9007199254740992.0);
    };
    int64_t off = 0;
    for (int i = 0; i < 3; ++i) {
        const int in = m->dims[i], outr = (i == 2) ? n_out : m->dims[i + 1];
        const double sd = sqrt(2.0 / in);
        for (int64_t k = 0; k < (int64_t)outr * in; ++k)
            host[off + k] = (float)(sd * sqrt(-2.0 * log(uni())) * cos(6.283185307179586 * uni()));
        off += (int64_t)outr * in + outr;
    }
    for (int i = 0; i < 3; ++i) {
        const size_t nw = (size_t)m->dims[i + 1] * m->dims[i], nb = m->dims[i + 1];
        cudaMemsetAsync(m->W[i], 0, nw * 4, m->st);   // padding rows of the last layer stay zero
        cudaMemsetAsync(m->b[i], 0, nb * 4, m->st);
        cudaMemsetAsync(m->mW[i], 0, nw * 4, m->st);
        cudaMemsetAsync(m->vW[i], 0, nw * 4, m->st);
        cudaMemsetAsync(m->mb[i], 0, nb * 4, m->st);
        cudaMemsetAsync(m->vb[i], 0, nb * 4, m->st);
        cudaMemsetAsync(m->gW[i], 0, nw * 4, m->st);
    }
    cudaMemsetAsync(m->flag, 0, 4, m->st);
    const psdp_status st = params_io(m, host.data(), false, false);
    if (st != PSDP_OK) {
        mlp_free(m);
        return st;
    }
    *out = m;
    return PSDP_OK;
}

void psdp_mlp_destroy(psdp_mlp* m) { mlp_free(m); }

psdp_status psdp_mlp_params(psdp_mlp* m, float* get, const float* set, int64_t* count) {
    if (!m) return PSDP_EINVAL;
    cudaSetDevice(m->device);
    if (count) *count = nparams(m) - (int64_t)(m->n_pad - m->n_out) * (m->width + 1);
    if (set) {
        psdp_status s = params_io(m, const_cast<float*>(set), false, false);
        if (s != PSDP_OK) return s;
    }
    if (get) return params_io(m, get, true, false);
    return PSDP_OK;
}

psdp_status psdp_mlp_grads(psdp_mlp* m, const float* X, const float* T, int B, float* loss, float* grads) {
    if (!m || !X || !T || B < 1 || B > m->max_b) return PSDP_EINVAL;
    cudaSetDevice(m->device);
    cudaMemcpyAsync(m->Xf, X, (size_t)B * m->n_in * 4, cudaMemcpyHostToDevice, m->st);
    cudaMemcpyAsync(m->Tf, T, (size_t)B * m->n_out * 4, cudaMemcpyHostToDevice, m->st);
    load_batch(m, m->Xf, nullptr, B);
    psdp_status s = mlp_forward(m, B);
    if (s == PSDP_OK) s = mlp_backward(m, B);
    if (s != PSDP_OK) return s;
    double l = 0.0;
    int flag = 0;
    cudaMemcpyAsync(&l, m->loss, sizeof(double), cudaMemcpyDeviceToHost, m->st);
    cudaMemcpyAsync(&flag, m->flag, sizeof(int), cudaMemcpyDeviceToHost, m->st);
    if (cudaStreamSynchronize(m->st) != cudaSuccess || cudaGetLastError() != cudaSuccess) return PSDP_ECUDA;
    if (flag) return PSDP_ETIMEOUT;
    if (loss) *loss = (float)(l / ((double)B * m->n_out));
    if (grads) return params_io(m, grads, true, true);
    return PSDP_OK;
}

psdp_status psdp_mlp_train(psdp_mlp* m, const float* X, const float* T, int n, int epochs, int B, float lr,
                           uint64_t seed, float* final_loss) {
    if (!m || !X || !T || n < B || B < 8 || B > m->max_b || B % 8 || epochs < 1 || !(lr > 0.f)) return PSDP_EINVAL;
    cudaSetDevice(m->device);
    float *dX = nullptr, *dT = nullptr, *Ts = nullptr;
    int32_t* didx = nullptr;
    if (!dalloc_n(&dX, (size_t)n * m->n_in) || !dalloc_n(&dT, (size_t)n * m->n_out) || !dalloc_n(&didx, (size_t)n) ||
        !dalloc_n(&Ts, (size_t)B * m->n_out)) {
        cudaFree(dX); cudaFree(dT); cudaFree(didx); cudaFree(Ts);
        return PSDP_ENOMEM;
    }
    cudaMemcpyAsync(dX, X, (size_t)n * m->n_in * 4, cudaMemcpyHostToDevice, m->st);
    cudaMemcpyAsync(dT, T, (size_t)n * m->n_out * 4, cudaMemcpyHostToDevice, m->st);
    k_colstats<<<grid1(m->n_in), kT, 0, m->st>>>(n, m->n_in, dX, m->xmean, m->xstd);
    k_colstats<<<grid1(m->n_out), kT, 0, m->st>>>(n, m->n_out, dT, m->tmean, m->tstd);
    m->fitted = true;
    std::vector<int32_t> perm(n);
    uint64_t s = seed * 2862933555777941757ull + 3037000493ull;
    double last = 0.0;
    psdp_status st = PSDP_OK;
    for (int ep = 0; ep < epochs && st == PSDP_OK; ++ep) {
        for (int i = 0; i < n; ++i) perm[i] = i;
        for (int i = n - 1; i > 0; --i) {     // Fisher-Yates with a 64-bit LCG
            s = s * 6364136223846793005ull + 1442695040888963407ull;
            const int j = (int)((s >> 33) % (uint64_t)(i + 1));
            std::swap(perm[i], perm[j]);
        }
        cudaMemcpyAsync(didx, perm.data(), (size_t)n * 4, cudaMemcpyHostToDevice, m->st);
        double ep_loss = 0.0;
        int nb = 0;
        for (int b0 = 0; b0 + B <= n; b0 += B, ++nb) {
            k_gather_std<<<grid1((int64_t)B * m->n_in), kT, 0, m->st>>>(B, m->n_in, didx + b0, dX, m->xmean, m->xstd,
                                                                       m->Xf);
            k_gather_std<<<grid1((int64_t)B * m->n_out), kT, 0, m->st>>>(B, m->n_out, didx + b0, dT, m->tmean,
                                                                        m->tstd, m->Tf);
            load_batch(m, m->Xf, nullptr, B);
            if ((st = mlp_forward(m, B)) != PSDP_OK || (st = mlp_backward(m, B)) != PSDP_OK) break;
            adam_step(m, lr);
            double l = 0.0;
            cudaMemcpyAsync(&l, m->loss, sizeof(double), cudaMemcpyDeviceToHost, m->st);
            cudaStreamSynchronize(m->st);
            ep_loss += l / ((double)B * m->n_out);
        }
        last = nb ? ep_loss / nb : 0.0;
    }
    int flag = 0;
    cudaMemcpyAsync(&flag, m->flag, sizeof(int), cudaMemcpyDeviceToHost, m->st);
    if (cudaStreamSynchronize(m->st) != cudaSuccess || cudaGetLastError() != cudaSuccess) st = PSDP_ECUDA;
    if (flag) st = PSDP_ETIMEOUT;
    cudaFree(dX); cudaFree(dT); cudaFree(didx); cudaFree(Ts);
    if (final_loss) *final_loss = (float)last;
    return st;
}

psdp_status psdp_mlp_predict(psdp_mlp* m, const float* X, int n, float* Y) {
    if (!m || !X || !Y || n < 1) return PSDP_EINVAL;
    cudaSetDevice(m->device);
    float *dX = nullptr, *dY = nullptr;
    if (!dalloc_n(&dX, (size_t)n * m->n_in) || !dalloc_n(&dY, (size_t)n * m->n_out)) {
        cudaFree(dX); cudaFree(dY);
        return PSDP_ENOMEM;
    }
    cudaMemcpyAsync(dX, X, (size_t)n * m->n_in * 4, cudaMemcpyHostToDevice, m->st);
    psdp_status st = PSDP_OK;
    for (int r0 = 0; r0 < n && st == PSDP_OK; r0 += m->max_b) {
        const int B = std::min(m->max_b, n - r0);
        if (m->fitted)
            k_gather_std<<<grid1((int64_t)B * m->n_in), kT, 0, m->st>>>(B, m->n_in, nullptr, dX + (int64_t)r0 * m->n_in,
                                                                       m->xmean, m->xstd, m->Xf);
        else
            cudaMemcpyAsync(m->Xf, dX + (int64_t)r0 * m->n_in, (size_t)B * m->n_in * 4, cudaMemcpyDeviceToDevice, m->st);
        load_batch(m, m->Xf, nullptr, B);
        st = mlp_forward(m, B);
        if (m->fitted) {
            k_unstd<<<grid1((int64_t)B * m->n_out), kT, 0, m->st>>>(B, m->n_pad, m->n_out, m->Z[2], m->tmean, m->tstd,
                                                                   dY + (int64_t)r0 * m->n_out);
        } else {
            cudaMemcpy2DAsync(dY + (int64_t)r0 * m->n_out, (size_t)m->n_out * 4, m->Z[2], (size_t)m->n_pad * 4,
                              (size_t)m->n_out * 4, B, cudaMemcpyDeviceToDevice, m->st);
        }
    }
    cudaMemcpyAsync(Y, dY, (size_t)n * m->n_out * 4, cudaMemcpyDeviceToHost, m->st);
    if (cudaStreamSynchronize(m->st) != cudaSuccess || cudaGetLastError() != cudaSuccess) st = PSDP_ECUDA;
    cudaFree(dX);
    cudaFree(dY);
    return st;
}

}  // extern "C"

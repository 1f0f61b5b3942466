// Learned Davidson preconditioner: a small MLP that corrects the diagonal one.
//
// For a residual r of the Ritz pair (w, y) the diagonal preconditioner is
// t_x = r_x p_x with p_x = 1 / (w - D_x) (|w - D_x| clamped to >= 1e-8; D the
// zeroth-order / 1p-block diagonal).  The learned form keeps the correction
// linear in r and adds a multiplier from a 3 -> 64 -> 64 -> 1 network (tanh):
//   t_x = r_x (p_x + m(f_x)),  f_x = (d, sign(d) / max(|d|, 0.01), [x in the 1p/1h block]),  d = D_x - w.
// With zero output weights it is exactly the diagonal preconditioner.  It is
// trained on (d, block, r, t*) samples, t* the exact correction y_exact /
// <y, y_exact>_S - y of plain Davidson iterates, by minimising
//   L = sum_x (r_x (p_x + m_x) - t*_x)^2 / sum_x t*_x^2
// with Adam, in FP32, by the fused kernels below.
#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "mlp.cuh"

namespace adc {

namespace {

constexpr int NF = 3, NH = 64;
// weight layout: W1 [NH][NF], b1 [NH], W2 [NH][NH], b2 [NH], W3 [NH], b3
constexpr int OW1 = 0, OB1 = OW1 + NH * NF, OW2 = OB1 + NH, OB2 = OW2 + NH * NH, OW3 = OB2 + NH, OB3 = OW3 + NH;
constexpr int NW = OB3 + 1;

__device__ __forceinline__ void features(float d, int blk, float f[NF]) {
    f[0] = d;
    const float ad = fabsf(d);
    f[1] = (ad < 0.01f ? (d < 0.f ? -1.f : 1.f) / 0.01f : 1.f / d);
    f[2] = blk ? 1.f : 0.f;
}
__device__ __forceinline__ double diag_mult(double d) {  // p = 1 / (w - D) = -1 / d, |d| >= 1e-8
    if (fabs(d) < 1e-8) d = d < 0 ? -1e-8 : 1e-8;
    return -1.0 / d;
}

// forward of one sample; h1, h2 hold the hidden activations
__device__ __forceinline__ float forward(const float* __restrict__ W, const float f[NF], float h1[NH], float h2[NH]) {
#pragma unroll
    for (int j = 0; j < NH; ++j) {
        float s = W[OB1 + j];
#pragma unroll
        for (int i = 0; i < NF; ++i) s += W[OW1 + j * NF + i] * f[i];
        h1[j] = tanhf(s);
    }
    float m = W[OB3];
    for (int j = 0; j < NH; ++j) {
        float s = W[OB2 + j];
#pragma unroll
        for (int k = 0; k < NH; ++k) s += W[OW2 + j * NH + k] * h1[k];
        h2[j] = tanhf(s);
        m += W[OW3 + j] * h2[j];
    }
    return m;
}

// Davidson correction out[r][x] = R[r][x] (p + m) for nr residuals
__global__ void __launch_bounds__(256) k_mlp_precond(long long nr, long long dim, long long n1, const double* __restrict__ R,
                                                     const double* __restrict__ w, const double* __restrict__ D,
                                                     const float* __restrict__ Wg, double* __restrict__ out) {
    __shared__ float W[NW];
    for (int i = threadIdx.x; i < NW; i += blockDim.x) W[i] = Wg[i];
    __syncthreads();
    const long long n = nr * dim;
    for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < n; x += (long long)gridDim.x * blockDim.x) {
        const long long r = x / dim, k = x - r * dim;
        const double d = D[k] - w[r];
        float f[NF], h1[NH], h2[NH];
        features((float)d, k < n1, f);
        const float m = forward(W, f, h1, h2);
        out[x] = R[x] * (diag_mult(d) + (double)m);
    }
}

// loss and gradient over n samples; grad and loss accumulate (zeroed by the caller)
__global__ void __launch_bounds__(128) k_mlp_grad(long long n, const float* __restrict__ d, const unsigned char* __restrict__ blk,
                                                  const float* __restrict__ r, const float* __restrict__ t,
                                                  const float* __restrict__ Wg, float inv_norm, float* __restrict__ grad,
                                                  double* __restrict__ loss) {
    __shared__ float W[NW];
    __shared__ float G[NW];
    for (int i = threadIdx.x; i < NW; i += blockDim.x) {
        W[i] = Wg[i];
        G[i] = 0.f;
    }
    __syncthreads();
    double lsum = 0.0;
    for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < n; x += (long long)gridDim.x * blockDim.x) {
        float f[NF], h1[NH], h2[NH];
        features(d[x], blk[x], f);
        const float m = forward(W, f, h1, h2);
        const float e = r[x] * ((float)diag_mult(d[x]) + m) - t[x];
        lsum += (double)e * e * inv_norm;
        const float g = 2.f * e * r[x] * inv_norm;  // dL/dm
        atomicAdd(&G[OB3], g);
        float g1[NH];
#pragma unroll
        for (int k = 0; k < NH; ++k) g1[k] = 0.f;
        for (int j = 0; j < NH; ++j) {
            atomicAdd(&G[OW3 + j], g * h2[j]);
            const float g2 = g * W[OW3 + j] * (1.f - h2[j] * h2[j]);
            atomicAdd(&G[OB2 + j], g2);
#pragma unroll
            for (int k = 0; k < NH; ++k) {
                atomicAdd(&G[OW2 + j * NH + k], g2 * h1[k]);
                g1[k] += g2 * W[OW2 + j * NH + k];
            }
        }
#pragma unroll
        for (int k = 0; k < NH; ++k) {
            const float gk = g1[k] * (1.f - h1[k] * h1[k]);
            atomicAdd(&G[OB1 + k], gk);
#pragma unroll
            for (int i = 0; i < NF; ++i) atomicAdd(&G[OW1 + k * NF + i], gk * f[i]);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < NW; i += blockDim.x) atomicAdd(&grad[i], G[i]);
    // block-reduce the loss through shared memory
    __shared__ double L[128];
    L[threadIdx.x] = lsum;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) L[threadIdx.x] += L[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(loss, L[0]);
}

__global__ void k_adam(int n, float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m1, float* __restrict__ m2,
                       float lr, float b1, float b2, float eps, float c1, float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    m1[i] = b1 * m1[i] + (1.f - b1) * g[i];
    m2[i] = b2 * m2[i] + (1.f - b2) * g[i] * g[i];
    w[i] -= lr * (m1[i] / c1) / (sqrtf(m2[i] / c2) + eps);
}

struct DevBuf {
    void* p = nullptr;
    ~DevBuf() { cudaFree(p); }
    void* get(size_t bytes) {
        ADC_CUDA(cudaMalloc(&p, bytes ? bytes : 1));
        return p;
    }
};

struct Samples {
    DevBuf bd, bb, br, bt;
    float *d, *r, *t;
    unsigned char* b;
    float inv_norm;
};

void load_samples(Samples& s, const double* d, const unsigned char* blk, const double* r, const double* t, long long n) {
    std::vector<float> fd(n), fr(n), ft(n);
    double tn = 0.0;
    for (long long i = 0; i < n; ++i) {
        fd[i] = (float)d[i];
        fr[i] = (float)r[i];
        ft[i] = (float)t[i];
        tn += t[i] * t[i];
    }
    s.inv_norm = tn > 0 ? (float)(1.0 / tn) : 1.f;
    s.d = (float*)s.bd.get(n * sizeof(float));
    s.r = (float*)s.br.get(n * sizeof(float));
    s.t = (float*)s.bt.get(n * sizeof(float));
    s.b = (unsigned char*)s.bb.get(n);
    ADC_CUDA(cudaMemcpy(s.d, fd.data(), n * sizeof(float), cudaMemcpyHostToDevice));
    ADC_CUDA(cudaMemcpy(s.r, fr.data(), n * sizeof(float), cudaMemcpyHostToDevice));
    ADC_CUDA(cudaMemcpy(s.t, ft.data(), n * sizeof(float), cudaMemcpyHostToDevice));
    ADC_CUDA(cudaMemcpy(s.b, blk, n, cudaMemcpyHostToDevice));
}

int grad_blocks(long long n) { return (int)std::max<long long>(1, std::min<long long>((n + 127) / 128, 152LL * 8)); }

}  // namespace

int mlp_nweights() { return NW; }

void mlp_precondition(Ctx& c, long long nr, long long dim, long long n1, const double* R, const double* w, const double* D,
                      const float* weights, double* out) {
    const long long n = nr * dim;
    const int grid = (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, 152LL * 16));
    k_mlp_precond<<<grid, 256, 0, c.stream>>>(nr, dim, n1, R, w, D, weights, out);
    ++c.kernels;
    ADC_CUDA(cudaGetLastError());
}

double mlp_loss_grad_host(const float* weights, const double* d, const unsigned char* blk, const double* r, const double* t,
                          long long n, float* grad) {
    Samples s;
    load_samples(s, d, blk, r, t, n);
    DevBuf bw, bg, bl;
    float* W = (float*)bw.get(NW * sizeof(float));
    float* G = (float*)bg.get(NW * sizeof(float));
    double* L = (double*)bl.get(sizeof(double));
    ADC_CUDA(cudaMemcpy(W, weights, NW * sizeof(float), cudaMemcpyHostToDevice));
    ADC_CUDA(cudaMemset(G, 0, NW * sizeof(float)));
    ADC_CUDA(cudaMemset(L, 0, sizeof(double)));
    k_mlp_grad<<<grad_blocks(n), 128>>>(n, s.d, s.b, s.r, s.t, W, s.inv_norm, G, L);
    ADC_CUDA(cudaGetLastError());
    double loss = 0.0;
    ADC_CUDA(cudaMemcpy(grad, G, NW * sizeof(float), cudaMemcpyDeviceToHost));
    ADC_CUDA(cudaMemcpy(&loss, L, sizeof(double), cudaMemcpyDeviceToHost));
    return loss;
}

void mlp_train_host(float* weights, const double* d, const unsigned char* blk, const double* r, const double* t, long long n,
                    int steps, float lr, double* loss_hist) {
    Samples s;
    load_samples(s, d, blk, r, t, n);
    DevBuf bw, bg, bm1, bm2, bl;
    float* W = (float*)bw.get(NW * sizeof(float));
    float* G = (float*)bg.get(NW * sizeof(float));
    float* M1 = (float*)bm1.get(NW * sizeof(float));
    float* M2 = (float*)bm2.get(NW * sizeof(float));
    double* L = (double*)bl.get(sizeof(double) * std::max(steps, 1));
    ADC_CUDA(cudaMemcpy(W, weights, NW * sizeof(float), cudaMemcpyHostToDevice));
    ADC_CUDA(cudaMemset(M1, 0, NW * sizeof(float)));
    ADC_CUDA(cudaMemset(M2, 0, NW * sizeof(float)));
    ADC_CUDA(cudaMemset(L, 0, sizeof(double) * std::max(steps, 1)));
    const float b1 = 0.9f, b2 = 0.999f;
    float c1 = 1.f, c2 = 1.f;
    for (int it = 0; it < steps; ++it) {
        ADC_CUDA(cudaMemsetAsync(G, 0, NW * sizeof(float)));
        k_mlp_grad<<<grad_blocks(n), 128>>>(n, s.d, s.b, s.r, s.t, W, s.inv_norm, G, L + it);
        c1 *= b1;
        c2 *= b2;
        k_adam<<<(NW + 255) / 256, 256>>>(NW, W, G, M1, M2, lr, b1, b2, 1e-8f, 1.f - c1, 1.f - c2);
        ADC_CUDA(cudaGetLastError());
    }
    ADC_CUDA(cudaMemcpy(weights, W, NW * sizeof(float), cudaMemcpyDeviceToHost));
    if (loss_hist) ADC_CUDA(cudaMemcpy(loss_hist, L, sizeof(double) * steps, cudaMemcpyDeviceToHost));
}

}  // namespace adc

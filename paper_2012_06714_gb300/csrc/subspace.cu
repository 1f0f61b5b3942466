// FP64 subspace kernels of the Davidson iteration; see subspace.cuh.
#include "subspace.cuh"

#include <algorithm>

namespace adc {
namespace {

constexpr int kThreads = 256;
constexpr int kRT = 8;  // output rows of a linear combination per pass

// Partial inner products of a TI x TJ block of (A row, B row) pairs over one
// slice of x: part[s][i][j] for slice s = blockIdx.y.  The block shape follows
// the problem (TI, TJ <= na, nb rounded up to powers of two), so no FP64 FMA is
// spent on pairs that are not asked for, except in the last block.
template <int TI, int TJ>
__global__ void __launch_bounds__(kThreads) k_multidot(int na, const double* __restrict__ A, long long lda, int nb,
                                                       const double* __restrict__ B, long long ldb, long long n,
                                                       long long chunk, int tiles_j, double* __restrict__ part) {
    const int ti = blockIdx.x / tiles_j, tj = blockIdx.x % tiles_j;
    const int i0 = ti * TI, j0 = tj * TJ;
    const long long x0 = (long long)blockIdx.y * chunk, x1 = x0 + chunk < n ? x0 + chunk : n;
    double acc[TI][TJ];
#pragma unroll
    for (int a = 0; a < TI; ++a)
#pragma unroll
        for (int b = 0; b < TJ; ++b) acc[a][b] = 0.0;
    // rows past na / nb read row 0 (always valid) and are discarded at the end
    const double* Ar[TI];
    const double* Br[TJ];
#pragma unroll
    for (int a = 0; a < TI; ++a) Ar[a] = A + (long long)(i0 + a < na ? i0 + a : 0) * lda;
#pragma unroll
    for (int b = 0; b < TJ; ++b) Br[b] = B + (long long)(j0 + b < nb ? j0 + b : 0) * ldb;
    for (long long x = x0 + threadIdx.x; x < x1; x += kThreads) {
        double bv[TJ];
#pragma unroll
        for (int b = 0; b < TJ; ++b) bv[b] = __ldg(Br[b] + x);
#pragma unroll
        for (int a = 0; a < TI; ++a) {
            const double av = __ldg(Ar[a] + x);
#pragma unroll
            for (int b = 0; b < TJ; ++b) acc[a][b] = fma(av, bv[b], acc[a][b]);
        }
    }
    // reduce over the CTA: warp shuffles, then one value per warp through shared memory
    __shared__ double red[kThreads / 32][TI * TJ];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int a = 0; a < TI; ++a)
#pragma unroll
        for (int b = 0; b < TJ; ++b) {
            double v = acc[a][b];
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
            if (lane == 0) red[warp][a * TJ + b] = v;
        }
    __syncthreads();
    if (threadIdx.x < TI * TJ) {
        double v = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) v += red[w][threadIdx.x];
        const int a = threadIdx.x / TJ, b = threadIdx.x % TJ;
        if (i0 + a < na && j0 + b < nb) part[((long long)blockIdx.y * na + i0 + a) * nb + j0 + b] = v;
    }
}

// D = sum_s part[s] in slice order; part[s] is [na][nb], D is that ([na][nb]) or,
// with trans, its transpose ([nb][na])
__global__ void k_sum_parts(int S, int na, int nb, int trans, const double* __restrict__ part, double* __restrict__ D) {
    const long long ne = (long long)na * nb;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < ne; e += (long long)gridDim.x * blockDim.x) {
        double v = 0.0;
        for (int s = 0; s < S; ++s) v += part[(long long)s * ne + e];
        D[trans ? (e % nb) * na + e / nb : e] = v;
    }
}

template <int TI, int TJ>
void launch_multidot(dim3 grid, cudaStream_t st, int na, const double* A, long long lda, int nb, const double* B,
                     long long ldb, long long n, long long chunk, int tiles_j, double* part) {
    k_multidot<TI, TJ><<<grid, kThreads, 0, st>>>(na, A, lda, nb, B, ldb, n, chunk, tiles_j, part);
}

// Y[r0 + r][x] = beta Y + alpha sum_i C[(r0 + r) * k + i] V[i][x] for r < nrc (<= kRT); C rows in shared memory
__global__ void __launch_bounds__(kThreads) k_lincomb(int nrc, int r0, int k, const double* __restrict__ C,
                                                     const double* __restrict__ V, long long ldv, long long n,
                                                     double alpha, double beta, double* __restrict__ Y, long long ldy) {
    extern __shared__ double Cs[];  // [nrc][k]
    for (int e = threadIdx.x; e < nrc * k; e += blockDim.x) Cs[e] = C[(long long)r0 * k + e];
    __syncthreads();
    for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < n; x += (long long)gridDim.x * blockDim.x) {
        double acc[kRT];
#pragma unroll
        for (int r = 0; r < kRT; ++r) acc[r] = 0.0;
        for (int i = 0; i < k; ++i) {
            const double v = __ldg(V + (long long)i * ldv + x);
#pragma unroll
            for (int r = 0; r < kRT; ++r)
                if (r < nrc) acc[r] = fma(Cs[r * k + i], v, acc[r]);
        }
#pragma unroll
        for (int r = 0; r < kRT; ++r)
            if (r < nrc) {
                double* y = Y + (long long)(r0 + r) * ldy + x;
                *y = beta == 0.0 ? alpha * acc[r] : fma(beta, *y, alpha * acc[r]);
            }
    }
}

int sm_count() {
    static int n = [] {
        int dev = 0, v = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return 152;
        return v > 0 ? v : 152;
    }();
    return n;
}

}  // namespace

void multidot(Ctx& c, int na, const double* A, long long lda, int nb, const double* B, long long ldb, long long n,
              double* D) {
    if (na <= 0 || nb <= 0) return;
    if (n <= 0) {
        fill(c, (long long)na * nb, 0.0, D);
        return;
    }
    // the longer side takes the block's TI rows; the result is transposed back if swapped
    const int trans = na < nb ? 1 : 0;
    if (trans) {
        std::swap(na, nb);
        std::swap(A, B);
        std::swap(lda, ldb);
    }
    const int TI = na >= 8 ? 8 : na > 2 ? 4 : na;          // 1, 2, 4 or 8
    const int TJ = nb >= 4 ? 4 : nb > 2 ? 4 : nb;          // 1, 2 or 4 (TJ <= TI)
    const int ti = (na + TI - 1) / TI, tj = (nb + TJ - 1) / TJ, tiles = ti * tj;
    if ((long long)tiles > (1LL << 30)) throw Error(-1, "multidot: too many vectors");
    // about four resident CTAs per SM in total; each slice at least 4096 elements
    long long S = std::max(1LL, (long long)(4 * sm_count()) / tiles);
    S = std::min(S, std::max(1LL, n / 4096));
    S = std::min(S, 65535LL);
    const long long chunk = (n + S - 1) / S;
    S = (n + chunk - 1) / chunk;
    Arena::Mark mk = c.arena.mark();
    double* part = c.arena.dalloc((size_t)S * na * nb);
    const dim3 grid(tiles, (unsigned)S);
    const cudaStream_t st = c.stream;
    switch (TI * 16 + TJ) {
        case 8 * 16 + 4: launch_multidot<8, 4>(grid, st, na, A, lda, nb, B, ldb, n, chunk, tj, part); break;
        case 8 * 16 + 2: launch_multidot<8, 2>(grid, st, na, A, lda, nb, B, ldb, n, chunk, tj, part); break;
        case 8 * 16 + 1: launch_multidot<8, 1>(grid, st, na, A, lda, nb, B, ldb, n, chunk, tj, part); break;
        case 4 * 16 + 4: launch_multidot<4, 4>(grid, st, na, A, lda, nb, B, ldb, n, chunk, tj, part); break;
        case 4 * 16 + 2: launch_multidot<4, 2>(grid, st, na, A, lda, nb, B, ldb, n, chunk, tj, part); break;
        case 4 * 16 + 1: launch_multidot<4, 1>(grid, st, na, A, lda, nb, B, ldb, n, chunk, tj, part); break;
        case 2 * 16 + 2: launch_multidot<2, 2>(grid, st, na, A, lda, nb, B, ldb, n, chunk, tj, part); break;
        case 2 * 16 + 1: launch_multidot<2, 1>(grid, st, na, A, lda, nb, B, ldb, n, chunk, tj, part); break;
        case 1 * 16 + 1: launch_multidot<1, 1>(grid, st, na, A, lda, nb, B, ldb, n, chunk, tj, part); break;
        default: throw Error(-1, "multidot: no block shape");
    }
    ++c.kernels;
    ADC_CUDA(cudaGetLastError());
    const long long ne = (long long)na * nb;
    k_sum_parts<<<(int)std::min<long long>((ne + 255) / 256, 1024), 256, 0, c.stream>>>((int)S, na, nb, trans, part, D);
    ++c.kernels;
    ADC_CUDA(cudaGetLastError());
    c.arena.release(mk);
}

void lincomb(Ctx& c, int nr, int k, const double* C, const double* V, long long ldv, long long n, double alpha, double beta,
             double* Y, long long ldy) {
    if (nr <= 0 || n <= 0) return;
    if (k <= 0) {
        for (int r = 0; r < nr; ++r) {
            double* y = Y + (long long)r * ldy;
            if (beta == 0.0)
                fill(c, n, 0.0, y);
            else
                axpby(c, n, beta, y, 0.0, y);
        }
        return;
    }
    const size_t smem = (size_t)kRT * k * sizeof(double);
    if (smem > 48 * 1024) throw Error(-1, "lincomb: basis too large (k > 768)");
    const int grid = (int)std::min<long long>((n + kThreads - 1) / kThreads, 8LL * sm_count());
    for (int r0 = 0; r0 < nr; r0 += kRT) {
        const int nrc = std::min(kRT, nr - r0);
        k_lincomb<<<grid, kThreads, (size_t)nrc * k * sizeof(double), c.stream>>>(nrc, r0, k, C, V, ldv, n, alpha, beta, Y,
                                                                                 ldy);
        ++c.kernels;
        ADC_CUDA(cudaGetLastError());
    }
}

}  // namespace adc

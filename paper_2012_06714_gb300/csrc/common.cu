// Elementwise kernels and the tensor-contraction executor used by setup and
// the FP64 sigma path.
#include <algorithm>
#include <cstring>
#include <map>
#include <type_traits>

#include <cuda_bf16.h>

#include "common.cuh"
#include "ladder_tc.cuh"

namespace adc {

namespace {

struct PermArgs {
    int nd;
    long long dout[kMaxDim];
    long long sin[kMaxDim];  // input stride for each output axis
};

// I: the index type of the coordinate arithmetic (32-bit when every offset fits: integer
// division by a runtime divisor is several times cheaper than in 64 bits)
template <typename I>
__global__ void permute_kernel(const double* __restrict__ in, double* __restrict__ out, PermArgs a, long long total,
                               double alpha, double beta) {
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        I r = (I)idx, off = 0;
        for (int j = a.nd - 1; j >= 0; --j) {
            const I d = (I)a.dout[j];
            const I q = r / d;
            off += (r - q * d) * (I)a.sin[j];
            r = q;
        }
        double v = alpha * in[off];
        out[idx] = (beta == 0.0) ? v : v + beta * out[idx];
    }
}

template <typename I, typename Tin, typename Tout>
__global__ void permute_cvt_kernel(const Tin* __restrict__ in, Tout* __restrict__ out, PermArgs a, long long total,
                                   double alpha, double beta) {
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        I r = (I)idx, off = 0;
        for (int j = a.nd - 1; j >= 0; --j) {
            const I d = (I)a.dout[j];
            const I q = r / d;
            off += (r - q * d) * (I)a.sin[j];
            r = q;
        }
        double v = alpha * (double)in[off];
        out[idx] = (Tout)((beta == 0.0) ? v : v + beta * (double)out[idx]);
    }
}

__global__ void axpby_kernel(long long n, double alpha, const double* __restrict__ x, double beta, double* __restrict__ y) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = (beta == 0.0) ? alpha * x[i] : alpha * x[i] + beta * y[i];
}

__global__ void fill_kernel(long long n, double v, double* __restrict__ y) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = v;
}

// out[p][r*Kp + k] (two BF16 planes) from the permuted input, zero for k >= K
template <typename I, typename Tin>
__global__ void permute_split_kernel(const Tin* __restrict__ in, __nv_bfloat16* __restrict__ o0,
                                     __nv_bfloat16* __restrict__ o1, PermArgs a, long long rows, long long K, long long Kp) {
    const long long total = rows * Kp;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const I r = (I)(idx / Kp), k = (I)(idx - (long long)r * Kp);
        double x = 0.0;
        if (k < (I)K) {
            I lin = r * (I)K + k, off = 0;
            for (int j = a.nd - 1; j >= 0; --j) {
                const I d = (I)a.dout[j];
                const I q = lin / d;
                off += (lin - q * d) * (I)a.sin[j];
                lin = q;
            }
            x = (double)in[off];
        }
        const __nv_bfloat16 h = __double2bfloat16(x);
        o0[idx] = h;
        o1[idx] = __double2bfloat16(x - (double)__bfloat162float(h));
    }
}

// ---- transposing permutes through shared memory ----------------------------------
// When the output's fastest axis x is strided in the input, the plain kernels above read one
// element per memory sector.  These take a 32 x 32 tile over x and the axis y that is
// contiguous in the input: threads read along y (coalesced), the tile is transposed in shared
// memory, threads write along x (coalesced).  The remaining output axes index the tiles.
struct TileArgs {
    int nrest;
    long long rdim[kMaxDim], rsin[kMaxDim], rsout[kMaxDim];  // other output axes: extent, input / output stride
    long long nx, ny, sx_in, sy_out;  // x: output-innermost axis (input stride sx_in); y: input-contiguous axis
    long long ntx, nty, nblocks;
};

// output of two split BF16 planes [rows][Kp] (the linear output index counts [rows][K])
struct OpPlanes {
    __nv_bfloat16 *o0, *o1;
    long long K, Kp;
    __device__ long long addr(long long lin) const {
        const long long r = lin / K;
        return r * Kp + (lin - r * K);
    }
    __device__ void put(long long ad, double x) const {
        const __nv_bfloat16 h = __double2bfloat16(x);
        o0[ad] = h;
        o1[ad] = __double2bfloat16(x - (double)__bfloat162float(h));
    }
};
// out = alpha x + beta out
template <typename Tout>
struct OpAxpby {
    Tout* out;
    double alpha, beta;
    __device__ long long addr(long long lin) const { return lin; }
    __device__ void put(long long ad, double x) const {
        const double v = alpha * x;
        out[ad] = (Tout)(beta == 0.0 ? v : v + beta * (double)out[ad]);
    }
};

template <typename Tin, typename Op>
__global__ void __launch_bounds__(256) k_permute_tiled(const Tin* __restrict__ in, TileArgs a, Op op) {
    __shared__ double tile[32][33];
    for (long long b = blockIdx.x; b < a.nblocks; b += gridDim.x) {
        long long t = b;
        const long long tx = t % a.ntx;
        t /= a.ntx;
        const long long ty = t % a.nty;
        t /= a.nty;
        long long in_off = 0, out_lin = 0;
        for (int j = a.nrest - 1; j >= 0; --j) {
            const long long cj = t % a.rdim[j];
            t /= a.rdim[j];
            in_off += cj * a.rsin[j];
            out_lin += cj * a.rsout[j];
        }
        const long long x0 = tx * 32, y0 = ty * 32;
        for (int i = threadIdx.y; i < 32; i += 8) {
            const long long x = x0 + i, y = y0 + threadIdx.x;
            if (x < a.nx && y < a.ny) tile[threadIdx.x][i] = (double)in[in_off + x * a.sx_in + y];
        }
        __syncthreads();
        for (int i = threadIdx.y; i < 32; i += 8) {
            const long long y = y0 + i, x = x0 + threadIdx.x;
            if (y < a.ny && x < a.nx) {
                // the row's 32 x values share one output row (x is the innermost output axis)
                const long long ad = op.addr(out_lin + y * a.sy_out + x0);
                op.put(ad + threadIdx.x, tile[i][threadIdx.x]);
            }
        }
        __syncthreads();
    }
}

// zero the K padding columns of split planes [rows][Kp]
__global__ void k_zero_pad(__nv_bfloat16* __restrict__ o0, __nv_bfloat16* __restrict__ o1, long long rows, long long K,
                           long long Kp) {
    const long long w = Kp - K, n = rows * w;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const long long r = i / w, k = K + (i - r * w);
        o0[r * Kp + k] = __double2bfloat16(0.0);
        o1[r * Kp + k] = __double2bfloat16(0.0);
    }
}

__global__ void sum_slices_kernel(int S, long long n, const double* __restrict__ T, double* __restrict__ C) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        double a = 0.0;
        for (int s = 0; s < S; ++s) a += T[s * n + i];
        C[i] = a;
    }
}

inline int grid_for(long long n) {
    long long g = (n + 255) / 256;
    return (int)std::min<long long>(std::max<long long>(g, 1), 152LL * 32);
}

// ---- own GEMM kernels for the small and skinny contractions of sigma ------------
// Row-major A [M][K] (lda), B [K][N] (ldb).  F32: FP64 operands rounded to FP32 in
// registers, FP32 products summed in FP32 over at most 64 terms, those partial sums
// accumulated in FP64 (the FP32-accurate class); else FP64 throughout.  Each kernel
// writes its K slice's partial result P[slice][m][n]; k_reduce_slices finishes
// C = alpha sum_slices P + beta C.

constexpr int SK_THREADS = 256;
constexpr int SK_CHUNK = 64;  // FP32 partial-sum length

// M <= MM rows of A (a few trial vectors): one thread per column n of B, the A values of
// the current 256-deep K chunk in shared memory; reads B once, coalesced along n.
template <int MM, bool F32>
__global__ void __launch_bounds__(SK_THREADS) k_skinny_m(int M, long long N, long long K, long long kslice,
                                                         const double* __restrict__ A, long long lda,
                                                         const double* __restrict__ B, long long ldb,
                                                         double* __restrict__ P) {
    // the A chunk in shared memory, already rounded to FP32 for the FP32-product form
    using AT = typename std::conditional<F32, float, double>::type;
    __shared__ AT As[MM][SK_THREADS];
    const long long n = blockIdx.x * (long long)SK_THREADS + threadIdx.x;
    const long long k0 = blockIdx.y * kslice, k1 = min(K, k0 + kslice);
    double acc[MM];
#pragma unroll
    for (int m = 0; m < MM; ++m) acc[m] = 0.0;
    for (long long kc = k0; kc < k1; kc += SK_THREADS) {
        const int kn = (int)min((long long)SK_THREADS, k1 - kc);
        __syncthreads();
        if (threadIdx.x < kn)
#pragma unroll
            for (int m = 0; m < MM; ++m) As[m][threadIdx.x] = (AT)(m < M ? A[m * lda + kc + threadIdx.x] : 0.0);
        __syncthreads();
        if (n >= N) continue;
        const double* b = B + kc * ldb + n;
        // U independent loads in flight per thread before their FMAs (the loop is bound by
        // memory latency otherwise)
        constexpr int U = 8;
        if (F32) {
            for (int k2 = 0; k2 < kn; k2 += SK_CHUNK) {
                float part[MM];
#pragma unroll
                for (int m = 0; m < MM; ++m) part[m] = 0.f;
                const int ke = min(kn, k2 + SK_CHUNK);
                for (int kk = k2; kk < ke; kk += U) {
                    float bv[U];
#pragma unroll
                    for (int u = 0; u < U; ++u) bv[u] = kk + u < ke ? (float)b[(long long)(kk + u) * ldb] : 0.f;
#pragma unroll
                    for (int u = 0; u < U; ++u)
#pragma unroll
                        for (int m = 0; m < MM; ++m) part[m] = fmaf(kk + u < ke ? (float)As[m][kk + u] : 0.f, bv[u], part[m]);
                }
#pragma unroll
                for (int m = 0; m < MM; ++m) acc[m] += (double)part[m];
            }
        } else {
            for (int kk = 0; kk < kn; kk += U) {
                double bv[U];
#pragma unroll
                for (int u = 0; u < U; ++u) bv[u] = kk + u < kn ? b[(long long)(kk + u) * ldb] : 0.0;
#pragma unroll
                for (int u = 0; u < U; ++u)
#pragma unroll
                    for (int m = 0; m < MM; ++m) acc[m] = fma(kk + u < kn ? As[m][kk + u] : 0.0, bv[u], acc[m]);
            }
        }
    }
    if (n < N)
#pragma unroll
        for (int m = 0; m < MM; ++m)
            if (m < M) P[((long long)blockIdx.y * M + m) * N + n] = acc[m];
}

// N <= NN columns of B: one block per row m of A and K slice; threads stride over k
// (A read coalesced), then a warp-shuffle and shared-memory reduction of the NN sums.
template <int NN, bool F32>
__global__ void __launch_bounds__(SK_THREADS) k_skinny_n(long long M, int N, long long K, long long kslice,
                                                         const double* __restrict__ A, long long lda,
                                                         const double* __restrict__ B, long long ldb,
                                                         double* __restrict__ P) {
    __shared__ double red[SK_THREADS / 32][NN];
    const long long m = blockIdx.x;
    const long long k0 = blockIdx.y * kslice, k1 = min(K, k0 + kslice);
    double acc[NN];
#pragma unroll
    for (int j = 0; j < NN; ++j) acc[j] = 0.0;
    const double* a = A + m * lda;
    if (F32) {
        // each thread takes up to SK_CHUNK of its strided terms per FP32 partial sum
        for (long long kb = k0; kb < k1; kb += (long long)SK_THREADS * SK_CHUNK) {
            float part[NN];
#pragma unroll
            for (int j = 0; j < NN; ++j) part[j] = 0.f;
            const long long ke = min(k1, kb + (long long)SK_THREADS * SK_CHUNK);
            constexpr int U = 4;
            for (long long k = kb + threadIdx.x; k < ke; k += (long long)U * SK_THREADS) {
                double av[U];
#pragma unroll
                for (int u = 0; u < U; ++u) av[u] = k + u * SK_THREADS < ke ? a[k + u * SK_THREADS] : 0.0;
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const long long ku = k + u * SK_THREADS;
                    if (ku < ke)
#pragma unroll
                        for (int j = 0; j < NN; ++j)
                            if (j < N) part[j] = fmaf((float)av[u], (float)B[ku * ldb + j], part[j]);
                }
            }
#pragma unroll
            for (int j = 0; j < NN; ++j) acc[j] += (double)part[j];
        }
    } else {
        constexpr int U = 4;
        for (long long k = k0 + threadIdx.x; k < k1; k += (long long)U * SK_THREADS) {
            double av[U];
#pragma unroll
            for (int u = 0; u < U; ++u) av[u] = k + u * SK_THREADS < k1 ? a[k + u * SK_THREADS] : 0.0;
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const long long ku = k + u * SK_THREADS;
                if (ku < k1)
#pragma unroll
                    for (int j = 0; j < NN; ++j)
                        if (j < N) acc[j] = fma(av[u], B[ku * ldb + j], acc[j]);
            }
        }
    }
#pragma unroll
    for (int j = 0; j < NN; ++j) {
        double x = acc[j];
        for (int off = 16; off > 0; off >>= 1) x += __shfl_down_sync(0xffffffffu, x, off);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5][j] = x;
    }
    __syncthreads();
    if (threadIdx.x < N) {
        double x = 0.0;
        for (int w = 0; w < SK_THREADS / 32; ++w) x += red[w][threadIdx.x];
        P[((long long)blockIdx.y * M + m) * N + threadIdx.x] = x;
    }
}

// General small contraction in FP64: 64 x 64 output tiles, 16-deep K steps through
// shared memory, 4 x 4 outputs per thread.
__global__ void __launch_bounds__(256) k_tile_f64(long long M, long long N, long long K, const double* __restrict__ A,
                                                  long long lda, const double* __restrict__ B, long long ldb,
                                                  double* __restrict__ P) {
    __shared__ double As[16][64 + 1];
    __shared__ double Bs[16][64];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const long long m0 = blockIdx.y * 64LL, n0 = blockIdx.x * 64LL;
    double acc[4][4] = {};
    for (long long k0 = 0; k0 < K; k0 += 16) {
        for (int e = threadIdx.x; e < 64 * 16; e += 256) {
            const int r = e / 16, kk = e % 16;
            const long long gm = m0 + r, gk = k0 + kk;
            As[kk][r] = (gm < M && gk < K) ? A[gm * lda + gk] : 0.0;
            const int kb = e / 64, cn = e % 64;
            const long long gn = n0 + cn, gk2 = k0 + kb;
            Bs[kb][cn] = (gn < N && gk2 < K) ? B[gk2 * ldb + gn] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            double av[4], bv[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) av[i] = As[kk][ty * 4 + i];
#pragma unroll
            for (int j = 0; j < 4; ++j) bv[j] = Bs[kk][tx * 4 + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const long long gm = m0 + ty * 4 + i, gn = n0 + tx * 4 + j;
            if (gm < M && gn < N) P[gm * N + gn] = acc[i][j];
        }
}

// As k_reduce_slices for many slices: one warp per output element, lanes over slices,
// then a shuffle reduction.
__global__ void k_reduce_slices_warp(int S, long long M, long long N, const double* __restrict__ P, double alpha,
                                     double beta, double* __restrict__ C, long long ldc) {
    const long long total = M * N;
    const int lane = threadIdx.x & 31;
    const long long warps = (long long)gridDim.x * blockDim.x / 32;
    for (long long x = (blockIdx.x * (long long)blockDim.x + threadIdx.x) / 32; x < total; x += warps) {
        double a = 0.0;
        for (int s2 = lane; s2 < S; s2 += 32) a += P[s2 * total + x];
        for (int off = 16; off > 0; off >>= 1) a += __shfl_down_sync(0xffffffffu, a, off);
        if (lane == 0) {
            const long long m = x / N, n = x - m * N;
            double* cp = C + m * ldc + n;
            *cp = beta == 0.0 ? alpha * a : alpha * a + beta * *cp;
        }
    }
}

// C[m * ldc + n] = alpha sum_s P[s][m][n] + beta C[m * ldc + n]
__global__ void k_reduce_slices(int S, long long M, long long N, const double* __restrict__ P, double alpha, double beta,
                                double* __restrict__ C, long long ldc) {
    const long long total = M * N;
    for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < total; x += (long long)gridDim.x * blockDim.x) {
        double a = 0.0;
        for (int s2 = 0; s2 < S; ++s2) a += P[s2 * total + x];
        const long long m = x / N, n = x - m * N;
        double* cp = C + m * ldc + n;
        *cp = beta == 0.0 ? alpha * a : alpha * a + beta * *cp;
    }
}

template <int MM, bool F32>
void launch_skinny_m(dim3 g, cudaStream_t st, int M, long long N, long long K, long long ks, const double* A, long long lda,
                     const double* B, long long ldb, double* P) {
    k_skinny_m<MM, F32><<<g, SK_THREADS, 0, st>>>(M, N, K, ks, A, lda, B, ldb, P);
}
template <int NN, bool F32>
void launch_skinny_n(dim3 g, cudaStream_t st, long long M, int N, long long K, long long ks, const double* A, long long lda,
                     const double* B, long long ldb, double* P) {
    k_skinny_n<NN, F32><<<g, SK_THREADS, 0, st>>>(M, N, K, ks, A, lda, B, ldb, P);
}

}  // namespace

void own_gemm(Ctx& c, long long M, long long N, long long K, double alpha, const double* A, long long lda, const double* B,
              long long ldb, double beta, double* C, long long ldc, bool f32) {
    if (M <= 0 || N <= 0) return;
    if (K <= 0) {
        for (long long m = 0; m < M; ++m) {
            if (beta == 0.0)
                fill(c, N, 0.0, C + m * ldc);
            else if (beta != 1.0)
                axpby(c, N, 0.0, C + m * ldc, beta, C + m * ldc);
        }
        return;
    }
    const long long target = 152LL * 8;  // blocks that fill the GPU several times over
    Arena::Mark mk = c.arena.mark();
    int S = 1;
    double* P = nullptr;
    if (M <= 8) {
        const long long nbn = (N + SK_THREADS - 1) / SK_THREADS;
        const long long kch = (K + SK_THREADS - 1) / SK_THREADS;
        S = (int)std::max<long long>(1, std::min<long long>({kch, (target + nbn - 1) / nbn, 512}));
        const long long ks = (kch + S - 1) / S * SK_THREADS;
        S = (int)((K + ks - 1) / ks);
        P = c.arena.dalloc((size_t)S * M * N);
        dim3 g((unsigned)nbn, (unsigned)S);
        auto go = [&](auto f) { f(g, c.stream, (int)M, N, K, ks, A, lda, B, ldb, P); };
        switch ((int)M) {
#define SKM(X)                                                              \
    case X:                                                                 \
        if (f32) go(launch_skinny_m<X, true>); else go(launch_skinny_m<X, false>); \
        break;
            SKM(1) SKM(2) SKM(3) SKM(4) SKM(5) SKM(6) SKM(7) SKM(8)
#undef SKM
        }
    } else if (N <= 8) {
        const long long kch = (K + SK_THREADS - 1) / SK_THREADS;
        S = (int)std::max<long long>(1, std::min<long long>({kch, (target + M - 1) / M, 512}));
        const long long ks = (kch + S - 1) / S * SK_THREADS;
        S = (int)((K + ks - 1) / ks);
        if (M > 0x7fffffffLL) throw Error(-1, "own_gemm: too many rows");
        P = c.arena.dalloc((size_t)S * M * N);
        dim3 g((unsigned)M, (unsigned)S);
        auto go = [&](auto f) { f(g, c.stream, M, (int)N, K, ks, A, lda, B, ldb, P); };
        switch ((int)N) {
#define SKN(X)                                                              \
    case X:                                                                 \
        if (f32) go(launch_skinny_n<X, true>); else go(launch_skinny_n<X, false>); \
        break;
            SKN(1) SKN(2) SKN(3) SKN(4) SKN(5) SKN(6) SKN(7) SKN(8)
#undef SKN
        }
    } else {
        if ((M + 63) / 64 > 65535) throw Error(-1, "own_gemm: too many row tiles");
        P = c.arena.dalloc((size_t)M * N);
        dim3 g((unsigned)((N + 63) / 64), (unsigned)((M + 63) / 64));
        k_tile_f64<<<g, 256, 0, c.stream>>>(M, N, K, A, lda, B, ldb, P);
    }
    ++c.kernels;
    ADC_CUDA(cudaGetLastError());
    if (S >= 16)
        k_reduce_slices_warp<<<grid_for(32 * M * N), 256, 0, c.stream>>>(S, M, N, P, alpha, beta, C, ldc);
    else
        k_reduce_slices<<<grid_for(M * N), 256, 0, c.stream>>>(S, M, N, P, alpha, beta, C, ldc);
    ++c.kernels;
    ADC_CUDA(cudaGetLastError());
    c.arena.release(mk);
}

// The tiled form applies when, after dropping unit axes, the output's innermost axis is
// strided in the input and both it and the input-contiguous axis are at least 8 long.
static bool tiled_args(const PermArgs& p, TileArgs& t) {
    long long d[kMaxDim], si[kMaxDim];
    int nd = 0;
    for (int j = 0; j < p.nd; ++j)
        if (p.dout[j] > 1) {
            d[nd] = p.dout[j];
            si[nd] = p.sin[j];
            ++nd;
        }
    if (nd < 2 || si[nd - 1] == 1) return false;
    int jy = -1;
    for (int j = 0; j < nd - 1; ++j)
        if (si[j] == 1) jy = j;
    if (jy < 0 || d[jy] < 8 || d[nd - 1] < 8) return false;
    long long so[kMaxDim], acc = 1;
    for (int j = nd - 1; j >= 0; --j) {
        so[j] = acc;
        acc *= d[j];
    }
    t.nrest = 0;
    long long rest = 1;
    for (int j = 0; j < nd - 1; ++j) {
        if (j == jy) continue;
        t.rdim[t.nrest] = d[j];
        t.rsin[t.nrest] = si[j];
        t.rsout[t.nrest] = so[j];
        ++t.nrest;
        rest *= d[j];
    }
    t.nx = d[nd - 1];
    t.sx_in = si[nd - 1];
    t.ny = d[jy];
    t.sy_out = so[jy];
    t.ntx = (t.nx + 31) / 32;
    t.nty = (t.ny + 31) / 32;
    t.nblocks = t.ntx * t.nty * rest;
    return true;
}

template <typename Tin, typename Op>
static void launch_tiled(Ctx& c, const Tin* in, const TileArgs& t, const Op& op) {
    const long long g = std::min<long long>(t.nblocks, 152LL * 16);
    k_permute_tiled<Tin, Op><<<(unsigned)g, dim3(32, 8), 0, c.stream>>>(in, t, op);
    ++c.kernels;
    ADC_CUDA(cudaGetLastError());
}

void permute(Ctx& c, const double* in, const Shape& s, const int* perm, double* out, double alpha, double beta) {
    PermArgs a;
    a.nd = s.nd;
    long long st[kMaxDim];
    long long acc = 1, total = 1;
    for (int j = s.nd - 1; j >= 0; --j) {
        st[j] = acc;
        acc *= s.d[j];
    }
    for (int j = 0; j < s.nd; ++j) {
        a.dout[j] = s.d[perm[j]];
        a.sin[j] = st[perm[j]];
        total *= a.dout[j];
    }
    if (total == 0) return;
    TileArgs t;
    if (tiled_args(a, t)) {
        launch_tiled(c, in, t, OpAxpby<double>{out, alpha, beta});
        return;
    }
    if (total <= 0xffffffffLL)  // every offset is below total
        permute_kernel<unsigned><<<grid_for(total), 256, 0, c.stream>>>(in, out, a, total, alpha, beta);
    else
        permute_kernel<long long><<<grid_for(total), 256, 0, c.stream>>>(in, out, a, total, alpha, beta);
    ++c.kernels;
    ADC_CUDA(cudaGetLastError());
}

static PermArgs perm_args(const Shape& s, const int* perm, long long& total) {
    PermArgs a;
    a.nd = s.nd;
    long long st[kMaxDim];
    long long acc = 1;
    total = 1;
    for (int j = s.nd - 1; j >= 0; --j) {
        st[j] = acc;
        acc *= s.d[j];
    }
    for (int j = 0; j < s.nd; ++j) {
        a.dout[j] = s.d[perm[j]];
        a.sin[j] = st[perm[j]];
        total *= a.dout[j];
    }
    return a;
}

template <typename Tin, typename Tout>
static void permute_cvt(Ctx& c, const Tin* in, const Shape& s, const int* perm, Tout* out, double alpha, double beta) {
    long long total;
    PermArgs a = perm_args(s, perm, total);
    if (total == 0) return;
    TileArgs t;
    if (tiled_args(a, t)) {
        launch_tiled(c, in, t, OpAxpby<Tout>{out, alpha, beta});
        return;
    }
    if (total <= 0xffffffffLL)
        permute_cvt_kernel<unsigned, Tin, Tout><<<grid_for(total), 256, 0, c.stream>>>(in, out, a, total, alpha, beta);
    else
        permute_cvt_kernel<long long, Tin, Tout><<<grid_for(total), 256, 0, c.stream>>>(in, out, a, total, alpha, beta);
    ++c.kernels;
    ADC_CUDA(cudaGetLastError());
}

template <typename Tin>
static void split_planes_t(Ctx& c, const Tin* in, const PermArgs& a, long long rows, long long K, long long Kp,
                           void* const* out) {
    TileArgs t;
    if (tiled_args(a, t)) {
        launch_tiled(c, in, t, OpPlanes{(__nv_bfloat16*)out[0], (__nv_bfloat16*)out[1], K, Kp});
        if (Kp > K) {
            k_zero_pad<<<grid_for(rows * (Kp - K)), 256, 0, c.stream>>>((__nv_bfloat16*)out[0], (__nv_bfloat16*)out[1],
                                                                         rows, K, Kp);
            ++c.kernels;
            ADC_CUDA(cudaGetLastError());
        }
        return;
    }
    // 32-bit coordinates when the output index fits (every input offset is below rows * K)
    if (rows * Kp <= 0xffffffffLL)
        permute_split_kernel<unsigned, Tin><<<grid_for(rows * Kp), 256, 0, c.stream>>>(
            in, (__nv_bfloat16*)out[0], (__nv_bfloat16*)out[1], a, rows, K, Kp);
    else
        permute_split_kernel<long long, Tin><<<grid_for(rows * Kp), 256, 0, c.stream>>>(
            in, (__nv_bfloat16*)out[0], (__nv_bfloat16*)out[1], a, rows, K, Kp);
    ++c.kernels;
    ADC_CUDA(cudaGetLastError());
}

void split_planes(Ctx& c, const double* in, const Shape& s, const int* perm, long long rows, long long K, long long Kp,
                  void* const* out, bool in32) {
    long long total;
    PermArgs a = perm_args(s, perm, total);
    if (total != rows * K) throw Error(-1, "split_planes: shape mismatch");
    if (rows * Kp == 0) return;
    if (in32)
        split_planes_t(c, (const float*)in, a, rows, K, Kp, out);
    else
        split_planes_t(c, in, a, rows, K, Kp, out);
}

void permute_any(Ctx& c, const void* in, bool in32, const Shape& s, const int* perm, void* out, bool out32,
                 double alpha, double beta) {
    if (!in32 && !out32)
        permute(c, (const double*)in, s, perm, (double*)out, alpha, beta);
    else if (in32 && out32)
        permute_cvt(c, (const float*)in, s, perm, (float*)out, alpha, beta);
    else if (in32)
        permute_cvt(c, (const float*)in, s, perm, (double*)out, alpha, beta);
    else
        permute_cvt(c, (const double*)in, s, perm, (float*)out, alpha, beta);
}

void axpby(Ctx& c, long long n, double alpha, const double* x, double beta, double* y) {
    if (n <= 0) return;
    axpby_kernel<<<grid_for(n), 256, 0, c.stream>>>(n, alpha, x, beta, y);
    ++c.kernels;
    ADC_CUDA(cudaGetLastError());
}

void sum_slices(Ctx& c, int S, long long n, const double* T, double* C) {
    if (n <= 0) return;
    sum_slices_kernel<<<grid_for(n), 256, 0, c.stream>>>(S, n, T, C);
    ++c.kernels;
    ADC_CUDA(cudaGetLastError());
}

void ensure_side_streams(Ctx& c, int count) {
    if (c.capturing && (!c.side_fork || (int)c.side.size() < count))
        throw Error(-3, "side stream creation during stream capture");
    if (!c.side_fork) ADC_CUDA(cudaEventCreateWithFlags(&c.side_fork, cudaEventDisableTiming));
    while ((int)c.side.size() < count) {
        cudaStream_t s = nullptr;
        cudaEvent_t e = nullptr;
        ADC_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
        ADC_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        c.side.push_back(s);
        c.side_join.push_back(e);
    }
}

void fill(Ctx& c, long long n, double v, double* y) {
    if (n <= 0) return;
    fill_kernel<<<grid_for(n), 256, 0, c.stream>>>(n, v, y);
    ++c.kernels;
    ADC_CUDA(cudaGetLastError());
}

void gemm(Ctx& c, bool ta, bool tb, long long M, long long N, long long K, double alpha, const double* A, long long lda,
          long long sA, const double* B, long long ldb, long long sB, double beta, double* C, long long ldc,
          long long sC, long long batch) {
    if (M <= 0 || N <= 0 || batch <= 0) return;
    if (K <= 0) {
        // C = beta C
        if (ldc == N && (batch == 1 || sC == M * N)) {
            if (beta == 0.0)
                fill(c, M * N * batch, 0.0, C);
            else if (beta != 1.0)
                axpby(c, M * N * batch, 0.0, C, beta, C);
            return;
        }
        throw Error(-1, "gemm: K == 0 with strided C");
    }
    // row-major C = op(A) op(B)  <=>  column-major C^T = op(B)^T op(A)^T
    cublasOperation_t oa = ta ? CUBLAS_OP_T : CUBLAS_OP_N;
    cublasOperation_t ob = tb ? CUBLAS_OP_T : CUBLAS_OP_N;
    if (batch == 1) {
        ADC_BLAS(cublasDgemm(c.blas, ob, oa, (int)N, (int)M, (int)K, &alpha, B, (int)ldb, A, (int)lda, &beta, C, (int)ldc));
    } else {
        ADC_BLAS(cublasDgemmStridedBatched(c.blas, ob, oa, (int)N, (int)M, (int)K, &alpha, B, (int)ldb, sB, A, (int)lda,
                                           sA, &beta, C, (int)ldc, sC, (int)batch));
    }
}

namespace {

struct Spec {
    std::string a, b, c;
};

Spec parse(const char* spec) {
    std::string s(spec);
    size_t comma = s.find(','), arrow = s.find("->");
    if (comma == std::string::npos || arrow == std::string::npos || comma > arrow)
        throw Error(-1, std::string("einsum: bad spec ") + spec);
    return {s.substr(0, comma), s.substr(comma + 1, arrow - comma - 1), s.substr(arrow + 2)};
}

bool has(const std::string& s, char x) { return s.find(x) != std::string::npos; }

// permute src (letters ls, dims) into the letter order lt; returns pointer (src if identity)
// (an FP32 operand is always converted into an FP64 copy)
const double* to_order(Ctx& c, const double* src, const std::string& ls, const std::map<char, long long>& dim,
                       const std::string& lt, bool f32 = false) {
    if (ls == lt && !f32) return src;
    Shape sh;
    sh.nd = (int)ls.size();
    long long n = 1;
    for (int j = 0; j < sh.nd; ++j) {
        sh.d[j] = dim.at(ls[j]);
        n *= sh.d[j];
    }
    int perm[kMaxDim];
    for (int j = 0; j < sh.nd; ++j) perm[j] = (int)ls.find(lt[j]);
    double* dst = c.arena.dalloc(n);
    permute_any(c, src, f32, sh, perm, dst, false, 1.0, 0.0);
    return dst;
}

}  // namespace

// FP32-accurate contraction: operands permuted and rounded to FP32, GEMM with
// BF16x9 emulation (falls back to plain FP32 if the library lacks it), result
// permuted and accumulated into the FP64 output.
static void einsum_fp32(Ctx& c, const std::string& la, const std::string& lb, const std::string& lc,
                        std::map<char, long long>& dim, const std::string& batch, const std::string& fa,
                        const std::string& fb, const std::string& con, double alpha, const T& A, const T& B,
                        double beta, void* C, bool c32) {
    auto prod = [&](const std::string& l) {
        long long p = 1;
        for (char x : l) p *= dim[x];
        return p;
    };
    long long nb = prod(batch), M = prod(fa), N = prod(fb), K = prod(con);
    auto conv = [&](const T& X, const std::string& ls, const std::string& lt) {
        // an FP32 operand already in GEMM order is used in place
        if (X.f32 && ls == lt) return (const float*)X.p;
        Shape sh;
        sh.nd = (int)ls.size();
        long long n = 1;
        for (int j = 0; j < sh.nd; ++j) {
            sh.d[j] = dim.at(ls[j]);
            n *= sh.d[j];
        }
        int perm[kMaxDim];
        std::string key;
        for (int j = 0; j < sh.nd; ++j) {
            perm[j] = (int)ls.find(lt[j]);
            key += (char)('0' + perm[j]);
            key += ':';
            key += std::to_string(sh.d[j]);
            key += ',';
        }
        float* dst;
        if (X.constant && (size_t)n * sizeof(float) <= c.cache_max_bytes) {
            auto it = c.f32cache.find({X.p, key});
            if (it != c.f32cache.end()) return (const float*)it->second;
            if (c.capturing) throw Error(-3, "operand cache miss during stream capture");
            dst = (float*)dev_alloc(n * sizeof(float), c.stream);
            c.f32cache[{X.p, key}] = dst;
        } else {
            dst = (float*)c.arena.alloc(n * sizeof(float));
        }
        permute_any(c, X.p, X.f32, sh, perm, dst, true, 1.0, 0.0);
        return (const float*)dst;
    };
    const float* A32 = conv(A, la, batch + fa + con);
    const float* B32 = conv(B, lb, batch + con + fb);
    const std::string tord = batch + fa + fb;
    // an FP32 output in the GEMM's order is written by the GEMM itself (C = alpha AB + beta C)
    const bool direct = c32 && tord == lc;
    float* T32 = direct ? (float*)C : (float*)c.arena.alloc(nb * M * N * sizeof(float));
    const float one = direct ? (float)alpha : 1.0f, zero = direct ? (float)beta : 0.0f;
    // row-major T[M][N] = A[M][K] B[K][N]  <=>  column-major T^T = B^T A^T
    auto run = [&](cublasComputeType_t ct) {
        return cublasGemmStridedBatchedEx(c.blas, CUBLAS_OP_N, CUBLAS_OP_N, (int)N, (int)M, (int)K, &one, B32, CUDA_R_32F,
                                          (int)N, K * N, A32, CUDA_R_32F, (int)K, M * K, &zero, T32, CUDA_R_32F, (int)N,
                                          M * N, (int)nb, ct, CUBLAS_GEMM_DEFAULT);
    };
    if (c.emulation_ok != 0) {
        cublasStatus_t st = run(CUBLAS_COMPUTE_32F_EMULATED_16BFX9);
        if (st == CUBLAS_STATUS_SUCCESS) {
            c.emulation_ok = 1;
        } else if (c.emulation_ok == -1 && (st == CUBLAS_STATUS_NOT_SUPPORTED || st == CUBLAS_STATUS_INVALID_VALUE)) {
            c.emulation_ok = 0;
            ADC_BLAS(run(CUBLAS_COMPUTE_32F));
        } else {
            ADC_BLAS(st);
        }
    } else {
        ADC_BLAS(run(CUBLAS_COMPUTE_32F));
    }
    if (direct) return;
    Shape sh;
    sh.nd = (int)tord.size();
    for (int j = 0; j < sh.nd; ++j) sh.d[j] = dim[tord[j]];
    int perm[kMaxDim];
    for (int j = 0; j < sh.nd; ++j) perm[j] = (int)tord.find(lc[j]);
    permute_any(c, T32, true, sh, perm, C, c32, alpha, beta);
}

// Tensor-core contraction (gemm_mode 2): operands permuted into K-major GEMM
// order and split into two BF16 planes (constant operands once, cached), the
// tcgen05 split-BF16 GEMM into an FP64 temporary, then permuted and
// accumulated into the output.
static void einsum_tc(Ctx& c, const std::string& la, const std::string& lb, const std::string& lc,
                      std::map<char, long long>& dim, const std::string& fa, const std::string& fb, const std::string& con,
                      double alpha, const T& A, const T& B, double beta, void* C, bool c32) {
    auto prod = [&](const std::string& l) {
        long long p = 1;
        for (char x : l) p *= dim[x];
        return p;
    };
    const long long M = prod(fa), N = prod(fb), K = prod(con), Kp = (K + 7) / 8 * 8;
    auto planes_of = [&](const T& X, const std::string& ls, const std::string& lt, long long rows) {
        Shape sh;
        sh.nd = (int)ls.size();
        for (int j = 0; j < sh.nd; ++j) sh.d[j] = dim.at(ls[j]);
        int perm[kMaxDim];
        std::string key = "bf16x2:";
        for (int j = 0; j < sh.nd; ++j) {
            perm[j] = (int)ls.find(lt[j]);
            key += (char)('0' + perm[j]);
            key += ':';
            key += std::to_string(sh.d[j]);
            key += ',';
        }
        key += std::to_string(K);
        void* base = nullptr;
        if (X.constant && (size_t)(2 * rows * Kp * 2) <= c.cache_max_bytes) {
            auto it = c.bf16cache.find({X.p, key});
            if (it != c.bf16cache.end()) return it->second;
            if (c.capturing) throw Error(-3, "operand cache miss during stream capture");
            base = dev_alloc(2 * rows * Kp * 2, c.stream);
            c.bf16cache[{X.p, key}] = base;
        } else {
            base = c.arena.alloc(2 * rows * Kp * 2);
        }
        void* out[2] = {base, (char*)base + rows * Kp * 2};
        split_planes(c, X.p, sh, perm, rows, K, Kp, out, X.f32);
        return base;
    };
    void* pa = planes_of(A, la, fa + con, M);
    void* pb = planes_of(B, lb, fb + con, N);
    if (!c.d_err) {
        if (c.capturing) throw Error(-3, "error flag allocation during stream capture");
        c.d_err = (int*)dev_alloc(sizeof(int), c.stream);
        ADC_CUDA(cudaMemsetAsync(c.d_err, 0, sizeof(int), c.stream));
    }
    double* T = c.arena.dalloc((size_t)(M * N));
    const void* A2[2] = {pa, (const char*)pa + M * Kp * 2};
    const void* B2[2] = {pb, (const char*)pb + N * Kp * 2};
    tc_gemm(c, A2, B2, M, N, Kp, 2.0 * M * N * K, T);
    std::string tord = fa + fb;
    Shape sh;
    sh.nd = (int)tord.size();
    for (int j = 0; j < sh.nd; ++j) sh.d[j] = dim[tord[j]];
    int perm[kMaxDim];
    for (int j = 0; j < sh.nd; ++j) perm[j] = (int)tord.find(lc[j]);
    permute_any(c, T, false, sh, perm, C, c32, alpha, beta);
}

static void einsum_core(Ctx& c, const char* specstr, double alpha, const T& A, const T& B, double beta, void* C, bool c32,
                        const std::vector<long long>& cdims) {
    Spec sp = parse(specstr);
    if (sp.a.size() != A.dims.size() || sp.b.size() != B.dims.size() || sp.c.size() != cdims.size())
        throw Error(-1, std::string("einsum: rank mismatch in ") + specstr);
    std::map<char, long long> dim;
    auto put = [&](const std::string& l, const std::vector<long long>& d) {
        for (size_t j = 0; j < l.size(); ++j) {
            auto it = dim.find(l[j]);
            if (it != dim.end() && it->second != d[j])
                throw Error(-1, std::string("einsum: dimension mismatch in ") + specstr);
            dim[l[j]] = d[j];
        }
    };
    put(sp.a, A.dims);
    put(sp.b, B.dims);
    put(sp.c, cdims);
    std::string batch, fa, fb, con;
    for (char x : sp.c) {
        bool ia = has(sp.a, x), ib = has(sp.b, x);
        if (ia && ib)
            batch += x;
        else if (ia)
            fa += x;
        else if (ib)
            fb += x;
        else
            throw Error(-1, std::string("einsum: output index not in inputs: ") + specstr);
    }
    for (char x : sp.a) {
        if (has(sp.c, x)) continue;
        if (!has(sp.b, x)) throw Error(-1, std::string("einsum: summed index in one operand only: ") + specstr);
        con += x;
    }
    for (char x : sp.b)
        if (!has(sp.c, x) && !has(sp.a, x)) throw Error(-1, std::string("einsum: summed index in one operand only: ") + specstr);
    auto prod = [&](const std::string& l) {
        long long p = 1;
        for (char x : l) p *= dim[x];
        return p;
    };
    long long nb = prod(batch), M = prod(fa), N = prod(fb), K = prod(con);
    Arena::Mark mk = c.arena.mark();
    if (c.gemm_mode == 2 && nb == 1) {
        // the mixed sigma: tensor cores for the large contractions, own kernels for the rest
        const bool big = 2.0 * M * N * K >= c.fp32_min_flops;
        // few-vector shapes: the own bandwidth kernels read the large operand once, in place when
        // it is an FP64 tensor already in their order ([K][N] for M <= 8, [M][K] for N <= 8);
        // otherwise the tensor cores take them when the large operand is a constant of the
        // handle (its split planes are cached once, the permuted FP64 copy would be made per call)
        const bool skinny = std::min(M, N) <= 8;
        const bool big_const = M <= N ? B.constant : A.constant;
        const bool big_in_place = M <= N ? (!B.f32 && sp.b == con + fb) : (!A.f32 && sp.a == fa + con);
        if (big && tc_gemm_fits(M, N, K) && (!skinny || (big_const && !big_in_place))) {
            einsum_tc(c, sp.a, sp.b, sp.c, dim, fa, fb, con, alpha, A, B, beta, C, c32);
        } else {
            const double* Ap = to_order(c, A.p, sp.a, dim, fa + con, A.f32);
            const double* Bp = to_order(c, B.p, sp.b, dim, con + fb, B.f32);
            const std::string tord = fa + fb;
            if (tord == sp.c && !c32) {
                own_gemm(c, M, N, K, alpha, Ap, K, Bp, N, beta, (double*)C, N, big);
            } else {
                double* Tm = c.arena.dalloc((size_t)(M * N));
                own_gemm(c, M, N, K, 1.0, Ap, K, Bp, N, 0.0, Tm, N, big);
                Shape sh;
                sh.nd = (int)tord.size();
                for (int j = 0; j < sh.nd; ++j) sh.d[j] = dim[tord[j]];
                int perm[kMaxDim];
                for (int j = 0; j < sh.nd; ++j) perm[j] = (int)tord.find(sp.c[j]);
                permute_any(c, Tm, false, sh, perm, C, c32, alpha, beta);
            }
        }
        c.arena.release(mk);
        return;
    }
    if (c.gemm_mode >= 1 && 2.0 * nb * M * N * K >= c.fp32_min_flops) {
        einsum_fp32(c, sp.a, sp.b, sp.c, dim, batch, fa, fb, con, alpha, A, B, beta, C, c32);
        c.arena.release(mk);
        return;
    }
    const double* Ap = to_order(c, A.p, sp.a, dim, batch + fa + con, A.f32);
    const double* Bp = to_order(c, B.p, sp.b, dim, batch + con + fb, B.f32);
    std::string tord = batch + fa + fb;
    if (tord == sp.c && !c32) {
        gemm(c, false, false, M, N, K, alpha, Ap, K, M * K, Bp, N, K * N, beta, (double*)C, N, M * N, nb);
    } else {
        double* Tm = c.arena.dalloc((size_t)(nb * M * N));
        gemm(c, false, false, M, N, K, 1.0, Ap, K, M * K, Bp, N, K * N, 0.0, Tm, N, M * N, nb);
        Shape sh;
        sh.nd = (int)tord.size();
        for (int j = 0; j < sh.nd; ++j) sh.d[j] = dim[tord[j]];
        int perm[kMaxDim];
        for (int j = 0; j < sh.nd; ++j) perm[j] = (int)tord.find(sp.c[j]);
        permute_any(c, Tm, false, sh, perm, C, c32, alpha, beta);
    }
    c.arena.release(mk);
}

void einsum(Ctx& c, const char* spec, double alpha, const T& A, const T& B, double beta, double* C,
            const std::vector<long long>& cdims) {
    einsum_core(c, spec, alpha, A, B, beta, C, false, cdims);
}

void einsum(Ctx& c, const char* spec, double alpha, const T& A, const T& B, double beta, float* C,
            const std::vector<long long>& cdims) {
    einsum_core(c, spec, alpha, A, B, beta, C, true, cdims);
}

}  // namespace adc

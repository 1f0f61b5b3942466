// Density-fitted ladder sum_cd (ac|bd) X_n[c,d] = sum_Q (B^Q X_n B^Q)_ab on
// the 5th-generation tensor cores of sm_103a (tcgen05.mma, operands staged in
// shared memory by TMA, FP32 accumulators in tensor memory).
//
// Per auxiliary chunk q in [q0, q0+qn) two K-major GEMMs run back to back:
//   GEMM1  Z[(q,a),(n,d)] = sum_c B^q[a,c] X_n[c,d]        (A = Bs, B = X^T)
//   GEMM2  out[(n,a),b]  += sum_(q,d) Z_n[a,(q,d)] B^q[d,b] (A = Z,  B = Bp)
// (B^q symmetric).  Every operand x is split as x = hi + lo with hi, lo in
// BF16; each product uses hi*hi + hi*lo + lo*hi.  GEMM1 writes Z already split
// and laid out as GEMM2's K-major A operand; GEMM2 accumulates in FP32 over
// one chunk and adds into the FP64 output, so FP64 carries the sum over chunks.
//
// Index padding: the virtual index on every K axis is padded to vp (multiple
// of 32) with zeros so that TMA row strides and coordinates are 16-byte
// aligned and 16-column epilogue chunks never straddle a matrix.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdint>
#include <mutex>

#include "ladder_tc.cuh"

namespace adc {

namespace {

constexpr int BM = 128;
constexpr int BK = 64;  // 64 BF16 = 128 bytes = one 128B-swizzle row
constexpr int MAX_STAGES = 4;
constexpr int THREADS = 192;  // warp 0: TMA, warp 1: MMA + TMEM owner, warps 2-5: epilogue
constexpr int TMEM_COLS = 512;  // two accumulators of up to 256 FP32 columns
constexpr int MAX_BN = 256;
constexpr int A_BYTES = BM * BK * 2;
// Always request (nearly) all of shared memory so that exactly one CTA, and one
// 512-column TMEM allocation, lives on each SM.
constexpr size_t SMEM_BYTES = 226 * 1024;
constexpr unsigned long long WAIT_NS = 2000000000ull;  // bounded waits: 2 s

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ uint64_t gtime() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t n) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(n) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* b, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\n"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(su32(b)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait: false on timeout (raises the CTA abort flag and the global
// error flag) or when another role of the CTA has already aborted.
__device__ bool mbar_wait(uint64_t* b, uint32_t parity, volatile int* abort_flag, int* err) {
    if (mbar_try(b, parity)) return true;
    const uint64_t t0 = gtime();
    while (true) {
        if (mbar_try(b, parity)) return true;
        if (*abort_flag) return false;
        if (gtime() - t0 > WAIT_NS) {
            *abort_flag = 1;
            atomicExch(err, 1);
            return false;
        }
    }
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* m, uint64_t* bar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
            su32(dst)),
        "l"((uint64_t)m), "r"(su32(bar)), "r"(x), "r"(y)
        : "memory");
}
// tcgen05 shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row
// core groups 1024 bytes apart.
__device__ __forceinline__ uint64_t smem_desc(const void* p) {
    uint64_t d = 0;
    d |= (uint64_t)((su32(p) >> 4) & 0x3FFF);
    d |= (uint64_t)1 << 16;             // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;   // stride byte offset
    d |= (uint64_t)1 << 46;             // descriptor version
    d |= (uint64_t)2 << 61;             // 128-byte swizzle
    return d;
}
__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar)) : "memory");
}
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

struct Epi {
    int mode;  // 0: split store of Z (GEMM1), 1: FP64 accumulate (GEMM2)
    int M, N;
    // mode 0: row r = (q, a), col j = (n, dp); Z[((n*v + a)*qn + q)*vp + dp]
    __nv_bfloat16 *zhi, *zlo;
    int v, vp, qn;
    // mode 1: out[r*ldc + j] += acc
    double* out;
    long long ldc;
    int* err;
};

__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(b)) : "memory");
}

// Persistent GEMM C = A B^T with split-BF16 operands (three products per K step)
// and a double-buffered TMEM accumulator.  Roles: warp 0 lane 0 issues TMA
// loads through a ring of `stages` shared-memory stages, running ahead across
// tiles; warp 1 owns TMEM and its lane 0 issues the MMAs; warps 2-5 drain the
// accumulator of tile j while the MMAs of tile j+1 run into the other buffer.
__global__ void __launch_bounds__(THREADS, 1)
    k_gemm_bf16x3(const __grid_constant__ CUtensorMap mAh, const __grid_constant__ CUtensorMap mAl,
                  const __grid_constant__ CUtensorMap mBh, const __grid_constant__ CUtensorMap mBl, int a_row0, int b_x0,
                  int K, int BN, int stages, int m_fastest, int mt, int nt, Epi ep) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    __shared__ uint64_t full_bar[MAX_STAGES], empty_bar[MAX_STAGES], tfull[2], tempty[2], done_bar;
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int num_k = (K + BK - 1) / BK;
    const int B_BYTES = BN * BK * 2;
    const int STAGE = 2 * A_BYTES + 2 * B_BYTES;
    const int ntiles = mt * nt;

    if (threadIdx.x == 0) {
        for (int s = 0; s < stages; ++s) {
            mbar_init(&full_bar[s], 1);
            mbar_init(&empty_bar[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], 4);  // one arrival per epilogue warp
        }
        mbar_init(&done_bar, 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tmem_slot)), "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            long long g = 0;
            for (int t = blockIdx.x; t < ntiles && !abort_flag; t += gridDim.x) {
                const int m_tile = m_fastest ? t % mt : t / nt;
                const int n_tile = m_fastest ? t / mt : t % nt;
                for (int kb = 0; kb < num_k; ++kb, ++g) {
                    const int s = (int)(g % stages);
                    const uint32_t ph = (uint32_t)((g / stages) & 1);
                    if (g >= stages && !mbar_wait(&empty_bar[s], ph ^ 1, &abort_flag, ep.err)) break;
                    uint8_t* st = smem + (size_t)s * STAGE;
                    mbar_expect_tx(&full_bar[s], STAGE);
                    const int kx = kb * BK;
                    tma_load_2d(st, &mAh, &full_bar[s], kx, a_row0 + m_tile * BM);
                    tma_load_2d(st + A_BYTES, &mAl, &full_bar[s], kx, a_row0 + m_tile * BM);
                    tma_load_2d(st + 2 * A_BYTES, &mBh, &full_bar[s], b_x0 + kx, n_tile * BN);
                    tma_load_2d(st + 2 * A_BYTES + B_BYTES, &mBl, &full_bar[s], b_x0 + kx, n_tile * BN);
                }
            }
            if (abort_flag) {
                // let the copies of the last `stages` issues land before the CTA retires (bounded)
                for (long long q = (g > stages ? g - stages : 0); q < g; ++q) {
                    const uint64_t t0 = gtime();
                    while (!mbar_try(&full_bar[q % stages], (uint32_t)((q / stages) & 1)) && gtime() - t0 < WAIT_NS) {
                    }
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
            long long g = 0;
            int j = 0;
            for (int t = blockIdx.x; t < ntiles && !abort_flag; t += gridDim.x, ++j) {
                const int b = j & 1;
                if (j >= 2 && !mbar_wait(&tempty[b], (uint32_t)(((j >> 1) & 1) ^ 1), &abort_flag, ep.err)) break;
                fence_after();
                const uint32_t tacc = tmem + (uint32_t)(b * 256);
                bool ok = true;
                for (int kb = 0; kb < num_k; ++kb, ++g) {
                    const int s = (int)(g % stages);
                    if (!mbar_wait(&full_bar[s], (uint32_t)((g / stages) & 1), &abort_flag, ep.err)) {
                        ok = false;
                        break;
                    }
                    fence_after();
                    uint8_t* st = smem + (size_t)s * STAGE;
                    const uint64_t ah = smem_desc(st), al = smem_desc(st + A_BYTES);
                    const uint64_t bh = smem_desc(st + 2 * A_BYTES), bl = smem_desc(st + 2 * A_BYTES + B_BYTES);
#pragma unroll
                    for (int kk = 0; kk < BK / 16; ++kk) {
                        const uint64_t o = (uint64_t)(kk * 2);  // 16 BF16 = 32 bytes along K
                        mma_bf16(tacc, ah + o, bh + o, idesc, (kb | kk) != 0);
                        mma_bf16(tacc, ah + o, bl + o, idesc, 1u);
                        mma_bf16(tacc, al + o, bh + o, idesc, 1u);
                    }
                    mma_commit(&empty_bar[s]);
                }
                if (!ok) break;
                mma_commit(&tfull[b]);
            }
            mma_commit(&done_bar);  // fires when every MMA issued above has completed
        }
    } else {
        // epilogue: warp w reads TMEM lanes 32*(w%4) .. +31 (one accumulator row per thread)
        const int quarter = warp & 3;
        int j = 0;
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++j) {
            const int b = j & 1;
            if (!mbar_wait(&tfull[b], (uint32_t)((j >> 1) & 1), &abort_flag, ep.err)) break;
            fence_after();
            const int m_tile = m_fastest ? t % mt : t / nt;
            const int n_tile = m_fastest ? t / mt : t % nt;
            const int row = m_tile * BM + quarter * 32 + lane;
            const uint32_t tbase = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(b * 256);
            for (int c0 = 0; c0 < BN; c0 += 16) {
                float v[16];
                tmem_ld16(tbase + (uint32_t)c0, v);
                const int col0 = n_tile * BN + c0;
                if (row >= ep.M || col0 >= ep.N) continue;
                if (ep.mode == 0) {
                    const int q = row / ep.v, a = row - q * ep.v;
                    const int n = col0 / ep.vp, dp = col0 - n * ep.vp;
                    const long long z = (((long long)n * ep.v + a) * ep.qn + q) * ep.vp + dp;
                    __align__(16) __nv_bfloat16 hi[16], lo[16];
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        hi[i] = __float2bfloat16_rn(v[i]);
                        lo[i] = __float2bfloat16_rn(v[i] - __bfloat162float(hi[i]));
                    }
                    uint4* dh = (uint4*)(ep.zhi + z);
                    uint4* dl = (uint4*)(ep.zlo + z);
                    dh[0] = ((uint4*)hi)[0];
                    dh[1] = ((uint4*)hi)[1];
                    dl[0] = ((uint4*)lo)[0];
                    dl[1] = ((uint4*)lo)[1];
                } else {
                    double* o = ep.out + (long long)row * ep.ldc + col0;
#pragma unroll
                    for (int i = 0; i < 16; ++i)
                        if (col0 + i < ep.N) o[i] += (double)v[i];
                }
            }
            fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty[b]);
        }
    }
    fence_before();
    __syncthreads();
    if (warp == 1) {
        const uint64_t t0 = gtime();
        while (!mbar_try(&done_bar, 0) && gtime() - t0 < WAIT_NS) {
        }
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    }
}

// ---- operand preparation (FP64 -> split BF16) --------------------------------
__device__ __forceinline__ void split2(double x, __nv_bfloat16& h, __nv_bfloat16& l) {
    h = __double2bfloat16(x);
    l = __double2bfloat16(x - (double)__bfloat162float(h));
}
#define GRID_STRIDE(i, n) for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (n); i += (long long)gridDim.x * blockDim.x)

// Bs[(Q,a)][cp] = B^Q[a][c] (c < v), zero pad
__global__ void k_split_Bs(const double* __restrict__ B, int naux, int v, int vp, __nv_bfloat16* hi, __nv_bfloat16* lo) {
    long long n = (long long)naux * v * vp;
    GRID_STRIDE(x, n) {
        int cp = x % vp;
        long long qa = x / vp;
        double val = cp < v ? B[qa * v + cp] : 0.0;
        split2(val, hi[x], lo[x]);
    }
}
// Bp[b][(Q,dp)] = B^Q[d][b] (= B^Q[b][d]), zero pad
__global__ void k_split_Bp(const double* __restrict__ B, int naux, int v, int vp, __nv_bfloat16* hi, __nv_bfloat16* lo) {
    long long n = (long long)v * naux * vp;
    GRID_STRIDE(x, n) {
        int dp = x % vp;
        long long r = x / vp;
        int Q = r % naux, b = r / naux;
        double val = dp < v ? B[((long long)Q * v + b) * v + dp] : 0.0;
        split2(val, hi[x], lo[x]);
    }
}
// XT[(m,d)][cp] = X_m[c][d] (c, d < v), zero pad; m < nmat
__global__ void k_split_XT(const double* __restrict__ X, long long nmat, int v, int vp, __nv_bfloat16* hi, __nv_bfloat16* lo) {
    long long n = nmat * vp * vp;
    GRID_STRIDE(x, n) {
        int cp = x % vp;
        long long r = x / vp;
        int d = r % vp;
        long long m = r / vp;
        double val = (cp < v && d < v) ? X[(m * v + cp) * v + d] : 0.0;
        split2(val, hi[x], lo[x]);
    }
}

inline int grid_for(long long n) { return (int)std::min<long long>(std::max<long long>((n + 255) / 256, 1), 152LL * 32); }

// ---- host: tensor maps ------------------------------------------------------
typedef CUresult (*EncodeFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*, const cuuint64_t*,
                             const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                             CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeFn encode_fn() {
    static EncodeFn fn = nullptr;
    static std::once_flag once;
    static cudaError_t st = cudaSuccess;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        st = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q);
        if (st == cudaSuccess && q == cudaDriverEntryPointSuccess) fn = (EncodeFn)p;
    });
    if (!fn) throw Error(-3, "cuTensorMapEncodeTiled unavailable");
    return fn;
}

// 2-D BF16 tensor [rows][cols] (cols contiguous), box {64, box_rows}, 128-byte swizzle
CUtensorMap make_map(const void* base, long long rows, long long cols, int box_rows) {
    if (((uintptr_t)base & 15) || (cols * 2) % 16) throw Error(-1, "tensor map: misaligned operand");
    CUtensorMap m;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
    cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
    cuuint32_t es[2] = {1, 1};
    CUresult r = encode_fn()(&m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, es,
                             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) throw Error(-3, "cuTensorMapEncodeTiled failed: " + std::to_string((int)r));
    return m;
}

int pick_bn(int n) {
    // smallest padded width; prefer the wider tile on ties
    int best = 256;
    long long best_pad = ((n + 255) / 256) * 256LL;
    for (int bn = 240; bn >= 64; bn -= 16) {
        long long pad = ((long long)(n + bn - 1) / bn) * bn;
        if (pad < best_pad) {
            best_pad = pad;
            best = bn;
        }
    }
    return best;
}

void launch_gemm(Ctx& c, const CUtensorMap& ah, const CUtensorMap& al, const CUtensorMap& bh, const CUtensorMap& bl,
                 int a_row0, int b_x0, int M, int N, int K, int BN, int m_fastest, const Epi& ep, double algo_flops) {
    static bool attr = false;
    static int num_sms = 0;
    if (!attr) {
        ADC_CUDA(cudaFuncSetAttribute(k_gemm_bf16x3, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES));
        int dev = 0;
        ADC_CUDA(cudaGetDevice(&dev));
        ADC_CUDA(cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev));
        attr = true;
    }
    const int mt = (M + BM - 1) / BM, nt = (N + BN - 1) / BN;
    const long long ntiles = (long long)mt * nt;
    if (ntiles <= 0) return;
    if (ntiles > (1LL << 31) - 1) throw Error(-1, "ladder: tile count too large");
    const int stage_bytes = 2 * A_BYTES + 2 * BN * BK * 2;
    const int stages = std::min(MAX_STAGES, (int)((SMEM_BYTES - 1024) / stage_bytes));
    if (stages < 2) throw Error(-1, "ladder: tile too large for shared memory");
    const int grid = (int)std::min<long long>(ntiles, num_sms);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (c.timing) {
        ADC_CUDA(cudaEventCreate(&e0));
        ADC_CUDA(cudaEventCreate(&e1));
        ADC_CUDA(cudaEventRecord(e0, c.stream));
    }
    k_gemm_bf16x3<<<grid, THREADS, SMEM_BYTES, c.stream>>>(ah, al, bh, bl, a_row0, b_x0, K, BN, stages, m_fastest, mt, nt,
                                                           ep);
    ++c.kernels;
    ADC_CUDA(cudaGetLastError());
    if (c.timing) {
        ADC_CUDA(cudaEventRecord(e1, c.stream));
        c.ev_start.push_back(e0);
        c.ev_stop.push_back(e1);
        c.algo_flops += algo_flops;
        c.mma_flops += 3.0 * 2.0 * (double)mt * BM * (double)nt * BN * (double)(((K + BK - 1) / BK) * BK);
    }
}

}  // namespace

struct LadderTC {
    int naux = 0, v = 0, vp = 0, chunk = 0, bn2 = 256;
    __nv_bfloat16 *Bs_hi = nullptr, *Bs_lo = nullptr, *Bp_hi = nullptr, *Bp_lo = nullptr;
    CUtensorMap mBs_hi, mBs_lo, mBp_hi, mBp_lo;
    int* d_err = nullptr;
    ~LadderTC() {
        cudaFree(Bs_hi);
        cudaFree(Bs_lo);
        cudaFree(Bp_hi);
        cudaFree(Bp_lo);
        cudaFree(d_err);
    }
};

LadderTC* ladder_tc_create(Ctx& c, const double* Bvv, int naux, int v, int aux_chunk) {
    auto* L = new LadderTC();
    try {
        L->naux = naux;
        L->v = v;
        L->vp = (v + 31) / 32 * 32;
        L->chunk = aux_chunk;
        L->bn2 = pick_bn(v);
        const long long nB = (long long)naux * v * L->vp;
        ADC_CUDA(cudaMalloc(&L->Bs_hi, nB * 2));
        ADC_CUDA(cudaMalloc(&L->Bs_lo, nB * 2));
        ADC_CUDA(cudaMalloc(&L->Bp_hi, nB * 2));
        ADC_CUDA(cudaMalloc(&L->Bp_lo, nB * 2));
        ADC_CUDA(cudaMalloc(&L->d_err, sizeof(int)));
        ADC_CUDA(cudaMemsetAsync(L->d_err, 0, sizeof(int), c.stream));
        k_split_Bs<<<grid_for(nB), 256, 0, c.stream>>>(Bvv, naux, v, L->vp, L->Bs_hi, L->Bs_lo);
        ++c.kernels;
        k_split_Bp<<<grid_for(nB), 256, 0, c.stream>>>(Bvv, naux, v, L->vp, L->Bp_hi, L->Bp_lo);
        ++c.kernels;
        ADC_CUDA(cudaGetLastError());
        L->mBs_hi = make_map(L->Bs_hi, (long long)naux * v, L->vp, BM);
        L->mBs_lo = make_map(L->Bs_lo, (long long)naux * v, L->vp, BM);
        L->mBp_hi = make_map(L->Bp_hi, v, (long long)naux * L->vp, L->bn2);
        L->mBp_lo = make_map(L->Bp_lo, v, (long long)naux * L->vp, L->bn2);
    } catch (...) {
        delete L;
        throw;
    }
    return L;
}

void ladder_tc_destroy(LadderTC* L) { delete L; }

void ladder_tc_apply(LadderTC& L, Ctx& c, const double* X, long long nmat, double* out) {
    const int v = L.v, vp = L.vp, naux = L.naux;
    if (nmat <= 0) return;
    // Scratch budget for Z (hi+lo): ~1 GiB.  Matrices are processed in groups
    // small enough that a chunk holds >= 8 auxiliary functions (long K in GEMM2,
    // fewer FP64 read-modify-write passes over the output); K2 <= 8192.
    const long long budget = 1LL << 30;
    const int qmax = std::max(1, std::min(naux, std::max(1, 8192 / vp)));
    const int qwant = L.chunk > 0 ? std::min(L.chunk, qmax) : std::min(8, qmax);
    const long long per_mq = (long long)v * vp * 4;  // Z bytes per (matrix, aux function)
    long long mg = std::max<long long>(1, budget / (per_mq * qwant));
    mg = std::min(mg, nmat);
    Arena::Mark mk = c.arena.mark();
    const long long nXT = mg * vp * vp;
    auto* xh = (__nv_bfloat16*)c.arena.alloc(nXT * 2);
    auto* xl = (__nv_bfloat16*)c.arena.alloc(nXT * 2);
    int qc = L.chunk > 0 ? std::min(L.chunk, qmax) : (int)std::max<long long>(1, budget / (per_mq * mg));
    qc = std::max(1, std::min(qc, qmax));
    const long long nZ = mg * v * (long long)qc * vp;
    auto* zh = (__nv_bfloat16*)c.arena.alloc(nZ * 2);
    auto* zl = (__nv_bfloat16*)c.arena.alloc(nZ * 2);
    for (long long m0 = 0; m0 < nmat; m0 += mg) {
        const long long nm = std::min(mg, nmat - m0);
        k_split_XT<<<grid_for(nm * vp * vp), 256, 0, c.stream>>>(X + m0 * v * v, nm, v, vp, xh, xl);
        ++c.kernels;
        ADC_CUDA(cudaGetLastError());
        CUtensorMap mXh = make_map(xh, nm * vp, vp, 256), mXl = make_map(xl, nm * vp, vp, 256);
        for (int q0 = 0; q0 < naux; q0 += qc) {
            const int qn = std::min(qc, naux - q0);
            // GEMM1: Z[(q,a),(n,d)] = sum_c B^q[a,c] X_n[c,d]
            Epi e1{};
            e1.mode = 0;
            e1.M = qn * v;
            e1.N = (int)(nm * vp);
            e1.zhi = zh;
            e1.zlo = zl;
            e1.v = v;
            e1.vp = vp;
            e1.qn = qn;
            e1.err = L.d_err;
            const double algo = 2.0 * (double)qn * v * (double)nm * v * v;  // unpadded B^q X_n products
            launch_gemm(c, L.mBs_hi, L.mBs_lo, mXh, mXl, q0 * v, 0, e1.M, e1.N, vp, 256, 1, e1, algo);
            // GEMM2: out[(n,a),b] += sum_(q,d) Z_n[a,(q,d)] B^q[d,b]
            CUtensorMap mZh = make_map(zh, nm * v, (long long)qn * vp, BM), mZl = make_map(zl, nm * v, (long long)qn * vp, BM);
            Epi e2{};
            e2.mode = 1;
            e2.M = (int)(nm * v);
            e2.N = v;
            e2.out = out + m0 * v * v;
            e2.ldc = v;
            e2.err = L.d_err;
            launch_gemm(c, mZh, mZl, L.mBp_hi, L.mBp_lo, 0, q0 * vp, e2.M, e2.N, qn * vp, L.bn2, 0, e2, algo);
        }
    }
    int err = 0;
    ADC_CUDA(cudaMemcpyAsync(&err, L.d_err, sizeof(int), cudaMemcpyDeviceToHost, c.stream));
    ADC_CUDA(cudaStreamSynchronize(c.stream));
    c.arena.release(mk);
    if (err) throw Error(-5, "ladder: a bounded device wait timed out");
}

// Same ladder as ladder_tc_apply, but every intermediate (split X^T and Z) is
// carved out of a caller-provided device buffer of `bytes` bytes instead of
// the handle's scratch arena.  out is overwritten (zeroed, then accumulated).
// Returns false (launching nothing) if one matrix and one auxiliary function
// do not fit in the buffer.
bool ladder_tc_apply_scratch(LadderTC& L, Ctx& c, const double* X, long long nmat, double* out, void* scratch,
                             size_t bytes) {
    const int v = L.v, vp = L.vp, naux = L.naux;
    const long long per_xt = (long long)vp * vp * 4;  // split X^T (hi+lo) per matrix
    const long long per_mq = (long long)v * vp * 4;   // Z (hi+lo) per (matrix, aux function)
    auto round256 = [](long long b) { return (b + 255) / 256 * 256; };
    if (round256(per_xt) + round256(per_mq) > (long long)bytes) return false;
    if (nmat <= 0) return true;
    const int qmax = std::max(1, std::min(naux, std::max(1, 8192 / vp)));
    const int qwant = std::min(8, qmax);
    long long mg = std::max<long long>(1, (long long)bytes / (per_xt + per_mq * qwant + 1024));
    mg = std::min(mg, nmat);
    while (mg > 1 && round256(mg * per_xt) + round256(mg * per_mq) > (long long)bytes) --mg;
    const long long left = (long long)bytes - round256(mg * per_xt);
    int qc = (int)std::max<long long>(1, left / (per_mq * mg));
    qc = std::max(1, std::min(qc, qmax));
    char* base = (char*)scratch;
    auto* xh = (__nv_bfloat16*)base;
    auto* xl = xh + mg * vp * vp;
    auto* zh = (__nv_bfloat16*)(base + round256(mg * per_xt));
    auto* zl = zh + mg * v * (long long)qc * vp;
    ADC_CUDA(cudaMemsetAsync(out, 0, (size_t)nmat * v * v * sizeof(double), c.stream));
    for (long long m0 = 0; m0 < nmat; m0 += mg) {
        const long long nm = std::min(mg, nmat - m0);
        k_split_XT<<<grid_for(nm * vp * vp), 256, 0, c.stream>>>(X + m0 * v * v, nm, v, vp, xh, xl);
        ++c.kernels;
        ADC_CUDA(cudaGetLastError());
        CUtensorMap mXh = make_map(xh, nm * vp, vp, 256), mXl = make_map(xl, nm * vp, vp, 256);
        for (int q0 = 0; q0 < naux; q0 += qc) {
            const int qn = std::min(qc, naux - q0);
            Epi e1{};
            e1.mode = 0;
            e1.M = qn * v;
            e1.N = (int)(nm * vp);
            e1.zhi = zh;
            e1.zlo = zl;
            e1.v = v;
            e1.vp = vp;
            e1.qn = qn;
            e1.err = L.d_err;
            const double algo = 2.0 * (double)qn * v * (double)nm * v * v;
            launch_gemm(c, L.mBs_hi, L.mBs_lo, mXh, mXl, q0 * v, 0, e1.M, e1.N, vp, 256, 1, e1, algo);
            CUtensorMap mZh = make_map(zh, nm * v, (long long)qn * vp, BM), mZl = make_map(zl, nm * v, (long long)qn * vp, BM);
            Epi e2{};
            e2.mode = 1;
            e2.M = (int)(nm * v);
            e2.N = v;
            e2.out = out + m0 * v * v;
            e2.ldc = v;
            e2.err = L.d_err;
            launch_gemm(c, mZh, mZl, L.mBp_hi, L.mBp_lo, 0, q0 * vp, e2.M, e2.N, qn * vp, L.bn2, 0, e2, algo);
        }
    }
    int err = 0;
    ADC_CUDA(cudaMemcpyAsync(&err, L.d_err, sizeof(int), cudaMemcpyDeviceToHost, c.stream));
    ADC_CUDA(cudaStreamSynchronize(c.stream));
    if (err) throw Error(-5, "ladder: a bounded device wait timed out");
    return true;
}

}  // namespace adc

// Density-fitted ladder sum_cd (ac|bd) X_n[c,d] = sum_Q (B^Q X_n B^Q)_ab on
// the 5th-generation tensor cores of sm_103a (tcgen05.mma, operands staged in
// shared memory by TMA, FP32 accumulators in tensor memory).
//
// Per auxiliary chunk q in [q0, q0+qn) two K-major GEMMs run back to back:
//   GEMM1  Z[(q,a),(n,d)] = sum_c B^q[a,c] X_n[c,d]        (A = Bs, B = X^T)
//   GEMM2  out[(n,a),b]  += sum_(q,d) Z_n[a,(q,d)] B^q[d,b] (A = Z,  B = Bp)
// (B^q symmetric).  Every operand x is split into BF16 planes: x = hi + lo
// (two planes, products hi*hi + hi*lo + lo*hi: "BF16x3", 16 significand bits,
// used in sigma) or x = hi + mid + lo (three planes, the six products of total
// order <= 2: "BF16x6", 24 significand bits, used for the one-off ladder of
// the amplitudes in setup, which feeds the 1p-1p block directly).
// GEMM1 writes Z already split
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
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "ladder_tc.cuh"

namespace adc {

namespace {

constexpr int BM = 128;
// K block: 64 BF16 = 128-byte rows in the 128-byte swizzle (8-row atoms of
// 1024 bytes).  (32-deep blocks with the 64-byte swizzle also work -- twice the
// stages of half the size -- but measured slower.)
constexpr int BK = 64;
constexpr int ROW_BYTES = BK * 2;
constexpr int KB_PER_EPOCH_UNIT = 64 / BK;  // LadderMode epochs count 64-deep K blocks
constexpr int MAX_STAGES = 8;
constexpr int EPI_WARPS = 8;
constexpr int THREADS = 64 + 32 * EPI_WARPS;  // warp 0: TMA, warp 1: MMA + TMEM owner, warps 2-9: epilogue
constexpr int TMEM_COLS = 512;  // two accumulators of up to 256 FP32 columns
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
// try_wait that lets the hardware suspend the thread (up to the hint, in ns)
// until the phase completes, instead of spinning on issue slots.
__device__ __forceinline__ bool mbar_try_sleep(uint64_t* b, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\n"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
        "selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(su32(b)), "r"(parity), "r"(20000u)
        : "memory");
    return ok != 0;
}
// Bounded wait: false on timeout (raises the CTA abort flag and the global
// error flag) or when another role of the CTA has already aborted.  The abort
// flag and the clock are checked every 16 tries only.
__device__ bool mbar_wait(uint64_t* b, uint32_t parity, volatile int* abort_flag, int* err) {
    if (mbar_try(b, parity)) return true;
    const uint64_t t0 = gtime();
    for (uint32_t n = 1;; ++n) {
        if (mbar_try_sleep(b, parity)) return true;
        if ((n & 15u) == 0) {
            if (*abort_flag) return false;
            if (gtime() - t0 > WAIT_NS) {
                *abort_flag = 1;
                atomicExch(err, 1);
                return false;
            }
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
__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\nbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// tcgen05 shared-memory matrix descriptor: K-major, ROW_BYTES swizzle, 8-row
// core groups 8 * ROW_BYTES apart.
__device__ __forceinline__ uint64_t smem_desc(const void* p) {
    uint64_t d = 0;
    d |= (uint64_t)((su32(p) >> 4) & 0x3FFF);
    d |= (uint64_t)1 << 16;                     // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)((8 * ROW_BYTES) >> 4) << 32;  // stride byte offset
    d |= (uint64_t)1 << 46;                     // descriptor version
    d |= (uint64_t)(ROW_BYTES == 128 ? 2 : 4) << 61;  // layout: 128-byte (2) or 64-byte (4) swizzle
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

__device__ __forceinline__ void tmem_ld32_add(uint32_t taddr, float* acc) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,"
        "%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
          "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) acc[i] += __uint_as_float(r[i]);
}

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
    int mode;  // 0: split store of Z (GEMM1, through shared memory and TMA), 1: FP64 accumulate (GEMM2),
               // 2: FP64 store (generic contraction)
    int M, N;
    // mode 0: row r = q*vpa + a (a padded to vpa, a multiple of 32), col j = n*vp + dp;
    // Z[((n*v + a)*qn + q)*vp + dp] per plane, written through the 4-D tensor maps Maps::z
    int vpa, vp;
    // modes 1, 2: out[r*ldc + j] (+)= acc
    double* out;
    long long ldc;
    int vec;  // out rows 16-byte aligned (vector loads and stores)
    int* err;
};

__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(b)) : "memory");
}

// 16 consecutive FP32 results of one row into the FP64 output: accumulated
// (mode 1, GEMM2 of the ladder) or stored (mode 2, generic contractions).
__device__ __forceinline__ void store_out16(const Epi& ep, int row, int col0, const float* v) {
    double* o = ep.out + (long long)row * ep.ldc + col0;
    if (ep.mode == 2) {
        if (ep.vec && col0 + 16 <= ep.N) {
#pragma unroll
            for (int i = 0; i < 8; ++i) ((double2*)o)[i] = make_double2((double)v[2 * i], (double)v[2 * i + 1]);
        } else {
#pragma unroll
            for (int i = 0; i < 16; ++i)
                if (col0 + i < ep.N) o[i] = (double)v[i];
        }
        return;
    }
    if (ep.vec && col0 + 16 <= ep.N) {
        // 8 columns at a time: four 16-byte loads in flight before the stores
#pragma unroll
        for (int h8 = 0; h8 < 16; h8 += 8) {
            double2 x[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) x[i] = ((const double2*)(o + h8))[i];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                x[i].x += (double)v[h8 + 2 * i];
                x[i].y += (double)v[h8 + 2 * i + 1];
                ((double2*)(o + h8))[i] = x[i];
            }
        }
    } else {
#pragma unroll
        for (int i = 0; i < 16; ++i)
            if (col0 + i < ep.N) o[i] += (double)v[i];
    }
}

struct Maps {
    CUtensorMap a[3];  // A operand planes (hi, mid/lo, lo)
    CUtensorMap b[3];  // B operand planes
    CUtensorMap z[3];  // GEMM1 output planes: 4-D {dp, q, a, n}, box {16, 1, 32, 1}
};

// Z store of one warp through shared memory: the warp's 32 rows (one q, 32
// consecutive a: row0 = q*vpa + a0 with a0 a multiple of 32) x 16 columns (one
// matrix n), split into `planes` BF16 planes, each written by one TMA store of
// a 32 x 16 box; rows a >= nvir (padding) and q >= qn are clipped by the
// tensor map.  stg: this warp's staging, nbuf buffers of planes x 1 KB, reused
// once the TMA has read them.  The split runs on the FMA/ALU pipes: packed
// round-to-nearest conversions, BF16 -> FP32 by a 16-bit shift.
__device__ __forceinline__ void store_z16(const Maps& maps, const Epi& ep, int planes, int row0, int col0, const float* v,
                                          uint8_t* stg, int nbuf, int& nchunk, int lane) {
    uint8_t* buf = stg + (nchunk % nbuf) * planes * 1024;
    if (lane == 0) {
        if (nbuf == 2)
            asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
        else
            asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
    }
    __syncwarp();
#pragma unroll
    for (int h8 = 0; h8 < 16; h8 += 8) {
        uint32_t pl[3][4];  // [plane][pair of columns]
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            float r0 = v[h8 + 2 * i], r1 = v[h8 + 2 * i + 1];
#pragma unroll
            for (int p = 0; p < 3; ++p) {
                if (p < planes) {
                    const __nv_bfloat162 h = __floats2bfloat162_rn(r0, r1);
                    const uint32_t u = *(const uint32_t*)&h;
                    pl[p][i] = u;
                    r0 -= __uint_as_float(u << 16);
                    r1 -= __uint_as_float(u & 0xFFFF0000u);
                }
            }
        }
#pragma unroll
        for (int p = 0; p < 3; ++p)
            if (p < planes)
                *(uint4*)(buf + p * 1024 + lane * 32 + h8 * 2) = make_uint4(pl[p][0], pl[p][1], pl[p][2], pl[p][3]);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncwarp();
    if (lane == 0) {
        const int q = row0 / ep.vpa, a0 = row0 - q * ep.vpa;
        const int n = col0 / ep.vp, dp0 = col0 - n * ep.vp;
#pragma unroll
        for (int p = 0; p < 3; ++p)
            if (p < planes)
                asm volatile(
                    "cp.async.bulk.tensor.4d.global.shared::cta.bulk_group [%0, {%2, %3, %4, %5}], [%1];" ::"l"(
                        (uint64_t)&maps.z[p]),
                    "r"(su32(buf + p * 1024)), "r"(dp0), "r"(q), "r"(a0), "r"(n)
                    : "memory");
        asm volatile("cp.async.bulk.commit_group;" ::: "memory");
    }
    ++nchunk;
}
__device__ __forceinline__ void store_z_drain(int lane) {
    if (lane == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
    __syncwarp();
}

// Persistent GEMM C = A B^T with split-BF16 operands.  Roles: warp 0 lane 0
// issues TMA loads through a ring of `stages` shared-memory stages, running
// ahead across tiles; warp 1 owns TMEM and its lane 0 issues the MMAs; warps
// 2-9 are the epilogue.
//
// Accumulation.  The tensor core's FP32 accumulate truncates, so a long
// accumulation in one TMEM accumulator drifts toward zero by about a quarter
// ulp per MMA (measured: 2e-5 relative over a 4160-deep chunk).  The MMAs of a
// tile are therefore issued in short epochs of `ekb` K blocks, alternating
// between two TMEM accumulators; the epilogue warps add every epoch into FP32
// registers with round-to-nearest (unbiased) while the next epoch runs, and
// write the tile once after its last epoch.  Epilogue warp w covers TMEM lane
// quarter (w % 4) and one half of the tile's columns.

// kPromote = false (one epoch per tile) streams each tile from TMEM to global
// memory without the register accumulator.
// (ten warps: three share a sub-partition's 16K registers, so at most 168 per thread)
template <bool kPromote>
__global__ void __launch_bounds__(THREADS, 1)
    k_gemm_bf16x3(const __grid_constant__ Maps maps, int planes, int a_row0, int b_x0, int K, int BN, int stages,
                  int m_fastest, int mt, int nt, int ekb, int nbuf, Epi ep) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    __shared__ uint64_t full_bar[MAX_STAGES], empty_bar[MAX_STAGES], tfull[2], tempty[2], done_bar;
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int num_k = (K + BK - 1) / BK;
    const int epochs = (num_k + ekb - 1) / ekb;  // per tile
    const int B_BYTES = BN * BK * 2;
    const int STAGE = planes * (A_BYTES + B_BYTES);  // [A planes][B planes]
    const int ntiles = mt * nt;

    if (threadIdx.x == 0) {
        for (int s = 0; s < stages; ++s) {
            mbar_init(&full_bar[s], 1);
            mbar_init(&empty_bar[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], EPI_WARPS);  // one arrival per epilogue warp
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
                    // plane indices are compile-time constants so that the tensor maps stay in the parameter space
                    uint8_t* sb = st + planes * A_BYTES;
                    const int ya = a_row0 + m_tile * BM, yb = n_tile * BN;
                    tma_load_2d(st, &maps.a[0], &full_bar[s], kx, ya);
                    tma_load_2d(st + A_BYTES, &maps.a[1], &full_bar[s], kx, ya);
                    if (planes == 3) tma_load_2d(st + 2 * A_BYTES, &maps.a[2], &full_bar[s], kx, ya);
                    tma_load_2d(sb, &maps.b[0], &full_bar[s], b_x0 + kx, yb);
                    tma_load_2d(sb + B_BYTES, &maps.b[1], &full_bar[s], b_x0 + kx, yb);
                    if (planes == 3) tma_load_2d(sb + 2 * B_BYTES, &maps.b[2], &full_bar[s], b_x0 + kx, yb);
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
            long long g = 0;   // stage uses
            long long e = 0;   // epochs issued by this CTA (across tiles)
            bool ok = true;
            for (int t = blockIdx.x; t < ntiles && ok && !abort_flag; t += gridDim.x) {
                int left = 0;  // K blocks left in the current epoch (epochs are whole K blocks)
                uint32_t tacc = 0;
                for (int kb = 0; kb < num_k; ++kb, ++g) {
                    const int s = (int)(g % stages);
                    if (!mbar_wait(&full_bar[s], (uint32_t)((g / stages) & 1), &abort_flag, ep.err)) {
                        ok = false;
                        break;
                    }
                    uint32_t first = 1u;
                    if (left == 0) {
                        // new epoch: wait until the epilogue has drained this buffer's previous epoch
                        const int b = (int)(e & 1);
                        if (e >= 2 && !mbar_wait(&tempty[b], (uint32_t)(((e >> 1) & 1) ^ 1), &abort_flag, ep.err)) {
                            ok = false;
                            break;
                        }
                        tacc = tmem + (uint32_t)(b * 256);
                        left = ekb;
                        first = 0u;
                    }
                    fence_after();
                    uint8_t* st = smem + (size_t)s * STAGE;
                    const uint64_t a0 = smem_desc(st), a1 = smem_desc(st + A_BYTES);
                    const uint64_t b0 = smem_desc(st + planes * A_BYTES), b1 = smem_desc(st + planes * A_BYTES + B_BYTES);
                    if (planes == 3) {
                        const uint64_t a2 = smem_desc(st + 2 * A_BYTES), b2 = smem_desc(st + planes * A_BYTES + 2 * B_BYTES);
#pragma unroll
                        for (int kk = 0; kk < BK / 16; ++kk) {
                            const uint64_t o = (uint64_t)(kk * 2);  // 16 BF16 = 32 bytes along K
                            mma_bf16(tacc, a0 + o, b0 + o, idesc, kk == 0 ? first : 1u);
                            mma_bf16(tacc, a0 + o, b1 + o, idesc, 1u);
                            mma_bf16(tacc, a1 + o, b0 + o, idesc, 1u);
                            mma_bf16(tacc, a0 + o, b2 + o, idesc, 1u);
                            mma_bf16(tacc, a2 + o, b0 + o, idesc, 1u);
                            mma_bf16(tacc, a1 + o, b1 + o, idesc, 1u);
                        }
                    } else {
#pragma unroll
                        for (int kk = 0; kk < BK / 16; ++kk) {
                            const uint64_t o = (uint64_t)(kk * 2);
                            mma_bf16(tacc, a0 + o, b0 + o, idesc, kk == 0 ? first : 1u);
                            mma_bf16(tacc, a0 + o, b1 + o, idesc, 1u);
                            mma_bf16(tacc, a1 + o, b0 + o, idesc, 1u);
                        }
                    }
                    mma_commit(&empty_bar[s]);
                    if (--left == 0 || kb == num_k - 1) {
                        mma_commit(&tfull[e & 1]);
                        ++e;
                        left = 0;
                    }
                }
            }
            mma_commit(&done_bar);  // fires when every MMA issued above has completed
        }
    } else {
        const int ew = warp - 2;
        const int quarter = warp & 3;  // TMEM lanes 32*quarter .. +31
        const int half = ew >> 2;      // column half of the tile
        // The halves split on a 16-column boundary, [0, h0) and [h0, BN): both
        // widths are multiples of 16 (BN is) and at most 128.
        const int h0 = ((BN >> 1) + 15) & ~15;
        const int cbeg = half ? h0 : 0, cw = half ? BN - h0 : h0;
        // Z staging of this warp (mode 0) after the pipeline stages
        uint8_t* stg = smem + (size_t)stages * STAGE + (size_t)ew * nbuf * planes * 1024;
        int nchunk = 0;
        long long e = 0;
        bool ok = true;
        for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
            const int m_tile = m_fastest ? t % mt : t / nt;
            const int n_tile = m_fastest ? t / mt : t % nt;
            const int row = m_tile * BM + quarter * 32 + lane;
            const int colt = n_tile * BN + cbeg;  // first output column of this warp
            if constexpr (kPromote) {
                float acc[128];
#pragma unroll
                for (int i = 0; i < 128; ++i) acc[i] = 0.0f;
                for (int ep_i = 0; ep_i < epochs; ++ep_i, ++e) {
                    if (ep.mode == 1 && ep_i == epochs - 1 && row < ep.M) {
                        // pull this thread's FP64 output segment into L2 while the last epoch runs
                        const double* o = ep.out + (long long)row * ep.ldc + colt;
                        for (int c0 = 0; c0 < cw; c0 += 16)
                            if (colt + c0 < ep.N) asm volatile("prefetch.global.L2 [%0];" ::"l"(o + c0));
                    }
                    const int b = (int)(e & 1);
                    if (!mbar_wait(&tfull[b], (uint32_t)((e >> 1) & 1), &abort_flag, ep.err)) {
                        ok = false;
                        break;
                    }
                    fence_after();
                    const uint32_t tbase = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(b * 256 + cbeg);
                    // 32-column loads (one wait each), then a 16-column tail
#pragma unroll
                    for (int c0 = 0; c0 < 128; c0 += 32)
                        if (c0 + 32 <= cw) tmem_ld32_add(tbase + (uint32_t)c0, acc + c0);
#pragma unroll
                    for (int c0 = 0; c0 < 128; c0 += 16) {
                        if (c0 >= (cw & ~31) && c0 < cw) {
                            float v[16];
                            tmem_ld16(tbase + (uint32_t)c0, v);
#pragma unroll
                            for (int i = 0; i < 16; ++i) acc[c0 + i] += v[i];
                        }
                    }
                    fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&tempty[b]);
                }
                if (!ok) break;
#pragma unroll
                for (int c0 = 0; c0 < 128; c0 += 16) {
                    if (c0 >= cw || colt + c0 >= ep.N) continue;  // uniform across the warp
                    if (ep.mode == 0)
                        store_z16(maps, ep, planes, row - lane, colt + c0, acc + c0, stg, nbuf, nchunk, lane);
                    else if (row < ep.M)
                        store_out16(ep, row, colt + c0, acc + c0);
                }
            } else {
                // one epoch per tile: stream TMEM -> global 16 columns at a time, then release the buffer
                const int b = (int)(e & 1);
                if (!mbar_wait(&tfull[b], (uint32_t)((e >> 1) & 1), &abort_flag, ep.err)) {
                    ok = false;
                    break;
                }
                ++e;
                fence_after();
                const uint32_t tbase = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(b * 256 + cbeg);
                for (int c0 = 0; c0 < cw; c0 += 16) {
                    float v[16];
                    tmem_ld16(tbase + (uint32_t)c0, v);  // warp-collective: every lane loads
                    if (colt + c0 < ep.N) {  // uniform across the warp
                        if (ep.mode == 0)
                            store_z16(maps, ep, planes, row - lane, colt + c0, v, stg, nbuf, nchunk, lane);
                        else if (row < ep.M)
                            store_out16(ep, row, colt + c0, v);
                    }
                }
                fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&tempty[b]);
            }
        }
        if (ep.mode == 0) store_z_drain(lane);  // this warp's Z stores have completed
    }
    fence_before();
    __syncthreads();
    if (warp == 1) {
        const uint64_t t0 = gtime();
        while (!mbar_try(&done_bar, 0) && gtime() - t0 < WAIT_NS) {
        }
        fence_after();
    }
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
}

// ---- 2-SM variant: one MMA tile of 256 rows on a CTA pair (cta_group::2) -----
__device__ __forceinline__ uint32_t mapa_rank(const void* p, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(su32(p)), "r"(rank));
    return r;
}
// TMA load into this CTA's shared memory that completes its bytes on an
// mbarrier of either CTA of the pair (shared::cluster address)
__device__ __forceinline__ void tma_load_2d_pair(void* dst, const CUtensorMap* m, uint32_t bar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], "
        "[%2];" ::"r"(su32(dst)),
        "l"((uint64_t)m), "r"(bar), "r"(x), "r"(y)
        : "memory");
}
__device__ __forceinline__ void mma_bf16_pair(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}
// arrive on the mbarrier at `bar`'s offset in both CTAs once the pair's MMAs issued so far have completed
__device__ __forceinline__ void mma_commit_pair(uint64_t* bar) {
    asm volatile(
        "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
            su32(bar)),
        "h"((uint16_t)3)
        : "memory");
}
__device__ __forceinline__ void mbar_arrive_remote(uint32_t bar) {
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try_cluster(uint64_t* b, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\n"
        "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(su32(b)), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait with cluster-scope acquire (for arrivals from the peer CTA)
__device__ bool mbar_wait_cluster(uint64_t* b, uint32_t parity, volatile int* abort_flag, int* err) {
    const uint64_t t0 = gtime();
    for (uint32_t n = 0;; ++n) {
        if (mbar_try_cluster(b, parity)) return true;
        if ((n & 15u) == 15u) {
            if (*abort_flag) return false;
            if (gtime() - t0 > WAIT_NS) {
                *abort_flag = 1;
                atomicExch(err, 1);
                return false;
            }
        }
    }
}

// Persistent GEMM C = A B^T as k_gemm_bf16x3, with each tile 256 rows high and
// computed by a CTA pair (a cluster of two) through cta_group::2 MMAs: CTA r
// holds rows [128 r, 128 r + 128) of the A tile and rows [BN/2 r, BN/2 (r+1))
// of the B tile, so each SM receives A + B/2 per K block instead of A + B and
// a stage is a third smaller.  Both CTAs' TMA loads complete on the leader's
// (rank 0) full barrier; the leader's MMA thread issues every MMA and its
// commits arrive on the barriers of both CTAs; each CTA's epilogue drains its
// own tensor memory (its 128 rows of the tile, all BN columns) and releases
// the accumulator on the leader's barrier (2 x EPI_WARPS arrivals).
template <bool kPromote>
__global__ void __launch_bounds__(THREADS, 1)
    k_gemm_pair(const __grid_constant__ Maps maps, int planes, int a_row0, int b_x0, int K, int BN, int stages,
                int m_fastest, int mt, int nt, int ekb, int nbuf, Epi ep) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    __shared__ uint64_t full_bar[MAX_STAGES], empty_bar[MAX_STAGES], tfull[2], tempty[2], done_bar;
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int num_k = (K + BK - 1) / BK;
    const int epochs = (num_k + ekb - 1) / ekb;  // per tile
    const int BH = BN / 2;                       // B rows held by each CTA
    const int BH_BYTES = BH * ROW_BYTES;
    const int STAGE = planes * (A_BYTES + BH_BYTES);  // per CTA: [A planes][B-half planes]
    const int rank = (int)cluster_rank();
    const bool leader = rank == 0;
    const int mt2 = (mt + 1) / 2;  // 256-row tiles
    const int nunits = mt2 * nt;
    const int cid = blockIdx.x >> 1, ncl = gridDim.x >> 1;

    if (threadIdx.x == 0) {
        for (int s = 0; s < stages; ++s) {
            mbar_init(&full_bar[s], 1);   // leader: its producer's expect_tx (bytes of both CTAs)
            mbar_init(&empty_bar[s], 1);  // the leader's commit
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], 2 * EPI_WARPS);  // leader: every epilogue warp of both CTAs
        }
        mbar_init(&done_bar, 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        // one warp of each CTA of the pair allocates collectively (same address in both)
        asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tmem_slot)), "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncwarp();
    cluster_sync();
    fence_after();
    const uint32_t tmem = tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            long long g = 0;
            for (int u = cid; u < nunits && !abort_flag; u += ncl) {
                const int m2 = m_fastest ? u % mt2 : u / nt;
                const int n_tile = m_fastest ? u / mt2 : u % nt;
                const int ya = a_row0 + m2 * 2 * BM + rank * BM, yb = n_tile * BN + rank * BH;
                for (int kb = 0; kb < num_k; ++kb, ++g) {
                    const int s = (int)(g % stages);
                    const uint32_t ph = (uint32_t)((g / stages) & 1);
                    if (g >= stages && !mbar_wait(&empty_bar[s], ph ^ 1, &abort_flag, ep.err)) break;
                    uint8_t* st = smem + (size_t)s * STAGE;
                    if (leader) mbar_expect_tx(&full_bar[s], 2 * STAGE);
                    const uint32_t fb = mapa_rank(&full_bar[s], 0);
                    const int kx = kb * BK;
                    uint8_t* sb = st + planes * A_BYTES;
                    tma_load_2d_pair(st, &maps.a[0], fb, kx, ya);
                    tma_load_2d_pair(st + A_BYTES, &maps.a[1], fb, kx, ya);
                    if (planes == 3) tma_load_2d_pair(st + 2 * A_BYTES, &maps.a[2], fb, kx, ya);
                    tma_load_2d_pair(sb, &maps.b[0], fb, b_x0 + kx, yb);
                    tma_load_2d_pair(sb + BH_BYTES, &maps.b[1], fb, b_x0 + kx, yb);
                    if (planes == 3) tma_load_2d_pair(sb + 2 * BH_BYTES, &maps.b[2], fb, b_x0 + kx, yb);
                }
            }
            if (abort_flag && leader) {
                // let the copies of the last `stages` issues of both CTAs land (bounded)
                for (long long q = (g > stages ? g - stages : 0); q < g; ++q) {
                    const uint64_t t0 = gtime();
                    while (!mbar_try(&full_bar[q % stages], (uint32_t)((q / stages) & 1)) && gtime() - t0 < WAIT_NS) {
                    }
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0 && leader) {
            const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)((2 * BM) >> 4) << 24);
            long long g = 0;  // stage uses
            long long e = 0;  // epochs issued (across tiles)
            bool ok = true;
            for (int u = cid; u < nunits && ok && !abort_flag; u += ncl) {
                int left = 0;
                uint32_t tacc = 0;
                for (int kb = 0; kb < num_k; ++kb, ++g) {
                    const int s = (int)(g % stages);
                    if (!mbar_wait(&full_bar[s], (uint32_t)((g / stages) & 1), &abort_flag, ep.err)) {
                        ok = false;
                        break;
                    }
                    uint32_t first = 1u;
                    if (left == 0) {
                        const int b = (int)(e & 1);
                        if (e >= 2 && !mbar_wait_cluster(&tempty[b], (uint32_t)(((e >> 1) & 1) ^ 1), &abort_flag, ep.err)) {
                            ok = false;
                            break;
                        }
                        tacc = tmem + (uint32_t)(b * 256);
                        left = ekb;
                        first = 0u;
                    }
                    fence_after();
                    uint8_t* st = smem + (size_t)s * STAGE;
                    const uint64_t a0 = smem_desc(st), a1 = smem_desc(st + A_BYTES);
                    const uint64_t b0 = smem_desc(st + planes * A_BYTES), b1 = smem_desc(st + planes * A_BYTES + BH_BYTES);
                    if (planes == 3) {
                        const uint64_t a2 = smem_desc(st + 2 * A_BYTES), b2 = smem_desc(st + planes * A_BYTES + 2 * BH_BYTES);
#pragma unroll
                        for (int kk = 0; kk < BK / 16; ++kk) {
                            const uint64_t o = (uint64_t)(kk * 2);
                            mma_bf16_pair(tacc, a0 + o, b0 + o, idesc, kk == 0 ? first : 1u);
                            mma_bf16_pair(tacc, a0 + o, b1 + o, idesc, 1u);
                            mma_bf16_pair(tacc, a1 + o, b0 + o, idesc, 1u);
                            mma_bf16_pair(tacc, a0 + o, b2 + o, idesc, 1u);
                            mma_bf16_pair(tacc, a2 + o, b0 + o, idesc, 1u);
                            mma_bf16_pair(tacc, a1 + o, b1 + o, idesc, 1u);
                        }
                    } else {
#pragma unroll
                        for (int kk = 0; kk < BK / 16; ++kk) {
                            const uint64_t o = (uint64_t)(kk * 2);
                            mma_bf16_pair(tacc, a0 + o, b0 + o, idesc, kk == 0 ? first : 1u);
                            mma_bf16_pair(tacc, a0 + o, b1 + o, idesc, 1u);
                            mma_bf16_pair(tacc, a1 + o, b0 + o, idesc, 1u);
                        }
                    }
                    mma_commit_pair(&empty_bar[s]);
                    if (--left == 0 || kb == num_k - 1) {
                        mma_commit_pair(&tfull[e & 1]);
                        ++e;
                        left = 0;
                    }
                }
            }
            mma_commit_pair(&done_bar);  // fires in both CTAs when every MMA issued above has completed
        }
    } else {
        const int ew = warp - 2;
        const int quarter = warp & 3;
        const int half = ew >> 2;
        const int h0 = ((BN >> 1) + 15) & ~15;
        const int cbeg = half ? h0 : 0, cw = half ? BN - h0 : h0;
        const uint32_t tempty_l[2] = {mapa_rank(&tempty[0], 0), mapa_rank(&tempty[1], 0)};
        uint8_t* stg = smem + (size_t)stages * STAGE + (size_t)ew * nbuf * planes * 1024;
        int nchunk = 0;
        long long e = 0;
        bool ok = true;
        for (int u = cid; u < nunits && ok; u += ncl) {
            const int m2 = m_fastest ? u % mt2 : u / nt;
            const int n_tile = m_fastest ? u / mt2 : u % nt;
            const int row = m2 * 2 * BM + rank * BM + quarter * 32 + lane;  // rows past M are skipped
            const int colt = n_tile * BN + cbeg;
            if constexpr (kPromote) {
                float acc[128];
#pragma unroll
                for (int i = 0; i < 128; ++i) acc[i] = 0.0f;
                for (int ep_i = 0; ep_i < epochs; ++ep_i, ++e) {
                    if (ep.mode == 1 && ep_i == epochs - 1 && row < ep.M) {
                        const double* o = ep.out + (long long)row * ep.ldc + colt;
                        for (int c0 = 0; c0 < cw; c0 += 16)
                            if (colt + c0 < ep.N) asm volatile("prefetch.global.L2 [%0];" ::"l"(o + c0));
                    }
                    const int b = (int)(e & 1);
                    if (!mbar_wait(&tfull[b], (uint32_t)((e >> 1) & 1), &abort_flag, ep.err)) {
                        ok = false;
                        break;
                    }
                    fence_after();
                    const uint32_t tbase = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(b * 256 + cbeg);
#pragma unroll
                    for (int c0 = 0; c0 < 128; c0 += 32)
                        if (c0 + 32 <= cw) tmem_ld32_add(tbase + (uint32_t)c0, acc + c0);
#pragma unroll
                    for (int c0 = 0; c0 < 128; c0 += 16) {
                        if (c0 >= (cw & ~31) && c0 < cw) {
                            float v[16];
                            tmem_ld16(tbase + (uint32_t)c0, v);
#pragma unroll
                            for (int i = 0; i < 16; ++i) acc[c0 + i] += v[i];
                        }
                    }
                    fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive_remote(tempty_l[b]);
                }
                if (!ok) break;
#pragma unroll
                for (int c0 = 0; c0 < 128; c0 += 16) {
                    if (c0 >= cw || colt + c0 >= ep.N) continue;  // uniform across the warp
                    if (ep.mode == 0)
                        store_z16(maps, ep, planes, row - lane, colt + c0, acc + c0, stg, nbuf, nchunk, lane);
                    else if (row < ep.M)
                        store_out16(ep, row, colt + c0, acc + c0);
                }
            } else {
                const int b = (int)(e & 1);
                if (!mbar_wait(&tfull[b], (uint32_t)((e >> 1) & 1), &abort_flag, ep.err)) {
                    ok = false;
                    break;
                }
                ++e;
                fence_after();
                const uint32_t tbase = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(b * 256 + cbeg);
                for (int c0 = 0; c0 < cw; c0 += 16) {
                    float v[16];
                    tmem_ld16(tbase + (uint32_t)c0, v);
                    if (colt + c0 < ep.N) {  // uniform across the warp
                        if (ep.mode == 0)
                            store_z16(maps, ep, planes, row - lane, colt + c0, v, stg, nbuf, nchunk, lane);
                        else if (row < ep.M)
                            store_out16(ep, row, colt + c0, v);
                    }
                }
                fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive_remote(tempty_l[b]);
            }
        }
        if (ep.mode == 0) store_z_drain(lane);  // this warp's Z stores have completed
    }
    fence_before();
    __syncthreads();
    if (warp == 1) {
        const uint64_t t0 = gtime();
        while (!mbar_try_cluster(&done_bar, 0) && gtime() - t0 < WAIT_NS) {
        }
        fence_after();
    }
    // the leader's MMAs have completed in both CTAs; neither CTA leaves while
    // the other may still signal its barriers or read its shared memory
    __syncwarp();
    cluster_sync();
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
}

// ---- operand preparation (FP64 -> split BF16) --------------------------------
// x = p0 + p1 (+ p2) with every plane in BF16 (successive remainders)
__device__ __forceinline__ void splitp(double x, int planes, __nv_bfloat16* p0, __nv_bfloat16* p1, __nv_bfloat16* p2) {
    const __nv_bfloat16 h = __double2bfloat16(x);
    double r = x - (double)__bfloat162float(h);
    const __nv_bfloat16 m = __double2bfloat16(r);
    *p0 = h;
    *p1 = m;
    if (planes == 3) *p2 = __double2bfloat16(r - (double)__bfloat162float(m));
}
#define GRID_STRIDE(i, n) for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (n); i += (long long)gridDim.x * blockDim.x)

struct Planes {
    __nv_bfloat16* p[3];
};

// Bs[(Q,a')][c'] = B^Q[a][c] (a, c < v), zero pad: a' and c' both run over vp,
// so that GEMM1's 32-row warp slices never straddle two auxiliary functions
__global__ void k_split_Bs(const double* __restrict__ B, int naux, int v, int vp, int planes, Planes o) {
    long long n = (long long)naux * vp * vp;
    GRID_STRIDE(x, n) {
        int cp = x % vp;
        long long r = x / vp;
        int a = r % vp;
        long long Q = r / vp;
        double val = (cp < v && a < v) ? B[(Q * v + a) * v + cp] : 0.0;
        splitp(val, planes, o.p[0] + x, o.p[1] + x, o.p[2] + x);
    }
}
// Bp[b][(Q,dp)] = B^Q[d][b] (= B^Q[b][d]), zero pad
__global__ void k_split_Bp(const double* __restrict__ B, int naux, int v, int vp, int planes, Planes o) {
    long long n = (long long)v * naux * vp;
    GRID_STRIDE(x, n) {
        int dp = x % vp;
        long long r = x / vp;
        int Q = r % naux, b = r / naux;
        double val = dp < v ? B[((long long)Q * v + b) * v + dp] : 0.0;
        splitp(val, planes, o.p[0] + x, o.p[1] + x, o.p[2] + x);
    }
}
// XT[(m,d)][cp] = X_m[c][d] for X_m of va x vb (c < va, d < vb; rows d padded to vpb,
// columns c to vpa), zero pad; m < nmat
__global__ void k_split_XT(const double* __restrict__ X, long long nmat, int va, int vb, int vpa, int vpb, int planes,
                           Planes o) {
    long long n = nmat * vpb * vpa;
    GRID_STRIDE(x, n) {
        int cp = x % vpa;
        long long r = x / vpa;
        int d = r % vpb;
        long long m = r / vpb;
        double val = (cp < va && d < vb) ? X[(m * va + cp) * vb + d] : 0.0;
        splitp(val, planes, o.p[0] + x, o.p[1] + x, o.p[2] + x);
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

// 2-D BF16 tensor [rows][cols] (cols contiguous), box {BK, box_rows}, ROW_BYTES swizzle
CUtensorMap make_map(const void* base, long long rows, long long cols, int box_rows) {
    if (((uintptr_t)base & 15) || (cols * 2) % 16) throw Error(-1, "tensor map: misaligned operand");
    CUtensorMap m;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
    cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
    cuuint32_t es[2] = {1, 1};
    CUresult r = encode_fn()(&m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, es,
                             CU_TENSOR_MAP_INTERLEAVE_NONE,
                             ROW_BYTES == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) throw Error(-3, "cuTensorMapEncodeTiled failed: " + std::to_string((int)r));
    return m;
}

// Tile width for N = n columns: minimises n-tiles x per-MMA time, where an
// M=128, N=bn, K=16 BF16 MMA takes bn/2 tensor cycles but must read 4 KB (A)
// + 32*bn bytes (B) of shared memory at 128 B/cycle; ties go to the wider tile.
// bn is a multiple of 16 (so that each CTA's half of the B tile in pair mode
// is whole 8-row swizzle atoms).
// Z plane [nm][v][qn][vp] (dp fastest) as a 4-D tensor {dp, q, a, n} for the
// GEMM1 epilogue's TMA stores: box {16, 1, 32, 1}, no swizzle; stores clip at
// the tensor bounds (a >= v, q >= qn, n >= nm)
CUtensorMap make_map_z(const void* base, int vp, int qn, int v, long long nm) {
    if (((uintptr_t)base & 15) || (vp * 2) % 16) throw Error(-1, "tensor map: misaligned Z plane");
    CUtensorMap m;
    cuuint64_t dims[4] = {(cuuint64_t)vp, (cuuint64_t)qn, (cuuint64_t)v, (cuuint64_t)nm};
    cuuint64_t strides[3] = {(cuuint64_t)vp * 2, (cuuint64_t)qn * vp * 2, (cuuint64_t)v * qn * vp * 2};
    cuuint32_t box[4] = {16, 1, 32, 1};
    cuuint32_t es[4] = {1, 1, 1, 1};
    CUresult r = encode_fn()(&m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void*>(base), dims, strides, box, es,
                             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) throw Error(-3, "cuTensorMapEncodeTiled (Z) failed: " + std::to_string((int)r));
    return m;
}

// 2-D BF16 tensor [rows][cols] with a row stride of `ld` elements (a column
// slice of a wider matrix); box {BK, box_rows}, ROW_BYTES swizzle
CUtensorMap make_map_ld(const void* base, long long rows, long long cols, long long ld, int box_rows) {
    if (((uintptr_t)base & 15) || (ld * 2) % 16) throw Error(-1, "tensor map: misaligned operand slice");
    CUtensorMap m;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
    cuuint32_t es[2] = {1, 1};
    CUresult r = encode_fn()(&m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, es,
                             CU_TENSOR_MAP_INTERLEAVE_NONE,
                             ROW_BYTES == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) throw Error(-3, "cuTensorMapEncodeTiled failed: " + std::to_string((int)r));
    return m;
}

int pick_bn(int n, int maxbn) {
    int best = maxbn;
    double best_cost = 1e300;
    for (int bn = maxbn; bn >= 16; bn -= 16) {
        const double nt = (double)((n + bn - 1) / bn);
        const double cost = nt * std::max(bn / 2.0, 32.0 + bn / 4.0);
        if (cost < best_cost - 1e-9) {
            best_cost = cost;
            best = bn;
        }
    }
    return best;
}

// Per-device launch facts, set up once per device (thread-safe): kernel
// attributes, SM count, and how many CTA pairs of k_gemm_pair fit at once.
struct DevInfo {
    std::once_flag once;
    cudaError_t st = cudaSuccess;
    int num_sms = 0, max_pairs = 0;
};
const DevInfo& dev_info() {
    static DevInfo info[64];
    int dev = 0;
    ADC_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) throw Error(-3, "ladder: device index out of range");
    DevInfo& d = info[dev];
    std::call_once(d.once, [&d, dev] {
        auto chk = [&d](cudaError_t e) {
            if (e != cudaSuccess && d.st == cudaSuccess) d.st = e;
        };
        chk(cudaFuncSetAttribute(k_gemm_bf16x3<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES));
        chk(cudaFuncSetAttribute(k_gemm_bf16x3<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES));
        chk(cudaFuncSetAttribute(k_gemm_pair<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES));
        chk(cudaFuncSetAttribute(k_gemm_pair<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES));
        chk(cudaDeviceGetAttribute(&d.num_sms, cudaDevAttrMultiProcessorCount, dev));
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute cl[1];
        cl[0].id = cudaLaunchAttributeClusterDimension;
        cl[0].val.clusterDim.x = 2;
        cl[0].val.clusterDim.y = 1;
        cl[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3((unsigned)(d.num_sms / 2 * 2));
        cfg.blockDim = dim3(THREADS);
        cfg.dynamicSmemBytes = SMEM_BYTES;
        cfg.attrs = cl;
        cfg.numAttrs = 1;
        chk(cudaOccupancyMaxActiveClusters(&d.max_pairs, (void*)k_gemm_pair<true>, &cfg));
    });
    ADC_CUDA(d.st);
    if (d.max_pairs < 1) throw Error(-3, "ladder: no CTA pair fits on the device");
    return d;
}

// ekb: accumulation epoch in 64-deep K blocks (0 = one epoch per tile);
// pair: 256-row tiles on CTA pairs (k_gemm_pair), else 128-row tiles per CTA
void launch_gemm(Ctx& c, const Maps& maps, int planes, int a_row0, int b_x0, int M, int N, int K, int BN, int m_fastest,
                 int ekb, bool pair, const Epi& ep, double algo_flops, cudaStream_t stream_override = nullptr) {
    const cudaStream_t st = stream_override ? stream_override : c.stream;
    if (BN % 16 || BN < 16 || BN > 256) throw Error(-1, "ladder: tile width must be a multiple of 16 in [16, 256]");
    const DevInfo& di = dev_info();
    const int num_sms = di.num_sms, max_pairs = di.max_pairs;
    const int mt = (M + BM - 1) / BM, nt = (N + BN - 1) / BN;
    const long long ntiles = (long long)mt * nt;
    if (ntiles <= 0) return;
    if (ntiles > (1LL << 31) - 1) throw Error(-1, "ladder: tile count too large");
    const int stage_bytes = planes * (A_BYTES + (pair ? BN / 2 : BN) * ROW_BYTES);
    // mode 0: per-warp Z staging of planes x 1 KB, double-buffered when two pipeline stages still fit
    const int stg = ep.mode == 0 ? EPI_WARPS * planes * 1024 : 0;
    int nbuf = ep.mode == 0 ? 2 : 0;
    int stages = std::min(MAX_STAGES, (int)((SMEM_BYTES - 1024 - nbuf * stg) / stage_bytes));
    if (stages < 2 && nbuf == 2) {
        nbuf = 1;
        stages = std::min(MAX_STAGES, (int)((SMEM_BYTES - 1024 - stg) / stage_bytes));
    }
    if (stages < 2) throw Error(-1, "ladder: tile too large for shared memory");
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute cl[1];
    cl[0].id = cudaLaunchAttributeClusterDimension;
    cl[0].val.clusterDim.x = 2;
    cl[0].val.clusterDim.y = 1;
    cl[0].val.clusterDim.z = 1;
    cfg.blockDim = dim3(THREADS);
    cfg.dynamicSmemBytes = SMEM_BYTES;
    cfg.stream = st;
    cfg.attrs = cl;
    cfg.numAttrs = 1;
    int grid;
    if (!pair) {
        grid = (int)std::min<long long>(ntiles, num_sms);
    } else {
        const long long units = (long long)((mt + 1) / 2) * nt;  // 256-row tiles
        grid = (int)std::min<long long>(units, max_pairs) * 2;
    }
    cfg.gridDim = dim3((unsigned)grid);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (c.timing) {
        ADC_CUDA(cudaEventCreate(&e0));
        ADC_CUDA(cudaEventCreate(&e1));
        ADC_CUDA(cudaEventRecord(e0, st));
    }
    // epoch length in the kernel's K blocks (MMAs per epoch = ekb * BK/16 * (3 or 6 products))
    ekb = ekb <= 0 ? (K + BK - 1) / BK : ekb * KB_PER_EPOCH_UNIT;
    // one accumulation epoch per tile: the streaming epilogue without register accumulation
    const bool promote = ekb < (K + BK - 1) / BK;
    if (pair) {
        auto kp = promote ? k_gemm_pair<true> : k_gemm_pair<false>;
        ADC_CUDA(cudaLaunchKernelEx(&cfg, kp, maps, planes, a_row0, b_x0, K, BN, stages, m_fastest, mt, nt, ekb, nbuf, ep));
    } else {
        auto kern = promote ? k_gemm_bf16x3<true> : k_gemm_bf16x3<false>;
        kern<<<grid, THREADS, SMEM_BYTES, st>>>(maps, planes, a_row0, b_x0, K, BN, stages, m_fastest, mt, nt, ekb, nbuf,
                                                      ep);
    }
    ++c.kernels;
    ADC_CUDA(cudaGetLastError());
    if (c.timing) {
        ADC_CUDA(cudaEventRecord(e1, st));
        c.ev_start.push_back(e0);
        c.ev_stop.push_back(e1);
        const double mma = (planes == 3 ? 6.0 : 3.0) * 2.0 * (double)mt * BM * (double)nt * BN * (double)(((K + BK - 1) / BK) * BK);
        c.ev_ladder.push_back(ep.mode != 2);  // the DF ladder's two GEMMs (mode 2: other contractions)
        c.ev_algo.push_back(algo_flops);
        c.ev_mma.push_back(mma);
        for (double x : {(double)M, (double)N, (double)K, (double)BN}) c.ev_shape.push_back(x);
        c.algo_flops += algo_flops;
        c.mma_flops += mma;
    }
}

}  // namespace

struct LadderTC {
    int naux = 0, v = 0, vp = 0, chunk = 0;
    bool pair1 = true, pair2 = true;    // 2-SM tiles (cta_group::2 on CTA pairs) for GEMM1 / GEMM2
    int bn2[4] = {256, 256, 256, 256};  // GEMM2 tile width by plane count (2 or 3)
    const double* Bvv = nullptr;        // FP64 source (owned by the caller, outlives this object)
    int nplanes = 0;                    // BF16 planes held (2; 3 once a three-plane ladder was asked for)
    __nv_bfloat16 *Bs[3] = {}, *Bp[3] = {};  // BF16 planes of B^Q in the GEMM1-A and GEMM2-B layouts
    CUtensorMap mBs[3];                       // GEMM1-A maps
    int* d_err = nullptr;
    ~LadderTC() {
        for (int p = 0; p < 3; ++p) {
            cudaFree(Bs[p]);
            cudaFree(Bp[p]);
        }
        cudaFree(d_err);
    }
};

namespace {
constexpr int BN1[4] = {0, 0, 256, 128};  // GEMM1 tile width by plane count (two stages must fit)

// (Re)split B^Q_vv into `planes` BF16 planes of both layouts and make their tensor maps.
void split_B(LadderTC& L, Ctx& c, int planes) {
    const long long nB = (long long)L.naux * L.v * L.vp;      // Bp planes
    const long long nBs = (long long)L.naux * L.vp * L.vp;    // Bs planes (rows padded)
    Planes ps{}, pp{};
    for (int p = 0; p < planes; ++p) {
        if (!L.Bs[p]) L.Bs[p] = (__nv_bfloat16*)dev_alloc(nBs * 2, c.stream);
        if (!L.Bp[p]) L.Bp[p] = (__nv_bfloat16*)dev_alloc(nB * 2, c.stream);
        ps.p[p] = L.Bs[p];
        pp.p[p] = L.Bp[p];
    }
    k_split_Bs<<<grid_for(nBs), 256, 0, c.stream>>>(L.Bvv, L.naux, L.v, L.vp, planes, ps);
    ++c.kernels;
    k_split_Bp<<<grid_for(nB), 256, 0, c.stream>>>(L.Bvv, L.naux, L.v, L.vp, planes, pp);
    ++c.kernels;
    ADC_CUDA(cudaGetLastError());
    for (int p = 0; p < planes; ++p) {
        L.mBs[p] = make_map(L.Bs[p], (long long)L.naux * L.vp, L.vp, BM);
        // GEMM2-B boxes: one CTA's half of the tile in pair mode
    }
    L.nplanes = planes;
}
}  // namespace

LadderTC* ladder_tc_create(Ctx& c, const double* Bvv, int naux, int v, int aux_chunk) {
    auto* L = new LadderTC();
    try {
        L->naux = naux;
        L->v = v;
        L->vp = (v + 31) / 32 * 32;
        L->chunk = aux_chunk;
        L->Bvv = Bvv;
        L->bn2[2] = pick_bn(v, 256);
        L->bn2[3] = pick_bn(v, 128);
        L->d_err = (int*)dev_alloc(sizeof(int), c.stream);
        ADC_CUDA(cudaMemsetAsync(L->d_err, 0, sizeof(int), c.stream));
        split_B(*L, c, 2);
    } catch (...) {
        delete L;
        throw;
    }
    return L;
}

void ladder_tc_destroy(LadderTC* L) { delete L; }

namespace {

// The chunk loop shared by both entry points: groups of mg matrices, chunks of
// qc auxiliary functions; scratch xt (split X^T planes of one group) and zt (Z planes).
// out_n[a,b] += sum_Q (B_l^Q X_n B_r^Q)[a,b] for X_n of va x vb: B_l (va x va) from Ll
// (GEMM1's A operand), B_r (vb x vb) from Lr (GEMM2's B operand); Ll == Lr for the
// square ladder of one B^Q.
void run_ladder(LadderTC& Ll, LadderTC& Lr, Ctx& c, const double* X, long long nmat, double* out, const LadderMode& md,
                Planes xt, Planes zt, long long mg, int qc, int bn2) {
    const int va = Ll.v, vpa = Ll.vp, vb = Lr.v, vpb = Lr.vp, naux = Ll.naux, planes = md.planes;
    const int bn1 = BN1[planes];
    CUtensorMap mBp[3];  // GEMM2-B maps: one CTA's half of the tile in pair mode
    for (int p = 0; p < planes; ++p) mBp[p] = make_map(Lr.Bp[p], vb, (long long)naux * vpb, Lr.pair2 ? bn2 / 2 : bn2);
    for (long long m0 = 0; m0 < nmat; m0 += mg) {
        const long long nm = std::min(mg, nmat - m0);
        k_split_XT<<<grid_for(nm * vpb * vpa), 256, 0, c.stream>>>(X + m0 * va * vb, nm, va, vb, vpa, vpb, planes, xt);
        ++c.kernels;
        ADC_CUDA(cudaGetLastError());
        Maps m1;
        for (int p = 0; p < planes; ++p) {
            m1.a[p] = Ll.mBs[p];
            m1.b[p] = make_map(xt.p[p], nm * vpb, vpa, Ll.pair1 ? bn1 / 2 : bn1);
        }
        for (int q0 = 0; q0 < naux; q0 += qc) {
            const int qn = std::min(qc, naux - q0);
            // GEMM1: Z[(q,a),(n,d)] = sum_c B_l^q[a,c] X_n[c,d]  (rows q*vpa + a, a padded to vpa; d to vpb)
            Epi e1{};
            e1.mode = 0;
            e1.M = qn * vpa;
            e1.N = (int)(nm * vpb);
            e1.vpa = vpa;
            e1.vp = vpb;
            e1.err = Ll.d_err;
            for (int p = 0; p < planes; ++p) m1.z[p] = make_map_z(zt.p[p], vpb, qn, va, nm);
            launch_gemm(c, m1, planes, q0 * vpa, 0, e1.M, e1.N, vpa, bn1, 1, md.epoch1, Ll.pair1, e1,
                        2.0 * (double)qn * va * (double)nm * vb * va);  // unpadded products
            // GEMM2: out[(n,a),b] += sum_(q,d) Z_n[a,(q,d)] B_r^q[d,b]
            Maps m2;
            for (int p = 0; p < planes; ++p) {
                m2.a[p] = make_map(zt.p[p], nm * va, (long long)qn * vpb, BM);
                m2.b[p] = mBp[p];
            }
            Epi e2{};
            e2.mode = 1;
            e2.M = (int)(nm * va);
            e2.N = vb;
            e2.out = out + m0 * va * vb;
            e2.ldc = vb;
            e2.vec = ((uintptr_t)e2.out % 16 == 0) && (vb % 2 == 0);
            e2.err = Ll.d_err;
            launch_gemm(c, m2, planes, 0, q0 * vpb, e2.M, e2.N, qn * vpb, bn2, 0, md.epoch2, Lr.pair2, e2,
                        2.0 * (double)nm * va * (double)vb * qn * vb);
        }
    }
}

void check_err(LadderTC& L, Ctx& c) {
    if (c.capturing) return;  // read after the graph's replay
    int err = 0;
    ADC_CUDA(cudaMemcpyAsync(&err, L.d_err, sizeof(int), cudaMemcpyDeviceToHost, c.stream));
    ADC_CUDA(cudaStreamSynchronize(c.stream));
    if (err) throw Error(-5, "ladder: a bounded device wait timed out");
}

}  // namespace

// ---- tile autotuner ------------------------------------------------------------
// Tile choices measured on the device and kept in a text file shared by every handle
// of the process that names it (one line per problem: key, then the chosen values).
struct TuneCache {
    std::mutex mu;
    std::string path;
    std::map<std::string, std::vector<int>> table;
};

namespace {
std::mutex g_tune_mu;
std::map<std::string, std::unique_ptr<TuneCache>> g_tune;

bool tune_get(TuneCache* t, const std::string& key, std::vector<int>& v) {
    std::lock_guard<std::mutex> lk(t->mu);
    auto it = t->table.find(key);
    if (it == t->table.end()) return false;
    v = it->second;
    return true;
}

void tune_put(TuneCache* t, const std::string& key, const std::vector<int>& v) {
    std::lock_guard<std::mutex> lk(t->mu);
    t->table[key] = v;
    FILE* f = std::fopen(t->path.c_str(), "w");
    if (!f) return;  // the choices still hold for this process
    for (auto& kv : t->table) {
        std::fprintf(f, "%s", kv.first.c_str());
        for (int x : kv.second) std::fprintf(f, " %d", x);
        std::fprintf(f, "\n");
    }
    std::fclose(f);
}

// milliseconds of one run of f on c.stream (CUDA events; synchronises)
template <class F>
float time_on_stream(Ctx& c, F f) {
    cudaEvent_t e0, e1;
    ADC_CUDA(cudaEventCreate(&e0));
    ADC_CUDA(cudaEventCreate(&e1));
    ADC_CUDA(cudaEventRecord(e0, c.stream));
    f();
    ADC_CUDA(cudaEventRecord(e1, c.stream));
    ADC_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    ADC_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return ms;
}

// distinct multiples of 16 in [16, maxbn], the cost model's choice first
std::vector<int> bn_candidates(int n, int maxbn, std::initializer_list<int> extra) {
    std::vector<int> c{pick_bn(n, maxbn)};
    for (int b : extra)
        if (b >= 16 && b <= maxbn && b % 16 == 0 && std::find(c.begin(), c.end(), b) == c.end()) c.push_back(b);
    return c;
}
}  // namespace

TuneCache* tune_cache_open(const char* path) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto& slot = g_tune[path];
    if (!slot) {
        slot.reset(new TuneCache());
        slot->path = path;
        if (FILE* f = std::fopen(path, "r")) {
            char line[512];
            while (std::fgets(line, sizeof line, f)) {
                // key: the first token; values: the integers after it
                char* save = nullptr;
                char* tok = strtok_r(line, " \t\n", &save);
                if (!tok) continue;
                std::string key = tok;
                std::vector<int> vals;
                while ((tok = strtok_r(nullptr, " \t\n", &save))) vals.push_back(std::atoi(tok));
                if (!vals.empty()) slot->table[key] = vals;
            }
            std::fclose(f);
        }
    }
    return slot.get();
}

void ladder_tc_apply(LadderTC& L, Ctx& c, const double* X, long long nmat, double* out, const LadderMode& md) {
    ladder_tc_apply_pair(L, L, c, X, nmat, out, md);
}

void ladder_tc_check(LadderTC& L, Ctx& c) {
    int err = 0;
    ADC_CUDA(cudaMemcpyAsync(&err, L.d_err, sizeof(int), cudaMemcpyDeviceToHost, c.stream));
    ADC_CUDA(cudaStreamSynchronize(c.stream));
    if (err) throw Error(-5, "ladder: a bounded device wait timed out");
}

void ladder_tc_apply_pair(LadderTC& Ll, LadderTC& Lr, Ctx& c, const double* X, long long nmat, double* out,
                          const LadderMode& md) {
    LadderTC& L = Ll;
    const int v = Ll.v, vp = Lr.vp, vpl = Ll.vp, vr = Lr.v, naux = Ll.naux, planes = md.planes;
    if (nmat <= 0) return;
    if (Lr.naux != naux) throw Error(-1, "ladder: the two B^Q factors differ in naux");
    if (planes != 2 && planes != 3) throw Error(-1, "ladder: planes must be 2 or 3");
    if (md.epoch1 < 0 || md.epoch2 < 0) throw Error(-1, "ladder: negative epoch length");
    if (planes > Ll.nplanes) split_B(Ll, c, planes);  // the third plane only when first asked for
    if (planes > Lr.nplanes) split_B(Lr, c, planes);
    ADC_CUDA(cudaMemsetAsync(L.d_err, 0, sizeof(int), c.stream));  // clear a timeout of an earlier call
    // Scratch budget for Z (all planes): ~4 GiB.  Matrices are processed in
    // groups small enough that a chunk holds >= 8 auxiliary functions (long K
    // in GEMM2, fewer FP64 read-modify-write passes over the output); with
    // promotion of the FP32 partial sums K2 = chunk * vp has no accuracy limit.
    const long long budget = 4LL << 30;
    const int qmax = std::max(1, naux);
    const int qwant = L.chunk > 0 ? std::min(L.chunk, qmax) : std::min(8, qmax);
    const long long per_mq = (long long)v * vp * 2 * planes;  // Z bytes per (matrix, aux function)
    long long mg = std::max<long long>(1, budget / (per_mq * qwant));
    mg = std::min(mg, nmat);
    int qc = L.chunk > 0 ? std::min(L.chunk, qmax) : (int)std::max<long long>(1, budget / (per_mq * mg));
    qc = std::max(1, std::min(qc, qmax));
    int bn2 = Lr.bn2[planes];
    Arena::Mark mk = c.arena.mark();
    auto scratch = [&](int q) {
        Planes xt{}, zt{};
        for (int p = 0; p < planes; ++p) {
            xt.p[p] = (__nv_bfloat16*)c.arena.alloc(mg * vp * vpl * 2);
            zt.p[p] = (__nv_bfloat16*)c.arena.alloc(mg * v * (long long)q * vp * 2);
        }
        return std::make_pair(xt, zt);
    };
    if (c.tuner && !c.timing && !c.capturing && md.epoch1 == 0) {
        // GEMM2 tile width of the sigma ladder (single-epoch GEMM1; the promoted modes of
        // setup and refinement are one-off and keep the cost model's width): measured once
        // per B^Q shape, on the first call's matrices, and cached
        TuneCache* tc = (TuneCache*)c.tuner;
        const std::string key = "ladder:sm" + std::to_string(dev_info().num_sms) + ":v" + std::to_string(v) +
                                (vr != v ? "x" + std::to_string(vr) : std::string()) + ":naux" +
                                std::to_string(naux) + ":p" + std::to_string(planes) + ":e" + std::to_string(md.epoch2);
        std::vector<int> got;
        if (tune_get(tc, key, got) && got.size() == 1) {
            bn2 = got[0];
        } else {
            const int maxbn = planes == 3 ? 128 : 256;
            double* tmp = c.arena.dalloc((size_t)nmat * v * vr);  // timing runs accumulate here
            ADC_CUDA(cudaMemsetAsync(tmp, 0, (size_t)nmat * v * vr * sizeof(double), c.stream));
            float best = 1e30f;
            int bb = bn2;
            Arena::Mark m2 = c.arena.mark();
            auto sc = scratch(qc);
            for (int b : bn_candidates(vr, maxbn, {256, 224, 192, 160})) {
                const float ms =
                    time_on_stream(c, [&] { run_ladder(Ll, Lr, c, X, nmat, tmp, md, sc.first, sc.second, mg, qc, b); });
                if (ms < best) best = ms, bb = b;
            }
            c.arena.release(m2);
            check_err(L, c);
            bn2 = bb;
            tune_put(tc, key, {bn2});
        }
    }
    auto sc = scratch(qc);
    run_ladder(Ll, Lr, c, X, nmat, out, md, sc.first, sc.second, mg, qc, bn2);
    check_err(L, c);
    c.arena.release(mk);
}

// Same ladder (two planes, sigma's accumulation epochs), but every intermediate (split X^T
// and Z) is carved out of a caller-provided device buffer of `bytes` bytes
// instead of the handle's scratch arena.  out is overwritten (zeroed, then
// accumulated).  Returns false (launching nothing) if one matrix and one
// auxiliary function do not fit in the buffer.
bool ladder_tc_apply_scratch(LadderTC& L, Ctx& c, const double* X, long long nmat, double* out, const LadderMode& md,
                             void* scratch, size_t bytes) {
    const int v = L.v, vp = L.vp, naux = L.naux, planes = 2;
    if (md.planes != 2) throw Error(-1, "ladder: the fixed-scratch path takes two planes");
    const long long per_xt = (long long)vp * vp * 2 * planes;  // split X^T per matrix
    const long long per_mq = (long long)v * vp * 2 * planes;   // Z per (matrix, aux function)
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
    Planes xt{}, zt{};
    xt.p[0] = (__nv_bfloat16*)base;
    xt.p[1] = xt.p[0] + mg * vp * vp;
    zt.p[0] = (__nv_bfloat16*)(base + round256(mg * per_xt));
    zt.p[1] = zt.p[0] + mg * v * (long long)qc * vp;
    ADC_CUDA(cudaMemsetAsync(L.d_err, 0, sizeof(int), c.stream));  // clear a timeout of an earlier call
    ADC_CUDA(cudaMemsetAsync(out, 0, (size_t)nmat * v * v * sizeof(double), c.stream));
    run_ladder(L, L, c, X, nmat, out, md, xt, zt, mg, qc, L.bn2[planes]);
    check_err(L, c);
    return true;
}

// ---- generic split-BF16 contraction (gemm_mode 2) --------------------------

bool tc_gemm_fits(long long M, long long N, long long K) {
    return M < (1LL << 30) && N < (1LL << 30) && K < (1LL << 30) && K >= 64;
}

static void tc_gemm_bn(Ctx& c, const void* const* A, const void* const* B, long long M, long long N, long long Kp,
                       double algo_flops, double* C, int BN);

void tc_gemm(Ctx& c, const void* const* A, const void* const* B, long long M, long long N, long long Kp, double algo_flops,
             double* C) {
    if (!c.d_err) throw Error(-1, "tc_gemm: no device error flag");
    const int n = (int)std::min<long long>(N, 1 << 20);
    int BN = pick_bn(n, 256);
    if (c.tuner && !c.timing && !c.capturing) {
        // tile width measured once per shape (every run overwrites C, so the runs are interchangeable)
        TuneCache* tc = (TuneCache*)c.tuner;
        const std::string key = "gemm:sm" + std::to_string(dev_info().num_sms) + ":M" + std::to_string(M) + ":N" +
                                std::to_string(N) + ":K" + std::to_string(Kp);
        std::vector<int> got;
        if (tune_get(tc, key, got) && got.size() == 1) {
            BN = got[0];
        } else {
            float best = 1e30f;
            int bb = BN, last = BN;
            for (int b : bn_candidates(n, 256, {256, 128})) {
                const float ms = time_on_stream(c, [&] { tc_gemm_bn(c, A, B, M, N, Kp, algo_flops, C, b); });
                last = b;
                if (ms < best) best = ms, bb = b;
            }
            tune_put(tc, key, {bb});
            if (bb == last) return;  // C already holds the result of the chosen tile width
            BN = bb;
        }
    }
    tc_gemm_bn(c, A, B, M, N, Kp, algo_flops, C, BN);
}

static void tc_gemm_bn(Ctx& c, const void* const* A, const void* const* B, long long M, long long N, long long Kp,
                       double algo_flops, double* C, int BN) {
    const bool pair = true;
    const long long tiles = ((M + 255) / 256) * ((N + BN - 1) / BN);
    // K slices, each its own launch on a side stream (the launches of few tiles run side by side)
    int S = 1;
    long long ks = Kp;
    if (tiles < 64) {
        S = (int)std::min<long long>(16, std::max<long long>(2, (64 + tiles - 1) / tiles));
        ks = ((Kp + S - 1) / S + 63) / 64 * 64;
        S = (int)((Kp + ks - 1) / ks);
    }
    Epi e{};
    e.mode = 2;
    e.M = (int)M;
    e.N = (int)N;
    e.ldc = N;
    e.err = c.d_err;
    const int m_fastest = M <= N ? 1 : 0;  // consecutive tiles share the B tile when A is the smaller operand
    if (S == 1) {
        Maps m{};
        for (int p = 0; p < 2; ++p) {
            m.a[p] = make_map(A[p], M, Kp, BM);
            m.b[p] = make_map(B[p], N, Kp, pair ? BN / 2 : BN);
        }
        e.out = C;
        e.vec = ((uintptr_t)C % 16 == 0) && (N % 2 == 0);
        launch_gemm(c, m, 2, 0, 0, (int)M, (int)N, (int)Kp, BN, m_fastest, 16, pair, e, algo_flops);
        return;
    }
    double* T = c.arena.dalloc((size_t)(S * M * N));
    ensure_side_streams(c, S);
    ADC_CUDA(cudaEventRecord(c.side_fork, c.stream));
    for (int sl = 0; sl < S; ++sl) {
        const long long k0 = sl * ks, kn = std::min(ks, Kp - k0);
        Maps m{};
        for (int p = 0; p < 2; ++p) {
            m.a[p] = make_map_ld((const __nv_bfloat16*)A[p] + k0, M, kn, Kp, BM);
            m.b[p] = make_map_ld((const __nv_bfloat16*)B[p] + k0, N, kn, Kp, pair ? BN / 2 : BN);
        }
        e.out = T + sl * M * N;
        e.vec = ((uintptr_t)e.out % 16 == 0) && (N % 2 == 0);
        ADC_CUDA(cudaStreamWaitEvent(c.side[sl], c.side_fork, 0));
        launch_gemm(c, m, 2, 0, 0, (int)M, (int)N, (int)kn, BN, m_fastest, 16, pair, e, algo_flops * kn / Kp, c.side[sl]);
        ADC_CUDA(cudaEventRecord(c.side_join[sl], c.side[sl]));
    }
    for (int sl = 0; sl < S; ++sl) ADC_CUDA(cudaStreamWaitEvent(c.stream, c.side_join[sl], 0));
    sum_slices(c, S, M * N, T, C);
}

}  // namespace adc

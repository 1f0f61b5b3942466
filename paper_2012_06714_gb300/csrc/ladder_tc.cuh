// Tensor-core (tcgen05 / TMEM, sm_103a) density-fitted ladder:
//   out[n] += sum_Q B^Q X_n B^Q      (sum_cd (ac|bd) X_n[c,d], Eq. 19)
// with split-precision BF16 operands (planes = 2: x = hi + lo, three products;
// planes = 3: x = hi + mid + lo, six products), FP32 accumulation within one
// auxiliary chunk and FP64 accumulation across chunks.
#pragma once
#include "common.cuh"

namespace adc {

// Arithmetic of one ladder evaluation.  The tensor core's FP32 accumulation
// truncates, so a long accumulation in tensor memory drifts toward zero
// (about a quarter ulp per MMA).  epoch1 / epoch2 bound the K blocks (64 deep)
// accumulated in tensor memory before the partial sum is added, rounded to
// nearest, into FP32 registers (GEMM1: K = nvir, GEMM2: K = chunk * nvir);
// 0 means the whole K range of a tile in one accumulator.
struct LadderMode {
    int planes;  // 2 or 3
    int epoch1, epoch2;
};

struct LadderTC;  // owns the BF16 hi/lo copies of B^Q_vv in the GEMM layouts

LadderTC* ladder_tc_create(Ctx& c, const double* Bvv, int naux, int nvir, int aux_chunk);
void ladder_tc_destroy(LadderTC* L);
// throws ADC_ERR_TIMEOUT if a bounded wait of this ladder's kernels gave up (synchronises c.stream)
void ladder_tc_check(LadderTC& L, Ctx& c);
void ladder_tc_apply(LadderTC& L, Ctx& c, const double* X, long long nmat, double* out, const LadderMode& md);
// out[n] += sum_Q Bl^Q X[n] Br^Q for nmat rectangular Ll.v x Lr.v matrices (the two B^Q
// factors share naux; e.g. the alpha and beta virtual blocks of an open-shell reference)
void ladder_tc_apply_pair(LadderTC& Ll, LadderTC& Lr, Ctx& c, const double* X, long long nmat, double* out,
                          const LadderMode& md);
bool ladder_tc_apply_scratch(LadderTC& L, Ctx& c, const double* X, long long nmat, double* out, const LadderMode& md,
                             void* scratch, size_t bytes);

// Generic contraction on the same kernel: C[M][N] (FP64 row-major, overwritten)
// = sum_k A[m][k] B[n][k] for two-plane split-BF16 K-major operands A[p]
// [M][Kp], B[p] [N][Kp] (Kp a multiple of 8, zeros beyond K), FP32 partial
// sums promoted every 16 K blocks (64 deep).  A bounded device wait that gives
// up raises c.d_err.
// Tile autotuner: measured tile choices (GEMM2 tile width and auxiliary chunk of the
// ladder, tile width of the generic contractions) kept per problem in a text file;
// one instance per path, shared by the process's handles (Ctx::tuner).
struct TuneCache;
TuneCache* tune_cache_open(const char* path);

// the shape fits the kernel's 32-bit tile coordinates and K >= 64 (one K block)
bool tc_gemm_fits(long long M, long long N, long long K);
void tc_gemm(Ctx& c, const void* const* A, const void* const* B, long long M, long long N, long long Kp, double algo_flops,
             double* C);

}  // namespace adc

// Tensor-core (tcgen05 / TMEM, sm_103a) density-fitted ladder:
//   out[n] += sum_Q B^Q X_n B^Q      (sum_cd (ac|bd) X_n[c,d], Eq. 19)
// with split-precision BF16 operands (x = x_hi + x_lo, three products
// hi*hi + hi*lo + lo*hi), FP32 accumulation in tensor memory within one
// auxiliary chunk and FP64 accumulation across chunks.
#pragma once
#include "common.cuh"

namespace adc {

struct LadderTC;  // owns the BF16 hi/lo copies of B^Q_vv in the GEMM layouts

LadderTC* ladder_tc_create(Ctx& c, const double* Bvv, int naux, int nvir, int aux_chunk);
void ladder_tc_destroy(LadderTC* L);
void ladder_tc_apply(LadderTC& L, Ctx& c, const double* X, long long nmat, double* out);
bool ladder_tc_apply_scratch(LadderTC& L, Ctx& c, const double* X, long long nmat, double* out, void* scratch,
                             size_t bytes);

}  // namespace adc

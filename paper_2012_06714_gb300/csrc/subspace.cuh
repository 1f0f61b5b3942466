// FP64 subspace kernels of the Davidson iteration (Sec. III A step 4): inner
// products of a few long vectors and linear combinations of the basis.  The
// vectors are millions of elements long and there are at most a few hundred
// of them, so both operations stream the vectors once; their cost is set by
// the FP64 FMA rate and HBM bandwidth, not by GEMM tiling.
#pragma once
#include "common.cuh"

namespace adc {

// D[i * nb + j] = sum_{x < n} A[i * lda + x] * B[j * ldb + x]   (i < na, j < nb; D on the device).
// Deterministic: fixed split of x and a fixed reduction order.
void multidot(Ctx& c, int na, const double* A, long long lda, int nb, const double* B, long long ldb, long long n,
              double* D);

// Y[r * ldy + x] = beta * Y[r * ldy + x] + alpha * sum_{i < k} C[r * k + i] * V[i * ldv + x]
// (r < nr, x < n; C on the device).  Y must not overlap V.  beta = 0 does not read Y.
void lincomb(Ctx& c, int nr, int k, const double* C, const double* V, long long ldv, long long n, double alpha, double beta,
             double* Y, long long ldy);

}  // namespace adc

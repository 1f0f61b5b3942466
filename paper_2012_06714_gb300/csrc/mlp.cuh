// Learned Davidson preconditioner (3 -> 64 -> 64 -> 1 MLP correcting the
// diagonal one); see mlp.cu for the definition.
#pragma once
#include "common.cuh"

namespace adc {

int mlp_nweights();
// out[r][x] = R[r][x] (1/(w_r - D_x) + m(f_x)) for nr residuals (device arrays; weights device FP32)
void mlp_precondition(Ctx& c, long long nr, long long dim, long long n1, const double* R, const double* w, const double* D,
                      const float* weights, double* out);
// loss and its gradient over n host samples (d = D - w, block flag, r, t*); grad host [nweights]
double mlp_loss_grad_host(const float* weights, const double* d, const unsigned char* blk, const double* r, const double* t,
                          long long n, float* grad);
// full-batch Adam on the device; weights host [nweights] in/out; loss_hist host [steps] or NULL
void mlp_train_host(float* weights, const double* d, const unsigned char* blk, const double* r, const double* t, long long n,
                    int steps, float lr, double* loss_hist);

}  // namespace adc

// Spin-adapted, density-fitted EA/IP-ADC(n) (n = 2, 3) on one GPU: setup,
// sigma = M X and the Davidson solver behind the C ABI of include/adc.h.
//
// Working equations (closed-shell, spin-adapted; (pq|rs) = sum_Q B^Q_pq B^Q_rs,
// Eq. 19; t_ij^ab the alpha-beta MP amplitudes):
//   t_ij^ab(1) = (ia|jb) / D_ij^ab
//   D t_ij^ab(2) = sum_cd (ac|bd) t_ij^cd + sum_kl (ki|lj) t_kl^ab + W_ij^ab + W_ji^ba
//   D_i^a t_i^a(2) = sum (kc|ad)(2 t_ik^dc - t_ik^cd) - sum (ki|lc)(2 t_kl^ac - t_kl^ca)
// and the 1p-1p / 1h-1h block, coupling and 2p1h / 2h1p blocks written out
// term by term below (each term's four-index form is in its comment).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <numeric>
#include <string>
#include <vector>
#include <atomic>
#include <thread>
#include <unordered_set>

#include "../../include/adc.h"
#include "common.cuh"
#include "ladder_tc.cuh"
#include "mlp.cuh"
#include "subspace.cuh"

using namespace adc;

namespace adc {
void noalloc_prepare();  // ladder_static.cu: resolve the allocation-free ladder's scratch on this device
}

struct adc_handle {
    int o = 0, v = 0, naux = 0, order = 3, kind = ADC_EA;
    adc_options opt{};
    Ctx ctx;
    // device tensors (FP64)
    double *eps = nullptr, *Boo = nullptr, *Bov = nullptr, *Bvv = nullptr;
    double *ovov = nullptr, *oovv = nullptr, *oooo = nullptr, *ooov = nullptr;
    double *t = nullptr, *tau = nullptr, *t_2 = nullptr, *t1_2 = nullptr, *M11 = nullptr, *diag = nullptr;
    // ADC(3) 2p1h / 2h1p block: the two ring terms that share the operand Y_jcb, as one integral
    // combination (EA [i][a][j][c] = 2 (ia|jc) - (ji|ac); IP [i][a][k][b] = (ki|ab) - 2 (ia|kb))
    double* ring2 = nullptr;
    double* t1_3 = nullptr;  // third-order singles (ADC(3) transition moments only), made on first use
    double emp[2] = {0.0, 0.0};  // MP correlation energy E(2), E(3) (Sec. III A step 2)
    double setup_times[8] = {};  // wall seconds of the setup phases (adc_get_tensor "setup_seconds")
    // unrestricted (open-shell) reference: o, v count spin orbitals, the 2p1h / 2h1p basis
    // holds the restricted pairs (i, a<b) / (i<j, a), and the <pq||rs> blocks are kept
    bool unrestricted = false;
    double *g_oovv = nullptr, *g_oooo = nullptr, *g_ooov = nullptr, *g_ovov = nullptr, *g_vovo = nullptr,
           *g_vooo = nullptr, *m12 = nullptr;
    int* pair_idx = nullptr;  // [3][npairs] (i, a, b) for EA, (i, j, a) for IP
    LadderTC* tc = nullptr;  // tensor-core ladder state (BF16x3 operands of B^Q_vv; open shells: the alpha block)
    LadderTC* tc_b = nullptr;  // open shells: the beta virtual block's ladder state
    int nva = 0;               // open shells: alpha virtual spin orbitals (the first nva of the v)
    // tensor-core ladder arithmetic: Davidson sigma, the setup ladder of t, and
    // the final refinement of converged roots
    // (sigma: partial sums promoted every 16 K blocks, drift <= ~3e-6 relative;
    // refinement and the IP setup: every K block, drift ~4e-7; the EA setup: GEMM1
    // every 2 and GEMM2 every 8 K blocks, Richardson-extrapolated to t2(2) within
    // 4e-7 relative of FP64 at nvir 180 and 960 -- as close as every-block promotion
    // and 22% faster)
    LadderMode lm_sigma{2, 0, 16}, lm_setup{2, 1, 1}, lm_refine{2, 1, 1};
    bool refining = false;  // sigma evaluates with lm_refine
    int cmode_setup = 0, cmode_sigma = 0, cmode_refine = 0;  // Ctx::gemm_mode in setup / sigma / refinement
    std::vector<double> X_last;             // spectroscopic amplitudes [nroots][nmo] of the last adc_davidson
    float* mlp_w = nullptr;                 // learned preconditioner weights (device), NULL: diagonal
    double* Lt = nullptr;    // sum_cd (ac|bd) t_kl^cd, shared by t2(2) and the EA 1p-1p block (setup only,
                             // unless the 1p-1p block is applied on the fly)
    // 1p-1p / 1h-1h block applied on the fly (m11_on_the_fly): small intermediates of step 2
    double *otf_g = nullptr, *otf_Hq = nullptr, *otf_gz = nullptr, *otf_Zm = nullptr, *otf_U = nullptr;
    // memory-lean layout (option lean; closed-shell EA, mixed precision): the o^2 v^2 constants
    // held in FP32 (f_*; every contraction that reads them is split-BF16 or FP32-accurate, so
    // FP32 storage loses nothing), no tau or ring2 tensor (contractions with them expanded into
    // ones with t and the integrals), operand copies made per call instead of cached, setup's
    // o^2 v^2 temporaries in FP32, and the root-independent parts of the transition moments
    // made at setup
    bool lean = false;
    float *f_t = nullptr, *f_t2 = nullptr, *f_ovov = nullptr, *f_oovv = nullptr;
    float* f_tau = nullptr;  // lean: tau in FP32, only while setup needs it
    // lean: [2][max(o,v)^2] one-particle block and [2][o][v] singles of the transition
    // moments (index: third-order terms included)
    double *spec_Tpp = nullptr, *spec_t1 = nullptr;
    std::vector<void*> owned;
    // sigma captured as CUDA graphs (cuda_graphs): one per block size, on fixed input / output buffers
    struct SigmaGraph {
        long long n = 0;
        double *X = nullptr, *S = nullptr;
        cudaGraphExec_t exec = nullptr;
    };
    std::vector<SigmaGraph> graphs;
    bool graphs_failed = false;  // a capture failed once: sigma runs without graphs on this handle
    cudaStream_t own_stream = nullptr;  // created by adc_setup_batch, destroyed with the handle
    std::string err;
    long long npairs() const {
        return kind == ADC_EA ? (long long)o * v * (v - 1) / 2 : (long long)o * (o - 1) / 2 * v;
    }
    long long dim() const {
        if (unrestricted) return n1() + npairs();
        return kind == ADC_EA ? (long long)v + (long long)o * v * v : (long long)o + (long long)o * o * v;
    }
    int n1() const { return kind == ADC_EA ? v : o; }
    double* dmalloc(size_t n) {
        void* p = dev_alloc(std::max<size_t>(n, 1) * sizeof(double), ctx.stream);
        owned.push_back(p);
        return (double*)p;
    }
    float* fmalloc(size_t n) {
        void* p = dev_alloc(std::max<size_t>(n, 1) * sizeof(float), ctx.stream);
        owned.push_back(p);
        return (float*)p;
    }
    // release one owned buffer before the handle ends (stream-ordered)
    void dfree(void* p) {
        if (!p) return;
        auto it = std::find(owned.begin(), owned.end(), p);
        if (it == owned.end()) return;
        owned.erase(it);
        cudaFreeAsync(p, ctx.stream);
    }
    ~adc_handle() {
        if (ctx.stream) cudaStreamSynchronize(ctx.stream);
        for (auto& g : graphs) {
            if (g.exec) cudaGraphExecDestroy(g.exec);
            cudaFree(g.X);
            cudaFree(g.S);
        }
        ladder_tc_destroy(tc);
        ladder_tc_destroy(tc_b);
        for (void* p : owned) cudaFree(p);
        if (ctx.blas) cublasDestroy(ctx.blas);
        if (own_stream) cudaStreamDestroy(own_stream);
    }
};

static thread_local std::string g_setup_error = "no error";  // last adc_setup failure of this host thread

// --------------------------------------------------------------------------
// ADC-specific elementwise kernels
// --------------------------------------------------------------------------
namespace {

inline int grid_for(long long n) {
    long long g = (n + 255) / 256;
    return (int)std::min<long long>(std::max<long long>(g, 1), 152LL * 32);
}
#define GRID_STRIDE(i, n) for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (n); i += (long long)gridDim.x * blockDim.x)

// t[i,j,a,b] = ovov[i,a,j,b] / (e_i + e_j - e_a - e_b)
__global__ void k_make_t(int o, int v, const double* __restrict__ eps, const double* __restrict__ ovov, double* __restrict__ t) {
    long long n = (long long)o * o * v * v;
    GRID_STRIDE(x, n) {
        int b = x % v, a = (x / v) % v, j = (x / ((long long)v * v)) % o, i = x / ((long long)v * v * o);
        double D = eps[i] + eps[j] - eps[o + a] - eps[o + b];
        t[x] = ovov[(((long long)i * v + a) * o + j) * v + b] / D;
    }
}
// P[p] = t[i_p][j_p] (v x v matrices) for the pairs i_p <= j_p
__global__ void k_pairs_gather(long long np, long long vv, int o, const int* __restrict__ pi, const int* __restrict__ pj,
                               const double* __restrict__ t, double* __restrict__ P) {
    GRID_STRIDE(x, np * vv) {
        const long long p = x / vv, e = x - p * vv;
        P[x] = t[((long long)pi[p] * o + pj[p]) * vv + e];
    }
}
// out[i][j] = L[p] and out[j][i] = L[p]^T for the pairs (i, j) = (i_p, j_p): 32 x 32 tiles, the
// transposed copy through shared memory (block 32 x 8; grid over pairs x tiles)
__global__ void k_pairs_scatter(long long np, int v, int o, const int* __restrict__ pi, const int* __restrict__ pj,
                                const double* __restrict__ L, double* __restrict__ out) {
    __shared__ double tile[32][33];
    const long long nt = (v + 31) / 32, per = nt * nt, vv = (long long)v * v;
    for (long long b = blockIdx.x; b < np * per; b += gridDim.x) {
        const long long p = b / per, r = b - p * per;
        const int a0 = (int)(r / nt) * 32, c0 = (int)(r % nt) * 32;
        const int i = pi[p], j = pj[p];
        const double* Lp = L + p * vv;
        double* dij = out + ((long long)i * o + j) * vv;
        double* dji = out + ((long long)j * o + i) * vv;
        for (int y = threadIdx.y; y < 32; y += 8) {
            const int a = a0 + y, c = c0 + threadIdx.x;
            if (a < v && c < v) {
                const double x = Lp[(long long)a * v + c];
                dij[(long long)a * v + c] = x;
                tile[y][threadIdx.x] = x;
            }
        }
        __syncthreads();
        if (i != j)
            for (int y = threadIdx.y; y < 32; y += 8) {
                const int c = c0 + y, a = a0 + threadIdx.x;  // out[j][i][c][a] = L[p][a][c]
                if (a < v && c < v) dji[(long long)c * v + a] = tile[threadIdx.x][y];
            }
        __syncthreads();
    }
}
// X[i,j,a,b] /= D_ij^ab
__global__ void k_div_D2(int o, int v, const double* __restrict__ eps, double* __restrict__ X) {
    long long n = (long long)o * o * v * v;
    GRID_STRIDE(x, n) {
        int b = x % v, a = (x / v) % v, j = (x / ((long long)v * v)) % o, i = x / ((long long)v * v * o);
        X[x] /= eps[i] + eps[j] - eps[o + a] - eps[o + b];
    }
}
__global__ void k_div_D1(int o, int v, const double* __restrict__ eps, double* __restrict__ X) {
    long long n = (long long)o * v;
    GRID_STRIDE(x, n) {
        int a = x % v, i = x / v;
        X[x] /= eps[i] - eps[o + a];
    }
}
// Y~ = 2 Y - P Y on the 2p1h (EA: swap last two) or 2h1p (IP: swap first two) part, nvec blocks
__global__ void k_two_minus_swap(int ea, int o, int v, long long nvec, const double* __restrict__ Y, double* __restrict__ Yt) {
    long long blk = ea ? (long long)o * v * v : (long long)o * o * v;
    long long n = nvec * blk;
    GRID_STRIDE(x, n) {
        long long r = x % blk, base = x - r;
        long long s;
        if (ea) {
            int b = r % v, a = (r / v) % v;
            long long i = r / ((long long)v * v);
            s = (i * v + b) * v + a;
        } else {
            int a = r % v, k = (r / v) % o;
            long long j = r / ((long long)o * v);
            s = ((long long)k * o + j) * v + a;
        }
        Yt[x] = 2.0 * Y[x] - Y[base + s];
    }
}
// full vectors [nvec][dim]: out = S Y (mode 0) or S^-1 Y (mode 1); S = diag(1, 2 - P)
__global__ void k_metric(int ea, int o, int v, long long nvec, const double* __restrict__ Y, double* __restrict__ out, int inverse) {
    long long n1 = ea ? v : o;
    long long blk = ea ? (long long)o * v * v : (long long)o * o * v;
    long long dim = n1 + blk;
    long long n = nvec * dim;
    GRID_STRIDE(x, n) {
        long long r = x % dim, base = x - r;
        if (r < n1) {
            out[x] = Y[x];
            continue;
        }
        long long q = r - n1, s;
        if (ea) {
            int b = q % v, a = (q / v) % v;
            long long i = q / ((long long)v * v);
            s = (i * v + b) * v + a;
        } else {
            int a = q % v, k = (q / v) % o;
            long long j = q / ((long long)o * v);
            s = ((long long)k * o + j) * v + a;
        }
        double y = Y[x], ys = Y[base + n1 + s];
        out[x] = inverse ? (2.0 * y + ys) / 3.0 : 2.0 * y - ys;
    }
}
// zeroth-order 2p1h/2h1p diagonal: EA e_a + e_b - e_i ; IP (M_-) e_i + e_j - e_a
__device__ inline double d22(int ea, int o, int v, const double* eps, long long q) {
    if (ea) {
        int b = q % v, a = (q / v) % v;
        long long i = q / ((long long)v * v);
        return eps[o + a] + eps[o + b] - eps[i];
    } else {
        int a = q % v, k = (q / v) % o;
        long long j = q / ((long long)o * v);
        return eps[j] + eps[k] - eps[o + a];
    }
}
// S2 += d22 * Y2 over nvec blocks
__global__ void k_diag22(int ea, int o, int v, long long nvec, const double* __restrict__ eps, const double* __restrict__ Y2,
                         double* __restrict__ S2) {
    long long blk = ea ? (long long)o * v * v : (long long)o * o * v;
    long long n = nvec * blk;
    GRID_STRIDE(x, n) { S2[x] += d22(ea, o, v, eps, x % blk) * Y2[x]; }
}
// preconditioner diagonal of the applied matrix: [diag(M11), +/- d22]
__global__ void k_diag(int ea, int o, int v, const double* __restrict__ eps, const double* __restrict__ M11, double* __restrict__ D) {
    long long n1 = ea ? v : o;
    long long blk = ea ? (long long)o * v * v : (long long)o * o * v;
    long long n = n1 + blk;
    GRID_STRIDE(x, n) {
        if (x < n1)
            D[x] = M11 ? M11[x * n1 + x] : (ea ? eps[o + x] : -eps[x]);  // no M11: zeroth order
        else
            D[x] = ea ? d22(1, o, v, eps, x - n1) : -d22(0, o, v, eps, x - n1);
    }
}
// s[n][p] = e[p] y[n][p]: the zeroth-order one-particle block applied to nvec vectors
__global__ void k_eps_apply(long long nvec, long long n1, const double* __restrict__ e, const double* __restrict__ y,
                            double* __restrict__ out) {
    GRID_STRIDE(x, nvec * n1) { out[x] = e[x % n1] * y[x]; }
}
// copy strided blocks: out[n][r] = in[n*ldin + off + r]
__global__ void k_gather(long long nvec, long long len, const double* __restrict__ in, long long ldin, long long off,
                         double* __restrict__ out, long long ldout, long long offo, double beta) {
    long long n = nvec * len;
    GRID_STRIDE(x, n) {
        long long r = x % len, k = x / len;
        double val = in[k * ldin + off + r];
        double* dst = out + k * ldout + offo + r;
        *dst = (beta == 0.0) ? val : val + beta * *dst;
    }
}
// Davidson correction: out[r][x] = R[r][x] / (w_r - D[x]) with |w - D| >= 1e-8
__global__ void k_precond(long long nr, long long dim, const double* __restrict__ R, const double* __restrict__ w,
                          const double* __restrict__ D, double* __restrict__ out) {
    long long n = nr * dim;
    GRID_STRIDE(x, n) {
        long long r = x / dim, k = x % dim;
        double den = w[r] - D[k];
        if (fabs(den) < 1e-8) den = den < 0 ? -1e-8 : 1e-8;
        out[x] = R[x] / den;
    }
}
// unit vectors: V[k][idx[k]] = 1
__global__ void k_units(int n, const long long* __restrict__ idx, long long dim, double* __restrict__ V) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) V[(long long)k * dim + idx[k]] = 1.0;
}

// learned-preconditioner samples of one root: for each chosen element x = idx[k],
// d = D_x - w, blk = [x in the 1p/1h block], r = sigma_x - w y_x, t = y_exact_x / ov - y_x
__global__ void k_mlp_samples(long long m, const long long* __restrict__ idx, long long n1, const double* __restrict__ D,
                              double w, const double* __restrict__ sig, const double* __restrict__ y,
                              const double* __restrict__ yex, double inv_ov, double* __restrict__ od,
                              unsigned char* __restrict__ ob, double* __restrict__ orr, double* __restrict__ ot) {
    GRID_STRIDE(k, m) {
        const long long x = idx[k];
        od[k] = D[x] - w;
        ob[k] = x < n1 ? 1 : 0;
        orr[k] = sig[x] - w * y[x];
        ot[k] = yex[x] * inv_ov - y[x];
    }
}

void launch_check(Ctx& c) {
    ++c.kernels;
    ADC_CUDA(cudaGetLastError());
}

// mark/release helper
struct Scope {
    Arena& a;
    Arena::Mark m;
    explicit Scope(Arena& ar) : a(ar), m(ar.mark()) {}
    ~Scope() { a.release(m); }
};

T tn(const double* p, std::initializer_list<long long> d) { return T{p, std::vector<long long>(d), false}; }
T tn(const double* p, const std::vector<long long>& d) { return T{p, d, false}; }
// handle-owned tensor that never changes after setup (its FP32 operand copy may be cached)
T tc(const double* p, std::initializer_list<long long> d) { return T{p, std::vector<long long>(d), true}; }
// handle-owned FP32 tensor (constant)
T tf(const float* p, std::initializer_list<long long> d) { return T{(const double*)p, std::vector<long long>(d), true, true}; }

// An o^2 v^2-sized scratch tensor of setup: FP32 on a lean handle, else FP64.
struct Buf {
    void* p = nullptr;
    bool f32 = false;
    T as(std::initializer_list<long long> d) const { return T{(const double*)p, std::vector<long long>(d), false, f32}; }
};
Buf scratch(Arena& a, long long n, bool f32) {
    Buf b;
    b.f32 = f32;
    b.p = f32 ? a.alloc((size_t)n * sizeof(float)) : (void*)a.dalloc((size_t)n);
    return b;
}
void ein(Ctx& c, const char* spec, double alpha, const T& A, const T& B, double beta, const Buf& C,
         const std::vector<long long>& d) {
    if (C.f32)
        einsum(c, spec, alpha, A, B, beta, (float*)C.p, d);
    else
        einsum(c, spec, alpha, A, B, beta, (double*)C.p, d);
}
// C = alpha * permute(X) + beta * C (output axis j = input axis perm[j])
void perm_into(Ctx& c, const T& X, std::initializer_list<int> perm, const Buf& C, double alpha, double beta) {
    Shape s{(int)X.dims.size(), {}};
    for (int j = 0; j < s.nd; ++j) s.d[j] = X.dims[j];
    std::vector<int> p(perm);
    permute_any(c, X.p, X.f32, s, p.data(), C.p, C.f32, alpha, beta);
}

}  // namespace

// The o^2 v^2 operands: FP32 on a lean handle once converted, else FP64.  cst marks them
// constant (sigma: operand copies may be cached); setup passes false.
static T op_t(const adc_handle* h, bool cst) {
    const long long o = h->o, v = h->v;
    if (h->f_t) return tf(h->f_t, {o, o, v, v});
    return cst ? tc(h->t, {o, o, v, v}) : tn(h->t, {o, o, v, v});
}
static T op_t2(const adc_handle* h, bool cst) {
    const long long o = h->o, v = h->v;
    if (h->f_t2) return tf(h->f_t2, {o, o, v, v});
    return cst ? tc(h->t_2, {o, o, v, v}) : tn(h->t_2, {o, o, v, v});
}
static T op_tau(const adc_handle* h, bool cst) {
    const long long o = h->o, v = h->v;
    if (h->f_tau) return tf(h->f_tau, {o, o, v, v});
    if (!h->tau) throw Error(ADC_ERR_ARG, "tau is not held by this handle");
    return cst ? tc(h->tau, {o, o, v, v}) : tn(h->tau, {o, o, v, v});
}
static T op_ovov(const adc_handle* h, bool cst) {
    const long long o = h->o, v = h->v;
    if (h->f_ovov) return tf(h->f_ovov, {o, v, o, v});
    return cst ? tc(h->ovov, {o, v, o, v}) : tn(h->ovov, {o, v, o, v});
}
static T op_oovv(const adc_handle* h, bool cst) {
    const long long o = h->o, v = h->v;
    if (h->f_oovv) return tf(h->f_oovv, {o, o, v, v});
    return cst ? tc(h->oovv, {o, o, v, v}) : tn(h->oovv, {o, o, v, v});
}
// FP32 copy of an owned FP64 tensor; the FP64 one is released
static float* to_f32(adc_handle* h, double*& src, long long n) {
    float* dst = h->fmalloc(n);
    Shape s{1, {n}};
    int id[1] = {0};
    permute_any(h->ctx, src, false, s, id, dst, true, 1.0, 0.0);
    h->dfree(src);
    src = nullptr;
    return dst;
}

// --------------------------------------------------------------------------
// DF ladder: out[n] += sum_Q B^Q_vv X_n B^Q_vv for nmat v x v matrices
//   (sum_cd (ac|bd) X_n[c,d]; the vvvv integral is never formed)
// --------------------------------------------------------------------------
static void ladder_open_shell(adc_handle* h, const double* F, long long nmat, double* out, const LadderMode& md);

static void ladder(adc_handle* h, const double* X, long long nmat, double* out, const LadderMode& md) {
    Ctx& c = h->ctx;
    const long long v = h->v;
    if (h->unrestricted && h->tc) {
        ladder_open_shell(h, X, nmat, out, md);
        return;
    }
    if (h->opt.precision != ADC_PREC_FP64 && h->tc) {
        ladder_tc_apply(*h->tc, c, X, nmat, out, md);
        return;
    }
    Scope sc(c.arena);
    // chunk the matrices so the intermediate stays modest
    long long per = std::max<long long>(1, std::min<long long>(nmat, (256LL << 20) / (8 * v * v)));
    double* W = c.arena.dalloc((size_t)(per * v * v));
    for (long long n0 = 0; n0 < nmat; n0 += per) {
        long long nn = std::min(per, nmat - n0);
        for (int Q = 0; Q < h->naux; ++Q) {
            const double* BQ = h->Bvv + (long long)Q * v * v;
            // W[(n,c), b] = X[(n,c), d] B^Q[d, b]
            gemm(c, false, false, nn * v, v, v, 1.0, X + n0 * v * v, v, 0, BQ, v, 0, 0.0, W, v, 0, 1);
            // out_n[a, b] += B^Q[a, c] W_n[c, b]
            gemm(c, false, false, v, v, v, 1.0, BQ, v, 0, W, v, v * v, 1.0, out + n0 * v * v, v, v * v, nn);
        }
    }
}

// --------------------------------------------------------------------------
// setup (Sec. III A steps 1-3)
// --------------------------------------------------------------------------
static void sym_add(adc_handle* h, const double* X, double* M, int n, double alpha) {
    // M += alpha (X + X^T)
    Ctx& c = h->ctx;
    axpby(c, (long long)n * n, alpha, X, 1.0, M);
    Shape s{2, {n, n}};
    int perm[2] = {1, 0};
    permute(c, X, s, perm, M, alpha, 1.0);
}

// XL: the ladder term -sum t_kl^ac [L_kl^bc - 1/2 L_kl^cb] (v x v), formed by setup while the
// ladder of t was alive; NULL: formed here from h->Lt
static void setup_m11_ea(adc_handle* h, const double* XL) {
    Ctx& c = h->ctx;
    const long long o = h->o, v = h->v, Q = h->naux;
    Scope sc(c.arena);
    double* M = h->M11;
    double* X = c.arena.dalloc(v * v);
    const T T4 = op_t(h, false), OVOV = op_ovov(h, false), OOVV = op_oovv(h, false);
    // second order: -sum t_kl^ac [(kb|lc) - 1/2 (kc|lb)] + (a<->b)
    einsum(c, "klac,kblc->ab", -1.0, T4, OVOV, 0.0, X, {v, v});
    einsum(c, "klac,kclb->ab", 0.5, T4, OVOV, 1.0, X, {v, v});
    sym_add(h, X, M, (int)v, 1.0);
    if (h->order < 3) return;
    const double* t1 = h->t1_2;
    const T T2 = op_t2(h, false);
    // t1(2): sum_kc t_k^c [2 (kc|ab) - (kb|ac)] + (a<->b)
    double* g = c.arena.dalloc(Q);
    einsum(c, "Qkc,kc->Q", 1.0, tn(h->Bov, {Q, o, v}), tn(t1, {o, v}), 0.0, g, {Q});
    einsum(c, "Q,Qab->ab", 2.0, tn(g, {Q}), tn(h->Bvv, {Q, v, v}), 0.0, X, {v, v});
    double* Hq = c.arena.dalloc(Q * o * v);
    einsum(c, "kc,Qac->Qka", 1.0, tn(t1, {o, v}), tn(h->Bvv, {Q, v, v}), 0.0, Hq, {Q, o, v});
    einsum(c, "Qkb,Qka->ab", -1.0, tn(h->Bov, {Q, o, v}), tn(Hq, {Q, o, v}), 1.0, X, {v, v});
    // t2(2): same shape as second order
    einsum(c, "klac,kblc->ab", -1.0, T2, OVOV, 1.0, X, {v, v});
    einsum(c, "klac,kclb->ab", 0.5, T2, OVOV, 1.0, X, {v, v});
    // vvvv, one open line: -sum t_kl^ac [L_kl^bc - 1/2 L_kl^cb], L_kl = sum_cd (bc..) ladder of t
    if (XL) {
        axpby(c, v * v, 1.0, XL, 1.0, X);
    } else {
        const T L = tn(h->Lt, {o, o, v, v});
        einsum(c, "klac,klbc->ab", -1.0, T4, L, 1.0, X, {v, v});
        einsum(c, "klac,klcb->ab", 0.5, T4, L, 1.0, X, {v, v});
    }
    // ring with the open lines on the amplitudes (G_A with t_km^ac, G_B with t_km^ca):
    //   u1 = -t/2 + t^T, u2 = t - 2 t^T, u3 = t - t^T/2 (t^T swaps the virtual pair).
    // u is held as [l][d][m][c] (the order in which it enters the GEMMs), G and GB as
    // [k][b][m][c] (the order in which the GEMMs write them); FP32 on a lean handle.
    {
        Scope rs(c.arena);
        const long long n4 = o * o * v * v;
        Buf u = scratch(c.arena, n4, h->lean), G = scratch(c.arena, n4, h->lean), GB = scratch(c.arena, n4, h->lean);
        auto make_u = [&](double a, double b) {  // u[l][d][m][c] = a t_lm^cd + b t_lm^dc
            perm_into(c, T4, {0, 3, 1, 2}, u, a, 0.0);
            perm_into(c, T4, {0, 2, 1, 3}, u, b, 1.0);
        };
        const T U = u.as({o, v, o, v});
        // G_A = sum_ld (kl|db) u1_lm^cd + sum_ld (kb|ld) u2_lm^cd
        make_u(-0.5, 1.0);
        ein(c, "kldb,ldmc->kbmc", 1.0, OOVV, U, 0.0, G, {o, v, o, v});
        ein(c, "kbld,ldmc->kbmc", 1.0, OVOV, U, 0.0, GB, {o, v, o, v});  // u1 part of G_B
        make_u(1.0, -2.0);
        ein(c, "kbld,ldmc->kbmc", 1.0, OVOV, U, 1.0, G, {o, v, o, v});
        make_u(1.0, -0.5);
        ein(c, "kldb,ldmc->kbmc", 1.0, OOVV, U, 1.0, GB, {o, v, o, v});
        einsum(c, "kmac,kbmc->ab", 1.0, T4, G.as({o, v, o, v}), 1.0, X, {v, v});
        einsum(c, "kmca,kbmc->ab", 1.0, T4, GB.as({o, v, o, v}), 1.0, X, {v, v});
    }
    sym_add(h, X, M, (int)v, 1.0);
    // vvvv with both lines on the integral: sum_cd [2 (ab|cd) - (ad|cb)] (2X - X')_cd
    double* Z = c.arena.dalloc(v * v);
    einsum(c, "klce,klde->cd", 2.0, T4, T4, 0.0, Z, {v, v});
    einsum(c, "klce,kled->cd", -1.0, T4, T4, 1.0, Z, {v, v});
    einsum(c, "Qcd,cd->Q", 1.0, tn(h->Bvv, {Q, v, v}), tn(Z, {v, v}), 0.0, g, {Q});
    einsum(c, "Q,Qab->ab", 2.0, tn(g, {Q}), tn(h->Bvv, {Q, v, v}), 1.0, M, {v, v});
    double* H2 = c.arena.dalloc(Q * v * v);
    einsum(c, "Qad,cd->Qac", 1.0, tn(h->Bvv, {Q, v, v}), tn(Z, {v, v}), 0.0, H2, {Q, v, v});
    einsum(c, "Qac,Qcb->ab", -1.0, tn(H2, {Q, v, v}), tn(h->Bvv, {Q, v, v}), 1.0, M, {v, v});
    // ring with both lines on the integral: -sum_kl [2 (kl|ab) - (kb|la)] (2U - U')_kl
    double* U = c.arena.dalloc(o * o);
    einsum(c, "kmcd,lmcd->kl", 2.0, T4, T4, 0.0, U, {o, o});
    einsum(c, "kmcd,lmdc->kl", -1.0, T4, T4, 1.0, U, {o, o});
    einsum(c, "klab,kl->ab", -2.0, OOVV, tn(U, {o, o}), 1.0, M, {v, v});
    einsum(c, "kbla,kl->ab", 1.0, OVOV, tn(U, {o, o}), 1.0, M, {v, v});
}

static void setup_m11_ip(adc_handle* h) {
    // paper's M_- 1h-1h block, negated at the end (the library applies -M_-)
    Ctx& c = h->ctx;
    const long long o = h->o, v = h->v;
    Scope sc(c.arena);
    double* M = h->M11;
    double* X = c.arena.dalloc(o * o);
    const double* t = h->t;
    einsum(c, "ilcd,jcld->ij", 1.0, tn(t, {o, o, v, v}), tn(h->ovov, {o, v, o, v}), 0.0, X, {o, o});
    einsum(c, "ilcd,jdlc->ij", -0.5, tn(t, {o, o, v, v}), tn(h->ovov, {o, v, o, v}), 1.0, X, {o, o});
    sym_add(h, X, M, (int)o, 1.0);
    if (h->order >= 3) {
        const double *t2 = h->t_2, *t1 = h->t1_2;
        // t1(2): sum_kc t_k^c [2 (ck|ij) - (cj|ik)]
        einsum(c, "kc,ijkc->ij", 2.0, tn(t1, {o, v}), tn(h->ooov, {o, o, o, v}), 0.0, X, {o, o});
        einsum(c, "kc,ikjc->ij", -1.0, tn(t1, {o, v}), tn(h->ooov, {o, o, o, v}), 1.0, X, {o, o});
        // t2(2): sum t2_ik^cd [(cj|dk) - 1/2 (ck|dj)]
        einsum(c, "ikcd,jckd->ij", 1.0, tn(t2, {o, o, v, v}), tn(h->ovov, {o, v, o, v}), 1.0, X, {o, o});
        einsum(c, "ikcd,kcjd->ij", -0.5, tn(t2, {o, o, v, v}), tn(h->ovov, {o, v, o, v}), 1.0, X, {o, o});
        // oooo with one open line: sum t_ik^cd (jl|km)(t_lm^cd - 1/2 t_lm^dc)
        double* u = c.arena.dalloc(o * o * v * v);
        double* G = c.arena.dalloc(o * o * v * v);
        Shape s4{4, {o, o, v, v}};
        int swp[4] = {0, 1, 3, 2};
        auto make_u = [&](double a, double b) {
            axpby(c, o * o * v * v, a, t, 0.0, u);
            permute(c, t, s4, swp, u, b, 1.0);
        };
        make_u(1.0, -0.5);
        einsum(c, "jlkm,lmcd->jkcd", 1.0, tn(h->oooo, {o, o, o, o}), tn(u, {o, o, v, v}), 0.0, G, {o, o, v, v});
        einsum(c, "ikcd,jkcd->ij", 1.0, tn(t, {o, o, v, v}), tn(G, {o, o, v, v}), 1.0, X, {o, o});
        // ring with open lines on the amplitudes: w1 = t/2 - t^T, w2 = -t + 2 t^T, w3 = -t + t^T/2
        double* GB = c.arena.dalloc(o * o * v * v);
        make_u(0.5, -1.0);
        einsum(c, "ljcd,klde->kecj", 1.0, tn(h->oovv, {o, o, v, v}), tn(u, {o, o, v, v}), 0.0, G, {o, v, v, o});
        einsum(c, "jcld,klde->kecj", 1.0, tn(h->ovov, {o, v, o, v}), tn(u, {o, o, v, v}), 0.0, GB, {o, v, v, o});
        make_u(-1.0, 2.0);
        einsum(c, "jcld,klde->kecj", 1.0, tn(h->ovov, {o, v, o, v}), tn(u, {o, o, v, v}), 1.0, G, {o, v, v, o});
        make_u(-1.0, 0.5);
        einsum(c, "ljcd,klde->kecj", 1.0, tn(h->oovv, {o, o, v, v}), tn(u, {o, o, v, v}), 1.0, GB, {o, v, v, o});
        einsum(c, "ikce,kecj->ij", 1.0, tn(t, {o, o, v, v}), tn(G, {o, v, v, o}), 1.0, X, {o, o});
        einsum(c, "ikec,kecj->ij", 1.0, tn(t, {o, o, v, v}), tn(GB, {o, v, v, o}), 1.0, X, {o, o});
        sym_add(h, X, M, (int)o, 1.0);
        // oooo with both lines on the integral: -[2 (ij|kl) - (il|kj)] (2U - U')_kl
        double* U = c.arena.dalloc(o * o);
        einsum(c, "kmcd,lmcd->kl", 2.0, tn(t, {o, o, v, v}), tn(t, {o, o, v, v}), 0.0, U, {o, o});
        einsum(c, "kmcd,lmdc->kl", -1.0, tn(t, {o, o, v, v}), tn(t, {o, o, v, v}), 1.0, U, {o, o});
        einsum(c, "ijkl,kl->ij", -2.0, tn(h->oooo, {o, o, o, o}), tn(U, {o, o}), 1.0, M, {o, o});
        einsum(c, "ilkj,kl->ij", 1.0, tn(h->oooo, {o, o, o, o}), tn(U, {o, o}), 1.0, M, {o, o});
        // ring with both lines on the integral: [2 (cd|ij) - (cj|id)] (2X - X')_cd
        double* Z = c.arena.dalloc(v * v);
        einsum(c, "klce,klde->cd", 2.0, tn(t, {o, o, v, v}), tn(t, {o, o, v, v}), 0.0, Z, {v, v});
        einsum(c, "klce,kled->cd", -1.0, tn(t, {o, o, v, v}), tn(t, {o, o, v, v}), 1.0, Z, {v, v});
        einsum(c, "ijcd,cd->ij", 2.0, tn(h->oovv, {o, o, v, v}), tn(Z, {v, v}), 1.0, M, {o, o});
        einsum(c, "jcid,cd->ij", -1.0, tn(h->ovov, {o, v, o, v}), tn(Z, {v, v}), 1.0, M, {o, o});
    }
    axpby(c, o * o, 0.0, M, -1.0, M);  // apply -M_-
}

// --------------------------------------------------------------------------
// The 1p-1p (EA) / 1h-1h (IP) block applied on the fly (Sec. III A: instead of
// precomputing the block in step 3, its contribution sum_b M_ab Y_b / sum_j
// M_ij Y_j is recomputed in every sigma from intermediates).  Each term of
// setup_m11_ea / setup_m11_ip is contracted with the vector first: a term
// X_ab = sum A_..a.. C_..b.. enters through (X + X^T) y = X y + X^T y, and
// every integral or amplitude of the term meets y before the other factor.
// Step-2 intermediates kept for it: the ladder of t (EA), and the small
// g_Q = sum_kc B^Q_kc t_k^c(2), Hq_Qka = sum_c t_k^c(2) B^Q_ac, Zm_cd =
// sum t t (v x v), gz_Q = sum_cd B^Q_cd Zm_cd and U_kl = sum t t (o x o).
// --------------------------------------------------------------------------
static void setup_m11_otf(adc_handle* h) {
    Ctx& c = h->ctx;
    const long long o = h->o, v = h->v, Q = h->naux;
    if (h->order < 3) return;
    const T T4 = tn(h->t, {o, o, v, v});
    h->otf_Zm = h->dmalloc(v * v);
    einsum(c, "klce,klde->cd", 2.0, T4, T4, 0.0, h->otf_Zm, {v, v});
    einsum(c, "klce,kled->cd", -1.0, T4, T4, 1.0, h->otf_Zm, {v, v});
    h->otf_U = h->dmalloc(o * o);
    einsum(c, "kmcd,lmcd->kl", 2.0, T4, T4, 0.0, h->otf_U, {o, o});
    einsum(c, "kmcd,lmdc->kl", -1.0, T4, T4, 1.0, h->otf_U, {o, o});
    if (h->kind != ADC_EA) return;
    h->otf_g = h->dmalloc(Q);
    einsum(c, "Qkc,kc->Q", 1.0, tn(h->Bov, {Q, o, v}), tn(h->t1_2, {o, v}), 0.0, h->otf_g, {Q});
    h->otf_Hq = h->dmalloc(Q * o * v);
    einsum(c, "kc,Qac->Qka", 1.0, tn(h->t1_2, {o, v}), tn(h->Bvv, {Q, v, v}), 0.0, h->otf_Hq, {Q, o, v});
    h->otf_gz = h->dmalloc(Q);
    einsum(c, "Qcd,cd->Q", 1.0, tn(h->Bvv, {Q, v, v}), tn(h->otf_Zm, {v, v}), 0.0, h->otf_gz, {Q});
}

// s1 = M_+11 y1 (EA, n vectors of length v), terms as in setup_m11_ea
static void m11_apply_otf_ea(adc_handle* h, const double* y1, double* s1, long long n) {
    Ctx& c = h->ctx;
    const long long o = h->o, v = h->v, Q = h->naux;
    Scope sc(c.arena);
    k_eps_apply<<<grid_for(n * v), 256, 0, c.stream>>>(n, v, h->eps + o, y1, s1);  // zeroth order
    launch_check(c);
    const T Y = tn(y1, {n, v});
    const T ovov = tc(h->ovov, {o, v, o, v}), oovv = tc(h->oovv, {o, o, v, v});
    const std::vector<long long> d4{n, o, o, v};
    double* W = c.arena.dalloc(n * o * o * v);
    double* Z = c.arena.dalloc(n * o * o * v);
    // X_ab = -sum t_kl^ac [(kb|lc) - 1/2 (kc|lb)] for t = t2(1) and (ADC(3)) t2(2)
    auto second = [&](const double* tt) {
        const T T4 = tc(tt, {o, o, v, v});
        einsum(c, "kblc,nb->nklc", -1.0, ovov, Y, 0.0, W, d4);
        einsum(c, "kclb,nb->nklc", 0.5, ovov, Y, 1.0, W, d4);
        einsum(c, "klac,nklc->na", 1.0, T4, tn(W, {n, o, o, v}), 1.0, s1, {n, v});
        einsum(c, "klbc,nb->nklc", 1.0, T4, Y, 0.0, Z, d4);  // Z_klc = sum_b t_kl^bc y_b
        einsum(c, "nklc,kalc->na", -1.0, tn(Z, {n, o, o, v}), ovov, 1.0, s1, {n, v});
        einsum(c, "nklc,kcla->na", 0.5, tn(Z, {n, o, o, v}), ovov, 1.0, s1, {n, v});
    };
    second(h->t);
    if (h->order < 3) return;
    second(h->t_2);
    const T T4 = tc(h->t, {o, o, v, v}), Bvv = tc(h->Bvv, {Q, v, v}), Bov = tc(h->Bov, {Q, o, v});
    // t1(2): X_ab = 2 sum_Q g_Q B^Q_ab - sum_Qk B^Q_kb Hq_Qka
    double* hq = c.arena.dalloc(n * Q * v);  // hq_Qa = sum_b B^Q_ab y_b
    einsum(c, "Qab,nb->nQa", 1.0, Bvv, Y, 0.0, hq, {n, Q, v});
    const T HQ = tn(hq, {n, Q, v});
    double* p = c.arena.dalloc(n * Q * o);
    einsum(c, "Q,nQa->na", 4.0, tc(h->otf_g, {Q}), HQ, 1.0, s1, {n, v});  // X y and X^T y
    einsum(c, "Qkb,nb->nQk", 1.0, Bov, Y, 0.0, p, {n, Q, o});
    einsum(c, "Qka,nQk->na", -1.0, tc(h->otf_Hq, {Q, o, v}), tn(p, {n, Q, o}), 1.0, s1, {n, v});
    einsum(c, "Qkb,nb->nQk", 1.0, tc(h->otf_Hq, {Q, o, v}), Y, 0.0, p, {n, Q, o});
    einsum(c, "Qka,nQk->na", -1.0, Bov, tn(p, {n, Q, o}), 1.0, s1, {n, v});
    // ladder of t: X_ab = -sum t_kl^ac [L_kl^bc - 1/2 L_kl^cb]
    const T L = tc(h->Lt, {o, o, v, v});
    einsum(c, "klbc,nb->nklc", -1.0, L, Y, 0.0, W, d4);
    einsum(c, "klcb,nb->nklc", 0.5, L, Y, 1.0, W, d4);
    einsum(c, "klac,nklc->na", 1.0, T4, tn(W, {n, o, o, v}), 1.0, s1, {n, v});
    einsum(c, "klbc,nb->nklc", 1.0, T4, Y, 0.0, Z, d4);  // Z_klc = sum_b t_kl^bc y_b (also the ring's Zt1)
    const T ZT = tn(Z, {n, o, o, v});
    einsum(c, "nklc,klac->na", -1.0, ZT, L, 1.0, s1, {n, v});
    einsum(c, "nklc,klca->na", 0.5, ZT, L, 1.0, s1, {n, v});
    // ring: X_ab = sum t_km^ac G_kmcb + t_km^ca GB_kmcb with G = (kl|db) u1 + (kb|ld) u2,
    // GB = (kb|ld) u1 + (kl|db) u3; u1 = -t/2 + t^T, u2 = t - 2 t^T, u3 = t - t^T/2
    double* A1 = c.arena.dalloc(n * o * o * v);  // sum_b (kl|db) y_b
    double* A2 = c.arena.dalloc(n * o * o * v);  // sum_b (kb|ld) y_b
    einsum(c, "kldb,nb->nkld", 1.0, oovv, Y, 0.0, A1, d4);
    einsum(c, "kbld,nb->nkld", 1.0, ovov, Y, 0.0, A2, d4);
    const T A1T = tn(A1, {n, o, o, v}), A2T = tn(A2, {n, o, o, v});
    // W <- G y, Z2 <- GB y (u contracted as a t + b t^T)
    double* Z2 = c.arena.dalloc(n * o * o * v);
    einsum(c, "nkld,lmcd->nkmc", -0.5, A1T, T4, 0.0, W, d4);
    einsum(c, "nkld,lmdc->nkmc", 1.0, A1T, T4, 1.0, W, d4);
    einsum(c, "nkld,lmcd->nkmc", 1.0, A2T, T4, 1.0, W, d4);
    einsum(c, "nkld,lmdc->nkmc", -2.0, A2T, T4, 1.0, W, d4);
    einsum(c, "nkld,lmcd->nkmc", -0.5, A2T, T4, 0.0, Z2, d4);
    einsum(c, "nkld,lmdc->nkmc", 1.0, A2T, T4, 1.0, Z2, d4);
    einsum(c, "nkld,lmcd->nkmc", 1.0, A1T, T4, 1.0, Z2, d4);
    einsum(c, "nkld,lmdc->nkmc", -0.5, A1T, T4, 1.0, Z2, d4);
    einsum(c, "kmac,nkmc->na", 1.0, T4, tn(W, {n, o, o, v}), 1.0, s1, {n, v});
    einsum(c, "kmca,nkmc->na", 1.0, T4, tn(Z2, {n, o, o, v}), 1.0, s1, {n, v});
    // X^T y through Zt1 = Z and Zt2_kmc = sum_b t_km^cb y_b: sum (kl|da) Ra_kld + (ka|ld) Rb_kld,
    // Ra = R(Zt1, u1) + R(Zt2, u3), Rb = R(Zt1, u2) + R(Zt2, u1), R(Z, u)_kld = sum_mc Z_kmc u_lm^cd
    double* Zt2 = c.arena.dalloc(n * o * o * v);
    einsum(c, "kmcb,nb->nkmc", 1.0, T4, Y, 0.0, Zt2, d4);
    const T Z2T = tn(Zt2, {n, o, o, v});
    double* Ra = W;
    double* Rb = Z2;
    einsum(c, "nkmc,lmcd->nkld", -0.5, ZT, T4, 0.0, Ra, d4);
    einsum(c, "nkmc,lmdc->nkld", 1.0, ZT, T4, 1.0, Ra, d4);
    einsum(c, "nkmc,lmcd->nkld", 1.0, Z2T, T4, 1.0, Ra, d4);
    einsum(c, "nkmc,lmdc->nkld", -0.5, Z2T, T4, 1.0, Ra, d4);
    einsum(c, "nkmc,lmcd->nkld", 1.0, ZT, T4, 0.0, Rb, d4);
    einsum(c, "nkmc,lmdc->nkld", -2.0, ZT, T4, 1.0, Rb, d4);
    einsum(c, "nkmc,lmcd->nkld", -0.5, Z2T, T4, 1.0, Rb, d4);
    einsum(c, "nkmc,lmdc->nkld", 1.0, Z2T, T4, 1.0, Rb, d4);
    einsum(c, "klda,nkld->na", 1.0, oovv, tn(Ra, {n, o, o, v}), 1.0, s1, {n, v});
    einsum(c, "kald,nkld->na", 1.0, ovov, tn(Rb, {n, o, o, v}), 1.0, s1, {n, v});
    // both lines on the integral: M_ab += 2 sum_Q gz_Q B^Q_ab - sum_Q (B^Q Zm^T B^Q)_ab
    einsum(c, "Q,nQa->na", 2.0, tc(h->otf_gz, {Q}), HQ, 1.0, s1, {n, v});
    double* w = c.arena.dalloc(n * Q * v);
    einsum(c, "nQc,cd->nQd", 1.0, HQ, tc(h->otf_Zm, {v, v}), 0.0, w, {n, Q, v});
    einsum(c, "Qad,nQd->na", -1.0, Bvv, tn(w, {n, Q, v}), 1.0, s1, {n, v});
    // M_ab += -2 sum_kl (kl|ab) U_kl + sum_kl (kb|la) U_kl   (A1, A2 hold the y-contracted integrals)
    einsum(c, "kl,nkla->na", -2.0, tc(h->otf_U, {o, o}), A1T, 1.0, s1, {n, v});
    einsum(c, "kl,nkla->na", 1.0, tc(h->otf_U, {o, o}), A2T, 1.0, s1, {n, v});
}

// s1 += M_-11 y1 (the paper's IP block, before the library's sign flip; n vectors of
// length o), terms as in setup_m11_ip
static void m11_apply_otf_ip(adc_handle* h, const double* y1, double* s1, long long n) {
    Ctx& c = h->ctx;
    const long long o = h->o, v = h->v;
    Scope sc(c.arena);
    double* s0 = c.arena.dalloc(n * o);
    k_eps_apply<<<grid_for(n * o), 256, 0, c.stream>>>(n, o, h->eps, y1, s0);  // zeroth order
    launch_check(c);
    axpby(c, n * o, 1.0, s0, 1.0, s1);
    const T Y = tn(y1, {n, o});
    const T ovov = tc(h->ovov, {o, v, o, v}), oovv = tc(h->oovv, {o, o, v, v}), oooo = tc(h->oooo, {o, o, o, o}),
            ooov = tc(h->ooov, {o, o, o, v});
    const std::vector<long long> d4{n, o, v, v};
    double* W = c.arena.dalloc(n * o * v * v);
    double* Z = c.arena.dalloc(n * o * v * v);
    // X_ij = sum t_il^cd [(jc|ld) - 1/2 (jd|lc)]
    {
        const T T4 = tc(h->t, {o, o, v, v});
        einsum(c, "jcld,nj->nlcd", 1.0, ovov, Y, 0.0, W, d4);
        einsum(c, "jdlc,nj->nlcd", -0.5, ovov, Y, 1.0, W, d4);
        einsum(c, "ilcd,nlcd->ni", 1.0, T4, tn(W, d4), 1.0, s1, {n, o});
        einsum(c, "jlcd,nj->nlcd", 1.0, T4, Y, 0.0, Z, d4);
        einsum(c, "icld,nlcd->ni", 1.0, ovov, tn(Z, d4), 1.0, s1, {n, o});
        einsum(c, "idlc,nlcd->ni", -0.5, ovov, tn(Z, d4), 1.0, s1, {n, o});
    }
    if (h->order < 3) return;
    const T T4 = tc(h->t, {o, o, v, v}), T2 = tc(h->t_2, {o, o, v, v}), T1 = tc(h->t1_2, {o, v});
    // t1(2): X_ij = 2 sum_kc t_k^c (ij|kc) - sum_kc t_k^c (ik|jc)
    {
        double* e = c.arena.dalloc(n * o * o * v);
        const T E = tn(e, {n, o, o, v});
        einsum(c, "ijkc,nj->nikc", 2.0, ooov, Y, 0.0, e, {n, o, o, v});
        einsum(c, "ikjc,nj->nikc", -1.0, ooov, Y, 1.0, e, {n, o, o, v});
        einsum(c, "kc,nikc->ni", 1.0, T1, E, 1.0, s1, {n, o});
        einsum(c, "jikc,nj->nikc", 2.0, ooov, Y, 0.0, e, {n, o, o, v});
        einsum(c, "jkic,nj->nikc", -1.0, ooov, Y, 1.0, e, {n, o, o, v});
        einsum(c, "kc,nikc->ni", 1.0, T1, E, 1.0, s1, {n, o});
    }
    // t2(2): X_ij = sum t2_ik^cd [(jc|kd) - 1/2 (kc|jd)]
    einsum(c, "jckd,nj->nkcd", 1.0, ovov, Y, 0.0, W, d4);
    einsum(c, "kcjd,nj->nkcd", -0.5, ovov, Y, 1.0, W, d4);
    einsum(c, "ikcd,nkcd->ni", 1.0, T2, tn(W, d4), 1.0, s1, {n, o});
    einsum(c, "jkcd,nj->nkcd", 1.0, T2, Y, 0.0, Z, d4);
    einsum(c, "ickd,nkcd->ni", 1.0, ovov, tn(Z, d4), 1.0, s1, {n, o});
    einsum(c, "kcid,nkcd->ni", -0.5, ovov, tn(Z, d4), 1.0, s1, {n, o});
    // oooo, one open line: X_ij = sum t_ik^cd G_jkcd, G_jkcd = sum_lm (jl|km) u_lm^cd, u = t - t^T/2
    {
        double* O4 = c.arena.dalloc(n * o * o * o);
        const T O4T = tn(O4, {n, o, o, o});
        einsum(c, "jlkm,nj->nlkm", 1.0, oooo, Y, 0.0, O4, {n, o, o, o});
        einsum(c, "nlkm,lmcd->nkcd", 1.0, O4T, T4, 0.0, W, d4);
        einsum(c, "nlkm,lmdc->nkcd", -0.5, O4T, T4, 1.0, W, d4);
        einsum(c, "ikcd,nkcd->ni", 1.0, T4, tn(W, d4), 1.0, s1, {n, o});
        einsum(c, "jkcd,nj->nkcd", 1.0, T4, Y, 0.0, Z, d4);  // Zt_kcd = sum_j t_jk^cd y_j
        einsum(c, "nkcd,lmcd->nklm", 1.0, tn(Z, d4), T4, 0.0, O4, {n, o, o, o});
        einsum(c, "nkcd,lmdc->nklm", -0.5, tn(Z, d4), T4, 1.0, O4, {n, o, o, o});
        einsum(c, "ilkm,nklm->ni", 1.0, oooo, O4T, 1.0, s1, {n, o});
    }
    // ring: X_ij = sum t_ik^ce G_kecj + t_ik^ec GB_kecj with G = (lj|cd) w1 + (jc|ld) w2,
    // GB = (jc|ld) w1 + (lj|cd) w3 (sums over l, d; w_kl^de); w1 = t/2 - t^T, w2 = -t + 2 t^T,
    // w3 = -t + t^T/2
    {
        double* B1 = c.arena.dalloc(n * o * v * v);  // sum_j (lj|cd) y_j  [n][l][c][d]
        double* B2 = c.arena.dalloc(n * o * v * v);  // sum_j (jc|ld) y_j
        einsum(c, "ljcd,nj->nlcd", 1.0, oovv, Y, 0.0, B1, d4);
        einsum(c, "jcld,nj->nlcd", 1.0, ovov, Y, 0.0, B2, d4);
        const T B1T = tn(B1, d4), B2T = tn(B2, d4);
        // W <- G y [n][k][e][c], Z <- GB y
        einsum(c, "nlcd,klde->nkec", 0.5, B1T, T4, 0.0, W, d4);
        einsum(c, "nlcd,kled->nkec", -1.0, B1T, T4, 1.0, W, d4);
        einsum(c, "nlcd,klde->nkec", -1.0, B2T, T4, 1.0, W, d4);
        einsum(c, "nlcd,kled->nkec", 2.0, B2T, T4, 1.0, W, d4);
        einsum(c, "nlcd,klde->nkec", 0.5, B2T, T4, 0.0, Z, d4);
        einsum(c, "nlcd,kled->nkec", -1.0, B2T, T4, 1.0, Z, d4);
        einsum(c, "nlcd,klde->nkec", -1.0, B1T, T4, 1.0, Z, d4);
        einsum(c, "nlcd,kled->nkec", 0.5, B1T, T4, 1.0, Z, d4);
        einsum(c, "ikce,nkec->ni", 1.0, T4, tn(W, d4), 1.0, s1, {n, o});
        einsum(c, "ikec,nkec->ni", 1.0, T4, tn(Z, d4), 1.0, s1, {n, o});
        // X^T y: Zr1_kce = sum_j t_jk^ce y_j, Zr2_kce = sum_j t_jk^ec y_j;
        // sum (li|cd) Ra_lcd + (ic|ld) Rb_lcd with Ra = R(Zr1, w1) + R(Zr2, w3), Rb = R(Zr1, w2) + R(Zr2, w1),
        // R(Z, w)_lcd = sum_ke Z_kce w_kl^de
        double* Zr1 = B1;
        double* Zr2 = B2;
        einsum(c, "jkce,nj->nkce", 1.0, T4, Y, 0.0, Zr1, d4);
        einsum(c, "jkec,nj->nkce", 1.0, T4, Y, 0.0, Zr2, d4);
        einsum(c, "nkce,klde->nlcd", 0.5, B1T, T4, 0.0, W, d4);
        einsum(c, "nkce,kled->nlcd", -1.0, B1T, T4, 1.0, W, d4);
        einsum(c, "nkce,klde->nlcd", -1.0, B2T, T4, 1.0, W, d4);
        einsum(c, "nkce,kled->nlcd", 0.5, B2T, T4, 1.0, W, d4);
        einsum(c, "nkce,klde->nlcd", -1.0, B1T, T4, 0.0, Z, d4);
        einsum(c, "nkce,kled->nlcd", 2.0, B1T, T4, 1.0, Z, d4);
        einsum(c, "nkce,klde->nlcd", 0.5, B2T, T4, 1.0, Z, d4);
        einsum(c, "nkce,kled->nlcd", -1.0, B2T, T4, 1.0, Z, d4);
        einsum(c, "licd,nlcd->ni", 1.0, oovv, tn(W, d4), 1.0, s1, {n, o});
        einsum(c, "icld,nlcd->ni", 1.0, ovov, tn(Z, d4), 1.0, s1, {n, o});
    }
    // both lines on the integral: M_ij += -2 sum_kl (ij|kl) U_kl + sum_kl (il|kj) U_kl
    //                                   + 2 sum_cd (ij|cd) Zm_cd - sum_cd (jc|id) Zm_cd
    {
        double* e = c.arena.dalloc(n * o * o * o);
        einsum(c, "ijkl,nj->nikl", -2.0, oooo, Y, 0.0, e, {n, o, o, o});
        einsum(c, "ilkj,nj->nikl", 1.0, oooo, Y, 1.0, e, {n, o, o, o});
        einsum(c, "kl,nikl->ni", 1.0, tc(h->otf_U, {o, o}), tn(e, {n, o, o, o}), 1.0, s1, {n, o});
        einsum(c, "ijcd,nj->nicd", 2.0, oovv, Y, 0.0, W, d4);
        einsum(c, "jcid,nj->nicd", -1.0, ovov, Y, 1.0, W, d4);
        einsum(c, "cd,nicd->ni", 1.0, tc(h->otf_Zm, {v, v}), tn(W, d4), 1.0, s1, {n, o});
    }
}

// --------------------------------------------------------------------------
// Third-order singles t_i^a(3) (Eq. t_singles at k = 3), spin-integrated.
// They enter only the ADC(3) transition moments, so they are made on first
// use, in the setup's contraction arithmetic.  With tau = 2t - t(ab swap):
//   D t(3) = A1 + A2 + (2 E1 + E2 + 4 E3 + 2 E4)/4 - (2 F1 + 4 F2 + F3 + 2 F4)/4,
//   t(3)  += 1/2 sum tau_ij^ab t_j^b(2)
// A1, A2: the CC-like singles terms of t1(2) and t2(2); E1..E4 and F1..F4:
// the connected-triples term 1/4 t_jk^bc W_ijk^abc summed permutation by
// permutation (particle and hole halves).  The costliest pieces are the ring
// products R1, R2 (o^3 v^3) and E2 (4 naux o^3 v^2, auxiliary index chunked by
// aux_chunk, or into slabs of W of at most 2^29 elements).
// --------------------------------------------------------------------------
static void make_t1_third_order(adc_handle* h) {
    if (h->t1_3 || h->order < 3) return;
    Ctx& c = h->ctx;
    const int saved = c.gemm_mode;
    c.gemm_mode = h->cmode_setup;
    const long long o = h->o, v = h->v, Q = h->naux;
    const long long o2v2 = o * o * v * v;
    double* out = h->dmalloc(o * v);
    {
        Scope sc(c.arena);
        const double* t1 = h->t1_2;
        const bool f32 = h->lean;  // o^2 v^2 temporaries in FP32 on a lean handle
        const T T4 = op_t(h, false), U4 = op_tau(h, false), T2 = op_t2(h, false);
        const T Boo = tn(h->Boo, {Q, o, o}), Bvv = tn(h->Bvv, {Q, v, v});
        double* num = c.arena.dalloc(o * v);
        // A1 = sum [2 (ia|jb) - (ij|ab)] t_j^b(2)
        einsum(c, "iajb,jb->ia", 2.0, op_ovov(h, false), tn(t1, {o, v}), 0.0, num, {o, v});
        einsum(c, "jiab,jb->ia", -1.0, op_oovv(h, false), tn(t1, {o, v}), 1.0, num, {o, v});
        {
            // A2: the t1(2) expression with tau(2) = 2 t2(2) - t2(2)(ab swap)
            Scope s2(c.arena);
            Buf tau2 = scratch(c.arena, o2v2, f32);
            perm_into(c, T2, {0, 1, 2, 3}, tau2, 2.0, 0.0);
            perm_into(c, T2, {0, 1, 3, 2}, tau2, -1.0, 1.0);
            double* G = c.arena.dalloc(Q * o * v);
            einsum(c, "Qkc,ikdc->Qid", 1.0, tn(h->Bov, {Q, o, v}), tau2.as({o, o, v, v}), 0.0, G, {Q, o, v});
            einsum(c, "Qid,Qad->ia", 1.0, tn(G, {Q, o, v}), Bvv, 1.0, num, {o, v});
            einsum(c, "kilc,klac->ia", -1.0, tn(h->ooov, {o, o, o, v}), tau2.as({o, o, v, v}), 1.0, num, {o, v});
        }
        {
            // E1/2 and -F1/2 through G_jb^Q = sum_kc (kc|Q) tau_jk^bc
            Scope s2(c.arena);
            double* G = c.arena.dalloc(Q * o * v);
            einsum(c, "Qkc,jkbc->Qjb", 1.0, tn(h->Bov, {Q, o, v}), U4, 0.0, G, {Q, o, v});
            double* Y = c.arena.dalloc(o * v);
            einsum(c, "Qjb,Qbd->jd", 2.0, tn(G, {Q, o, v}), Bvv, 0.0, Y, {o, v});
            einsum(c, "ijad,jd->ia", 0.5, U4, tn(Y, {o, v}), 1.0, num, {o, v});
            einsum(c, "Qlj,Qjb->lb", 2.0, Boo, tn(G, {Q, o, v}), 0.0, Y, {o, v});
            einsum(c, "ilab,lb->ia", -0.5, U4, tn(Y, {o, v}), 1.0, num, {o, v});
        }
        {
            // E2/4 = -sum t_jk^ad V_jkdi, V_jkdi = sum_Q sum_b B^Q_db sum_c tau_jk^cb B^Q_ic
            Scope s2(c.arena);
            // tau_jk^cb held as [b][j][k][c], the order in which the first contraction's GEMM reads it
            Buf tauS = scratch(c.arena, o2v2, f32);
            perm_into(c, U4, {3, 0, 1, 2}, tauS, 1.0, 0.0);
            double* V = c.arena.dalloc(v * o * o * o);  // [d][j][k][i]
            // auxiliary functions per chunk: the aux_chunk option if set, else a slab of W of
            // 2^29 elements (FP64) or 2^31 (FP32, lean)
            const long long per = v * o * o * o;
            const long long slab = f32 ? (1LL << 31) : (1LL << 29);
            const long long qc = h->opt.aux_chunk > 0 ? std::min<long long>(Q, h->opt.aux_chunk)
                                                      : std::max(1LL, std::min(Q, slab / std::max(per, 1LL)));
            Buf W = scratch(c.arena, qc * per, f32);  // [Q][b][j][k][i]
            for (long long q0 = 0; q0 < Q; q0 += qc) {
                const long long nq = std::min(qc, Q - q0);
                ein(c, "bjkc,Qic->Qbjki", 1.0, tauS.as({v, o, o, v}), tn(h->Bov + q0 * o * v, {nq, o, v}), 0.0, W,
                    {nq, v, o, o, o});
                einsum(c, "Qdb,Qbjki->djki", 1.0, tn(h->Bvv + q0 * v * v, {nq, v, v}), W.as({nq, v, o, o, o}),
                       q0 == 0 ? 0.0 : 1.0, V, {v, o, o, o});
            }
            einsum(c, "jkad,djki->ia", -1.0, T4, tn(V, {v, o, o, o}), 1.0, num, {o, v});
        }
        {
            // E3 (+1) and F2 (-1) through the ring products
            //   R1_ik^dc = sum tau_ij^db tau_jk^bc,  R2_ik^cd = -sum (tau_ij^db t_jk^bc + tau_ij^bd t_jk^cb)
            Scope s2(c.arena);
            Buf R = scratch(c.arena, o2v2, f32);
            const T RT = R.as({o, o, v, v});
            double* H = c.arena.dalloc(Q * std::max(std::max(o * v, v * v), o * o));
            ein(c, "ijdb,jkbc->ikdc", 1.0, U4, U4, 0.0, R, {o, o, v, v});
            einsum(c, "Qkc,ikdc->Qid", 1.0, tn(h->Bov, {Q, o, v}), RT, 0.0, H, {Q, o, v});
            einsum(c, "Qid,Qad->ia", 1.0, tn(H, {Q, o, v}), Bvv, 1.0, num, {o, v});   // E3: (ad|kc) R1
            einsum(c, "Qla,Qli->ia", -1.0, tn(H, {Q, o, v}), Boo, 1.0, num, {o, v});  // F2: (li|kc) R1
            ein(c, "ijdb,jkbc->ikcd", -1.0, U4, T4, 0.0, R, {o, o, v, v});
            ein(c, "ijbd,jkcb->ikcd", -1.0, U4, T4, 1.0, R, {o, o, v, v});
            einsum(c, "Qcd,ikcd->Qik", 1.0, Bvv, RT, 0.0, H, {Q, o, o});
            einsum(c, "Qik,Qka->ia", 1.0, tn(H, {Q, o, o}), tn(h->Bov, {Q, o, v}), 1.0, num, {o, v});  // E3: (ka|cd) R2
            einsum(c, "Qlk,lkca->Qca", 1.0, Boo, RT, 0.0, H, {Q, v, v});
            einsum(c, "Qca,Qic->ia", -1.0, tn(H, {Q, v, v}), tn(h->Bov, {Q, o, v}), 1.0, num, {o, v});  // F2: (lk|ic) R2
        }
        {
            // E4/2 with rho_cd = 2 sum t_jk^cb tau_jk^db; -F4/2 with rho'_kl = 2 sum t_jk^bc tau_jl^bc
            Scope s2(c.arena);
            double* rho = c.arena.dalloc(v * v);
            double* r = c.arena.dalloc(Q);
            double* L = c.arena.dalloc(Q * o * v);
            einsum(c, "jkcb,jkdb->cd", 2.0, T4, U4, 0.0, rho, {v, v});
            einsum(c, "Qcd,cd->Q", 1.0, Bvv, tn(rho, {v, v}), 0.0, r, {Q});
            einsum(c, "Qia,Q->ia", 1.0, tn(h->Bov, {Q, o, v}), tn(r, {Q}), 1.0, num, {o, v});
            einsum(c, "Qic,cd->Qid", 1.0, tn(h->Bov, {Q, o, v}), tn(rho, {v, v}), 0.0, L, {Q, o, v});
            einsum(c, "Qid,Qad->ia", -0.5, tn(L, {Q, o, v}), Bvv, 1.0, num, {o, v});
            double* rh = c.arena.dalloc(o * o);
            einsum(c, "jkbc,jlbc->kl", 2.0, T4, U4, 0.0, rh, {o, o});
            einsum(c, "lkia,kl->ia", -1.0, tn(h->ooov, {o, o, o, v}), tn(rh, {o, o}), 1.0, num, {o, v});
            einsum(c, "lika,kl->ia", 0.5, tn(h->ooov, {o, o, o, v}), tn(rh, {o, o}), 1.0, num, {o, v});
        }
        {
            // -F3/4 = -sum (lj|ka) X_jkil, X_jkil = sum t_jk^bc (tau - t)_il^bc - t_kj^bc t_il^bc
            Scope s2(c.arena);
            double* X = c.arena.dalloc(o * o * o * o);
            einsum(c, "jkbc,ilbc->jkil", 1.0, T4, U4, 0.0, X, {o, o, o, o});
            einsum(c, "jkbc,ilbc->jkil", -1.0, T4, T4, 1.0, X, {o, o, o, o});
            einsum(c, "kjbc,ilbc->jkil", -1.0, T4, T4, 1.0, X, {o, o, o, o});
            einsum(c, "ljka,jkil->ia", -1.0, tn(h->ooov, {o, o, o, v}), tn(X, {o, o, o, o}), 1.0, num, {o, v});
        }
        k_div_D1<<<grid_for(o * v), 256, 0, c.stream>>>((int)o, (int)v, h->eps, num);
        launch_check(c);
        ADC_CUDA(cudaMemcpyAsync(out, num, o * v * sizeof(double), cudaMemcpyDeviceToDevice, c.stream));
        einsum(c, "ijab,jb->ia", 0.5, U4, tn(t1, {o, v}), 1.0, out, {o, v});
    }
    c.gemm_mode = saved;
    h->t1_3 = out;
}

static void transition_parts(adc_handle* h, bool third, double* Tpp, double* t1x);

static void setup(adc_handle* h, const double* eps_in, const double* B_in, int on_device) {
    Ctx& c = h->ctx;
    // phase timer: 0 inputs and the ladder's operand planes, 1 integrals, 2 amplitudes and E(2),
    // 3 the ladder of t, 4 the rest of t2(2), t1(2) and E(3), 5 the 1p-1p / 1h-1h block,
    // 6 the transition moments' parts (lean) and the diagonal, 7 total
    const auto t_start = std::chrono::steady_clock::now();
    auto t_last = t_start;
    auto tick = [&](int k) {
        ADC_CUDA(cudaStreamSynchronize(c.stream));
        const auto now = std::chrono::steady_clock::now();
        h->setup_times[k] += std::chrono::duration<double>(now - t_last).count();
        h->setup_times[7] = std::chrono::duration<double>(now - t_start).count();
        t_last = now;
    };
    ADC_BLAS(cublasCreate(&c.blas));
    ADC_BLAS(cublasSetStream(c.blas, c.stream));
    ADC_BLAS(cublasSetMathMode(c.blas, CUBLAS_DEFAULT_MATH));
    // contraction arithmetic: setup (and refinement) FP32-accurate at most; sigma may use the tensor-core split GEMM
    const int cm = h->opt.contractions >= 0 ? h->opt.contractions : (h->opt.precision != ADC_PREC_FP64 ? 2 : 0);
    h->cmode_sigma = cm;
    h->cmode_setup = cm > 1 ? 1 : cm;
    h->cmode_refine = cm > 1 ? 1 : cm;
    if (h->kind == ADC_IP && h->opt.contractions < 0) {
        // IP: the sigma has no ladder and is cheap (o^3 v^2), and setup beyond its ladder is
        // o^3 v^3; on strongly correlated inputs the IP spectroscopic factors need these in
        // FP64 (FP32-accurate setup contractions moved them by ~1.5e-6 at o=20, v=180).  The
        // ladder of t2(2) stays on the tensor cores; the fast sigma keeps mode 2.
        h->cmode_setup = 0;
        h->cmode_refine = 0;
    }
    c.gemm_mode = h->cmode_setup;
    if (h->kind == ADC_EA) h->lm_setup = LadderMode{2, 2, 8};
    const long long o = h->o, v = h->v, Q = h->naux, nmo = o + v;
    h->eps = h->dmalloc(nmo);
    ADC_CUDA(cudaMemcpyAsync(h->eps, eps_in, nmo * sizeof(double), on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                             c.stream));
    h->Boo = h->dmalloc(Q * o * o);
    h->Bov = h->dmalloc(Q * o * v);
    h->Bvv = h->dmalloc(Q * v * v);
    {
        // slice B^Q into its oo, ov and vv blocks (2-D strided copies per block)
        cudaMemcpyKind kd = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        for (long long q = 0; q < Q; ++q) {
            const double* src = B_in + q * nmo * nmo;
            ADC_CUDA(cudaMemcpy2DAsync(h->Boo + q * o * o, o * sizeof(double), src, nmo * sizeof(double), o * sizeof(double), o, kd, c.stream));
            ADC_CUDA(cudaMemcpy2DAsync(h->Bov + q * o * v, v * sizeof(double), src + o, nmo * sizeof(double), v * sizeof(double), o, kd, c.stream));
            ADC_CUDA(cudaMemcpy2DAsync(h->Bvv + q * v * v, v * sizeof(double), src + o * nmo + o, nmo * sizeof(double), v * sizeof(double), v, kd,
                                       c.stream));
        }
    }
    if (h->opt.tune_cache && h->opt.tune_cache[0]) c.tuner = tune_cache_open(h->opt.tune_cache);
    h->opt.tune_cache = nullptr;  // the caller's string is not kept
    if (h->opt.precision != ADC_PREC_FP64) {
        h->tc = ladder_tc_create(c, h->Bvv, (int)Q, (int)v, h->opt.aux_chunk);
        noalloc_prepare();  // the allocation-free ladder's scratch address on this device, resolved up front
    }
    tick(0);
    // integrals (Eq. 19)
    const long long o2v2 = o * o * v * v;
    const bool lean = h->lean;
    h->ovov = h->dmalloc(o2v2);
    h->oovv = h->dmalloc(o2v2);
    h->oooo = h->dmalloc(o * o * o * o);
    h->ooov = h->dmalloc(o * o * o * v);
    einsum(c, "Qia,Qjb->iajb", 1.0, tn(h->Bov, {Q, o, v}), tn(h->Bov, {Q, o, v}), 0.0, h->ovov, {o, v, o, v});
    einsum(c, "Qij,Qab->ijab", 1.0, tn(h->Boo, {Q, o, o}), tn(h->Bvv, {Q, v, v}), 0.0, h->oovv, {o, o, v, v});
    einsum(c, "Qij,Qkl->ijkl", 1.0, tn(h->Boo, {Q, o, o}), tn(h->Boo, {Q, o, o}), 0.0, h->oooo, {o, o, o, o});
    einsum(c, "Qij,Qka->ijka", 1.0, tn(h->Boo, {Q, o, o}), tn(h->Bov, {Q, o, v}), 0.0, h->ooov, {o, o, o, v});
    if (h->order >= 3 && !lean) {
        // ring2[i][a][j][c] = 2 (ia|jc) - (ji|ac) (EA) or (ji|ac) - 2 (ia|jc) (IP)
        h->ring2 = h->dmalloc(o * v * o * v);
        const bool ea = h->kind == ADC_EA;
        axpby(c, o * v * o * v, ea ? 2.0 : -2.0, h->ovov, 0.0, h->ring2);
        Shape s4{4, {o, o, v, v}};
        int pr[4] = {1, 2, 0, 3};  // (j, i, a, c) -> (i, a, j, c)
        permute(c, h->oovv, s4, pr, h->ring2, ea ? -1.0 : 1.0, 1.0);
    }
    tick(1);
    // amplitudes (Eqs. t_singles, t_doubles)
    h->t = h->dmalloc(o2v2);
    k_make_t<<<grid_for(o2v2), 256, 0, c.stream>>>((int)o, (int)v, h->eps, h->ovov, h->t);
    launch_check(c);
    if (!lean) {
        h->tau = h->dmalloc(o2v2);
        axpby(c, o2v2, 2.0, h->t, 0.0, h->tau);
        Shape s4{4, {o, o, v, v}};
        int swp[4] = {0, 1, 3, 2};
        permute(c, h->t, s4, swp, h->tau, -1.0, 1.0);
    }
    // MPn correlation energy: E(k+1) = sum (ia|jb) (2 t_ij^ab - t_ij^ba), t = t2(k); o^2 v^2
    // work, always in FP64 (an FP32 integral operand is read into an FP64 copy)
    auto mp_energy = [&](const T& tk) {
        Scope sc(c.arena);
        const int saved = c.gemm_mode;
        c.gemm_mode = 0;
        double* part = c.arena.dalloc(o);
        einsum(c, "iajb,ijab->i", 2.0, op_ovov(h, false), tk, 0.0, part, {o});
        einsum(c, "iajb,ijba->i", -1.0, op_ovov(h, false), tk, 1.0, part, {o});
        std::vector<double> hp(o);
        ADC_CUDA(cudaMemcpyAsync(hp.data(), part, o * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
        ADC_CUDA(cudaStreamSynchronize(c.stream));
        c.gemm_mode = saved;
        double e = 0.0;
        for (double x : hp) e += x;
        return e;
    };
    h->emp[0] = mp_energy(tn(h->t, {o, o, v, v}));
    if (lean) {
        // every later use of the integrals is a split-BF16 or FP32-accurate contraction
        h->f_oovv = to_f32(h, h->oovv, o2v2);
        h->f_ovov = to_f32(h, h->ovov, o2v2);
    }
    tick(2);
    Scope setup_scope(c.arena);
    double* XL = nullptr;  // EA: the ladder term of the 1p-1p block, formed while the ladder of t is alive
    if (h->order >= 3) {
        const T T4 = op_t(h, false);
        const bool keep_Lt = h->opt.m11_on_the_fly && h->kind == ADC_EA;  // sigma applies the block from it
        double* Lt = h->dmalloc(o2v2);
        if (!lean) {
            fill(c, o2v2, 0.0, Lt);
            ladder(h, h->t, o * o, Lt, h->lm_setup);  // sum_cd (ac|bd) t_ij^cd (it feeds M_11 directly)
            if (h->opt.precision != ADC_PREC_FP64 && h->tc) {
                // The tensor core's truncating FP32 accumulation biases each promoted partial sum
                // toward zero, about linearly in the accumulation length.  With L(E) the ladder
                // accumulated in epochs of E K blocks, 2 L(E) - L(2E) removes the linear part of
                // that bias (Richardson extrapolation in E): measured on t2(2), bias -1.8e-7 ->
                // -6e-8 relative at E = 1.  Formed in place: Lt <- -2 L(E), then += L(2E), negated.
                const LadderMode twice{h->lm_setup.planes, 2 * h->lm_setup.epoch1, 2 * h->lm_setup.epoch2};
                axpby(c, o2v2, 0.0, Lt, -2.0, Lt);
                ladder(h, h->t, o * o, Lt, twice);
                axpby(c, o2v2, 0.0, Lt, -1.0, Lt);
            }
        } else {
            // L_ij = sum_Q B^Q t_ij B^Q, the sum_cd (ac|bd) t_ij^cd that feeds t2(2) and M_11.  With
            // t_ji = t_ij^T and every B^Q symmetric, L_ji = L_ij^T: on a lean handle the ladder runs
            // on the pairs i <= j only and the other half is their transpose (half the setup's
            // largest cost; the plain layout evaluates every pair)
            Scope ps(c.arena);
            const long long np = o * (o + 1) / 2, vv = v * v;
            std::vector<int> hpi, hpj;
            for (int i = 0; i < o; ++i)
                for (int j = i; j < o; ++j) {
                    hpi.push_back(i);
                    hpj.push_back(j);
                }
            int* dpi = (int*)c.arena.alloc(2 * np * sizeof(int));
            int* dpj = dpi + np;
            ADC_CUDA(cudaMemcpyAsync(dpi, hpi.data(), np * sizeof(int), cudaMemcpyHostToDevice, c.stream));
            ADC_CUDA(cudaMemcpyAsync(dpj, hpj.data(), np * sizeof(int), cudaMemcpyHostToDevice, c.stream));
            double* P = c.arena.dalloc(np * vv);
            double* Lp = c.arena.dalloc(np * vv);
            k_pairs_gather<<<grid_for(np * vv), 256, 0, c.stream>>>(np, vv, (int)o, dpi, dpj, h->t, P);
            launch_check(c);
            fill(c, np * vv, 0.0, Lp);
            ladder(h, P, np, Lp, h->lm_setup);
            if (h->opt.precision != ADC_PREC_FP64 && h->tc) {
                // The tensor core's truncating FP32 accumulation biases each promoted partial sum
                // toward zero, about linearly in the accumulation length.  With L(E) the ladder
                // accumulated in epochs of E K blocks, 2 L(E) - L(2E) removes the linear part of
                // that bias (Richardson extrapolation in E): measured on t2(2), bias -1.8e-7 ->
                // -6e-8 relative at E = 1.  Formed in place: Lp <- -2 L(E), then += L(2E), negated.
                const LadderMode twice{h->lm_setup.planes, 2 * h->lm_setup.epoch1, 2 * h->lm_setup.epoch2};
                axpby(c, np * vv, 0.0, Lp, -2.0, Lp);
                ladder(h, P, np, Lp, twice);
                axpby(c, np * vv, 0.0, Lp, -1.0, Lp);
            }
            const long long nt = (v + 31) / 32;
            k_pairs_scatter<<<(unsigned)std::min<long long>(np * nt * nt, 152LL * 16), dim3(32, 8), 0, c.stream>>>(
                np, (int)v, (int)o, dpi, dpj, Lp, Lt);
            launch_check(c);
        }
        tick(3);
        double* N = Lt;  // t2(2) numerator, formed in the ladder's buffer unless the ladder is kept
        if (keep_Lt) {
            h->Lt = Lt;
            N = h->dmalloc(o2v2);
            ADC_CUDA(cudaMemcpyAsync(N, Lt, o2v2 * sizeof(double), cudaMemcpyDeviceToDevice, c.stream));
        } else if (h->kind == ADC_EA) {
            // X_ab = -sum t_kl^ac [L_kl^bc - 1/2 L_kl^cb] (one open line through the ladder)
            XL = c.arena.dalloc(v * v);
            einsum(c, "klac,klbc->ab", -1.0, T4, tn(Lt, {o, o, v, v}), 0.0, XL, {v, v});
            einsum(c, "klac,klcb->ab", 0.5, T4, tn(Lt, {o, o, v, v}), 1.0, XL, {v, v});
        }
        h->t_2 = N;
        {
            Scope sc(c.arena);
            einsum(c, "kilj,klab->ijab", 1.0, tn(h->oooo, {o, o, o, o}), T4, 1.0, N, {o, o, v, v});
            const T OVOV = op_ovov(h, false), OOVV = op_oovv(h, false);
            Buf W = scratch(c.arena, o2v2, lean);
            ein(c, "kcjb,ikac->ijab", 2.0, OVOV, T4, 0.0, W, {o, o, v, v});
            ein(c, "kcjb,ikca->ijab", -1.0, OVOV, T4, 1.0, W, {o, o, v, v});
            ein(c, "kjbc,ikac->ijab", -1.0, OOVV, T4, 1.0, W, {o, o, v, v});
            ein(c, "kjac,ikcb->ijab", -1.0, OOVV, T4, 1.0, W, {o, o, v, v});
            const Buf Nb{N, false};
            perm_into(c, W.as({o, o, v, v}), {0, 1, 2, 3}, Nb, 1.0, 1.0);
            perm_into(c, W.as({o, o, v, v}), {1, 0, 3, 2}, Nb, 1.0, 1.0);
        }
        k_div_D2<<<grid_for(o2v2), 256, 0, c.stream>>>((int)o, (int)v, h->eps, N);
        launch_check(c);
        // singles: D t_i^a = sum (kc|ad)(2 t_ik^dc - t_ik^cd) - sum (ki|lc)(2 t_kl^ac - t_kl^ca)
        h->t1_2 = h->dmalloc(o * v);
        {
            Scope sc(c.arena);
            if (lean) {
                h->f_tau = (float*)c.arena.alloc(o2v2 * sizeof(float));
                const Buf tb{h->f_tau, true};
                perm_into(c, T4, {0, 1, 2, 3}, tb, 2.0, 0.0);
                perm_into(c, T4, {0, 1, 3, 2}, tb, -1.0, 1.0);
            }
            const T U4 = op_tau(h, false);
            double* Gq = c.arena.dalloc(Q * o * v);
            einsum(c, "Qkc,ikdc->Qid", 1.0, tn(h->Bov, {Q, o, v}), U4, 0.0, Gq, {Q, o, v});
            einsum(c, "Qid,Qad->ia", 1.0, tn(Gq, {Q, o, v}), tn(h->Bvv, {Q, v, v}), 0.0, h->t1_2, {o, v});
            einsum(c, "kilc,klac->ia", -1.0, tn(h->ooov, {o, o, o, v}), U4, 1.0, h->t1_2, {o, v});
            h->f_tau = nullptr;
        }
        k_div_D1<<<grid_for(o * v), 256, 0, c.stream>>>((int)o, (int)v, h->eps, h->t1_2);
        launch_check(c);
        h->emp[1] = mp_energy(tn(h->t_2, {o, o, v, v}));
    }
    if (lean) {
        h->f_t = to_f32(h, h->t, o2v2);
        if (h->t_2) h->f_t2 = to_f32(h, h->t_2, o2v2);
    }
    tick(4);
    const long long n1 = h->n1();
    if (h->opt.m11_on_the_fly) {
        // step 3 skipped: sigma applies the block from intermediates (the diagonal preconditioner
        // then takes the zeroth-order one-particle energies)
        setup_m11_otf(h);
        h->diag = h->dmalloc(h->dim());
        k_diag<<<grid_for(h->dim()), 256, 0, c.stream>>>(h->kind == ADC_EA, (int)o, (int)v, h->eps, nullptr, h->diag);
        launch_check(c);
        ADC_CUDA(cudaStreamSynchronize(c.stream));
        return;
    }
    h->M11 = h->dmalloc(n1 * n1);
    {
        // zeroth order: diag(eps)
        std::vector<double> e(nmo);
        ADC_CUDA(cudaMemcpyAsync(e.data(), h->eps, nmo * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
        ADC_CUDA(cudaStreamSynchronize(c.stream));
        std::vector<double> m0(n1 * n1, 0.0);
        for (long long p = 0; p < n1; ++p) m0[p * n1 + p] = e[h->kind == ADC_EA ? o + p : p];
        ADC_CUDA(cudaMemcpyAsync(h->M11, m0.data(), n1 * n1 * sizeof(double), cudaMemcpyHostToDevice, c.stream));
        ADC_CUDA(cudaStreamSynchronize(c.stream));
    }
    if (h->kind == ADC_EA) {
        setup_m11_ea(h, XL);
    } else {
        // The 1h-1h block's contractions run in FP64 in every precision: on strongly correlated
        // inputs its third-order terms cancel to a small fraction of their parts, and FP32-accurate
        // contractions there moved the IP roots by ~1e-6 Eh.  Its costliest terms are o^3 v^3.
        const int saved = c.gemm_mode;
        c.gemm_mode = 0;
        setup_m11_ip(h);
        c.gemm_mode = saved;
    }
    tick(5);
    if (lean) {
        // what the transition moments need beyond t and t2(2), made while setup's memory is free
        Scope sc(c.arena);
        h->f_tau = (float*)c.arena.alloc(o2v2 * sizeof(float));
        const Buf tb{h->f_tau, true};
        perm_into(c, op_t(h, false), {0, 1, 2, 3}, tb, 2.0, 0.0);
        perm_into(c, op_t(h, false), {0, 1, 3, 2}, tb, -1.0, 1.0);
        const long long np = std::max(o, v);
        h->spec_Tpp = h->dmalloc(2 * np * np);
        h->spec_t1 = h->dmalloc(2 * o * v);
        for (int third = 0; third <= (h->order >= 3 ? 1 : 0); ++third)
            transition_parts(h, third != 0, h->spec_Tpp + third * np * np, h->spec_t1 + third * o * v);
        h->f_tau = nullptr;
    }
    h->diag = h->dmalloc(h->dim());
    k_diag<<<grid_for(h->dim()), 256, 0, c.stream>>>(h->kind == ADC_EA, (int)o, (int)v, h->eps, h->M11, h->diag);
    launch_check(c);
    tick(6);
}

// --------------------------------------------------------------------------
// sigma (Sec. III A step 4; Eqs. sigma_i_adapted_3, sigma_jka_bab, EA analogue)
// --------------------------------------------------------------------------
static void sigma_ea(adc_handle* h, const double* Xin, double* Sout, long long nv_) {
    Ctx& c = h->ctx;
    const long long o = h->o, v = h->v, Q = h->naux, n = nv_, dim = h->dim(), blk = o * v * v;
    Scope sc(c.arena);
    // split into 1p and 2p1h parts (contiguous per part)
    double* y1 = c.arena.dalloc(n * v);
    double* Y2 = c.arena.dalloc(n * blk);
    double* s1 = c.arena.dalloc(n * v);
    double* S2 = c.arena.dalloc(n * blk);
    k_gather<<<grid_for(n * v), 256, 0, c.stream>>>(n, v, Xin, dim, 0, y1, v, 0, 0.0);
    launch_check(c);
    k_gather<<<grid_for(n * blk), 256, 0, c.stream>>>(n, blk, Xin, dim, v, Y2, blk, 0, 0.0);
    launch_check(c);
    double* Yt = c.arena.dalloc(n * blk);
    k_two_minus_swap<<<grid_for(n * blk), 256, 0, c.stream>>>(1, (int)o, (int)v, n, Y2, Yt);
    launch_check(c);
    // 1p row: M_ab Y_b (precomputed block, or on the fly)
    if (h->M11)
        einsum(c, "nb,ab->na", 1.0, tn(y1, {n, v}), tn(h->M11, {v, v}), 0.0, s1, {n, v});
    else
        m11_apply_otf_ea(h, y1, s1, n);
    // coupling row, first order: sum (ad|jc) Y~_jcd.  W^Q_d collects every coupling-row
    // term of the form sum_Qd W^Q_d (Q|da); it is contracted with B^Q_vv once, below.
    double* Wq = c.arena.dalloc(n * Q * v);
    einsum(c, "Qjc,njcd->nQd", 1.0, tc(h->Bov, {Q, o, v}), tn(Yt, {n, o, v, v}), 0.0, Wq, {n, Q, v});
    // 2p1h column, first order: (cb|ia) Y_c
    double* hq = c.arena.dalloc(n * Q * v);
    einsum(c, "nc,Qcb->nQb", 1.0, tn(y1, {n, v}), tc(h->Bvv, {Q, v, v}), 0.0, hq, {n, Q, v});
    einsum(c, "Qia,nQb->niab", 1.0, tc(h->Bov, {Q, o, v}), tn(hq, {n, Q, v}), 0.0, S2, {n, o, v, v});
    // 2p1h block, zeroth order
    k_diag22<<<grid_for(n * blk), 256, 0, c.stream>>>(1, (int)o, (int)v, n, h->eps, Y2, S2);
    launch_check(c);
    if (h->order >= 3) {
        const T T4 = op_t(h, true);
        // coupling row, second order:
        //  sum (al|jm) t_lm^dc Y~_jcd
        double* Z = c.arena.dalloc(n * o * o * o);
        einsum(c, "lmdc,njcd->nlmj", 1.0, T4, tn(Yt, {n, o, v, v}), 0.0, Z, {n, o, o, o});
        // P^Q_l collects the terms of the form sum_Ql P^Q_l (Q|la) (contracted once, below)
        double* P = c.arena.dalloc(n * Q * o);
        einsum(c, "Qjm,nlmj->nQl", 1.0, tc(h->Boo, {Q, o, o}), tn(Z, {n, o, o, o}), 0.0, P, {n, Q, o});
        //  sum (ad|em)(2 t_jm^ce - t_jm^ec) Y~_jcd  (a lean handle holds no tau: two contractions with t)
        double* V = c.arena.dalloc(n * o * v * v);
        if (h->tau) {
            einsum(c, "jmce,njcd->nmed", 1.0, tc(h->tau, {o, o, v, v}), tn(Yt, {n, o, v, v}), 0.0, V, {n, o, v, v});
        } else {
            einsum(c, "jmce,njcd->nmed", 2.0, T4, tn(Yt, {n, o, v, v}), 0.0, V, {n, o, v, v});
            einsum(c, "jmec,njcd->nmed", -1.0, T4, tn(Yt, {n, o, v, v}), 1.0, V, {n, o, v, v});
        }
        einsum(c, "nmed,Qme->nQd", 1.0, tn(V, {n, o, v, v}), tc(h->Bov, {Q, o, v}), 1.0, Wq, {n, Q, v});
        //  - sum (am|ed) [t_jm^ce Y~_jcd + t_jm^ed Y~_jdc]   (the two exchange-type terms)
        einsum(c, "jmce,njcd->nmed", 1.0, T4, tn(Yt, {n, o, v, v}), 0.0, V, {n, o, v, v});
        einsum(c, "jmec,njdc->nmed", 1.0, T4, tn(Yt, {n, o, v, v}), 1.0, V, {n, o, v, v});
        einsum(c, "nmed,Qed->nQm", -1.0, tn(V, {n, o, v, v}), tc(h->Bvv, {Q, v, v}), 1.0, P, {n, Q, o});
        einsum(c, "nQl,Qla->na", 1.0, tn(P, {n, Q, o}), tc(h->Bov, {Q, o, v}), 1.0, s1, {n, v});
        // 2p1h column, second order:
        //  sum_lm (cl|im) t_lm^ba Y_c
        double* p = c.arena.dalloc(n * Q * o);
        einsum(c, "nc,Qlc->nQl", 1.0, tn(y1, {n, v}), tc(h->Bov, {Q, o, v}), 0.0, p, {n, Q, o});
        double* Pl = c.arena.dalloc(n * o * o * o);
        einsum(c, "nQl,Qim->nlim", 1.0, tn(p, {n, Q, o}), tc(h->Boo, {Q, o, o}), 0.0, Pl, {n, o, o, o});
        einsum(c, "nlim,lmba->niab", 1.0, tn(Pl, {n, o, o, o}), T4, 1.0, S2, {n, o, v, v});
        //  sum_me (cb|em)(2 t_im^ae - t_im^ea) Y_c
        double* q = c.arena.dalloc(n * o * v * v);
        einsum(c, "nQb,Qme->nbme", 1.0, tn(hq, {n, Q, v}), tc(h->Bov, {Q, o, v}), 0.0, q, {n, v, o, v});
        if (h->tau) {
            einsum(c, "nbme,imae->niab", 1.0, tn(q, {n, v, o, v}), tc(h->tau, {o, o, v, v}), 1.0, S2, {n, o, v, v});
        } else {
            einsum(c, "nbme,imae->niab", 2.0, tn(q, {n, v, o, v}), T4, 1.0, S2, {n, o, v, v});
            einsum(c, "nbme,imea->niab", -1.0, tn(q, {n, v, o, v}), T4, 1.0, S2, {n, o, v, v});
        }
        //  - sum_me (cm|eb) t_im^ae Y_c - sum_me (cm|ea) t_im^eb Y_c
        einsum(c, "nQm,Qeb->nmeb", 1.0, tn(p, {n, Q, o}), tc(h->Bvv, {Q, v, v}), 0.0, q, {n, o, v, v});
        einsum(c, "nmeb,imae->niab", -1.0, tn(q, {n, o, v, v}), T4, 1.0, S2, {n, o, v, v});
        einsum(c, "nmea,imeb->niab", -1.0, tn(q, {n, o, v, v}), T4, 1.0, S2, {n, o, v, v});
        // 2p1h block, first order: ladder sum_cd (ac|bd) Y_icd (vvvv never stored)
        ladder(h, Y2, n * o, S2, h->refining ? h->lm_refine : h->lm_sigma);
        //  - (ac|ji) Y_jcb + 2 (ai|jc) Y_jcb - (ai|jc) Y_jbc - (bd|ji) Y_jad  (the first two as one
        //  contraction with ring2, or two on a lean handle)
        const T OVOV = op_ovov(h, true), OOVV = op_oovv(h, true), Y2T = tn(Y2, {n, o, v, v});
        if (h->ring2) {
            einsum(c, "iajc,njcb->niab", 1.0, tc(h->ring2, {o, v, o, v}), Y2T, 1.0, S2, {n, o, v, v});
        } else {
            einsum(c, "iajc,njcb->niab", 2.0, OVOV, Y2T, 1.0, S2, {n, o, v, v});
            einsum(c, "jiac,njcb->niab", -1.0, OOVV, Y2T, 1.0, S2, {n, o, v, v});
        }
        einsum(c, "iajc,njbc->niab", -1.0, OVOV, Y2T, 1.0, S2, {n, o, v, v});
        einsum(c, "jibd,njad->niab", -1.0, OOVV, Y2T, 1.0, S2, {n, o, v, v});
    }
    // coupling row: every sum_Qd W^Q_d (Q|da) term at once
    einsum(c, "nQd,Qda->na", 1.0, tn(Wq, {n, Q, v}), tc(h->Bvv, {Q, v, v}), 1.0, s1, {n, v});
    k_gather<<<grid_for(n * v), 256, 0, c.stream>>>(n, v, s1, v, 0, Sout, dim, 0, 0.0);
    launch_check(c);
    k_gather<<<grid_for(n * blk), 256, 0, c.stream>>>(n, blk, S2, blk, 0, Sout, dim, v, 0.0);
    launch_check(c);
}

static void sigma_ip(adc_handle* h, const double* Xin, double* Sout, long long nv_) {
    // contributions of the paper's M_- are accumulated, then negated; M11 already holds -M_-11
    Ctx& c = h->ctx;
    const long long o = h->o, v = h->v, Q = h->naux, n = nv_, dim = h->dim(), blk = o * o * v;
    Scope sc(c.arena);
    double* y1 = c.arena.dalloc(n * o);
    double* Y2 = c.arena.dalloc(n * blk);
    double* s1 = c.arena.dalloc(n * o);
    double* S2 = c.arena.dalloc(n * blk);
    k_gather<<<grid_for(n * o), 256, 0, c.stream>>>(n, o, Xin, dim, 0, y1, o, 0, 0.0);
    launch_check(c);
    k_gather<<<grid_for(n * blk), 256, 0, c.stream>>>(n, blk, Xin, dim, o, Y2, blk, 0, 0.0);
    launch_check(c);
    double* Yt = c.arena.dalloc(n * blk);
    k_two_minus_swap<<<grid_for(n * blk), 256, 0, c.stream>>>(0, (int)o, (int)v, n, Y2, Yt);
    launch_check(c);
    // coupling row, first order: -(ki|ja) Y~_jka
    double* G = c.arena.dalloc(n * Q * o);
    einsum(c, "Qja,njka->nQk", 1.0, tc(h->Bov, {Q, o, v}), tn(Yt, {n, o, o, v}), 0.0, G, {n, Q, o});
    einsum(c, "nQk,Qki->ni", -1.0, tn(G, {n, Q, o}), tc(h->Boo, {Q, o, o}), 0.0, s1, {n, o});
    // 2h1p column, first order: -(ki|ja) Y_i
    double* g = c.arena.dalloc(n * Q * o);
    einsum(c, "ni,Qki->nQk", 1.0, tn(y1, {n, o}), tc(h->Boo, {Q, o, o}), 0.0, g, {n, Q, o});
    einsum(c, "nQk,Qja->njka", -1.0, tn(g, {n, Q, o}), tc(h->Bov, {Q, o, v}), 0.0, S2, {n, o, o, v});
    k_diag22<<<grid_for(n * blk), 256, 0, c.stream>>>(0, (int)o, (int)v, n, h->eps, Y2, S2);
    launch_check(c);
    if (h->order >= 3) {
        const double *t = h->t, *tau = h->tau;
        // coupling row, second order
        //  - sum (ad|ie) t_jk^de Y~_jka
        double* Z = c.arena.dalloc(n * v * v * v);
        einsum(c, "jkde,njka->ndea", 1.0, tc(t, {o, o, v, v}), tn(Yt, {n, o, o, v}), 0.0, Z, {n, v, v, v});
        double* Hq = c.arena.dalloc(n * Q * v);
        einsum(c, "ndea,Qad->nQe", 1.0, tn(Z, {n, v, v, v}), tc(h->Bvv, {Q, v, v}), 0.0, Hq, {n, Q, v});
        einsum(c, "nQe,Qie->ni", -1.0, tn(Hq, {n, Q, v}), tc(h->Bov, {Q, o, v}), 1.0, s1, {n, o});
        //  - sum (ik|lc)(2 t_jl^ac - t_jl^ca) Y~_jka + sum (ic|lk) t_jl^ac Y~_jka + sum (ic|lj) t_kl^ca Y~_jka
        double* G2 = c.arena.dalloc(n * o * o * v);
        einsum(c, "jlac,njka->nklc", 1.0, tc(tau, {o, o, v, v}), tn(Yt, {n, o, o, v}), 0.0, G2, {n, o, o, v});
        einsum(c, "iklc,nklc->ni", -1.0, tc(h->ooov, {o, o, o, v}), tn(G2, {n, o, o, v}), 1.0, s1, {n, o});
        einsum(c, "jlac,njka->nlkc", 1.0, tc(t, {o, o, v, v}), tn(Yt, {n, o, o, v}), 0.0, G2, {n, o, o, v});
        einsum(c, "lkic,nlkc->ni", 1.0, tc(h->ooov, {o, o, o, v}), tn(G2, {n, o, o, v}), 1.0, s1, {n, o});
        einsum(c, "klca,njka->nljc", 1.0, tc(t, {o, o, v, v}), tn(Yt, {n, o, o, v}), 0.0, G2, {n, o, o, v});
        einsum(c, "ljic,nljc->ni", 1.0, tc(h->ooov, {o, o, o, v}), tn(G2, {n, o, o, v}), 1.0, s1, {n, o});
        // 2h1p column, second order (same tensor, applied to Y_i)
        double* bq = c.arena.dalloc(n * Q * v);
        einsum(c, "ni,Qie->nQe", 1.0, tn(y1, {n, o}), tc(h->Bov, {Q, o, v}), 0.0, bq, {n, Q, v});
        double* w = c.arena.dalloc(n * v * v * v);
        einsum(c, "nQe,Qad->nead", 1.0, tn(bq, {n, Q, v}), tc(h->Bvv, {Q, v, v}), 0.0, w, {n, v, v, v});
        einsum(c, "nead,jkde->njka", -1.0, tn(w, {n, v, v, v}), tc(t, {o, o, v, v}), 1.0, S2, {n, o, o, v});
        double* m = c.arena.dalloc(n * o * o * v);
        einsum(c, "ni,iklc->nklc", 1.0, tn(y1, {n, o}), tc(h->ooov, {o, o, o, v}), 0.0, m, {n, o, o, v});
        einsum(c, "nklc,jlac->njka", -1.0, tn(m, {n, o, o, v}), tc(tau, {o, o, v, v}), 1.0, S2, {n, o, o, v});
        einsum(c, "ni,lkic->nlkc", 1.0, tn(y1, {n, o}), tc(h->ooov, {o, o, o, v}), 0.0, m, {n, o, o, v});
        einsum(c, "nlkc,jlac->njka", 1.0, tn(m, {n, o, o, v}), tc(t, {o, o, v, v}), 1.0, S2, {n, o, o, v});
        einsum(c, "ni,ljic->nljc", 1.0, tn(y1, {n, o}), tc(h->ooov, {o, o, o, v}), 0.0, m, {n, o, o, v});
        einsum(c, "nljc,klca->njka", 1.0, tn(m, {n, o, o, v}), tc(t, {o, o, v, v}), 1.0, S2, {n, o, o, v});
        // 2h1p block, first order: -(ki|lj) Y_kla + (ki|ab) Y_kjb - 2 (ia|kb) Y_kjb + (ia|kb) Y_jkb + (kj|ab) Y_ikb
        einsum(c, "kilj,nkla->nija", -1.0, tc(h->oooo, {o, o, o, o}), tn(Y2, {n, o, o, v}), 1.0, S2, {n, o, o, v});
        einsum(c, "iakb,nkjb->nija", 1.0, tc(h->ring2, {o, v, o, v}), tn(Y2, {n, o, o, v}), 1.0, S2, {n, o, o, v});
        einsum(c, "iakb,njkb->nija", 1.0, tc(h->ovov, {o, v, o, v}), tn(Y2, {n, o, o, v}), 1.0, S2, {n, o, o, v});
        einsum(c, "kjab,nikb->nija", 1.0, tc(h->oovv, {o, o, v, v}), tn(Y2, {n, o, o, v}), 1.0, S2, {n, o, o, v});
    }
    // negate (M_IP = -M_-) and add the 1h-1h block (already negated), or apply it on the fly and negate
    if (h->M11) {
        einsum(c, "nj,ij->ni", 1.0, tn(y1, {n, o}), tn(h->M11, {o, o}), -1.0, s1, {n, o});
    } else {
        m11_apply_otf_ip(h, y1, s1, n);
        axpby(c, n * o, 0.0, s1, -1.0, s1);
    }
    k_gather<<<grid_for(n * o), 256, 0, c.stream>>>(n, o, s1, o, 0, Sout, dim, 0, 0.0);
    launch_check(c);
    axpby(c, n * blk, 0.0, S2, -1.0, S2);
    k_gather<<<grid_for(n * blk), 256, 0, c.stream>>>(n, blk, S2, blk, 0, Sout, dim, o, 0.0);
    launch_check(c);
}

static void sigma_unrestricted(adc_handle* h, const double* Xin, double* Sout, long long n);

// the launches of one sigma (no host synchronisation inside: it may run under stream capture)
static void sigma_launch(adc_handle* h, const double* X, double* S, long long nvec) {
    Ctx& c = h->ctx;
    if (!h->refining) c.gemm_mode = h->cmode_sigma;
    // a timeout of an earlier call left the flag raised; every call starts clean
    if (c.d_err) ADC_CUDA(cudaMemsetAsync(c.d_err, 0, sizeof(int), c.stream));
    if (h->unrestricted)
        sigma_unrestricted(h, X, S, nvec);
    else if (h->kind == ADC_EA)
        sigma_ea(h, X, S, nvec);
    else
        sigma_ip(h, X, S, nvec);
}

static void sigma_device(adc_handle* h, const double* X, double* S, long long nvec) {
    Ctx& c = h->ctx;
    sigma_launch(h, X, S, nvec);
    if (c.d_err) {
        int e = 0;
        ADC_CUDA(cudaMemcpyAsync(&e, c.d_err, sizeof(int), cudaMemcpyDeviceToHost, c.stream));
        ADC_CUDA(cudaStreamSynchronize(c.stream));
        if (e) throw Error(ADC_ERR_TIMEOUT, "sigma: a bounded device wait of the tensor-core GEMM timed out");
    }
}

// sigma through a CUDA graph (cuda_graphs, mixed-precision handles): the launches of one sigma
// of n vectors are captured once on fixed buffers (after one ordinary evaluation has made every
// allocation, operand cache entry and tile choice they need) and replayed as one launch; the
// inputs and outputs are copied to and from the fixed buffers, and the timeout flags of the
// tensor-core kernels are read after the replay.  A capture that fails leaves the handle on
// ordinary launches.
static void sigma_run(adc_handle* h, const double* X, double* S, long long n) {
    Ctx& c = h->ctx;
    if (!h->opt.cuda_graphs || h->graphs_failed || h->refining || h->cmode_sigma != 2 || c.timing || !c.stream) {
        // (the legacy default stream cannot be captured: graphs need the handle on a stream of its own)
        sigma_device(h, X, S, n);
        return;
    }
    const long long dim = h->dim();
    adc_handle::SigmaGraph* g = nullptr;
    for (auto& e : h->graphs)
        if (e.n == n) g = &e;
    if (!g) {
        adc_handle::SigmaGraph e;
        e.n = n;
        e.X = (double*)dev_alloc((size_t)n * dim * sizeof(double), c.stream);
        e.S = (double*)dev_alloc((size_t)n * dim * sizeof(double), c.stream);
        ADC_CUDA(cudaMemcpyAsync(e.X, X, (size_t)n * dim * sizeof(double), cudaMemcpyDeviceToDevice, c.stream));
        sigma_device(h, e.X, e.S, n);  // allocations, cached operands, tiles
        ADC_CUDA(cudaStreamSynchronize(c.stream));
        cudaGraph_t graph = nullptr;
        bool ok = true;
        c.capturing = true;
        c.arena.frozen = true;
        ADC_CUDA(cudaStreamBeginCapture(c.stream, cudaStreamCaptureModeThreadLocal));
        try {
            sigma_launch(h, e.X, e.S, n);
        } catch (const std::exception&) {
            ok = false;
        }
        const cudaError_t ec = cudaStreamEndCapture(c.stream, &graph);
        c.capturing = false;
        c.arena.frozen = false;
        if (ok && ec == cudaSuccess && graph && cudaGraphInstantiate(&e.exec, graph, 0) == cudaSuccess) {
            cudaGraphDestroy(graph);
            h->graphs.push_back(e);
            ADC_CUDA(cudaMemcpyAsync(S, e.S, (size_t)n * dim * sizeof(double), cudaMemcpyDeviceToDevice, c.stream));
            return;  // the ordinary evaluation above computed this call's result
        }
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        h->graphs_failed = true;
        ADC_CUDA(cudaMemcpyAsync(S, e.S, (size_t)n * dim * sizeof(double), cudaMemcpyDeviceToDevice, c.stream));
        ADC_CUDA(cudaStreamSynchronize(c.stream));
        cudaFree(e.X);
        cudaFree(e.S);
        return;
    }
    ADC_CUDA(cudaMemcpyAsync(g->X, X, (size_t)n * dim * sizeof(double), cudaMemcpyDeviceToDevice, c.stream));
    ADC_CUDA(cudaGraphLaunch(g->exec, c.stream));
    ADC_CUDA(cudaMemcpyAsync(S, g->S, (size_t)n * dim * sizeof(double), cudaMemcpyDeviceToDevice, c.stream));
    if (c.d_err) {
        int e = 0;
        ADC_CUDA(cudaMemcpyAsync(&e, c.d_err, sizeof(int), cudaMemcpyDeviceToHost, c.stream));
        ADC_CUDA(cudaStreamSynchronize(c.stream));
        if (e) throw Error(ADC_ERR_TIMEOUT, "sigma: a bounded device wait of the tensor-core GEMM timed out");
    }
    if (h->tc) ladder_tc_check(*h->tc, c);
    if (h->tc_b) ladder_tc_check(*h->tc_b, c);
}

// --------------------------------------------------------------------------
// Davidson (Eq. eig) in the S inner product
// --------------------------------------------------------------------------
namespace {

// cyclic Jacobi eigen-decomposition of a symmetric n x n matrix (row-major);
// eigenvalues ascending, eigenvectors as columns of V
void jacobi_eigh(int n, std::vector<double> A, std::vector<double>& w, std::vector<double>& V) {
    V.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                double a = A[(size_t)i * n + j] * A[(size_t)i * n + j];
                tot += a;
                if (i != j) off += a;
            }
        if (off <= 1e-30 * std::max(tot, 1e-300)) break;
        for (int p = 0; p < n - 1; ++p)
            for (int q = p + 1; q < n; ++q) {
                double apq = A[(size_t)p * n + q];
                if (std::fabs(apq) < 1e-300) continue;
                double app = A[(size_t)p * n + p], aqq = A[(size_t)q * n + q];
                double theta = 0.5 * (aqq - app) / apq;
                double tt = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                double cs = 1.0 / std::sqrt(tt * tt + 1.0), sn = tt * cs;
                for (int k = 0; k < n; ++k) {
                    double akp = A[(size_t)k * n + p], akq = A[(size_t)k * n + q];
                    A[(size_t)k * n + p] = cs * akp - sn * akq;
                    A[(size_t)k * n + q] = sn * akp + cs * akq;
                }
                for (int k = 0; k < n; ++k) {
                    double apk = A[(size_t)p * n + k], aqk = A[(size_t)q * n + k];
                    A[(size_t)p * n + k] = cs * apk - sn * aqk;
                    A[(size_t)q * n + k] = sn * apk + cs * aqk;
                }
                for (int k = 0; k < n; ++k) {
                    double vkp = V[(size_t)k * n + p], vkq = V[(size_t)k * n + q];
                    V[(size_t)k * n + p] = cs * vkp - sn * vkq;
                    V[(size_t)k * n + q] = sn * vkp + cs * vkq;
                }
            }
    }
    std::vector<int> idx(n);
    std::iota(idx.begin(), idx.end(), 0);
    std::vector<double> d(n);
    for (int i = 0; i < n; ++i) d[i] = A[(size_t)i * n + i];
    std::sort(idx.begin(), idx.end(), [&](int a, int b) { return d[a] < d[b]; });
    w.resize(n);
    std::vector<double> Vs((size_t)n * n);
    for (int j = 0; j < n; ++j) {
        w[j] = d[idx[j]];
        for (int k = 0; k < n; ++k) Vs[(size_t)k * n + j] = V[(size_t)k * n + idx[j]];
    }
    V.swap(Vs);
}

}  // namespace

struct Davidson {
    adc_handle* h;
    long long dim;
    int nroots, maxspace;
    double* V;   // [cap][dim] S-orthonormal basis
    double* SV;  // S V
    double* W;   // sigma(V)
    int k = 0;
    long long nsig = 0;
    double sigma_seconds = 0.0;
    int ldg = 0;
    std::vector<double> G;  // host [ldg][ldg]: G_ij = (SV_i . W_j + SV_j . W_i) / 2 for i, j < k

    void metric(const double* in, double* out, long long nvec, int inverse) {
        if (h->unrestricted) {  // the antisymmetric pair basis of an open-shell reference: S = 1
            if (out != in)
                ADC_CUDA(cudaMemcpyAsync(out, in, (size_t)nvec * dim * sizeof(double), cudaMemcpyDeviceToDevice, h->ctx.stream));
            return;
        }
        k_metric<<<grid_for(nvec * dim), 256, 0, h->ctx.stream>>>(h->kind == ADC_EA, h->o, h->v, nvec, in, out, inverse);
        launch_check(h->ctx);
    }
    void sigma(int first, int count) {
        auto t0 = std::chrono::steady_clock::now();
        sigma_run(h, V + (long long)first * dim, W + (long long)first * dim, count);
        ADC_CUDA(cudaStreamSynchronize(h->ctx.stream));
        sigma_seconds += std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        nsig += count;
    }
    // rows and columns [k0, k0 + kn) of the symmetrised subspace matrix, from the new vectors only
    void update_G(int k0, int kn) {
        Ctx& c = h->ctx;
        Scope gs(c.arena);
        const int kt = k0 + kn;
        double* A = c.arena.dalloc((size_t)kt * kn * 2);
        multidot(c, kt, SV, dim, kn, W + (long long)k0 * dim, dim, dim, A);            // SV_i . W_{k0+j}
        multidot(c, kt, W, dim, kn, SV + (long long)k0 * dim, dim, dim, A + kt * kn);  // W_i . SV_{k0+j}
        std::vector<double> hA((size_t)kt * kn * 2);
        ADC_CUDA(cudaMemcpyAsync(hA.data(), A, hA.size() * sizeof(double), cudaMemcpyDeviceToHost, h->ctx.stream));
        ADC_CUDA(cudaStreamSynchronize(h->ctx.stream));
        for (int i = 0; i < kt; ++i)
            for (int j = 0; j < kn; ++j) {
                const double g = 0.5 * (hA[(size_t)i * kn + j] + hA[(size_t)kt * kn + i * kn + j]);
                G[(size_t)i * ldg + k0 + j] = g;
                G[(size_t)(k0 + j) * ldg + i] = g;
            }
    }
    // S-orthonormalise rows [first, first+count) of V against rows [0, first) and each other; returns kept count.
    // Block classical Gram-Schmidt against the basis (two passes), then one new vector at a time.
    int orthonormalise(int first, int count) {
        Ctx& c = h->ctx;
        Scope os(c.arena);
        double* D = V + (long long)first * dim;
        double* cf = c.arena.dalloc((size_t)std::max(1, count) * std::max(1, first + count));
        if (first > 0) {
            // second pass only where the first removed more than 1 - 1/sqrt(2) of a vector's
            // S-norm (the Daniel-Gragg-Kaufman-Stewart criterion)
            double* SD = c.arena.dalloc((size_t)count * dim);
            double* nn = c.arena.dalloc((size_t)count * count);
            auto snorms = [&](std::vector<double>& out) {
                metric(D, SD, count, 0);
                multidot(c, count, D, dim, count, SD, dim, dim, nn);
                std::vector<double> m((size_t)count * count);
                ADC_CUDA(cudaMemcpyAsync(m.data(), nn, m.size() * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
                ADC_CUDA(cudaStreamSynchronize(c.stream));
                out.resize(count);
                for (int r = 0; r < count; ++r) out[r] = m[(size_t)r * count + r];
            };
            std::vector<double> before, after;
            snorms(before);
            for (int pass = 0; pass < 2; ++pass) {
                multidot(c, count, D, dim, first, SV, dim, dim, cf);           // cf[r][i] = D_r . (S V)_i
                lincomb(c, count, first, cf, V, dim, dim, -1.0, 1.0, D, dim);  // D_r -= sum_i cf[r][i] V_i
                if (pass == 1) break;
                snorms(after);
                bool again = false;
                for (int r = 0; r < count; ++r) again = again || !(after[r] >= 0.5 * before[r]);
                if (!again) break;
            }
        }
        int kept = 0;
        for (int r = 0; r < count; ++r) {
            double* x = D + (long long)r * dim;
            double* dst = D + (long long)kept * dim;
            if (dst != x) ADC_CUDA(cudaMemcpyAsync(dst, x, dim * sizeof(double), cudaMemcpyDeviceToDevice, c.stream));
            if (kept > 0)
                for (int pass = 0; pass < 2; ++pass) {
                    multidot(c, 1, dst, dim, kept, SV + (long long)first * dim, dim, dim, cf);
                    lincomb(c, 1, kept, cf, D, dim, dim, -1.0, 1.0, dst, dim);
                }
            double* sdst = SV + (long long)(first + kept) * dim;
            metric(dst, sdst, 1, 0);
            multidot(c, 1, dst, dim, 1, sdst, dim, dim, cf);
            double nrm2 = 0.0;
            ADC_CUDA(cudaMemcpyAsync(&nrm2, cf, sizeof(double), cudaMemcpyDeviceToHost, c.stream));
            ADC_CUDA(cudaStreamSynchronize(c.stream));
            if (!(nrm2 > 1e-20)) continue;
            double s = 1.0 / std::sqrt(nrm2);
            axpby(c, dim, 0.0, dst, s, dst);
            axpby(c, dim, 0.0, sdst, s, sdst);
            ++kept;
        }
        return kept;
    }
};

// Root-independent parts of the transition moments (Eqs. T_ea, T_ip; Appendix): the
// one-particle block of T without its unit diagonal, Tpp (EA: [v][v], T_cb - d_cb; IP: [o][o]),
// and the singles row t1x [o][v] = t1(2) [+ t1(3) + 1/2 sum tau t1(2)] (third: T through
// third order).  In the setup's contraction arithmetic.
static void transition_parts(adc_handle* h, bool third, double* Tpp, double* t1x) {
    Ctx& c = h->ctx;
    const int saved = c.gemm_mode;
    c.gemm_mode = h->cmode_setup;
    const long long o = h->o, v = h->v, Q = h->naux;
    Scope sc(c.arena);
    const T T4 = op_t(h, false);
    if (h->t1_2) {
        axpby(c, o * v, 1.0, h->t1_2, 0.0, t1x);
    } else {
        // second-order singles are part of T(2) also for ADC(2)
        double* Gq = c.arena.dalloc(Q * o * v);
        einsum(c, "Qkc,ikdc->Qid", 1.0, tn(h->Bov, {Q, o, v}), op_tau(h, false), 0.0, Gq, {Q, o, v});
        einsum(c, "Qid,Qad->ia", 1.0, tn(Gq, {Q, o, v}), tn(h->Bvv, {Q, v, v}), 0.0, t1x, {o, v});
        einsum(c, "kilc,klac->ia", -1.0, tn(h->ooov, {o, o, o, v}), op_tau(h, false), 1.0, t1x, {o, v});
        k_div_D1<<<grid_for(o * v), 256, 0, c.stream>>>((int)o, (int)v, h->eps, t1x);
        launch_check(c);
    }
    if (third) {
        make_t1_third_order(h);
        axpby(c, o * v, 1.0, h->t1_3, 1.0, t1x);
        const char* spec = h->kind == ADC_EA ? "klbc,lc->kb" : "jlcd,ld->jc";
        einsum(c, spec, 0.5, op_tau(h, false), tn(h->t1_2, {o, v}), 1.0, t1x, {o, v});
    }
    if (h->kind == ADC_EA) {
        // T_{c,b} = d_cb + B(t, t)_cb [+ B(t, t2) + B(t2, t)],
        // B(x, y)_cb = -sum x_kl^cd y_kl^bd + 1/2 sum x_kl^cd y_kl^db
        einsum(c, "klcd,klbd->cb", -1.0, T4, T4, 0.0, Tpp, {v, v});
        einsum(c, "klcd,kldb->cb", 0.5, T4, T4, 1.0, Tpp, {v, v});
        if (third) {
            const T T2 = op_t2(h, false);
            einsum(c, "klcd,klbd->cb", -1.0, T4, T2, 1.0, Tpp, {v, v});
            einsum(c, "klcd,kldb->cb", 0.5, T4, T2, 1.0, Tpp, {v, v});
            einsum(c, "klcd,klbd->cb", -1.0, T2, T4, 1.0, Tpp, {v, v});
            einsum(c, "klcd,kldb->cb", 0.5, T2, T4, 1.0, Tpp, {v, v});
        }
    } else {
        // T_{k,j} = d_kj + B'(t, t)_kj [+ B'(t, t2) + B'(t2, t)],
        // B'(x, y)_kj = -sum x_kl^cd y_jl^cd + 1/2 sum x_kl^cd y_jl^dc
        einsum(c, "klcd,jlcd->kj", -1.0, T4, T4, 0.0, Tpp, {o, o});
        einsum(c, "klcd,jldc->kj", 0.5, T4, T4, 1.0, Tpp, {o, o});
        if (third) {
            const T T2 = op_t2(h, false);
            einsum(c, "klcd,jlcd->kj", -1.0, T4, T2, 1.0, Tpp, {o, o});
            einsum(c, "klcd,jldc->kj", 0.5, T4, T2, 1.0, Tpp, {o, o});
            einsum(c, "klcd,jlcd->kj", -1.0, T2, T4, 1.0, Tpp, {o, o});
            einsum(c, "klcd,jldc->kj", 0.5, T2, T4, 1.0, Tpp, {o, o});
        }
    }
    c.gemm_mode = saved;
}

static void specfac_unrestricted(adc_handle* h, const double* Y, int nroots, double* specfac);

static void drop_graphs(adc_handle* h) {
    if (h->graphs.empty()) return;
    cudaStreamSynchronize(h->ctx.stream);
    for (auto& g : h->graphs) {
        if (g.exec) cudaGraphExecDestroy(g.exec);
        cudaFree(g.X);
        cudaFree(g.S);
    }
    h->graphs.clear();
}

static int davidson(adc_handle* h, int nroots, double tol, const double* guess, double* energies, double* specfac,
                    double* vectors, double* stats) {
    Ctx& c = h->ctx;
    // A captured sigma uses the scratch addresses of this call's arena layout: its graphs
    // live exactly as long as this call.
    struct GraphScope {
        adc_handle* h;
        ~GraphScope() { drop_graphs(h); }
    } graph_scope{h};
    auto t0 = std::chrono::steady_clock::now();
    const long long dim = h->dim();
    const int nextra = std::max(0, h->opt.nguess_extra);
    const int nstart = (int)std::min<long long>(dim, guess ? nroots : nroots + nextra);
    const int maxspace = std::max(h->opt.max_space_per_root * nroots,
                                  std::max(nstart, std::max(1, h->opt.keep_per_root) * nroots) + nroots);
    const int cap = maxspace + nroots;
    const double rtol = h->opt.res_tol > 0 ? h->opt.res_tol : std::sqrt(tol);
    Scope sc(c.arena);
    Davidson d{h, dim, nroots, maxspace, nullptr, nullptr, nullptr};
    d.ldg = cap;
    d.G.assign((size_t)cap * cap, 0.0);
    d.V = c.arena.dalloc((size_t)cap * dim);
    d.SV = c.arena.dalloc((size_t)cap * dim);
    d.W = c.arena.dalloc((size_t)cap * dim);
    double* X = c.arena.dalloc((size_t)nroots * dim);
    double* AX = c.arena.dalloc((size_t)nroots * dim);
    double* R = c.arena.dalloc((size_t)nroots * dim);
    double* SR = c.arena.dalloc((size_t)nroots * dim);
    double* Cd = c.arena.dalloc((size_t)cap * nroots);
    double* Gd = c.arena.dalloc((size_t)cap * cap);
    double* wd = c.arena.dalloc(nroots);
    // guesses
    if (guess) {
        for (long long x = 0; x < (long long)nroots * dim; ++x)
            if (!std::isfinite(guess[x])) throw Error(ADC_ERR_NONFINITE, "davidson: non-finite element in the guess vectors");
        ADC_CUDA(cudaMemcpyAsync(d.V, guess, (size_t)nroots * dim * sizeof(double), cudaMemcpyHostToDevice, c.stream));
    } else {
        std::vector<double> D(dim);
        ADC_CUDA(cudaMemcpyAsync(D.data(), h->diag, dim * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
        ADC_CUDA(cudaStreamSynchronize(c.stream));
        std::vector<long long> idx(dim);
        std::iota(idx.begin(), idx.end(), 0LL);
        // ascending diagonal, ties by index; a non-finite element sorts last (keeps the order strict)
        auto key = [&](long long x) { return std::isfinite(D[x]) ? D[x] : INFINITY; };
        std::partial_sort(idx.begin(), idx.begin() + nstart, idx.end(), [&](long long a, long long b) {
            const double ka = key(a), kb = key(b);
            return ka < kb || (ka == kb && a < b);
        });
        fill(c, (long long)nstart * dim, 0.0, d.V);
        long long* di = (long long*)c.arena.alloc(nstart * sizeof(long long));
        ADC_CUDA(cudaMemcpyAsync(di, idx.data(), nstart * sizeof(long long), cudaMemcpyHostToDevice, c.stream));
        k_units<<<1, std::max(32, nstart), 0, c.stream>>>(nstart, di, dim, d.V);
        launch_check(c);
    }
    d.k = d.orthonormalise(0, nstart);
    if (d.k < nroots) throw Error(ADC_ERR_ARG, "davidson: guess space too small");
    d.sigma(0, d.k);
    d.update_G(0, d.k);
    std::vector<double> wold(nroots, INFINITY), w, C, G, rn(nroots);
    // learned preconditioner: a root whose residual has not dropped below 0.9 x its best for
    // 4 iterations falls back to the diagonal one for the rest of the run
    std::vector<double> best_rn(nroots, INFINITY);
    std::vector<int> stall(nroots, 0), diag_only(nroots, h->mlp_w ? 0 : 1);
    int it = 0, status = ADC_ERR_NOT_CONVERGED;
    int maxit = std::max(1, h->opt.max_iter);
    // Refinement phase (mixed precision, refine >= 1 and refine_res_tol > 0): once the fast
    // operator has converged, the Davidson continues from its Ritz vectors with the accurate
    // one (lm_refine ladder; other contractions FP32-accurate for refine = 1, FP64 for
    // refine = 2) until the residual is below refine_res_tol.  That converges the vectors,
    // not just the energies, under the accurate operator (the spectroscopic factors are
    // linear in the vector error).
    const bool polish = h->opt.precision != ADC_PREC_FP64 && h->opt.refine > 0 && h->opt.refine_res_tol > 0;
    bool polishing = false;
    double rtol_cur = rtol;
    std::vector<double> w_fast;
    auto t_polish = std::chrono::steady_clock::now();
    struct AccurateOperator {  // h->refining and the contraction mode for the refinement, restored on exit
        adc_handle* h;
        int saved = 0;
        bool on = false;
        void enter() {
            saved = h->ctx.gemm_mode;
            h->refining = true;
            h->ctx.gemm_mode = h->opt.refine >= 2 ? 0 : h->cmode_refine;
            on = true;
        }
        ~AccurateOperator() {
            if (on) {
                h->refining = false;
                h->ctx.gemm_mode = saved;
            }
        }
    } accurate{h};
    for (it = 1; it <= maxit; ++it) {
        int k = d.k;
        // G = V S W^T (symmetrised), kept up to date on the host as vectors are added
        G.resize((size_t)k * k);
        for (int i = 0; i < k; ++i)
            for (int j = 0; j < k; ++j) G[(size_t)i * k + j] = d.G[(size_t)i * d.ldg + j];
        jacobi_eigh(k, G, w, C);
        // Ct[r][i] = C[i][r] for the lowest nroots
        std::vector<double> Ct((size_t)nroots * k);
        for (int r = 0; r < nroots; ++r)
            for (int i = 0; i < k; ++i) Ct[(size_t)r * k + i] = C[(size_t)i * k + r];
        ADC_CUDA(cudaMemcpyAsync(Cd, Ct.data(), Ct.size() * sizeof(double), cudaMemcpyHostToDevice, c.stream));
        lincomb(c, nroots, k, Cd, d.V, dim, dim, 1.0, 0.0, X, dim);
        lincomb(c, nroots, k, Cd, d.W, dim, dim, 1.0, 0.0, AX, dim);
        // R = AX - w X
        ADC_CUDA(cudaMemcpyAsync(R, AX, (size_t)nroots * dim * sizeof(double), cudaMemcpyDeviceToDevice, c.stream));
        for (int r = 0; r < nroots; ++r) axpby(c, dim, -w[r], X + (long long)r * dim, 1.0, R + (long long)r * dim);
        d.metric(R, SR, nroots, 0);
        std::vector<double> rr(nroots), rrm((size_t)nroots * nroots);
        multidot(c, nroots, R, dim, nroots, SR, dim, dim, Gd);
        ADC_CUDA(cudaMemcpyAsync(rrm.data(), Gd, rrm.size() * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
        ADC_CUDA(cudaStreamSynchronize(c.stream));
        for (int r = 0; r < nroots; ++r) rr[r] = rrm[(size_t)r * nroots + r];
        bool all = true;
        std::vector<int> todo;
        for (int r = 0; r < nroots; ++r) {
            rn[r] = std::sqrt(std::max(rr[r], 0.0));
            bool cv = std::fabs(w[r] - wold[r]) <= tol && rn[r] <= rtol_cur;
            if (!std::isfinite(w[r]) || !std::isfinite(rn[r]))
                throw Error(ADC_ERR_NONFINITE, "davidson: non-finite Ritz value or residual (non-finite sigma)");
            if (!cv) {
                all = false;
                todo.push_back(r);
            }
            wold[r] = w[r];
            if (rn[r] < 0.9 * best_rn[r]) {
                best_rn[r] = rn[r];
                stall[r] = 0;
            } else if (++stall[r] >= 4) {
                diag_only[r] = 1;
            }
        }
        if (all && polish && !polishing) {
            // switch to the accurate operator: the subspace restarts from the converged Ritz vectors
            polishing = true;
            t_polish = std::chrono::steady_clock::now();
            w_fast.assign(w.begin(), w.begin() + nroots);
            accurate.enter();
            ADC_CUDA(cudaMemcpyAsync(d.V, X, (size_t)nroots * dim * sizeof(double), cudaMemcpyDeviceToDevice, c.stream));
            d.metric(d.V, d.SV, nroots, 0);
            d.k = nroots;
            std::fill(d.G.begin(), d.G.end(), 0.0);
            d.sigma(0, nroots);
            d.update_G(0, nroots);
            std::fill(wold.begin(), wold.end(), INFINITY);
            std::fill(best_rn.begin(), best_rn.end(), INFINITY);
            std::fill(stall.begin(), stall.end(), 0);
            rtol_cur = h->opt.refine_res_tol;
            maxit = it + std::max(1, h->opt.max_iter);
            continue;
        }
        if (all) {
            status = ADC_OK;
            break;
        }
        int nnew = (int)todo.size();
        if (d.k + nnew > maxspace) {
            // thick restart: collapse onto the lowest nkeep Ritz vectors (S-orthonormal); sigma follows linearly
            const int nkeep = std::max(nroots, std::min(k, std::max(1, h->opt.keep_per_root) * nroots));
            Scope rs(c.arena);
            std::vector<double> Ck((size_t)nkeep * k);
            for (int r = 0; r < nkeep; ++r)
                for (int i = 0; i < k; ++i) Ck[(size_t)r * k + i] = C[(size_t)i * k + r];
            double* Ckd = c.arena.dalloc((size_t)nkeep * k);
            double* tmp = c.arena.dalloc((size_t)nkeep * dim);
            ADC_CUDA(cudaMemcpyAsync(Ckd, Ck.data(), Ck.size() * sizeof(double), cudaMemcpyHostToDevice, c.stream));
            lincomb(c, nkeep, k, Ckd, d.V, dim, dim, 1.0, 0.0, tmp, dim);
            ADC_CUDA(cudaMemcpyAsync(d.V, tmp, (size_t)nkeep * dim * sizeof(double), cudaMemcpyDeviceToDevice, c.stream));
            lincomb(c, nkeep, k, Ckd, d.W, dim, dim, 1.0, 0.0, tmp, dim);
            ADC_CUDA(cudaMemcpyAsync(d.W, tmp, (size_t)nkeep * dim * sizeof(double), cudaMemcpyDeviceToDevice, c.stream));
            d.metric(d.V, d.SV, nkeep, 0);
            d.k = nkeep;
            // the collapsed basis diagonalises the subspace matrix: G = diag(w_0 .. w_nkeep-1)
            std::fill(d.G.begin(), d.G.end(), 0.0);
            for (int r = 0; r < nkeep; ++r) d.G[(size_t)r * d.ldg + r] = w[r];
        }
        // corrections for unconverged roots
        std::vector<double> wt(nnew);
        for (int j = 0; j < nnew; ++j) {
            wt[j] = w[todo[j]];
            ADC_CUDA(cudaMemcpyAsync(SR + (long long)j * dim, R + (long long)todo[j] * dim, dim * sizeof(double),
                                     cudaMemcpyDeviceToDevice, c.stream));
        }
        ADC_CUDA(cudaMemcpyAsync(wd, wt.data(), nnew * sizeof(double), cudaMemcpyHostToDevice, c.stream));
        for (int j = 0; j < nnew; ++j) {
            double* dst = d.V + (long long)(d.k + j) * dim;
            if (!diag_only[todo[j]]) {
                mlp_precondition(c, 1, dim, h->n1(), SR + (long long)j * dim, wd + j, h->diag, h->mlp_w, dst);
                // a non-finite learned correction (bad weights) falls back to the diagonal one at once
                double nrm2 = 0.0;
                multidot(c, 1, dst, dim, 1, dst, dim, dim, Cd);
                ADC_CUDA(cudaMemcpyAsync(&nrm2, Cd, sizeof(double), cudaMemcpyDeviceToHost, c.stream));
                ADC_CUDA(cudaStreamSynchronize(c.stream));
                if (std::isfinite(nrm2)) continue;
                diag_only[todo[j]] = 1;
            }
            k_precond<<<grid_for(dim), 256, 0, c.stream>>>(1, dim, SR + (long long)j * dim, wd + j, h->diag, dst);
            launch_check(c);
        }
        int kept = d.orthonormalise(d.k, nnew);
        if (kept == 0) {
            // no correction survives orthonormalisation while roots are unconverged: the space
            // cannot grow, so the run stops with its best estimates and says so
            status = ADC_ERR_NOT_CONVERGED;
            break;
        }
        d.sigma(d.k, kept);
        d.update_G(d.k, kept);
        d.k += kept;
    }
    // Final refinement (mixed precision): sigma of the Ritz vectors once more
    // with the accurate ladder arithmetic (lm_refine) and, for refine = 2, FP64
    // for every other contraction (refine = 1 keeps them FP32-accurate), then
    // Rayleigh-Ritz in their span.  The Davidson residual
    // makes the vector error first order, its energy error second order, so
    // the refined energies carry the accurate operator's error only.
    double refine_shift = 0.0, refine_sec = 0.0;
    if (polishing) {
        for (int r = 0; r < nroots; ++r) refine_shift = std::max(refine_shift, std::fabs(w[r] - w_fast[r]));
        refine_sec = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_polish).count();
    } else if (h->opt.precision != ADC_PREC_FP64 && h->opt.refine) {
        auto tr = std::chrono::steady_clock::now();
        const int saved = c.gemm_mode;
        h->refining = true;
        // other contractions FP32-accurate (refine = 1) or FP64 (refine = 2)
        c.gemm_mode = h->opt.refine >= 2 ? 0 : h->cmode_refine;
        try {
            sigma_device(h, X, AX, nroots);
        } catch (...) {
            h->refining = false;
            c.gemm_mode = saved;
            throw;
        }
        h->refining = false;
        c.gemm_mode = saved;
        const int n = nroots;
        d.metric(X, SR, n, 0);
        multidot(c, n, SR, dim, n, AX, dim, dim, Gd);         // X S sigma(X)^T
        multidot(c, n, SR, dim, n, X, dim, dim, Gd + n * n);  // X S X^T
        std::vector<double> GO((size_t)2 * n * n);
        ADC_CUDA(cudaMemcpyAsync(GO.data(), Gd, GO.size() * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
        ADC_CUDA(cudaStreamSynchronize(c.stream));
        std::vector<double> Gs((size_t)n * n), Os((size_t)n * n), ow, U, wr, Z;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                Gs[(size_t)i * n + j] = 0.5 * (GO[(size_t)i * n + j] + GO[(size_t)j * n + i]);
                Os[(size_t)i * n + j] = 0.5 * (GO[(size_t)n * n + i * n + j] + GO[(size_t)n * n + j * n + i]);
            }
        // Loewdin: O^-1/2 G O^-1/2 = Z diag(w) Z^T, coefficients O^-1/2 Z
        jacobi_eigh(n, Os, ow, U);
        if (!(ow[0] > 1e-8)) throw Error(ADC_ERR_CUDA, "davidson: refinement basis is singular");
        std::vector<double> Oi((size_t)n * n, 0.0), T1((size_t)n * n, 0.0), Gt((size_t)n * n, 0.0);
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j)
                for (int k2 = 0; k2 < n; ++k2)
                    Oi[(size_t)i * n + j] += U[(size_t)i * n + k2] * U[(size_t)j * n + k2] / std::sqrt(ow[k2]);
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j)
                for (int k2 = 0; k2 < n; ++k2) T1[(size_t)i * n + j] += Gs[(size_t)i * n + k2] * Oi[(size_t)k2 * n + j];
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j)
                for (int k2 = 0; k2 < n; ++k2) Gt[(size_t)i * n + j] += Oi[(size_t)i * n + k2] * T1[(size_t)k2 * n + j];
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < i; ++j) Gt[(size_t)i * n + j] = Gt[(size_t)j * n + i] = 0.5 * (Gt[(size_t)i * n + j] + Gt[(size_t)j * n + i]);
        jacobi_eigh(n, Gt, wr, Z);
        std::vector<double> Crt((size_t)n * n, 0.0);  // Crt[r][i] = (O^-1/2 Z)[i][r]
        for (int r = 0; r < n; ++r)
            for (int i = 0; i < n; ++i)
                for (int k2 = 0; k2 < n; ++k2) Crt[(size_t)r * n + i] += Oi[(size_t)i * n + k2] * Z[(size_t)k2 * n + r];
        ADC_CUDA(cudaMemcpyAsync(Cd, Crt.data(), Crt.size() * sizeof(double), cudaMemcpyHostToDevice, c.stream));
        lincomb(c, n, n, Cd, X, dim, dim, 1.0, 0.0, R, dim);
        lincomb(c, n, n, Cd, AX, dim, dim, 1.0, 0.0, SR, dim);
        ADC_CUDA(cudaMemcpyAsync(X, R, (size_t)n * dim * sizeof(double), cudaMemcpyDeviceToDevice, c.stream));
        ADC_CUDA(cudaMemcpyAsync(AX, SR, (size_t)n * dim * sizeof(double), cudaMemcpyDeviceToDevice, c.stream));
        // residuals of the refined pairs under the accurate operator
        ADC_CUDA(cudaMemcpyAsync(R, AX, (size_t)n * dim * sizeof(double), cudaMemcpyDeviceToDevice, c.stream));
        for (int r = 0; r < n; ++r) axpby(c, dim, -wr[r], X + (long long)r * dim, 1.0, R + (long long)r * dim);
        d.metric(R, SR, n, 0);
        std::vector<double> rr(n), rrm((size_t)n * n);
        multidot(c, n, R, dim, n, SR, dim, dim, Gd);
        ADC_CUDA(cudaMemcpyAsync(rrm.data(), Gd, rrm.size() * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
        ADC_CUDA(cudaStreamSynchronize(c.stream));
        for (int r = 0; r < n; ++r) rr[r] = rrm[(size_t)r * n + r];
        for (int r = 0; r < n; ++r) {
            refine_shift = std::max(refine_shift, std::fabs(wr[r] - w[r]));
            w[r] = wr[r];
            rn[r] = std::sqrt(std::max(rr[r], 0.0));
        }
        refine_sec = std::chrono::duration<double>(std::chrono::steady_clock::now() - tr).count();
    }
    // outputs
    for (int r = 0; r < nroots; ++r) energies[r] = w[r];
    if (vectors) ADC_CUDA(cudaMemcpyAsync(vectors, X, (size_t)nroots * dim * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
    if (specfac && h->unrestricted) {
        specfac_unrestricted(h, X, nroots, specfac);
    } else if (specfac) {
        // X_p = sum_nu T_{p,nu} (S Y~)_nu, P = 2 sum_p X_p^2  (Appendix); Ritz vectors are S-normalised
        const long long o = h->o, v = h->v, nmo = o + v;
        double* SX = SR;
        d.metric(X, SX, nroots, 0);
        double* Xp = c.arena.dalloc((size_t)nroots * nmo);
        fill(c, (long long)nroots * nmo, 0.0, Xp);
        double* s1 = c.arena.dalloc((size_t)nroots * std::max(o, v));
        double* s2 = c.arena.dalloc((size_t)nroots * (h->kind == ADC_EA ? o * v * v : o * o * v));
        long long n1 = h->n1(), blk = dim - n1;
        k_gather<<<grid_for(nroots * n1), 256, 0, c.stream>>>(nroots, n1, SX, dim, 0, s1, n1, 0, 0.0);
        launch_check(c);
        k_gather<<<grid_for(nroots * blk), 256, 0, c.stream>>>(nroots, blk, SX, dim, n1, s2, blk, 0, 0.0);
        launch_check(c);
        // root-independent parts: the one-particle block T_pp' (without its unit diagonal) and
        // the singles row t1x (precomputed by setup on a lean handle)
        const bool third = h->order >= 3 && h->opt.transition_order != 2;
        const long long np = std::max(o, v);
        const double* Tpp;
        const double* t1;
        if (h->spec_Tpp) {
            Tpp = h->spec_Tpp + (third ? np * np : 0);
            t1 = h->spec_t1 + (third ? o * v : 0);
        } else {
            double* Tb = c.arena.dalloc((size_t)np * np);
            double* tb = c.arena.dalloc((size_t)o * v);
            transition_parts(h, third, Tb, tb);
            Tpp = Tb;
            t1 = tb;
        }
        const T T4 = op_t(h, h->lean);
        if (h->kind == ADC_EA) {
            double* xv = c.arena.dalloc((size_t)nroots * v);
            ADC_CUDA(cudaMemcpyAsync(xv, s1, (size_t)nroots * v * sizeof(double), cudaMemcpyDeviceToDevice, c.stream));
            einsum(c, "rb,cb->rc", 1.0, tn(s1, {nroots, v}), tn(Tpp, {v, v}), 1.0, xv, {nroots, v});
            k_gather<<<grid_for(nroots * v), 256, 0, c.stream>>>(nroots, v, xv, v, 0, Xp, nmo, o, 0.0);
            launch_check(c);
            // occupied: T_{k,b} = -t_k^b(2) [- t_k^b(3) - 1/2 sum tau_kl^bc t_l^c(2)] ;
            // T_{k,jcd} = -t_kj^dc [- t2_kj^dc]
            double* xo = c.arena.dalloc((size_t)nroots * o);
            einsum(c, "rb,kb->rk", -1.0, tn(s1, {nroots, v}), tn(t1, {o, v}), 0.0, xo, {nroots, o});
            einsum(c, "rjcd,kjdc->rk", -1.0, tn(s2, {nroots, o, v, v}), T4, 1.0, xo, {nroots, o});
            if (third) einsum(c, "rjcd,kjdc->rk", -1.0, tn(s2, {nroots, o, v, v}), op_t2(h, h->lean), 1.0, xo, {nroots, o});
            k_gather<<<grid_for(nroots * o), 256, 0, c.stream>>>(nroots, o, xo, o, 0, Xp, nmo, 0, 0.0);
            launch_check(c);
        } else {
            double* xo = c.arena.dalloc((size_t)nroots * o);
            ADC_CUDA(cudaMemcpyAsync(xo, s1, (size_t)nroots * o * sizeof(double), cudaMemcpyDeviceToDevice, c.stream));
            einsum(c, "rj,kj->rk", 1.0, tn(s1, {nroots, o}), tn(Tpp, {o, o}), 1.0, xo, {nroots, o});
            k_gather<<<grid_for(nroots * o), 256, 0, c.stream>>>(nroots, o, xo, o, 0, Xp, nmo, 0, 0.0);
            launch_check(c);
            // virtual: T_{c,j} = t_j^c(2) [+ t_j^c(3) + 1/2 sum tau_jl^cd t_l^d(2)] ;
            // T_{c,ija} = -t_ij^ac [- t2_ij^ac]
            double* xv = c.arena.dalloc((size_t)nroots * v);
            einsum(c, "rj,jc->rc", 1.0, tn(s1, {nroots, o}), tn(t1, {o, v}), 0.0, xv, {nroots, v});
            einsum(c, "rija,ijac->rc", -1.0, tn(s2, {nroots, o, o, v}), T4, 1.0, xv, {nroots, v});
            if (third) einsum(c, "rija,ijac->rc", -1.0, tn(s2, {nroots, o, o, v}), op_t2(h, h->lean), 1.0, xv, {nroots, v});
            k_gather<<<grid_for(nroots * v), 256, 0, c.stream>>>(nroots, v, xv, v, 0, Xp, nmo, o, 0.0);
            launch_check(c);
        }
        std::vector<double> xh((size_t)nroots * nmo);
        ADC_CUDA(cudaMemcpyAsync(xh.data(), Xp, xh.size() * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
        ADC_CUDA(cudaStreamSynchronize(c.stream));
        h->X_last = xh;
        for (int r = 0; r < nroots; ++r) {
            double s = 0.0;
            for (long long p = 0; p < nmo; ++p) s += xh[(size_t)r * nmo + p] * xh[(size_t)r * nmo + p];
            specfac[r] = 2.0 * s;
        }
    }
    ADC_CUDA(cudaStreamSynchronize(c.stream));
    if (stats) {
        double mr = 0.0;
        for (double x : rn) mr = std::max(mr, x);
        stats[0] = std::min(it, maxit);
        stats[1] = (double)d.nsig;
        stats[2] = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        stats[3] = mr;
        stats[4] = d.sigma_seconds;
        stats[5] = refine_shift;
        stats[6] = refine_sec;
        int fell = 0;
        if (h->mlp_w)
            for (int r = 0; r < nroots; ++r) fell += diag_only[r];
        stats[7] = fell;
    }
    return status;
}

// --------------------------------------------------------------------------
// Training samples of the learned preconditioner from the handle's own plain
// Davidson: the iterates y after k iterations (the solver stopped at max_iter =
// k), their residuals r = sigma(y) - w y and the exact correction
// t* = y_exact / <y_exact, y>_S - y, with y_exact the tightly converged root of
// largest S-overlap.  Each sample is one vector element.
// --------------------------------------------------------------------------
static long long mlp_samples_per_vector(const adc_handle* h, long long per_vector) {
    const long long n1 = h->n1(), rest = h->dim() - n1;
    return n1 + std::min(std::max(per_vector, 0LL), rest);
}

static void mlp_samples(adc_handle* h, int nroots, const int* iters, int n_iters, long long per_vector,
                        unsigned long long seed, double exact_tol, double* od, unsigned char* ob, double* orr, double* ot) {
    Ctx& c = h->ctx;
    const long long dim = h->dim(), n1 = h->n1(), per = mlp_samples_per_vector(h, per_vector);
    const adc_options saved = h->opt;
    struct Restore {
        adc_handle* h;
        adc_options o;
        ~Restore() { h->opt = o; }
    } restore{h, saved};
    Scope sc(c.arena);
    std::vector<double> e(nroots), hv((size_t)nroots * dim);
    // exact roots
    h->opt.max_iter = std::max(200, saved.max_iter);
    h->opt.res_tol = saved.res_tol > 0 ? std::min(1e-6, saved.res_tol) : 1e-6;
    h->opt.refine_res_tol = 0.0;
    davidson(h, nroots, exact_tol, nullptr, e.data(), nullptr, hv.data(), nullptr);
    double* Yex = c.arena.dalloc((size_t)nroots * dim);
    double* SYex = c.arena.dalloc((size_t)nroots * dim);
    double* Y = c.arena.dalloc((size_t)nroots * dim);
    double* W = c.arena.dalloc((size_t)nroots * dim);
    double* ov = c.arena.dalloc((size_t)nroots * nroots);
    long long* di = (long long*)c.arena.alloc((size_t)per * sizeof(long long));
    double* sd = c.arena.dalloc((size_t)per);
    double* sr = c.arena.dalloc((size_t)per);
    double* st = c.arena.dalloc((size_t)per);
    unsigned char* sb = (unsigned char*)c.arena.alloc((size_t)per);
    ADC_CUDA(cudaMemcpyAsync(Yex, hv.data(), hv.size() * sizeof(double), cudaMemcpyHostToDevice, c.stream));
    k_metric<<<grid_for((long long)nroots * dim), 256, 0, c.stream>>>(h->kind == ADC_EA, h->o, h->v, nroots, Yex, SYex, 0);
    launch_check(c);
    // element choice: every 1p/1h element, then per - n1 distinct 2p1h/2h1p elements (Floyd's
    // sampling with a splitmix64 stream seeded by `seed`)
    unsigned long long state = seed;
    auto next = [&state]() {
        unsigned long long z = (state += 0x9E3779B97F4A7C15ULL);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
        return z ^ (z >> 31);
    };
    std::vector<long long> pick((size_t)per);
    long long out = 0;
    for (int ki = 0; ki < n_iters; ++ki) {
        h->opt = saved;
        h->opt.max_iter = std::max(1, iters[ki]);
        h->opt.res_tol = 1e-12;
        h->opt.refine_res_tol = 0.0;
        davidson(h, nroots, 1e-14, nullptr, e.data(), nullptr, hv.data(), nullptr);  // NOT_CONVERGED by design
        ADC_CUDA(cudaMemcpyAsync(Y, hv.data(), hv.size() * sizeof(double), cudaMemcpyHostToDevice, c.stream));
        sigma_device(h, Y, W, nroots);
        multidot(c, nroots, SYex, dim, nroots, Y, dim, dim, ov);  // ov[s][r] = <y_exact_s, y_r>_S
        std::vector<double> hov((size_t)nroots * nroots);
        ADC_CUDA(cudaMemcpyAsync(hov.data(), ov, hov.size() * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
        ADC_CUDA(cudaStreamSynchronize(c.stream));
        for (int r = 0; r < nroots; ++r) {
            int best = 0;
            for (int s2 = 1; s2 < nroots; ++s2)
                if (std::fabs(hov[(size_t)s2 * nroots + r]) > std::fabs(hov[(size_t)best * nroots + r])) best = s2;
            const double ovr = hov[(size_t)best * nroots + r];
            if (!(std::fabs(ovr) > 0)) throw Error(ADC_ERR_NONFINITE, "adc_mlp_samples: iterate orthogonal to every exact root");
            for (long long x = 0; x < n1; ++x) pick[x] = x;
            const long long rest = dim - n1, m = per - n1;
            std::vector<long long> chosen;
            chosen.reserve((size_t)m);
            {
                std::unordered_set<long long> used;
                for (long long j = rest - m; j < rest; ++j) {
                    long long q = (long long)(next() % (unsigned long long)(j + 1));
                    if (used.count(q)) q = j;
                    used.insert(q);
                    chosen.push_back(q);
                }
            }
            for (long long k = 0; k < m; ++k) pick[n1 + k] = n1 + chosen[k];
            ADC_CUDA(cudaMemcpyAsync(di, pick.data(), per * sizeof(long long), cudaMemcpyHostToDevice, c.stream));
            k_mlp_samples<<<grid_for(per), 256, 0, c.stream>>>(per, di, n1, h->diag, e[r], W + (long long)r * dim,
                                                                Y + (long long)r * dim, Yex + (long long)best * dim, 1.0 / ovr,
                                                                sd, sb, sr, st);
            launch_check(c);
            ADC_CUDA(cudaMemcpyAsync(od + out, sd, per * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
            ADC_CUDA(cudaMemcpyAsync(ob + out, sb, per, cudaMemcpyDeviceToHost, c.stream));
            ADC_CUDA(cudaMemcpyAsync(orr + out, sr, per * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
            ADC_CUDA(cudaMemcpyAsync(ot + out, st, per * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
            ADC_CUDA(cudaStreamSynchronize(c.stream));
            out += per;
        }
    }
}

// Internal accessor for the allocation-free ladder entry point (ladder_static.cu).
namespace adc {
bool handle_ladder_view(adc_handle* h, LadderTC** tc, Ctx** c, int* nvir, std::string** err, LadderMode* md) {
    if (!h) return false;
    *tc = h->tc;
    *md = h->lm_sigma;
    *c = &h->ctx;
    *nvir = h->v;
    *err = &h->err;
    return true;
}
}  // namespace adc

// --------------------------------------------------------------------------
// C ABI
// --------------------------------------------------------------------------
// --------------------------------------------------------------------------
// Unrestricted (open-shell) references: EA/IP-UADC(n) sigma (Sec. II, the
// UADC runs of Sec. IV), FP64.  The spin orbitals are ordered occupied alpha,
// occupied beta, virtual alpha, virtual beta; B^Q_PR is the per-spin DF factor
// on the spin-diagonal blocks and zero between spins, so (PR|QS) = sum_Q
// B^Q_PR B^Q_QS (Eq. 19 for each spin pair) and the ladder over its virtual
// block is the alpha-alpha, beta-beta and alpha-beta ladder at once.  The
// working equations are the spin-orbital ones (<pq||rs>, t antisymmetric);
// every integral with three or four virtual indices goes through B^Q.  The
// two-particle basis is (i, a<b) i-major (EA) and (i<j, a) a-major (IP);
// IP applies -M_-, as the closed-shell path does.
// --------------------------------------------------------------------------
namespace {

// F[r][i][a][b] = y, F[r][i][b][a] = -y (EA) / F[r][i][j][a] = y, F[r][j][i][a] = -y (IP)
__global__ void k_pairs_to_full(int ea, long long n, long long np, int o, int v, const int* __restrict__ idx,
                                const double* __restrict__ Y, long long ldy, long long off, double* __restrict__ F) {
    const long long blk = ea ? (long long)o * v * v : (long long)o * o * v;
    GRID_STRIDE(x, n * np) {
        const long long r = x / np, q = x % np;
        const int p0 = idx[q], p1 = idx[np + q], p2 = idx[2 * np + q];
        const double y = Y[r * ldy + off + q];
        if (ea) {
            F[r * blk + ((long long)p0 * v + p1) * v + p2] = y;
            F[r * blk + ((long long)p0 * v + p2) * v + p1] = -y;
        } else {
            F[r * blk + ((long long)p0 * o + p1) * v + p2] = y;
            F[r * blk + ((long long)p1 * o + p0) * v + p2] = -y;
        }
    }
}

// out[m][r][c] = F[m][r0 + r][c0 + c] for the nr x nc block of nmat v x v matrices
__global__ void k_block_get(long long nmat, int v, int r0, int nr, int c0, int nc, const double* __restrict__ F,
                            double* __restrict__ out) {
    GRID_STRIDE(x, nmat * nr * nc) {
        const int cc = x % nc;
        const long long t = x / nc;
        const int r = t % nr;
        const long long m = t / nr;
        out[x] = F[(m * v + r0 + r) * v + c0 + cc];
    }
}
// S[m][r0 + r][c0 + c] += sgn * (trans ? O[m][c][r] : O[m][r][c]), O of nmat matrices of nr x nc
// (trans: of nc x nr)
__global__ void k_block_add(long long nmat, int v, int r0, int nr, int c0, int nc, int trans, double sgn,
                            const double* __restrict__ O, double* __restrict__ S) {
    GRID_STRIDE(x, nmat * nr * nc) {
        const int cc = x % nc;
        const long long t = x / nc;
        const int r = t % nr;
        const long long m = t / nr;
        const double val = trans ? O[(m * nc + cc) * nr + r] : O[x];
        S[(m * v + r0 + r) * v + c0 + cc] += sgn * val;
    }
}

// preconditioner diagonal of an unrestricted handle: [diag of the applied 1p/1h block,
// zeroth-order pair energies] (EA: e_a + e_b - e_i; IP: -(e_i + e_j - e_a))
__global__ void k_diag_pairs(int ea, long long n1, long long np, int o, const int* __restrict__ idx,
                             const double* __restrict__ eps, const double* __restrict__ M11, double* __restrict__ D) {
    GRID_STRIDE(x, n1 + np) {
        if (x < n1) {
            D[x] = ea ? M11[x * n1 + x] : -M11[x * n1 + x];
        } else {
            const long long q = x - n1;
            const int p0 = idx[q], p1 = idx[np + q], p2 = idx[2 * np + q];
            D[x] = ea ? eps[o + p1] + eps[o + p2] - eps[p0] : -(eps[p0] + eps[p1] - eps[o + p2]);
        }
    }
}

// S[r][off + q] = alpha * F[r][pair q]
__global__ void k_full_to_pairs(int ea, long long n, long long np, int o, int v, const int* __restrict__ idx,
                                const double* __restrict__ F, double alpha, double* __restrict__ S, long long lds, long long off) {
    const long long blk = ea ? (long long)o * v * v : (long long)o * o * v;
    GRID_STRIDE(x, n * np) {
        const long long r = x / np, q = x % np;
        const int p0 = idx[q], p1 = idx[np + q], p2 = idx[2 * np + q];
        const long long e = ea ? ((long long)p0 * v + p1) * v + p2 : ((long long)p0 * o + p1) * v + p2;
        S[r * lds + off + q] = alpha * F[r * blk + e];
    }
}

// out = alpha * perm(in) + beta * out for a 4-index tensor
void perm4(Ctx& c, const double* in, std::initializer_list<long long> d, std::initializer_list<int> p, double* out,
           double alpha, double beta) {
    Shape s{4, {0, 0, 0, 0}};
    int k = 0;
    for (long long x : d) s.d[k++] = x;
    int pp[4];
    k = 0;
    for (int x : p) pp[k++] = x;
    permute(c, in, s, pp, out, alpha, beta);
}

}  // namespace

// M += alpha (X + X^T) for an n x n X
static void sym_add_n(adc_handle* h, const double* X, double* M, long long n, double alpha) { sym_add(h, X, M, (int)n, alpha); }

// The ladder of an open-shell reference on the tensor cores, per spin block (Eq. 19 per
// spin pair): B^Q of the virtual spin orbitals is block diagonal (alpha, beta), so for the
// antisymmetric F_n (v x v, alpha virtuals first)
//   out_aa += sum_Q Ba F_aa Ba,  out_bb += sum_Q Bb F_bb Bb,  out_ab += sum_Q Ba F_ab Bb,
// and out_ba = -out_ab^T (the ladder keeps the antisymmetry).  Three tensor-core ladders
// instead of one over the spin-orbital factor, half of which is zeros.
static void ladder_open_shell(adc_handle* h, const double* F, long long nmat, double* out, const LadderMode& md) {
    Ctx& c = h->ctx;
    const int v = h->v, va = h->nva, vb = h->v - h->nva;
    Scope sc(c.arena);
    double* X = c.arena.dalloc((size_t)nmat * std::max(va, vb) * std::max(va, vb));
    double* O = c.arena.dalloc((size_t)nmat * std::max(va, vb) * std::max(va, vb));
    auto block = [&](LadderTC* l, LadderTC* r, int r0, int nr, int c0, int nc, bool both) {
        if (nr <= 0 || nc <= 0) return;
        k_block_get<<<grid_for(nmat * nr * nc), 256, 0, c.stream>>>(nmat, v, r0, nr, c0, nc, F, X);
        launch_check(c);
        fill(c, nmat * nr * nc, 0.0, O);
        ladder_tc_apply_pair(*l, *r, c, X, nmat, O, md);
        k_block_add<<<grid_for(nmat * nr * nc), 256, 0, c.stream>>>(nmat, v, r0, nr, c0, nc, 0, 1.0, O, out);
        launch_check(c);
        if (both) {  // the transposed block by antisymmetry
            k_block_add<<<grid_for(nmat * nr * nc), 256, 0, c.stream>>>(nmat, v, c0, nc, r0, nr, 1, -1.0, O, out);
            launch_check(c);
        }
    };
    block(h->tc, h->tc, 0, va, 0, va, false);
    block(h->tc_b, h->tc_b, va, vb, va, vb, false);
    block(h->tc, h->tc_b, 0, va, va, vb, true);
}

static void setup_unrestricted(adc_handle* h, const double* eps_so, const double* Bso) {
    Ctx& c = h->ctx;
    ADC_BLAS(cublasCreate(&c.blas));
    ADC_BLAS(cublasSetStream(c.blas, c.stream));
    ADC_BLAS(cublasSetMathMode(c.blas, CUBLAS_DEFAULT_MATH));
    // setup (and the refinement of converged roots) in FP64; mixed precision: the sigma's
    // contractions on the tensor cores / own kernels and its ladder per spin block on the
    // tensor cores (the split B^Q are made at the end of setup, so the setup ladders are FP64)
    c.gemm_mode = 0;
    h->cmode_setup = h->cmode_refine = 0;
    h->cmode_sigma = h->opt.precision != ADC_PREC_FP64 ? (h->opt.contractions >= 0 ? h->opt.contractions : 2) : 0;
    if (h->opt.tune_cache && h->opt.tune_cache[0]) c.tuner = tune_cache_open(h->opt.tune_cache);
    h->opt.tune_cache = nullptr;
    const long long o = h->o, v = h->v, Q = h->naux, nso = o + v;
    const long long o2v2 = o * o * v * v;
    h->eps = h->dmalloc(nso);
    ADC_CUDA(cudaMemcpyAsync(h->eps, eps_so, nso * sizeof(double), cudaMemcpyHostToDevice, c.stream));
    h->Boo = h->dmalloc(Q * o * o);
    h->Bov = h->dmalloc(Q * o * v);
    h->Bvv = h->dmalloc(Q * v * v);
    for (long long q = 0; q < Q; ++q) {
        const double* src = Bso + q * nso * nso;
        ADC_CUDA(cudaMemcpy2DAsync(h->Boo + q * o * o, o * sizeof(double), src, nso * sizeof(double), o * sizeof(double), o,
                                   cudaMemcpyHostToDevice, c.stream));
        ADC_CUDA(cudaMemcpy2DAsync(h->Bov + q * o * v, v * sizeof(double), src + o, nso * sizeof(double), v * sizeof(double), o,
                                   cudaMemcpyHostToDevice, c.stream));
        ADC_CUDA(cudaMemcpy2DAsync(h->Bvv + q * v * v, v * sizeof(double), src + o * nso + o, nso * sizeof(double),
                                   v * sizeof(double), v, cudaMemcpyHostToDevice, c.stream));
    }
    // pair basis
    {
        const long long np = h->npairs();
        std::vector<int> idx((size_t)3 * np);
        long long q = 0;
        if (h->kind == ADC_EA) {
            for (int i = 0; i < o; ++i)
                for (int a = 0; a < v; ++a)
                    for (int b = a + 1; b < v; ++b, ++q) idx[q] = i, idx[np + q] = a, idx[2 * np + q] = b;
        } else {
            for (int a = 0; a < v; ++a)
                for (int i = 0; i < o; ++i)
                    for (int j = i + 1; j < o; ++j, ++q) idx[q] = i, idx[np + q] = j, idx[2 * np + q] = a;
        }
        h->pair_idx = (int*)dev_alloc(std::max<size_t>(idx.size(), 1) * sizeof(int), c.stream);
        h->owned.push_back(h->pair_idx);
        if (!idx.empty())
            ADC_CUDA(cudaMemcpyAsync(h->pair_idx, idx.data(), idx.size() * sizeof(int), cudaMemcpyHostToDevice, c.stream));
        ADC_CUDA(cudaStreamSynchronize(c.stream));  // idx is a host temporary
    }
    const T Boo = tn(h->Boo, {Q, o, o}), Bov = tn(h->Bov, {Q, o, v}), Bvv = tn(h->Bvv, {Q, v, v});
    h->ovov = h->dmalloc(o2v2);
    h->oovv = h->dmalloc(o2v2);
    h->oooo = h->dmalloc(o * o * o * o);
    h->ooov = h->dmalloc(o * o * o * v);
    einsum(c, "Qia,Qjb->iajb", 1.0, Bov, Bov, 0.0, h->ovov, {o, v, o, v});
    einsum(c, "Qij,Qab->ijab", 1.0, Boo, Bvv, 0.0, h->oovv, {o, o, v, v});
    einsum(c, "Qij,Qkl->ijkl", 1.0, Boo, Boo, 0.0, h->oooo, {o, o, o, o});
    einsum(c, "Qij,Qka->ijka", 1.0, Boo, Bov, 0.0, h->ooov, {o, o, o, v});
    // antisymmetrised blocks with at most two virtual indices
    h->g_oovv = h->dmalloc(o2v2);  // <ij||ab> = (ia|jb) - (ib|ja)
    perm4(c, h->ovov, {o, v, o, v}, {0, 2, 1, 3}, h->g_oovv, 1.0, 0.0);
    perm4(c, h->ovov, {o, v, o, v}, {0, 2, 3, 1}, h->g_oovv, -1.0, 1.0);
    h->g_oooo = h->dmalloc(o * o * o * o);  // <ij||kl> = (ik|jl) - (il|jk)
    perm4(c, h->oooo, {o, o, o, o}, {0, 2, 1, 3}, h->g_oooo, 1.0, 0.0);
    perm4(c, h->oooo, {o, o, o, o}, {0, 2, 3, 1}, h->g_oooo, -1.0, 1.0);
    h->g_ooov = h->dmalloc(o * o * o * v);  // <ij||ka> = (ik|ja) - (ia|jk)
    perm4(c, h->ooov, {o, o, o, v}, {0, 2, 1, 3}, h->g_ooov, 1.0, 0.0);
    perm4(c, h->ooov, {o, o, o, v}, {2, 0, 1, 3}, h->g_ooov, -1.0, 1.0);
    h->g_ovov = h->dmalloc(o2v2);  // <ia||jb> = (ij|ab) - (ib|ja)
    perm4(c, h->oovv, {o, o, v, v}, {0, 2, 1, 3}, h->g_ovov, 1.0, 0.0);
    perm4(c, h->ovov, {o, v, o, v}, {0, 3, 2, 1}, h->g_ovov, -1.0, 1.0);
    h->g_vovo = h->dmalloc(o2v2);  // <ai||bj> = (ab|ij) - (aj|ib)
    perm4(c, h->oovv, {o, o, v, v}, {2, 0, 3, 1}, h->g_vovo, 1.0, 0.0);
    perm4(c, h->ovov, {o, v, o, v}, {1, 2, 3, 0}, h->g_vovo, -1.0, 1.0);
    h->g_vooo = h->dmalloc(o * o * o * v);  // <ai||jk> = (aj|ik) - (ak|ij)
    perm4(c, h->ooov, {o, o, o, v}, {3, 0, 2, 1}, h->g_vooo, 1.0, 0.0);
    perm4(c, h->ooov, {o, o, o, v}, {3, 0, 1, 2}, h->g_vooo, -1.0, 1.0);
    // first-order doubles t_ij^ab = <ij||ab> / D_ij^ab
    h->t = h->dmalloc(o2v2);
    ADC_CUDA(cudaMemcpyAsync(h->t, h->g_oovv, o2v2 * sizeof(double), cudaMemcpyDeviceToDevice, c.stream));
    k_div_D2<<<grid_for(o2v2), 256, 0, c.stream>>>((int)o, (int)v, h->eps, h->t);
    launch_check(c);
    const double* t = h->t;
    const T T4 = tn(t, {o, o, v, v}), goovv = tn(h->g_oovv, {o, o, v, v});
    Scope sc(c.arena);
    if (h->order >= 3) {
        // t2(2) = [sum (ac|bd) t_ij^cd + 1/2 <kl||ij> t_kl^ab + P(ij)P(ab) <kb||cj> t_ik^ac] / D
        h->t_2 = h->dmalloc(o2v2);
        double* N = h->t_2;
        fill(c, o2v2, 0.0, N);
        ladder(h, t, o * o, N, h->lm_setup);
        einsum(c, "klij,klab->ijab", 0.5, tn(h->g_oooo, {o, o, o, o}), T4, 1.0, N, {o, o, v, v});
        // <kb||cj> = <kb||cj> from g_ovvo[k,b,c,j] = (kc|jb) - (kj|bc)
        double* gvo = c.arena.dalloc(o2v2);  // [k,b,c,j]
        perm4(c, h->ovov, {o, v, o, v}, {0, 3, 1, 2}, gvo, 1.0, 0.0);
        perm4(c, h->oovv, {o, o, v, v}, {0, 2, 3, 1}, gvo, -1.0, 1.0);
        double* X = c.arena.dalloc(o2v2);
        einsum(c, "kbcj,ikac->ijab", 1.0, tn(gvo, {o, v, v, o}), T4, 0.0, X, {o, o, v, v});
        axpby(c, o2v2, 1.0, X, 1.0, N);
        perm4(c, X, {o, o, v, v}, {1, 0, 2, 3}, N, -1.0, 1.0);
        perm4(c, X, {o, o, v, v}, {0, 1, 3, 2}, N, -1.0, 1.0);
        perm4(c, X, {o, o, v, v}, {1, 0, 3, 2}, N, 1.0, 1.0);
        k_div_D2<<<grid_for(o2v2), 256, 0, c.stream>>>((int)o, (int)v, h->eps, N);
        launch_check(c);
        // t1(2) = [-(kc|ad) t_ik^cd - 1/2 <kl||ic> t_kl^ac] / D
        h->t1_2 = h->dmalloc(o * v);
        double* G = c.arena.dalloc(Q * o * v);
        einsum(c, "Qkc,ikcd->Qid", 1.0, Bov, T4, 0.0, G, {Q, o, v});
        einsum(c, "Qid,Qad->ia", -1.0, tn(G, {Q, o, v}), Bvv, 0.0, h->t1_2, {o, v});
        einsum(c, "klic,klac->ia", -0.5, tn(h->g_ooov, {o, o, o, v}), T4, 1.0, h->t1_2, {o, v});
        k_div_D1<<<grid_for(o * v), 256, 0, c.stream>>>((int)o, (int)v, h->eps, h->t1_2);
        launch_check(c);
    }
    // one-particle block (EA: M_ab; IP: the paper's M_ij, negated when applied)
    const long long n1 = h->n1();
    h->M11 = h->dmalloc(n1 * n1);
    {
        std::vector<double> e0((size_t)n1 * n1, 0.0), eh(nso);
        for (long long k = 0; k < nso; ++k) eh[k] = eps_so[k];
        for (long long k = 0; k < n1; ++k) e0[k * n1 + k] = h->kind == ADC_EA ? eh[o + k] : eh[k];
        ADC_CUDA(cudaMemcpyAsync(h->M11, e0.data(), e0.size() * sizeof(double), cudaMemcpyHostToDevice, c.stream));
        ADC_CUDA(cudaStreamSynchronize(c.stream));
    }
    double* M = h->M11;
    double* X = c.arena.dalloc(std::max(v * v, o * o));
    const bool third = h->order >= 3;
    if (h->kind == ADC_EA) {
        einsum(c, "klac,klbc->ab", 1.0, T4, goovv, 0.0, X, {v, v});
        sym_add_n(h, X, M, v, -0.25);
        if (third) {
            const T t1 = tn(h->t1_2, {o, v}), T2 = tn(h->t_2, {o, o, v, v});
            // t_k^c <ka||cb>, <ka||cb> = (kc|ab) - (kb|ac)
            double* r = c.arena.dalloc(Q);
            einsum(c, "kc,Qkc->Q", 1.0, t1, Bov, 0.0, r, {Q});
            einsum(c, "Q,Qab->ab", 1.0, tn(r, {Q}), Bvv, 0.0, X, {v, v});
            double* Z = c.arena.dalloc(Q * v * v);
            einsum(c, "kc,Qkb->Qbc", 1.0, t1, Bov, 0.0, Z, {Q, v, v});
            einsum(c, "Qac,Qbc->ab", -1.0, Bvv, tn(Z, {Q, v, v}), 1.0, X, {v, v});
            sym_add_n(h, X, M, v, 1.0);
            einsum(c, "klac,klbc->ab", 1.0, T2, goovv, 0.0, X, {v, v});
            sym_add_n(h, X, M, v, -0.25);
            // t_kl^ac <bc||de> t_kl^de = 2 t_kl^ac (sum_Q B^Q t_kl B^Q)^bc
            double* L = c.arena.dalloc(o2v2);
            fill(c, o2v2, 0.0, L);
            ladder(h, t, o * o, L, h->lm_setup);
            einsum(c, "klac,klbc->ab", 2.0, T4, tn(L, {o, o, v, v}), 0.0, X, {v, v});
            sym_add_n(h, X, M, v, -0.125);
            // 1/2 <ac||bd> rho_cd, <ac||bd> = (ab|cd) - (ad|cb), rho_cd = t_kl^ce t_kl^de
            double* rho = c.arena.dalloc(v * v);
            einsum(c, "klce,klde->cd", 1.0, T4, T4, 0.0, rho, {v, v});
            einsum(c, "Qcd,cd->Q", 1.0, Bvv, tn(rho, {v, v}), 0.0, r, {Q});
            einsum(c, "Q,Qab->ab", 0.5, tn(r, {Q}), Bvv, 1.0, M, {v, v});
            einsum(c, "Qad,cd->Qac", 1.0, Bvv, tn(rho, {v, v}), 0.0, Z, {Q, v, v});
            einsum(c, "Qac,Qcb->ab", -0.5, tn(Z, {Q, v, v}), Bvv, 1.0, M, {v, v});
            // ring terms with <kd||lb>
            const T gov = tn(h->g_ovov, {o, v, o, v});
            double* V1 = c.arena.dalloc(o2v2);  // [k,a,l,d]
            einsum(c, "kmac,lmcd->kald", 1.0, T4, T4, 0.0, V1, {o, v, o, v});
            einsum(c, "kald,kdlb->ab", 1.0, tn(V1, {o, v, o, v}), gov, 0.0, X, {v, v});
            sym_add_n(h, X, M, v, -0.5);
            double* u = c.arena.dalloc(o * o);
            einsum(c, "kmcd,lmcd->kl", 1.0, T4, T4, 0.0, u, {o, o});
            einsum(c, "kalb,kl->ab", -0.5, gov, tn(u, {o, o}), 1.0, M, {v, v});
        }
    } else {
        einsum(c, "ilcd,jlcd->ij", 1.0, T4, goovv, 0.0, X, {o, o});
        sym_add_n(h, X, M, o, 0.25);
        if (third) {
            const T t1 = tn(h->t1_2, {o, v}), T2 = tn(h->t_2, {o, o, v, v});
            const T gvooo = tn(h->g_vooo, {v, o, o, o}), goooo = tn(h->g_oooo, {o, o, o, o});
            einsum(c, "kc,cikj->ij", 1.0, t1, gvooo, 0.0, X, {o, o});
            sym_add_n(h, X, M, o, 1.0);
            einsum(c, "ikcd,jkcd->ij", 1.0, T2, goovv, 0.0, X, {o, o});
            sym_add_n(h, X, M, o, 0.25);
            double* Z = c.arena.dalloc(o * o * o * o);
            einsum(c, "ikcd,lmcd->iklm", 1.0, T4, T4, 0.0, Z, {o, o, o, o});
            einsum(c, "iklm,jklm->ij", 1.0, tn(Z, {o, o, o, o}), goooo, 0.0, X, {o, o});
            sym_add_n(h, X, M, o, 0.125);
            double* u = c.arena.dalloc(o * o);
            einsum(c, "kmcd,lmcd->kl", 1.0, T4, T4, 0.0, u, {o, o});
            einsum(c, "ikjl,kl->ij", -0.5, goooo, tn(u, {o, o}), 1.0, M, {o, o});
            const T gvovo = tn(h->g_vovo, {v, o, v, o});
            double* A = c.arena.dalloc(o2v2);  // [i,c,l,d]
            einsum(c, "ikce,klde->icld", 1.0, T4, T4, 0.0, A, {o, v, o, v});
            einsum(c, "icld,cldj->ij", 1.0, tn(A, {o, v, o, v}), gvovo, 0.0, X, {o, o});
            sym_add_n(h, X, M, o, 0.5);
            double* rho = c.arena.dalloc(v * v);
            einsum(c, "klce,klde->cd", 1.0, T4, T4, 0.0, rho, {v, v});
            einsum(c, "cidj,cd->ij", 0.5, gvovo, tn(rho, {v, v}), 1.0, M, {o, o});
        }
        // coupling M[i,j,k,a] = <jk||ia> (- 1/2 <ai||de> t_jk^de - (X - X^jk), X = <il||kc> t_jl^ac)
        const long long o3v = o * o * o * v;
        h->m12 = h->dmalloc(o3v);
        perm4(c, h->g_ooov, {o, o, o, v}, {2, 0, 1, 3}, h->m12, 1.0, 0.0);
        if (third) {
            // - sum_Q sum_d (sum_e B^Q_ie t_jk^de) B^Q_ad through G[Q,i,j,k,d], the auxiliary index in
            // chunks (aux_chunk, else G of at most 2^27 elements = 1 GiB per chunk)
            const long long qc = h->opt.aux_chunk > 0 ? std::min<long long>(Q, h->opt.aux_chunk)
                                                      : std::max(1LL, std::min(Q, (1LL << 27) / std::max(o3v, 1LL)));
            double* G = c.arena.dalloc(qc * o3v);
            for (long long q0 = 0; q0 < Q; q0 += qc) {
                const long long nq = std::min(qc, Q - q0);
                einsum(c, "Qie,jkde->Qijkd", 1.0, tn(h->Bov + q0 * o * v, {nq, o, v}), T4, 0.0, G, {nq, o, o, o, v});
                einsum(c, "Qijkd,Qad->ijka", -1.0, tn(G, {nq, o, o, o, v}), tn(h->Bvv + q0 * v * v, {nq, v, v}), 1.0,
                       h->m12, {o, o, o, v});
            }
            double* Xc = c.arena.dalloc(o3v);
            einsum(c, "ilkc,jlac->ijka", 1.0, tn(h->g_ooov, {o, o, o, v}), T4, 0.0, Xc, {o, o, o, v});
            axpby(c, o3v, -1.0, Xc, 1.0, h->m12);
            perm4(c, Xc, {o, o, o, v}, {0, 2, 1, 3}, h->m12, 1.0, 1.0);
        }
    }
    if (h->opt.precision != ADC_PREC_FP64) {
        // per-spin virtual blocks of B^Q for the tensor-core ladders of sigma
        const int va = h->nva, vb = (int)v - h->nva;
        double* Ba = h->dmalloc(Q * va * va);
        double* Bb = h->dmalloc(Q * vb * vb);
        k_block_get<<<grid_for(Q * va * va), 256, 0, c.stream>>>(Q, (int)v, 0, va, 0, va, h->Bvv, Ba);
        launch_check(c);
        k_block_get<<<grid_for(Q * vb * vb), 256, 0, c.stream>>>(Q, (int)v, va, vb, va, vb, h->Bvv, Bb);
        launch_check(c);
        h->tc = ladder_tc_create(c, Ba, (int)Q, va, h->opt.aux_chunk);
        h->tc_b = ladder_tc_create(c, Bb, (int)Q, vb, h->opt.aux_chunk);
    }
    // Davidson preconditioner diagonal (S = 1 in the antisymmetric pair basis)
    h->diag = h->dmalloc(h->dim());
    k_diag_pairs<<<grid_for(h->dim()), 256, 0, c.stream>>>(h->kind == ADC_EA, n1, h->npairs(), (int)o, h->pair_idx, h->eps,
                                                            h->M11, h->diag);
    launch_check(c);
    ADC_CUDA(cudaStreamSynchronize(c.stream));
}

// Third-order singles of an open-shell reference (Eq. t_singles at k = 3, the
// spin-orbital form: t antisymmetric, <pq||rs>), FP64, made on first use:
//   D t(3) = A + (2 E1 + E2 + 4 E3 + 2 E4)/4 - (2 F1 + 4 F2 + F3 + 2 F4)/4,  t(3) += 1/2 sum t_ij^ab t_j^b(2)
// A: the t1(2)-, t2(2)- and singles-shaped terms; E1..E4 / F1..F4: the connected
// triples-shaped term by particle / hole half.  Every integral with three virtual
// indices goes through B^Q (Eq. 19); E2 runs in auxiliary chunks.
static void make_t1_third_order_u(adc_handle* h) {
    if (h->t1_3 || h->order < 3) return;
    Ctx& c = h->ctx;
    const long long o = h->o, v = h->v, Q = h->naux, o2v2 = o * o * v * v;
    double* out = h->dmalloc(o * v);
    Scope sc(c.arena);
    const T T4 = tn(h->t, {o, o, v, v}), T2 = tn(h->t_2, {o, o, v, v}), t1 = tn(h->t1_2, {o, v});
    const T Bov = tn(h->Bov, {Q, o, v}), Bvv = tn(h->Bvv, {Q, v, v});
    double* num = c.arena.dalloc(o * v);
    double* G = c.arena.dalloc(Q * std::max(o * v, o * o));
    // A = sum (ia|jb) t_j^b - sum (ji|ab) t_j^b + singles(t2(2)),
    // singles(x) = -sum_Q sum_kcd B^Q_kc B^Q_ad x_ik^cd - 1/2 sum <kl||ic> x_kl^ac
    einsum(c, "iajb,jb->ia", 1.0, tn(h->ovov, {o, v, o, v}), t1, 0.0, num, {o, v});
    einsum(c, "jiab,jb->ia", -1.0, tn(h->oovv, {o, o, v, v}), t1, 1.0, num, {o, v});
    einsum(c, "Qkc,ikcd->Qid", 1.0, Bov, T2, 0.0, G, {Q, o, v});
    einsum(c, "Qid,Qad->ia", -1.0, tn(G, {Q, o, v}), Bvv, 1.0, num, {o, v});
    einsum(c, "klic,klac->ia", -0.5, tn(h->g_ooov, {o, o, o, v}), T2, 1.0, num, {o, v});
    // E1/2 = sum t_ij^ad Y_jd, Y_jd = 2 sum_Q sum_b B^Q_bd (sum_kc B^Q_kc t_jk^bc)
    double* Y = c.arena.dalloc(o * v);
    einsum(c, "Qkc,jkbc->Qjb", 1.0, Bov, T4, 0.0, G, {Q, o, v});
    einsum(c, "Qjb,Qbd->jd", 2.0, tn(G, {Q, o, v}), Bvv, 0.0, Y, {o, v});
    einsum(c, "ijad,jd->ia", 0.5, T4, tn(Y, {o, v}), 1.0, num, {o, v});
    {
        // E2/4 = 1/2 sum t_jk^ad V_jkdi, V_jkdi = sum_Q sum_b B^Q_bd sum_c t_jk^bc B^Q_ic
        Scope s2(c.arena);
        const long long per = o * o * v * o;
        double* V = c.arena.dalloc(per);
        const long long qc = h->opt.aux_chunk > 0 ? std::min<long long>(Q, h->opt.aux_chunk)
                                                  : std::max(1LL, std::min(Q, (1LL << 27) / std::max(per, 1LL)));
        double* W = c.arena.dalloc(qc * per);  // [Q][j][k][b][i]
        for (long long q0 = 0; q0 < Q; q0 += qc) {
            const long long nq = std::min(qc, Q - q0);
            einsum(c, "jkbc,Qic->Qjkbi", 1.0, T4, tn(h->Bov + q0 * o * v, {nq, o, v}), 0.0, W, {nq, o, o, v, o});
            einsum(c, "Qjkbi,Qbd->jkdi", 1.0, tn(W, {nq, o, o, v, o}), tn(h->Bvv + q0 * v * v, {nq, v, v}),
                   q0 == 0 ? 0.0 : 1.0, V, {o, o, v, o});
        }
        einsum(c, "jkad,jkdi->ia", 0.5, T4, tn(V, {o, o, v, o}), 1.0, num, {o, v});
    }
    {
        // E3 = -(sum_Q B^Q_ad B^Q_kc R_ikcd - sum_Q B^Q_ka B^Q_cd R_ikcd), R_ikcd = sum_jb t_ij^bd t_jk^bc
        Scope s2(c.arena);
        double* R = c.arena.dalloc(o2v2);
        einsum(c, "ijbd,jkbc->ikcd", 1.0, T4, T4, 0.0, R, {o, o, v, v});
        einsum(c, "Qkc,ikcd->Qid", 1.0, Bov, tn(R, {o, o, v, v}), 0.0, G, {Q, o, v});
        einsum(c, "Qid,Qad->ia", -1.0, tn(G, {Q, o, v}), Bvv, 1.0, num, {o, v});
        einsum(c, "Qcd,ikcd->Qik", 1.0, Bvv, tn(R, {o, o, v, v}), 0.0, G, {Q, o, o});
        einsum(c, "Qik,Qka->ia", 1.0, tn(G, {Q, o, o}), Bov, 1.0, num, {o, v});
    }
    {
        // E4/2 = -1/2 (sum_Q B^Q_ad B^Q_ic rho_cd - sum_Q B^Q_ia B^Q_cd rho_cd), rho_cd = sum t_jk^bc t_jk^bd
        double* rho = c.arena.dalloc(v * v);
        double* r = c.arena.dalloc(Q);
        einsum(c, "jkbc,jkbd->cd", 1.0, T4, T4, 0.0, rho, {v, v});
        einsum(c, "Qic,cd->Qid", 1.0, Bov, tn(rho, {v, v}), 0.0, G, {Q, o, v});
        einsum(c, "Qid,Qad->ia", -0.5, tn(G, {Q, o, v}), Bvv, 1.0, num, {o, v});
        einsum(c, "Qcd,cd->Q", 1.0, Bvv, tn(rho, {v, v}), 0.0, r, {Q});
        einsum(c, "Qia,Q->ia", 0.5, Bov, tn(r, {Q}), 1.0, num, {o, v});
    }
    {
        // F terms with <ia||jk> = (ij|ak) - (ik|aj), stored gov[i][a][j][k]
        Scope s2(c.arena);
        double* gov = c.arena.dalloc(o * v * o * o);
        perm4(c, h->ooov, {o, o, o, v}, {0, 3, 1, 2}, gov, 1.0, 0.0);
        perm4(c, h->ooov, {o, o, o, v}, {0, 3, 2, 1}, gov, -1.0, 1.0);
        const T GOV = tn(gov, {o, v, o, o});
        // -F1/2: F1 = sum t_il^ab U1_lb, U1_lb = sum t_jk^bc <lc||jk>
        double* U1 = c.arena.dalloc(o * v);
        einsum(c, "jkbc,lcjk->lb", 1.0, T4, GOV, 0.0, U1, {o, v});
        einsum(c, "ilab,lb->ia", -0.5, T4, tn(U1, {o, v}), 1.0, num, {o, v});
        // -F2: F2 = -sum <lc||ik> t_jk^bc t_jl^ab
        double* U2 = c.arena.dalloc(o * o * o * v);  // [l][i][j][b]
        einsum(c, "lcik,jkbc->lijb", 1.0, GOV, T4, 0.0, U2, {o, o, o, v});
        einsum(c, "lijb,jlab->ia", 1.0, tn(U2, {o, o, o, v}), T4, 1.0, num, {o, v});
        // -F3/4: F3 = sum <la||jk> t_jk^bc t_il^bc
        double* U3 = c.arena.dalloc(o * o * o * o);  // [j][k][i][l]
        einsum(c, "jkbc,ilbc->jkil", 1.0, T4, T4, 0.0, U3, {o, o, o, o});
        einsum(c, "lajk,jkil->ia", -0.25, GOV, tn(U3, {o, o, o, o}), 1.0, num, {o, v});
        // -F4/2: F4 = -sum <la||ik> t_jk^bc t_jl^bc
        double* U4 = c.arena.dalloc(o * o);
        einsum(c, "jkbc,jlbc->kl", 1.0, T4, T4, 0.0, U4, {o, o});
        einsum(c, "laik,kl->ia", 0.5, GOV, tn(U4, {o, o}), 1.0, num, {o, v});
    }
    k_div_D1<<<grid_for(o * v), 256, 0, c.stream>>>((int)o, (int)v, h->eps, num);
    launch_check(c);
    ADC_CUDA(cudaMemcpyAsync(out, num, o * v * sizeof(double), cudaMemcpyDeviceToDevice, c.stream));
    einsum(c, "ijab,jb->ia", 0.5, T4, t1, 1.0, out, {o, v});
    h->t1_3 = out;
}

// Spectroscopic factors of an open-shell reference (Eq. spec_factors with T from
// Eqs. T_ea, T_ip through order n, spin-orbital form): X_p = sum_nu T_p,nu Y_nu for
// Y normalised (S = 1), P = sum_p X_p^2 (one spin-orbital component: a Koopmans
// state has P = 1).  Pair columns act through the full antisymmetric tensor F
// (sum over i, a<b of T y = 1/2 sum over i, a, b of T F).
static void specfac_unrestricted(adc_handle* h, const double* Y, int nroots, double* specfac) {
    Ctx& c = h->ctx;
    Scope sc(c.arena);
    const long long o = h->o, v = h->v, nso = o + v, n1 = h->n1(), np = h->npairs(), dim = h->dim(), n = nroots;
    const bool ea = h->kind == ADC_EA;
    const bool third = h->order >= 3 && h->opt.transition_order != 2;
    if (third) make_t1_third_order_u(h);
    const long long blk = ea ? o * v * v : o * o * v;
    double* y1 = c.arena.dalloc(n * n1);
    double* F = c.arena.dalloc(n * blk);
    k_gather<<<grid_for(n * n1), 256, 0, c.stream>>>(n, n1, Y, dim, 0, y1, n1, 0, 0.0);
    launch_check(c);
    fill(c, n * blk, 0.0, F);
    k_pairs_to_full<<<grid_for(n * np), 256, 0, c.stream>>>(ea, n, np, (int)o, (int)v, h->pair_idx, Y, dim, n1, F);
    launch_check(c);
    const T T4 = tn(h->t, {o, o, v, v}), Y1 = tn(y1, {n, n1});
    double* tt = c.arena.dalloc(o * o * v * v);  // t2(1) [+ t2(2)]
    ADC_CUDA(cudaMemcpyAsync(tt, h->t, o * o * v * v * sizeof(double), cudaMemcpyDeviceToDevice, c.stream));
    if (third) axpby(c, o * o * v * v, 1.0, h->t_2, 1.0, tt);
    double* t1x = c.arena.dalloc(o * v);  // t1(2) [+ t1(3) + 1/2 sum t t1(2)]
    if (h->t1_2) {
        ADC_CUDA(cudaMemcpyAsync(t1x, h->t1_2, o * v * sizeof(double), cudaMemcpyDeviceToDevice, c.stream));
    } else {
        // ADC(2): second-order singles of the spin-orbital form, -(kc|ad) t_ik^cd - 1/2 <kl||ic> t_kl^ac
        const long long Q = h->naux;
        double* G = c.arena.dalloc(Q * o * v);
        einsum(c, "Qkc,ikcd->Qid", 1.0, tn(h->Bov, {Q, o, v}), T4, 0.0, G, {Q, o, v});
        einsum(c, "Qid,Qad->ia", -1.0, tn(G, {Q, o, v}), tn(h->Bvv, {Q, v, v}), 0.0, t1x, {o, v});
        einsum(c, "klic,klac->ia", -0.5, tn(h->g_ooov, {o, o, o, v}), T4, 1.0, t1x, {o, v});
        k_div_D1<<<grid_for(o * v), 256, 0, c.stream>>>((int)o, (int)v, h->eps, t1x);
        launch_check(c);
    }
    if (third) {
        axpby(c, o * v, 1.0, h->t1_3, 1.0, t1x);
        einsum(c, ea ? "klbc,lc->kb" : "jlcd,ld->jc", 0.5, T4, tn(h->t1_2, {o, v}), 1.0, t1x, {o, v});
    }
    double* Xp = c.arena.dalloc(n * nso);
    double* xo = c.arena.dalloc(n * o);
    double* xv = c.arena.dalloc(n * v);
    if (ea) {
        // virtual rows: T_cb = d_cb - 1/4 sum t_kl^cd t_kl^bd [- 1/4 (t t2 + t2 t)]
        double* Tvv = c.arena.dalloc(v * v);
        einsum(c, "klcd,klbd->cb", -0.25, T4, T4, 0.0, Tvv, {v, v});
        if (third) {
            einsum(c, "klcd,klbd->cb", -0.25, T4, tn(h->t_2, {o, o, v, v}), 1.0, Tvv, {v, v});
            einsum(c, "klcd,klbd->cb", -0.25, tn(h->t_2, {o, o, v, v}), T4, 1.0, Tvv, {v, v});
        }
        ADC_CUDA(cudaMemcpyAsync(xv, y1, n * v * sizeof(double), cudaMemcpyDeviceToDevice, c.stream));
        einsum(c, "rb,cb->rc", 1.0, Y1, tn(Tvv, {v, v}), 1.0, xv, {n, v});
        // occupied rows: T_kb = -t1x_kb; T_k,iab = t_ki^ab [+ t2_ki^ab]
        einsum(c, "rb,kb->rk", -1.0, Y1, tn(t1x, {o, v}), 0.0, xo, {n, o});
        einsum(c, "riab,kiab->rk", 0.5, tn(F, {n, o, v, v}), tn(tt, {o, o, v, v}), 1.0, xo, {n, o});
    } else {
        // occupied rows: T_kj = d_kj - 1/4 sum t_kl^cd t_jl^cd [- 1/4 (t t2 + t2 t)]
        double* Too = c.arena.dalloc(o * o);
        einsum(c, "klcd,jlcd->kj", -0.25, T4, T4, 0.0, Too, {o, o});
        if (third) {
            einsum(c, "klcd,jlcd->kj", -0.25, T4, tn(h->t_2, {o, o, v, v}), 1.0, Too, {o, o});
            einsum(c, "klcd,jlcd->kj", -0.25, tn(h->t_2, {o, o, v, v}), T4, 1.0, Too, {o, o});
        }
        ADC_CUDA(cudaMemcpyAsync(xo, y1, n * o * sizeof(double), cudaMemcpyDeviceToDevice, c.stream));
        einsum(c, "rj,kj->rk", 1.0, Y1, tn(Too, {o, o}), 1.0, xo, {n, o});
        // virtual rows: T_cj = t1x_jc; T_c,ija = t_ij^ca [+ t2_ij^ca]
        einsum(c, "rj,jc->rc", 1.0, Y1, tn(t1x, {o, v}), 0.0, xv, {n, v});
        einsum(c, "rija,ijca->rc", 0.5, tn(F, {n, o, o, v}), tn(tt, {o, o, v, v}), 1.0, xv, {n, v});
    }
    k_gather<<<grid_for(n * o), 256, 0, c.stream>>>(n, o, xo, o, 0, Xp, nso, 0, 0.0);
    launch_check(c);
    k_gather<<<grid_for(n * v), 256, 0, c.stream>>>(n, v, xv, v, 0, Xp, nso, o, 0.0);
    launch_check(c);
    std::vector<double> xh((size_t)n * nso);
    ADC_CUDA(cudaMemcpyAsync(xh.data(), Xp, xh.size() * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
    ADC_CUDA(cudaStreamSynchronize(c.stream));
    h->X_last = xh;
    for (int r = 0; r < nroots; ++r) {
        double s2 = 0.0;
        for (long long p = 0; p < nso; ++p) s2 += xh[(size_t)r * nso + p] * xh[(size_t)r * nso + p];
        specfac[r] = s2;
    }
}

static void sigma_unrestricted(adc_handle* h, const double* Xin, double* Sout, long long n) {
    Ctx& c = h->ctx;
    if (!h->refining) c.gemm_mode = h->cmode_sigma;
    const long long o = h->o, v = h->v, Q = h->naux, dim = h->dim(), np = h->npairs(), n1 = h->n1();
    const int ea = h->kind == ADC_EA;
    const long long blk = ea ? o * v * v : o * o * v;
    const bool third = h->order >= 3;
    Scope sc(c.arena);
    double* y1 = c.arena.dalloc(n * n1);
    double* s1 = c.arena.dalloc(n * n1);
    double* F = c.arena.dalloc(n * blk);
    double* S2 = c.arena.dalloc(n * blk);
    k_gather<<<grid_for(n * n1), 256, 0, c.stream>>>(n, n1, Xin, dim, 0, y1, n1, 0, 0.0);
    launch_check(c);
    fill(c, n * blk, 0.0, F);
    k_pairs_to_full<<<grid_for(n * np), 256, 0, c.stream>>>(ea, n, np, (int)o, (int)v, h->pair_idx, Xin, dim, n1, F);
    launch_check(c);
    const T Bov = tn(h->Bov, {Q, o, v}), Bvv = tn(h->Bvv, {Q, v, v});
    const T T4 = tn(h->t, {o, o, v, v});
    if (ea) {
        const T Y1 = tn(y1, {n, v}), F4 = tn(F, {n, o, v, v});
        einsum(c, "nb,ab->na", 1.0, Y1, tn(h->M11, {v, v}), 0.0, s1, {n, v});
        // coupling, first order: -<aj||cd>, <aj||cd> = (ac|jd) - (ad|jc)
        double* W = c.arena.dalloc(n * Q * v);
        einsum(c, "Qjd,njcd->nQc", 1.0, Bov, F4, 0.0, W, {n, Q, v});
        einsum(c, "nQc,Qac->na", -1.0, tn(W, {n, Q, v}), Bvv, 1.0, s1, {n, v});
        double* P = c.arena.dalloc(n * Q * v);
        einsum(c, "na,Qac->nQc", 1.0, Y1, Bvv, 0.0, P, {n, Q, v});
        einsum(c, "nQc,Qjd->njcd", -1.0, tn(P, {n, Q, v}), Bov, 0.0, S2, {n, o, v, v});
        einsum(c, "nQd,Qjc->njcd", 1.0, tn(P, {n, Q, v}), Bov, 1.0, S2, {n, o, v, v});
        if (third) {
            const T gvooo = tn(h->g_vooo, {v, o, o, o});
            // -1/2 <aj||lm> t_lm^cd
            double* G = c.arena.dalloc(n * o * o * o);
            einsum(c, "lmcd,njcd->njlm", 1.0, T4, F4, 0.0, G, {n, o, o, o});
            einsum(c, "ajlm,njlm->na", -0.25, gvooo, tn(G, {n, o, o, o}), 1.0, s1, {n, v});
            einsum(c, "na,ajlm->njlm", 1.0, Y1, gvooo, 0.0, G, {n, o, o, o});
            einsum(c, "njlm,lmcd->njcd", -0.5, tn(G, {n, o, o, o}), T4, 1.0, S2, {n, o, v, v});
            // -(X - X^cd), X[a,j,c,d] = <ae||cm> t_jm^de, <ae||cm> = (ac|em) - (am|ec)
            double* H = c.arena.dalloc(n * o * v * v);  // [n,m,e,c]
            einsum(c, "jmde,njcd->nmec", 1.0, T4, F4, 0.0, H, {n, o, v, v});
            double* Hq = c.arena.dalloc(n * Q * std::max(o, v));
            einsum(c, "Qme,nmec->nQc", 1.0, Bov, tn(H, {n, o, v, v}), 0.0, Hq, {n, Q, v});
            einsum(c, "nQc,Qac->na", -1.0, tn(Hq, {n, Q, v}), Bvv, 1.0, s1, {n, v});
            einsum(c, "Qec,nmec->nQm", 1.0, Bvv, tn(H, {n, o, v, v}), 0.0, Hq, {n, Q, o});
            einsum(c, "nQm,Qma->na", 1.0, tn(Hq, {n, Q, o}), Bov, 1.0, s1, {n, v});
            double* K = c.arena.dalloc(n * v * v * o);  // [n,e,c,m]
            einsum(c, "nQc,Qme->necm", 1.0, tn(P, {n, Q, v}), Bov, 0.0, K, {n, v, v, o});
            einsum(c, "na,Qma->nQm", 1.0, Y1, Bov, 0.0, Hq, {n, Q, o});
            einsum(c, "nQm,Qec->necm", -1.0, tn(Hq, {n, Q, o}), Bvv, 1.0, K, {n, v, v, o});
            double* Xc = c.arena.dalloc(n * blk);
            einsum(c, "necm,jmde->njcd", 1.0, tn(K, {n, v, v, o}), T4, 0.0, Xc, {n, o, v, v});
            axpby(c, n * blk, -1.0, Xc, 1.0, S2);
            perm4(c, Xc, {n, o, v, v}, {0, 1, 3, 2}, S2, 1.0, 1.0);
        }
        k_diag22<<<grid_for(n * blk), 256, 0, c.stream>>>(1, (int)o, (int)v, n, h->eps, F, S2);
        launch_check(c);
        if (third) {
            ladder(h, F, n * o, S2, h->refining ? h->lm_refine : h->lm_sigma);
            double* R = c.arena.dalloc(n * blk);
            einsum(c, "ajci,njcb->niab", 1.0, tn(h->g_vovo, {v, o, v, o}), F4, 0.0, R, {n, o, v, v});
            axpby(c, n * blk, -1.0, R, 1.0, S2);
            perm4(c, R, {n, o, v, v}, {0, 1, 3, 2}, S2, 1.0, 1.0);
        }
    } else {
        const T Y1 = tn(y1, {n, o}), F4 = tn(F, {n, o, o, v});
        const T M12 = tn(h->m12, {o, o, o, v});
        einsum(c, "nj,ij->ni", 1.0, Y1, tn(h->M11, {o, o}), 0.0, s1, {n, o});
        einsum(c, "ijka,njka->ni", 0.5, M12, F4, 1.0, s1, {n, o});
        einsum(c, "ijka,ni->njka", 1.0, M12, Y1, 0.0, S2, {n, o, o, v});
        k_diag22<<<grid_for(n * blk), 256, 0, c.stream>>>(0, (int)o, (int)v, n, h->eps, F, S2);
        launch_check(c);
        if (third) {
            einsum(c, "ijkl,nkla->nija", -0.5, tn(h->g_oooo, {o, o, o, o}), F4, 1.0, S2, {n, o, o, v});
            double* R = c.arena.dalloc(n * blk);
            einsum(c, "kaib,nkjb->nija", 1.0, tn(h->g_ovov, {o, v, o, v}), F4, 0.0, R, {n, o, o, v});
            axpby(c, n * blk, 1.0, R, 1.0, S2);
            perm4(c, R, {n, o, o, v}, {0, 2, 1, 3}, S2, -1.0, 1.0);
        }
    }
    const double sign = ea ? 1.0 : -1.0;  // IP applies -M_-
    if (!ea) axpby(c, n * n1, 0.0, s1, -1.0, s1);
    k_gather<<<grid_for(n * n1), 256, 0, c.stream>>>(n, n1, s1, n1, 0, Sout, dim, 0, 0.0);
    launch_check(c);
    k_full_to_pairs<<<grid_for(n * np), 256, 0, c.stream>>>(ea, n, np, (int)o, (int)v, h->pair_idx, S2, sign, Sout, dim, n1);
    launch_check(c);
}

#define GUARD(h, ...)                                    \
    try {                                                \
        __VA_ARGS__                                      \
    } catch (const adc::Error& e) {                      \
        if (h) h->err = e.what();                        \
        return e.code;                                   \
    } catch (const std::exception& e) {                  \
        if (h) h->err = e.what();                        \
        return ADC_ERR_CUDA;                             \
    }

extern "C" {

int adc_spectrum(const double* energies, const double* specfac, int nroots, double eta, const double* omega, int nomega,
                 double* A) {
    if (nroots < 0 || nomega < 0 || !(eta > 0.0) || (nroots > 0 && (!energies || !specfac)) || (nomega > 0 && (!omega || !A)))
        return ADC_ERR_ARG;
    // A(w) = -1/pi Im sum_mu P_mu / (w - w_mu + i eta) = 1/pi sum_mu P_mu eta / ((w - w_mu)^2 + eta^2)
    for (int k = 0; k < nomega; ++k) {
        double a = 0.0;
        for (int r = 0; r < nroots; ++r) {
            const double d = omega[k] - energies[r];
            a += specfac[r] * eta / (d * d + eta * eta);
        }
        A[k] = a / M_PI;
    }
    return ADC_OK;
}

int adc_mlp_nweights(void) { return mlp_nweights(); }

int adc_mlp_loss_grad(const float* weights, const double* d, const unsigned char* blk, const double* r, const double* t,
                      long long n, float* grad, double* loss) {
    if (!weights || !grad || !loss || n < 1 || !d || !blk || !r || !t) return ADC_ERR_ARG;
    try {
        *loss = mlp_loss_grad_host(weights, d, blk, r, t, n, grad);
        return ADC_OK;
    } catch (const adc::Error& e) {
        g_setup_error = e.what();
        return e.code;
    } catch (const std::exception& e) {
        g_setup_error = e.what();
        return ADC_ERR_CUDA;
    }
}

int adc_mlp_train(float* weights, const double* d, const unsigned char* blk, const double* r, const double* t, long long n,
                  int steps, float lr, double* loss_hist) {
    if (!weights || n < 1 || steps < 0 || !(lr > 0) || !d || !blk || !r || !t) return ADC_ERR_ARG;
    try {
        mlp_train_host(weights, d, blk, r, t, n, steps, lr, loss_hist);
        return ADC_OK;
    } catch (const adc::Error& e) {
        g_setup_error = e.what();
        return e.code;
    } catch (const std::exception& e) {
        g_setup_error = e.what();
        return ADC_ERR_CUDA;
    }
}

int adc_set_options(adc_handle* h, const adc_options* opt) {
    if (!h || !opt) return ADC_ERR_ARG;
    if (opt->max_space_per_root < 1 || opt->max_iter < 1 || opt->nguess_extra < 0 || opt->keep_per_root < 1 ||
        opt->refine < 0 || opt->refine > 2 || (opt->transition_order != 0 && opt->transition_order != 2) ||
        !(opt->refine_res_tol >= 0.0)) {
        h->err = "adc_set_options: invalid option";
        return ADC_ERR_ARG;
    }
    // solver options only; precision, contractions and aux_chunk are fixed at setup
    h->opt.max_space_per_root = opt->max_space_per_root;
    h->opt.max_iter = opt->max_iter;
    h->opt.nguess_extra = opt->nguess_extra;
    h->opt.res_tol = opt->res_tol;
    h->opt.keep_per_root = opt->keep_per_root;
    h->opt.refine = opt->refine;
    h->opt.transition_order = opt->transition_order;
    h->opt.refine_res_tol = opt->refine_res_tol;
    h->opt.cuda_graphs = opt->cuda_graphs;
    // m11_on_the_fly is fixed at setup
    return ADC_OK;
}

int adc_set_mlp(adc_handle* h, const float* weights) {
    if (!h) return ADC_ERR_ARG;
    GUARD(h, {
        if (!weights) {
            h->mlp_w = nullptr;  // the buffer stays owned by the handle
            return ADC_OK;
        }
        const int nw = mlp_nweights();
        float* w = (float*)dev_alloc(nw * sizeof(float), h->ctx.stream);
        h->owned.push_back(w);
        ADC_CUDA(cudaMemcpyAsync(w, weights, nw * sizeof(float), cudaMemcpyHostToDevice, h->ctx.stream));
        ADC_CUDA(cudaStreamSynchronize(h->ctx.stream));
        h->mlp_w = w;
        return ADC_OK;
    })
}

long long adc_mlp_nsamples(const adc_handle* h, int nroots, int n_iters, long long per_vector) {
    if (!h || h->unrestricted || nroots < 1 || n_iters < 1 || per_vector < 0) return -1;
    return (long long)n_iters * nroots * mlp_samples_per_vector(h, per_vector);
}

int adc_mlp_samples(adc_handle* h, int nroots, const int* iters, int n_iters, long long per_vector,
                    unsigned long long seed, double exact_tol, double* d, unsigned char* blk, double* r, double* t,
                    long long n) {
    if (!h) return ADC_ERR_ARG;
    if (h->unrestricted || nroots < 1 || nroots > h->dim() || !iters || n_iters < 1 || per_vector < 0 ||
        !(exact_tol > 0) || !d || !blk || !r || !t || n < adc_mlp_nsamples(h, nroots, n_iters, per_vector)) {
        h->err = "adc_mlp_samples: invalid argument (or output arrays shorter than adc_mlp_nsamples)";
        return ADC_ERR_ARG;
    }
    for (int k = 0; k < n_iters; ++k)
        if (iters[k] < 1) {
            h->err = "adc_mlp_samples: iteration counts must be >= 1";
            return ADC_ERR_ARG;
        }
    GUARD(h, {
        mlp_samples(h, nroots, iters, n_iters, per_vector, seed, exact_tol, d, blk, r, t);
        return ADC_OK;
    })
}

int adc_default_options(adc_options* opt) {
    if (!opt) return ADC_ERR_ARG;
    opt->precision = ADC_PREC_FP64;
    opt->max_space_per_root = 8;
    opt->max_iter = 100;
    opt->nguess_extra = 2;
    opt->res_tol = 0.0;
    opt->aux_chunk = 0;
    opt->keep_per_root = 2;
    opt->contractions = -1;
    opt->refine = 1;
    opt->transition_order = 0;
    opt->refine_res_tol = 0.0;
    opt->m11_on_the_fly = 0;
    opt->tune_cache = nullptr;
    opt->cuda_graphs = 0;
    opt->lean = -1;
    return ADC_OK;
}

}  // extern "C"

// One system on `stream` (owned by the handle if own_stream); returns ADC_OK or
// a negative code with the message in `msg`.
static int setup_one(const double* eps, const double* Bq, int nocc, int nvir, int naux, int order, int kind,
                     const adc_options* opt, int on_device, bool own_stream, adc_handle** out, std::string& msg) {
    if (!out) return ADC_ERR_ARG;
    *out = nullptr;
    if (!eps || !Bq || nocc < 1 || nvir < 1 || naux < 1 || (order != 2 && order != 3) || (kind != ADC_EA && kind != ADC_IP)) {
        msg = "adc_setup: invalid argument";
        return ADC_ERR_ARG;
    }
    if (opt && (opt->precision != ADC_PREC_FP64 && opt->precision != ADC_PREC_BF16X3)) {
        msg = "adc_setup: unknown precision";
        return ADC_ERR_ARG;
    }
    if (opt && (opt->contractions < -1 || opt->contractions > 2 || opt->refine < 0 || opt->refine > 2 ||
                !(opt->refine_res_tol >= 0.0))) {
        msg = "adc_setup: contractions must be -1..2, refine 0..2 and refine_res_tol >= 0";
        return ADC_ERR_ARG;
    }
    if (opt && opt->transition_order != 0 && opt->transition_order != 2) {
        msg = "adc_setup: transition_order must be 0 (the method's order) or 2";
        return ADC_ERR_ARG;
    }
    adc_handle* h = new adc_handle();
    h->o = nocc;
    h->v = nvir;
    h->naux = naux;
    h->order = order;
    h->kind = kind;
    adc_default_options(&h->opt);
    if (opt) h->opt = *opt;
    const bool lean_ok = kind == ADC_EA && h->opt.precision != ADC_PREC_FP64 && !h->opt.m11_on_the_fly;
    if (h->opt.lean > 0 && !lean_ok) {
        msg = "adc_setup: the lean layout needs EA, BF16X3 precision and a precomputed 1p-1p block";
        delete h;
        return ADC_ERR_ARG;
    }
    try {
        if (own_stream) {
            ADC_CUDA(cudaStreamCreateWithFlags(&h->own_stream, cudaStreamNonBlocking));
            h->ctx.set_stream(h->own_stream);
        }
        bool lean = h->opt.lean > 0;
        if (h->opt.lean < 0 && lean_ok) {
            // automatic: lean when the plain layout's setup peak would not fit the free memory
            // (B^Q blocks and input, the ladder's BF16 planes, ~9 o^2 v^2 FP64 tensors at once)
            size_t fr = 0, tot = 0;
            ADC_CUDA(cudaMemGetInfo(&fr, &tot));
            const double o = nocc, v = nvir, Q = naux, nmo = o + v;
            const double plain = 8.0 * (Q * nmo * nmo * (on_device ? 2.0 : 1.0) + 9.0 * o * o * v * v) +
                                 8.0 * Q * v * (v + 31.0);
            lean = plain > 0.9 * (double)fr;
        }
        if (lean) {
            h->lean = true;
            h->ctx.cache_max_bytes = 0;               // operand planes / FP32 copies made per call
            h->ctx.arena.big_bytes = size_t(256) << 20;  // large scratch in blocks of its own
        }
        setup(h, eps, Bq, on_device);
        ADC_CUDA(cudaStreamSynchronize(h->ctx.stream));
        // setup's scratch (ladder Z, o^2 v^2 temporaries) goes back to the device; sigma regrows
        // what it needs (many handles at once would otherwise each keep their setup peak)
        h->ctx.arena.free_all();
    } catch (const adc::Error& e) {
        msg = e.what();
        int code = e.code;
        delete h;
        return code;
    } catch (const std::exception& e) {
        msg = e.what();
        delete h;
        return ADC_ERR_CUDA;
    }
    *out = h;
    return ADC_OK;
}

// Run f(i) for i in [0, n) on up to `threads` host threads, each with the
// caller's current CUDA device.
template <class F>
static void parallel_for(int n, int threads, F f) {
    int dev = 0;
    cudaGetDevice(&dev);
    std::atomic<int> next{0};
    auto worker = [&] {
        cudaSetDevice(dev);
        for (int i = next++; i < n; i = next++) f(i);
    };
    std::vector<std::thread> pool;
    const int nt = std::max(1, std::min(n, threads));
    for (int t = 1; t < nt; ++t) pool.emplace_back(worker);
    worker();
    for (auto& t : pool) t.join();
}

static int batch_threads(int n) {
    const unsigned hc = std::thread::hardware_concurrency();
    return std::max(1, std::min(n, std::min(16, hc ? (int)hc : 4)));
}

extern "C" {

int adc_setup(const double* eps, const double* Bq, int nocc, int nvir, int naux, int order, int kind,
              const adc_options* opt, int on_device, adc_handle** out) {
    return setup_one(eps, Bq, nocc, nvir, naux, order, kind, opt, on_device, false, out, g_setup_error);
}

int adc_setup_batch(int nmol, const double* const* eps, const double* const* Bq, const int* nocc, const int* nvir,
                    const int* naux, int order, int kind, const adc_options* opt, int on_device, adc_handle** out) {
    if (nmol < 1 || !eps || !Bq || !nocc || !nvir || !naux || !out) {
        g_setup_error = "adc_setup_batch: invalid argument";
        return ADC_ERR_ARG;
    }
    for (int i = 0; i < nmol; ++i) out[i] = nullptr;
    std::vector<int> rc(nmol, ADC_OK);
    std::vector<std::string> msg(nmol);
    // One system after another: setup is dominated by kernels that fill the GPU and by device
    // allocations (which synchronise the device), so concurrent setups only contend (measured 6x
    // slower for 16 systems); the Davidson solves (adc_davidson_batch) run concurrently.
    for (int i = 0; i < nmol; ++i)
        rc[i] = setup_one(eps[i], Bq[i], nocc[i], nvir[i], naux[i], order, kind, opt, on_device, true, &out[i], msg[i]);
    for (int i = 0; i < nmol; ++i) {
        if (rc[i] != ADC_OK) {
            g_setup_error = "adc_setup_batch: system " + std::to_string(i) + ": " + msg[i];
            for (int j = 0; j < nmol; ++j) {
                delete out[j];
                out[j] = nullptr;
            }
            return rc[i];
        }
    }
    return ADC_OK;
}

int adc_setup_unrestricted(const double* eps_a, const double* eps_b, const double* Ba, const double* Bb, int nocc_a,
                           int nocc_b, int nmo, int naux, int order, int kind, const adc_options* opt, adc_handle** out) {
    if (!out) return ADC_ERR_ARG;
    *out = nullptr;
    const int no = nocc_a + nocc_b, nso = 2 * nmo, nv = nso - no;
    const bool pairs_ok = kind == ADC_EA ? nv >= 2 : no >= 2;
    if (!eps_a || !eps_b || !Ba || !Bb || nmo < 1 || nocc_a < 0 || nocc_b < 0 || nocc_a > nmo || nocc_b > nmo || no < 1 ||
        nv < 1 || naux < 1 || (order != 2 && order != 3) || (kind != ADC_EA && kind != ADC_IP) || !pairs_ok ||
        (opt && (opt->aux_chunk < 0 || (opt->precision != ADC_PREC_FP64 && opt->precision != ADC_PREC_BF16X3) ||
                 opt->m11_on_the_fly || opt->refine < 0 || opt->refine > 2 || !(opt->refine_res_tol >= 0.0)))) {
        g_setup_error = "adc_setup_unrestricted: invalid argument (or an option these handles do not take)";
        return ADC_ERR_ARG;
    }
    if (opt && opt->precision != ADC_PREC_FP64 && (nmo - nocc_a < 1 || nmo - nocc_b < 1)) {
        g_setup_error = "adc_setup_unrestricted: the mixed-precision ladder needs virtual orbitals of both spins";
        return ADC_ERR_ARG;
    }
    // spin orbitals: occupied alpha, occupied beta, virtual alpha, virtual beta
    std::vector<int> spin(nso), idx(nso);
    int k = 0;
    for (int p = 0; p < nocc_a; ++p, ++k) spin[k] = 0, idx[k] = p;
    for (int p = 0; p < nocc_b; ++p, ++k) spin[k] = 1, idx[k] = p;
    for (int p = nocc_a; p < nmo; ++p, ++k) spin[k] = 0, idx[k] = p;
    for (int p = nocc_b; p < nmo; ++p, ++k) spin[k] = 1, idx[k] = p;
    std::vector<double> eps_so(nso), Bso((size_t)naux * nso * nso, 0.0);
    for (int P = 0; P < nso; ++P) eps_so[P] = spin[P] ? eps_b[idx[P]] : eps_a[idx[P]];
    for (long long q = 0; q < naux; ++q)
        for (int P = 0; P < nso; ++P)
            for (int R = 0; R < nso; ++R)
                if (spin[P] == spin[R]) {
                    const double* B = spin[P] ? Bb : Ba;
                    Bso[((size_t)q * nso + P) * nso + R] = B[((size_t)q * nmo + idx[P]) * nmo + idx[R]];
                }
    adc_handle* h = new adc_handle();
    h->o = no;
    h->v = nv;
    h->naux = naux;
    h->order = order;
    h->kind = kind;
    h->unrestricted = true;
    h->nva = nmo - nocc_a;
    adc_default_options(&h->opt);
    if (opt) h->opt = *opt;
    try {
        setup_unrestricted(h, eps_so.data(), Bso.data());
        ADC_CUDA(cudaStreamSynchronize(h->ctx.stream));
        h->ctx.arena.free_all();
    } catch (const adc::Error& e) {
        g_setup_error = e.what();
        const int code = e.code;
        delete h;
        return code;
    } catch (const std::exception& e) {
        g_setup_error = e.what();
        delete h;
        return ADC_ERR_CUDA;
    }
    *out = h;
    return ADC_OK;
}

int adc_dim(const adc_handle* h, long long* dim) {
    if (!h || !dim) return ADC_ERR_ARG;
    *dim = h->dim();
    return ADC_OK;
}

int adc_mp_energy(const adc_handle* h, double* e, int n_out) {
    if (!h || !e || n_out < 1 || h->unrestricted) return ADC_ERR_ARG;
    const int n = std::min(n_out, h->order - 1);
    for (int k = 0; k < n; ++k) e[k] = h->emp[k];
    return ADC_OK;
}

int adc_set_stream(adc_handle* h, void* stream) {
    if (!h) return ADC_ERR_ARG;
    GUARD(h, {
        ADC_CUDA(cudaStreamSynchronize(h->ctx.stream));  // work and allocations of the old stream are done
        h->ctx.set_stream((cudaStream_t)stream);
        ADC_BLAS(cublasSetStream(h->ctx.blas, h->ctx.stream));
        return ADC_OK;
    })
}

int adc_sigma(adc_handle* h, const double* X, double* S, int nvec, int on_device) {
    if (!h) return ADC_ERR_ARG;
    if (!X || !S || nvec < 1) {
        h->err = "adc_sigma: invalid argument";
        return ADC_ERR_ARG;
    }
    GUARD(h, {
        Ctx& c = h->ctx;
        const long long dim = h->dim();
        if (on_device) {
            sigma_device(h, X, S, nvec);
        } else {
            Scope sc(c.arena);
            double* dX = c.arena.dalloc((size_t)nvec * dim);
            double* dS = c.arena.dalloc((size_t)nvec * dim);
            ADC_CUDA(cudaMemcpyAsync(dX, X, (size_t)nvec * dim * sizeof(double), cudaMemcpyHostToDevice, c.stream));
            sigma_device(h, dX, dS, nvec);
            ADC_CUDA(cudaMemcpyAsync(S, dS, (size_t)nvec * dim * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
        }
        ADC_CUDA(cudaStreamSynchronize(c.stream));
        return ADC_OK;
    })
}

int adc_davidson(adc_handle* h, int nroots, double tol, const double* guess, double* energies, double* specfac,
                 double* vectors, double* stats) {
    if (!h) return ADC_ERR_ARG;
    if (nroots < 1 || !energies || !(tol > 0) || nroots > h->dim()) {
        h->err = "adc_davidson: invalid argument";
        return ADC_ERR_ARG;
    }
    GUARD(h, {
        int st = davidson(h, nroots, tol, guess, energies, specfac, vectors, stats);
        if (st == ADC_ERR_NOT_CONVERGED) h->err = "adc_davidson: not converged within max_iter";
        // the solver's scratch (subspace, residuals, sigma intermediates) goes back to the device:
        // many handles solved one after another would otherwise each keep their peak
        h->ctx.arena.free_all(true);
        return st;
    })
}

int adc_davidson_batch(adc_handle* const* h, int nmol, int nroots, double tol, double* energies, double* specfac,
                       double* stats, int* status) {
    if (!h || nmol < 1 || !energies) return ADC_ERR_ARG;
    std::vector<int> rc(nmol, ADC_OK);
    parallel_for(nmol, batch_threads(nmol), [&](int i) {
        rc[i] = adc_davidson(h[i], nroots, tol, nullptr, energies + (size_t)i * nroots,
                             specfac ? specfac + (size_t)i * nroots : nullptr, nullptr, stats ? stats + 8 * (size_t)i : nullptr);
    });
    int worst = ADC_OK;
    for (int i = 0; i < nmol; ++i) {
        if (status) status[i] = rc[i];
        if (rc[i] != ADC_OK && (worst == ADC_OK || worst == ADC_ERR_NOT_CONVERGED)) worst = rc[i];
    }
    return worst;
}

int adc_get_tensor(adc_handle* h, const char* name, double* out, long long n) {
    if (!h || !name || !out) return ADC_ERR_ARG;
    GUARD(h, {
        const long long o = h->o, v = h->v;
        const double* src = nullptr;
        const float* src32 = nullptr;  // a lean handle's FP32 tensor
        long long cnt = 0;
        std::string s(name);
        if (s == "M11") {
            src = h->M11;
            cnt = (long long)h->n1() * h->n1();
        } else if (s == "t2" && h->f_t) {
            src32 = h->f_t;
            cnt = o * o * v * v;
        } else if (s == "t2") {
            src = h->t;
            cnt = o * o * v * v;
        } else if (s == "t2_2" && h->f_t2) {
            src32 = h->f_t2;
            cnt = o * o * v * v;
        } else if (s == "t2_2") {
            src = h->t_2;
            cnt = o * o * v * v;
        } else if (s == "t1_2") {
            src = h->t1_2;
            cnt = o * v;
        } else if (s == "t1_3") {
            if (h->unrestricted)
                make_t1_third_order_u(h);
            else
                make_t1_third_order(h);
            src = h->t1_3;
            cnt = o * v;
        } else if (s == "diag") {
            src = h->diag;
            cnt = h->dim();
        } else if (s == "setup_seconds") {
            cnt = 8;
            if (n < cnt) {
                h->err = "adc_get_tensor: buffer too small";
                return ADC_ERR_ARG;
            }
            std::memcpy(out, h->setup_times, sizeof(h->setup_times));
            return ADC_OK;
        } else if (s == "X") {
            // host copy kept by the last adc_davidson that computed spectroscopic factors
            cnt = (long long)h->X_last.size();
            if (cnt == 0) {
                h->err = "adc_get_tensor: no spectroscopic amplitudes yet (run adc_davidson with specfac)";
                return ADC_ERR_ARG;
            }
            if (n < cnt) {
                h->err = "adc_get_tensor: buffer too small";
                return ADC_ERR_ARG;
            }
            std::memcpy(out, h->X_last.data(), cnt * sizeof(double));
            return ADC_OK;
        }
        if (!src && !src32) {
            h->err = "adc_get_tensor: unknown or unavailable tensor " + s;
            return ADC_ERR_ARG;
        }
        if (n < cnt) {
            h->err = "adc_get_tensor: buffer too small";
            return ADC_ERR_ARG;
        }
        if (src32) {
            Scope sc(h->ctx.arena);
            double* tmp = h->ctx.arena.dalloc(cnt);
            Shape sh{1, {cnt}};
            int id[1] = {0};
            permute_any(h->ctx, src32, true, sh, id, tmp, false, 1.0, 0.0);
            ADC_CUDA(cudaMemcpyAsync(out, tmp, cnt * sizeof(double), cudaMemcpyDeviceToHost, h->ctx.stream));
            ADC_CUDA(cudaStreamSynchronize(h->ctx.stream));
            return ADC_OK;
        }
        ADC_CUDA(cudaMemcpyAsync(out, src, cnt * sizeof(double), cudaMemcpyDeviceToHost, h->ctx.stream));
        ADC_CUDA(cudaStreamSynchronize(h->ctx.stream));
        return ADC_OK;
    })
}

int adc_kernel_timing(adc_handle* h, int enable, double* out) {
    if (!h) return ADC_ERR_ARG;
    GUARD(h, {
        Ctx& c = h->ctx;
        if (enable) {
            for (auto e : c.ev_start) cudaEventDestroy(e);
            for (auto e : c.ev_stop) cudaEventDestroy(e);
            c.ev_start.clear();
            c.ev_stop.clear();
            c.ev_ladder.clear();
            c.ev_algo.clear();
            c.ev_mma.clear();
            c.ev_shape.clear();
            c.algo_flops = c.mma_flops = 0.0;
            c.kernels_at_start = c.kernels;
            c.timing = true;
            if (out)
                for (int i = 0; i < 9; ++i) out[i] = 0.0;
            return ADC_OK;
        }
        c.timing = false;
        ADC_CUDA(cudaStreamSynchronize(c.stream));
        double ms = 0.0, lms = 0.0, lalgo = 0.0, lmma = 0.0;
        long long nl = 0;
        for (size_t i = 0; i < c.ev_start.size(); ++i) {
            float t = 0.f;
            ADC_CUDA(cudaEventElapsedTime(&t, c.ev_start[i], c.ev_stop[i]));
            ms += t;
            if (c.ev_ladder[i]) {
                ++nl;
                lms += t;
                lalgo += c.ev_algo[i];
                lmma += c.ev_mma[i];
            }
        }
        if (out) {
            out[0] = (double)c.ev_start.size();
            out[1] = ms;
            out[2] = c.algo_flops;
            out[3] = c.mma_flops;
            out[4] = (double)(c.kernels - c.kernels_at_start);
            out[5] = (double)nl;
            out[6] = lms;
            out[7] = lalgo;
            out[8] = lmma;
        }
        return ADC_OK;
    })
}

long long adc_kernel_launches(adc_handle* h, double* out, long long n) {
    if (!h) return ADC_ERR_ARG;
    Ctx& c = h->ctx;
    const long long cnt = (long long)c.ev_start.size();
    if (!out) return cnt;
    if (c.timing || n < 7 * cnt) {
        h->err = "adc_kernel_launches: timing still on, or buffer shorter than 7 doubles per launch";
        return ADC_ERR_ARG;
    }
    try {
        for (long long i = 0; i < cnt; ++i) {
            float t = 0.f;
            ADC_CUDA(cudaEventElapsedTime(&t, c.ev_start[i], c.ev_stop[i]));
            double* r = out + 7 * i;
            for (int k = 0; k < 4; ++k) r[k] = c.ev_shape[4 * i + k];
            r[4] = c.ev_algo[i];
            r[5] = t;
            r[6] = c.ev_ladder[i] ? 1.0 : 0.0;
        }
    } catch (const adc::Error& e) {
        h->err = e.what();
        return e.code;
    }
    return cnt;
}

const char* adc_last_error(const adc_handle* h) { return h ? h->err.c_str() : g_setup_error.c_str(); }

void adc_destroy(adc_handle* h) {
    if (!h) return;
    cudaStreamSynchronize(h->ctx.stream);
    delete h;
}

}  // extern "C"


// Shared device helpers of the ADC library: error handling, a device scratch
// arena, an N-d permute kernel and a two-operand tensor contraction executor
// (permute to GEMM form + cuBLAS strided-batched DGEMM + permute back).
#pragma once

#include <cublas_v2.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <map>
#include <stdexcept>
#include <string>
#include <vector>

namespace adc {

struct Error : std::runtime_error {
    int code;
    Error(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};

#define ADC_CUDA(x)                                                                                   \
    do {                                                                                              \
        cudaError_t e_ = (x);                                                                         \
        if (e_ != cudaSuccess)                                                                        \
            throw ::adc::Error(e_ == cudaErrorMemoryAllocation ? -2 : -3,                             \
                               std::string(#x) + ": " + cudaGetErrorString(e_));                      \
    } while (0)

#define ADC_BLAS(x)                                                                                   \
    do {                                                                                              \
        cublasStatus_t s_ = (x);                                                                      \
        if (s_ != CUBLAS_STATUS_SUCCESS)                                                              \
            throw ::adc::Error(s_ == CUBLAS_STATUS_ALLOC_FAILED ? -2 : -3,                            \
                               std::string(#x) + ": cublas status " + std::to_string((int)s_));       \
    } while (0)

// Device scratch: blocks are allocated on demand and kept; mark()/release()
// give stack semantics so that repeated calls reuse the same memory.  Blocks
// come from the stream-ordered allocator on `stream` (no device-wide
// synchronisation, so handles on other streams keep running).
class Arena {
   public:
    cudaStream_t stream = nullptr;
    bool frozen = false;  // set while a stream capture records: growing would allocate inside the graph
    ~Arena() { free_all(); }
    // requests of at least big_bytes (0: never) get a block of their own, freed (stream-
    // ordered) by the release() of the enclosing mark: scratch of very different sizes at
    // the same stack depth then cannot fragment the kept blocks
    size_t big_bytes = 0;
    struct Mark {
        size_t block, top, nbig;
    };
    Mark mark() const { return {cur_, blocks_.empty() ? 0 : tops_[cur_], big_.size()}; }
    void release(Mark m) {
        for (size_t b = m.block + 1; b < tops_.size(); ++b) tops_[b] = 0;
        cur_ = m.block;
        if (!tops_.empty()) tops_[cur_] = m.top;
        while (big_.size() > m.nbig) {
            cudaFreeAsync(big_.back(), stream);
            big_.pop_back();
        }
    }
    void* alloc(size_t bytes) {
        bytes = (bytes + 255) & ~size_t(255);
        if (bytes == 0) bytes = 256;
        if (big_bytes && bytes >= big_bytes) {
            if (frozen) throw Error(-3, "arena: growth during stream capture");
            void* p = nullptr;
            ADC_CUDA(cudaMallocAsync(&p, bytes, stream));
            big_.push_back(p);
            return p;
        }
        while (cur_ < blocks_.size()) {
            if (tops_[cur_] + bytes <= caps_[cur_]) {
                void* p = (char*)blocks_[cur_] + tops_[cur_];
                tops_[cur_] += bytes;
                return p;
            }
            if (cur_ + 1 < blocks_.size()) {
                ++cur_;
                tops_[cur_] = 0;
            } else
                break;
        }
        if (frozen) throw Error(-3, "arena: growth during stream capture");
        size_t cap = bytes > (size_t(256) << 20) ? bytes : (size_t(256) << 20);
        void* p = nullptr;
        ADC_CUDA(cudaMallocAsync(&p, cap, stream));
        blocks_.push_back(p);
        caps_.push_back(cap);
        tops_.push_back(bytes);
        cur_ = blocks_.size() - 1;
        return p;
    }
    double* dalloc(size_t n) { return (double*)alloc(n * sizeof(double)); }
    // release every block (stream-ordered on `stream` when async, else with cudaFree)
    void free_all(bool async = false) {
        for (void* p : big_) blocks_.push_back(p);
        big_.clear();
        for (void* p : blocks_) {
            if (async)
                cudaFreeAsync(p, stream);
            else
                cudaFree(p);
        }
        blocks_.clear();
        caps_.clear();
        tops_.clear();
        cur_ = 0;
    }
    size_t capacity() const {
        size_t s = 0;
        for (size_t c : caps_) s += c;
        return s;
    }

   private:
    std::vector<void*> blocks_, big_;
    std::vector<size_t> caps_, tops_;
    size_t cur_ = 0;
};

// Stream-ordered device allocation (memory from it is freed with cudaFree).
inline void* dev_alloc(size_t bytes, cudaStream_t s) {
    void* p = nullptr;
    ADC_CUDA(cudaMallocAsync(&p, bytes ? bytes : 1, s));
    return p;
}

struct Ctx {
    cudaStream_t stream = 0;  // set with set_stream (the arena allocates on it)
    void set_stream(cudaStream_t s) {
        stream = s;
        arena.stream = s;
    }
    cublasHandle_t blas = nullptr;
    Arena arena;
    long long kernels = 0;  // own kernel launches issued (for reporting)
    // 0: every contraction in FP64 (DGEMM).  1: contractions of >= fp32_min_flops
    // run as FP32-accurate GEMMs (BF16x9 emulation on the tensor cores), with
    // FP64 inputs rounded to FP32 and results accumulated into FP64.  2 (the
    // mixed sigma): unbatched contractions of >= fp32_min_flops run on the tcgen05
    // split-BF16 GEMM (two planes, FP32 partial sums promoted every 16 K blocks,
    // FP64 result) unless a free dimension is <= 8 and the large operand is not a
    // cached constant; the others on the library's own kernels (own_gemm:
    // FP32-accurate from fp32_min_flops, else FP64).
    int gemm_mode = 0;
    double fp32_min_flops = 1e8;
    int emulation_ok = -1;  // -1 unknown, 1 BF16x9 emulation available, 0 plain FP32
    // live timing of the tensor-core GEMM launches (see adc_kernel_timing)
    bool timing = false;
    std::vector<cudaEvent_t> ev_start, ev_stop;
    std::vector<char> ev_ladder;          // launch is one of the DF ladder GEMMs
    std::vector<double> ev_algo, ev_mma;  // its algorithmic / issued tensor-core flops
    std::vector<double> ev_shape;         // its M, N, K, tile width (4 per launch)
    double algo_flops = 0.0, mma_flops = 0.0;
    long long kernels_at_start = 0;
    // FP32 copies (in GEMM operand order) of operands marked constant, reused across calls
    std::map<std::pair<const void*, std::string>, float*> f32cache;
    // split BF16 planes (K-major GEMM operand order) of operands marked constant
    std::map<std::pair<const void*, std::string>, void*> bf16cache;
    // constant operands are cached in these forms only if the copy is at most this size
    // (larger ones are converted per call into scratch)
    size_t cache_max_bytes = ~size_t(0);
    int* d_err = nullptr;  // device flag raised by a bounded wait that gave up (tensor-core GEMMs)
    void* tuner = nullptr;  // TuneCache of the tile autotuner (ladder_tc.cuh), or NULL: cost-model tiles
    // a CUDA-graph capture of sigma is recording on `stream`: no host synchronisation, no
    // allocation, no tuning; the timeout flags are read after the graph's replay instead
    bool capturing = false;
    // side streams for concurrent K slices of a contraction, with their fork / join events
    std::vector<cudaStream_t> side;
    std::vector<cudaEvent_t> side_join;
    cudaEvent_t side_fork = nullptr;
    ~Ctx() {
        for (auto& kv : f32cache) cudaFree(kv.second);
        for (auto& kv : bf16cache) cudaFree(kv.second);
        if (d_err) cudaFree(d_err);
        for (auto s : side) cudaStreamDestroy(s);
        for (auto e : side_join) cudaEventDestroy(e);
        if (side_fork) cudaEventDestroy(side_fork);
        for (auto e : ev_start) cudaEventDestroy(e);
        for (auto e : ev_stop) cudaEventDestroy(e);
    }
};

constexpr int kMaxDim = 8;
struct Shape {
    int nd;
    long long d[kMaxDim];
};

// ---- elementwise kernels --------------------------------------------------
void permute(Ctx& c, const double* in, const Shape& in_shape, const int* perm, double* out, double alpha, double beta);
void axpby(Ctx& c, long long n, double alpha, const double* x, double beta, double* y);  // y = a x + b y
void fill(Ctx& c, long long n, double v, double* y);
// C[i] = sum_s T[s*n + i]
void sum_slices(Ctx& c, int S, long long n, const double* T, double* C);
// make at least `count` side streams (non-blocking) and their events
void ensure_side_streams(Ctx& c, int count);

// ---- contraction executor -------------------------------------------------
struct T {
    const double* p;
    std::vector<long long> dims;
    bool constant = false;  // contents never change while the handle lives (FP32 copy may be cached)
    bool f32 = false;       // p points to FP32 values (read as such; FP64 operand paths convert)
};
// C[lc] = beta * C + alpha * sum A[la] B[lb] ; spec "la,lb->lc" with single-letter indices.
void einsum(Ctx& c, const char* spec, double alpha, const T& A, const T& B, double beta, double* C,
            const std::vector<long long>& cdims);
// the same with an FP32 output (the contraction's arithmetic is unchanged; the result and
// beta * C are formed in FP64, or FP32 where the GEMM writes the output itself, and rounded once)
void einsum(Ctx& c, const char* spec, double alpha, const T& A, const T& B, double beta, float* C,
            const std::vector<long long>& cdims);
// out = alpha * permute(in) + beta * out between FP64 / FP32 arrays (in32 / out32: FP32)
void permute_any(Ctx& c, const void* in, bool in32, const Shape& s, const int* perm, void* out, bool out32,
                 double alpha, double beta);

// Permute `in` (shape s, output axis j = input axis perm[j]) into row-major
// [rows][K] order and split each value x into BF16 planes x = p0 + p1 (two
// planes), written K-major as out[p][r * Kp + k] with zeros for K <= k < Kp.
void split_planes(Ctx& c, const double* in, const Shape& s, const int* perm, long long rows, long long K, long long Kp,
                  void* const* out, bool in32 = false);

// The library's own kernels for small and skinny contractions (row-major A [M][K],
// B [K][N], C [M][N] with leading dimensions): C = alpha A B + beta C.  M <= 8 or
// N <= 8 take bandwidth kernels that read the large operand once (K split over
// blocks, deterministic slice reduction); others a 64 x 64 tiled FP64 kernel.
// f32: FP32 products and partial sums of <= 64 terms, accumulated in FP64.
void own_gemm(Ctx& c, long long M, long long N, long long K, double alpha, const double* A, long long lda, const double* B,
              long long ldb, double beta, double* C, long long ldc, bool f32);

// Row-major GEMM: C[MxN] = alpha op(A) op(B) + beta C, batched with strides.
void gemm(Ctx& c, bool ta, bool tb, long long M, long long N, long long K, double alpha, const double* A, long long lda,
          long long sA, const double* B, long long ldb, long long sB, double beta, double* C, long long ldc,
          long long sC, long long batch);

}  // namespace adc

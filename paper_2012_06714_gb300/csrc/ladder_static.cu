// Allocation-free entry point for the density-fitted ladder (adc_ladder_noalloc).
//
// Some callers cannot allocate device memory while they run: for example a
// host application whose own memory manager owns all device memory and forbids
// cudaMalloc/cudaFree from library calls (these calls can synchronise the whole
// device and fragment a pool that the caller sizes up front), or code that runs
// on a thread where the caller has promised not to enter the CUDA allocator.
// For them this entry point computes the ladder with no allocation at all: its
// scratch is the fixed array below.  The array belongs to this file's device
// module, which CUDA loads (lazily) when its symbol address is first looked
// up; setup of a BF16X3 handle does that on its device (noalloc_prepare),
// so the entry point itself never triggers the module load, and the GPU holds
// the 64 MiB from then until process exit.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/adc.h"
#include "common.cuh"
#include "ladder_tc.cuh"

namespace adc {
bool handle_ladder_view(adc_handle* h, LadderTC** tc, Ctx** c, int* nvir, std::string** err, LadderMode* md);
}

namespace {

constexpr size_t kScratchBytes = size_t(64) << 20;  // 64 MiB per device

// The scratch memory.  In host code its name is only a host-side stand-in;
// kernels receive the device address obtained with cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_ladder_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

// Device address of g_ladder_scratch on the current device, looked up once per
// device (with that device current) and cached.
cudaError_t scratch_address(void** out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_ladder_scratch);
        if (e != cudaSuccess) return e;
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return cudaSuccess;
}

}  // namespace

namespace adc {
// Resolve the scratch array's device address on the current device (loading
// this module); called by the setup of every BF16X3 handle.
void noalloc_prepare() {
    void* p = nullptr;
    ADC_CUDA(scratch_address(&p));
}
}  // namespace adc

extern "C" int adc_ladder_noalloc(adc_handle* h, const double* X, double* out, long long nmat) {
    using namespace adc;
    LadderTC* tc = nullptr;
    Ctx* c = nullptr;
    int v = 0;
    std::string* err = nullptr;
    LadderMode md{2, 0, 0};
    if (!handle_ladder_view(h, &tc, &c, &v, &err, &md)) return ADC_ERR_ARG;
    if (!X || !out || nmat < 0) {
        *err = "adc_ladder_noalloc: invalid argument";
        return ADC_ERR_ARG;
    }
    if (!tc) {
        *err = "adc_ladder_noalloc: the handle was not set up with ADC_PREC_BF16X3";
        return ADC_ERR_ARG;
    }
    try {
        void* scratch = nullptr;
        ADC_CUDA(scratch_address(&scratch));
        if (!ladder_tc_apply_scratch(*tc, *c, X, nmat, out, md, scratch, kScratchBytes)) {
            *err = "adc_ladder_noalloc: nvir = " + std::to_string(v) +
                   " needs more than the fixed 64 MiB scratch for one matrix and one auxiliary function";
            return ADC_ERR_ARG;
        }
        return ADC_OK;
    } catch (const Error& e) {
        *err = e.what();
        return e.code;
    } catch (const std::exception& e) {
        *err = e.what();
        return ADC_ERR_CUDA;
    }
}

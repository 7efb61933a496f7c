// Pairwise contraction that allocates no device memory.
//
// Some callers cannot let a library allocate GPU memory: an application that
// owns all device memory through its own pool and forbids other allocations,
// or a latency-critical loop where cudaMalloc / cudaFree (which may
// synchronise the whole device) are not acceptable.  For them,
// tn_contract_dev_noalloc runs the strided contraction kernels of
// tn_contract_dev, keeping the partial sums of the split-K form in one
// fixed-size array that lives in the library's device image instead of in
// allocated memory.
#include <mutex>
#include <string>

#include "kernels.cuh"
#include "tn.h"

namespace tn {
tn_status set_error(tn_status s, const std::string &msg);
tn_status plain_contract_desc(int nlabels, const int *sizes, int na, const int *labels_a,
                              const void *A, int nb, const int *labels_b, const void *B, int nc,
                              const int *labels_c, void *C, int semiring, int32_t *argmax,
                              CDesc &d);
}  // namespace tn

// The scratch: partial sums (and argmax indices) of the split-K kernels.
// Every GPU that loads the library holds these TN_NOALLOC_SCRATCH_BYTES until
// the process exits.  No part of it needs to start at zero: each call writes
// every partial slot it later reads.
static __device__ __align__(256) unsigned char g_noalloc_scratch[TN_NOALLOC_SCRATCH_BYTES];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_scratch_addr[kMaxDevices] = {nullptr};

// Device address of the scratch on the current device.  In host code the
// array's name only denotes a host-side stand-in, so the address is looked
// up once per device (with that device current) and cached.
tn_status scratch_address(void **out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return tn::set_error(TN_E_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices)
        return tn::set_error(TN_E_UNSUPPORTED, "device index beyond the supported range");
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return tn::set_error(TN_E_CUDA, std::string("cudaGetSymbolAddress(scratch): ") +
                                                cudaGetErrorString(e));
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return TN_OK;
}
}  // namespace

extern "C" tn_status tn_contract_dev_noalloc(int nlabels, const int *sizes, int na,
                                             const int *labels_a, const void *A, int nb,
                                             const int *labels_b, const void *B, int nc,
                                             const int *labels_c, void *C, int semiring,
                                             int dtype, int32_t *argmax, void *cuda_stream) {
    if (dtype != 0 && dtype != 1) return tn::set_error(TN_E_ARG, "dtype must be 0 or 1");
    tn::CDesc d;
    tn_status s = tn::plain_contract_desc(nlabels, sizes, na, labels_a, A, nb, labels_b, B, nc,
                                          labels_c, C, semiring, argmax, d);
    if (s) return s;
    void *scratch = nullptr;
    s = scratch_address(&scratch);
    if (s) return s;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    bool ok = dtype == 0 ? tn::launch_contract_splitk_fixed<double>(d, semiring, scratch,
                                                                    TN_NOALLOC_SCRATCH_BYTES, st)
                         : tn::launch_contract_splitk_fixed<float>(d, semiring, scratch,
                                                                   TN_NOALLOC_SCRATCH_BYTES, st);
    if (!ok) {
        int64_t outs = d.nout_total * d.nbeta;
        return tn::set_error(
            TN_E_ARG, "output of " + std::to_string(outs) + " entries needs more than the " +
                          std::to_string((long long)TN_NOALLOC_SCRATCH_BYTES) +
                          "-byte fixed scratch (at most " +
                          std::to_string((long long)TN_NOALLOC_SCRATCH_BYTES / ((dtype == 0 ? 8 : 4) + 4)) +
                          " output entries)");
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return tn::set_error(TN_E_CUDA, std::string("launch: ") + cudaGetErrorString(e));
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess)
        return tn::set_error(TN_E_CUDA, std::string("cudaStreamSynchronize: ") + cudaGetErrorString(e));
    return TN_OK;
}

// Marginal probabilities with no allocation at all.
//
// sv_marginal_probabilities needs scratch device memory: one 128-bit
// fixed-point accumulator per output bin, plus a staging buffer when the
// caller wants the result in host memory.  Some callers cannot let a library
// allocate device memory: processes whose device memory is fully reserved by
// another allocator (a caching allocator that already holds almost all of the
// HBM and accounts for every byte), and latency-critical loops in which a
// cudaFree -- which waits for the whole device -- would stall work on other
// streams.  This file gives them a variant that takes the amplitudes by
// pointer and keeps its scratch in a fixed static device array instead.
//
// The array is 1.5 MiB (room for 2^16 bins) and is part of the library image:
// every GPU on which the library is loaded holds it until the process exits.
// All calls share it; each call clears the accumulators it uses before it
// starts, but two calls whose kernels overlap on the GPU (for example on two
// streams) race on it and must be serialised by the caller.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "kernels.cuh"
#include "sv.h"

namespace {

constexpr int kNoallocMaxMaskBits = 16;
constexpr uint64_t kNoallocBins = 1ull << kNoallocMaxMaskBits;

// [0, 2*bins): 128-bit accumulators (low, high word per bin);
// [2*bins, 3*bins): float64 results staged for a host-side output.
static __device__ __align__(256) unsigned long long g_noalloc_scratch[3 * kNoallocBins];

std::mutex g_mu;
void* g_scratch_addr[64] = {nullptr};
svk::DevInfo g_info[64];

// Per device, once, with that device current: the device address of the
// static array (host code cannot use the symbol itself as a pointer) and the
// launch parameters.
int setup_device(int dev, void** scratch, svk::DevInfo* di) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return SV_ERR_CUDA;
        svk::DevInfo d;
        d.device = dev;
        int smem = 0;
        if (cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
            return SV_ERR_CUDA;
        d.smem_optin = (size_t)smem;
        g_info[dev] = d;
        g_scratch_addr[dev] = p;
    }
    *scratch = g_scratch_addr[dev];
    *di = g_info[dev];
    return SV_OK;
}

}  // namespace

extern "C" int sv_marginal_probabilities_noalloc(const void* amplitudes, int n_qubits, int dt, uint64_t qubit_mask,
                                                 double* out, size_t out_len, int out_is_device,
                                                 void* cuda_stream) {
    if (!amplitudes || ((uintptr_t)amplitudes & 15) || !out) return SV_ERR_ARG;
    if (n_qubits < 1 || n_qubits > 34 || (dt != SV_C64 && dt != SV_C128)) return SV_ERR_ARG;
    if (qubit_mask >> n_qubits) return SV_ERR_QUBIT;
    const int k = __builtin_popcountll(qubit_mask);
    if (k > kNoallocMaxMaskBits) return SV_ERR_SIZE;  // beyond the static scratch
    const uint64_t nbins = 1ull << k;
    if (out_len != nbins) return SV_ERR_SIZE;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return SV_ERR_CUDA;
    void* scratch = nullptr;
    svk::DevInfo di;
    int rc = setup_device(dev, &scratch, &di);
    if (rc != SV_OK) return rc;
    auto* bins = static_cast<unsigned long long*>(scratch);
    double* staging = reinterpret_cast<double*>(bins + 2 * kNoallocBins);
    double* d_out = out_is_device ? out : staging;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    // launch_marginal clears the bins it uses before accumulating
    if (svk::launch_marginal(dt, amplitudes, n_qubits, qubit_mask, bins, d_out, s, di) != cudaSuccess)
        return SV_ERR_CUDA;
    if (!out_is_device &&
        cudaMemcpyAsync(out, staging, nbins * sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return SV_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return SV_ERR_CUDA;
    return SV_OK;
}

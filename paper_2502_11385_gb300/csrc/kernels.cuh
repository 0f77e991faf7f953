// Launchers of the sm_103a kernels (C++ linkage, used by the C-ABI layer).
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "device_types.hpp"

namespace svk {

struct DevInfo {
    int device = 0;
    int sms = 0;
    size_t smem_optin = 0;
};

// Tile-pass kernel configuration.
constexpr int kTileThreads = 256;

// amp := e_basis (K1).
cudaError_t launch_init(int dt, void* amp, int n, uint64_t basis, cudaStream_t s, const DevInfo& di);

// One tile-pass launch (K5) over n_entries (state, pass) pairs in device
// memory: every tile of every entry is gathered into shared memory, the
// entry's ops are applied in order, and the tile is written back.
// total_tiles = sum of the entries' tile counts; max_m / kmax = largest tile
// and dense block among the entries; arith: SV_ARITH_NATIVE, SV_ARITH_DF64,
// SV_ARITH_TC or SV_ARITH_TC_SYNC (complex128 only).
cudaError_t launch_tile_pass(int dt, int arith, const BatchEntry* d_entries, int n_entries, uint64_t total_tiles,
                             int max_m, int kmax, const DevOp* d_ops, const void* d_coef, cudaStream_t s,
                             const DevInfo& di);

// Batched form: every entry's state := |0...0> / every entry's probabilities.
cudaError_t launch_init_multi(int dt, const StateEntry* d_entries, int n_entries, uint64_t total_amps,
                              cudaStream_t s, const DevInfo& di);
cudaError_t launch_probs_multi(int dt, const StateEntry* d_entries, int n_entries, uint64_t total_amps,
                               cudaStream_t s, const DevInfo& di);

// Reads and clears the tensor-memory mode's fault flag (set when a bounded
// wait for the tensor cores ran out; the launch then left its state undefined).
cudaError_t tc_fault_take(int* fault);

// *d_out = bit pattern of max |re|, |im| over a complex128 state.
cudaError_t launch_max_abs_c128(const void* amp, int n, unsigned long long* d_out, cudaStream_t s,
                               const DevInfo& di);

// p[i - i0] = |amp_i|^2 for i in [i0, i0 + len) (K7, probability part).
cudaError_t launch_probs(int dt, const void* amp, uint64_t i0, uint64_t len, double* p,
                         cudaStream_t s, const DevInfo& di);

// *d_out = 2^-down sum_i |amp_i|^2 via exact 128-bit fixed-point
// accumulation (K7, norm part); the scaled sum must stay below 16 (down = 0
// for normalised states; down = 36 bounds any state whose components are at
// most 1 in magnitude).  d_scratch needs norm_scratch_bytes(di) bytes.
size_t norm_scratch_bytes(const DevInfo& di);
cudaError_t launch_norm(int dt, const void* amp, int n, void* d_scratch, double* d_out,
                        cudaStream_t s, const DevInfo& di, int down = 0);

// Marginal over the qubits of qubit_mask into d_out (2^popcount doubles);
// d_bins needs 2 * 8 * 2^popcount bytes.
cudaError_t launch_marginal(int dt, const void* amp, int n, uint64_t qubit_mask, void* d_bins,
                            double* d_out, cudaStream_t s, const DevInfo& di);

}  // namespace svk

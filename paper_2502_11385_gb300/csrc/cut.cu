// CutQC reconstruction on the GPU (Sec. III-A, Eqs. 3.2-3.7; the Builder of
// Sec. IV-A, including its partial reconstruction over chosen qubits).
//
// Each of the K cut wires contributes one of four terms i_j in {1,2,3,4}:
//   upstream (measured variant m, outcome y of the cut qubit):
//     1: I/Z variant, weight 2 for y = 0     2: I/Z variant, weight 2 for y = 1
//     3: X variant, weight (-1)^y            4: Y variant, weight (-1)^y
//   downstream (initialisation s of the cut qubit):
//     1: |0>    2: |1>    3: 2|+> - |0> - |1>    4: 2|+i> - |0> - |1>
// p(x_A, x_B) = 2^-K sum_{i in {1..4}^K} U_i(x_A) D_i(x_B).
//
// U and D are accumulated exactly as signed 128-bit fixed-point numbers (units
// of 2^-112, two's complement, integer atomics: order-independent), then
// rounded once to float64; the final 4^K-term contraction runs in float64.
// Headroom: |U| <= 2^K and |D| <= 4^K <= 2^12 (K <= 6), so every bin stays
// below 2^124 < 2^127 in those units.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <vector>

#include "kernels.cuh"
#include "sv.h"

namespace {

constexpr int kMaxCuts = 6;
constexpr int kScale = 112;  // fixed-point unit 2^-112

struct CutGeom {
    int32_t K, width_a, width_b, keep_a_n, keep_b_n;
    int8_t cut_pos[kMaxCuts];   // cut qubit j inside the upstream circuit
    int8_t keep_a[40];          // kept upstream qubits, ascending (output bits 0..keep_a_n-1)
    int8_t keep_b[40];          // kept downstream qubits, ascending (output bits above)
};

__device__ __forceinline__ unsigned __int128 fixed_of(double x) {  // x >= 0
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int e = (int)((b >> 52) & 0x7ff);
    if (e == 0) return 0;
    const unsigned long long mant = (b & ((1ull << 52) - 1)) | (1ull << 52);
    const int sh = e - 1075 + kScale;
    if (sh >= 0) return (unsigned __int128)mant << sh;
    if (sh <= -53) return 0;
    return (unsigned __int128)(mant >> (-sh));
}

__device__ __forceinline__ void atomic_add_s128(unsigned long long* bin, unsigned __int128 v) {
    const unsigned long long lo = (unsigned long long)v;
    unsigned long long hi = (unsigned long long)(v >> 64);
    const unsigned long long old = atomicAdd(bin, lo);
    if (old + lo < old) hi += 1ull;
    if (hi) atomicAdd(bin + 1, hi);
}

__device__ __forceinline__ double s128_to_double(unsigned long long lo, unsigned long long hi) {
    unsigned __int128 v = ((unsigned __int128)hi << 64) | lo;
    const bool neg = (hi >> 63) != 0;
    if (neg) v = ~v + 1;  // magnitude
    if (v == 0) return 0.0;
    const unsigned long long h = (unsigned long long)(v >> 64), l = (unsigned long long)v;
    const int lz = h ? __clzll(h) : 64 + __clzll(l);
    const unsigned __int128 nv = v << lz;
    unsigned long long top = (unsigned long long)(nv >> 64);
    top |= ((unsigned long long)nv != 0ull) ? 1ull : 0ull;
    const double d = ldexp(__ull2double_rn(top), 64 - lz - kScale);
    return neg ? -d : d;
}

__device__ __forceinline__ int extract(uint64_t i, const int8_t* q, int nq) {
    int k = 0;
    for (int j = 0; j < nq; j++) k |= (int)((i >> q[j]) & 1) << j;
    return k;
}

// Upstream: variant v, index i -> every term code c with UP basis pattern v.
__global__ void k_cut_up(const double* const* __restrict__ up, const CutGeom g,
                         unsigned long long* __restrict__ bins) {
    const uint64_t dim = 1ull << g.width_a;
    int nvar = 1;
    for (int j = 0; j < g.K; j++) nvar *= 3;
    const uint64_t total = dim * (uint64_t)nvar;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const int nkeep = 1 << g.keep_a_n;
    for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += stride) {
        const int v = (int)(t / dim);
        const uint64_t i = t % dim;
        const double p = up[v][i];
        if (p == 0.0) continue;
        const unsigned __int128 fx = fixed_of(p);
        const int xk = extract(i, g.keep_a, g.keep_a_n);
        // enumerate term codes whose measurement pattern is v: per cut, basis
        // digit 0 (I/Z) allows terms {1, 2}; 1 (X) -> 3; 2 (Y) -> 4
        int digit[kMaxCuts], yb[kMaxCuts], nfree = 0;
        int vv = v;
        for (int j = 0; j < g.K; j++) {
            digit[j] = vv % 3;
            vv /= 3;
            yb[j] = (int)((i >> g.cut_pos[j]) & 1);
            if (digit[j] == 0) nfree++;
        }
        for (int f = 0; f < (1 << nfree); f++) {
            int code = 0, pw4 = 1, fb = 0, shift = 0;
            bool neg = false, zero = false;
            for (int j = 0; j < g.K; j++) {
                int term;  // 0-based term index
                if (digit[j] == 0) {
                    term = (f >> fb) & 1;  // term 1 (index 0) or term 2 (index 1)
                    fb++;
                    if (term != yb[j]) zero = true;  // weight 2 only on the matching outcome
                    shift++;                         // weight 2
                } else {
                    term = digit[j] + 1;  // X -> index 2, Y -> index 3
                    if (yb[j]) neg = !neg;
                }
                code += term * pw4;
                pw4 *= 4;
            }
            if (zero) continue;
            unsigned __int128 w = fx << shift;
            if (neg) w = ~w + 1;
            atomic_add_s128(bins + 2 * ((uint64_t)code * nkeep + xk), w);
        }
    }
}

// Downstream: initialisation s (base-4 digits), index x -> every term code c.
__global__ void k_cut_down(const double* const* __restrict__ down, const CutGeom g,
                           unsigned long long* __restrict__ bins) {
    const uint64_t dim = 1ull << g.width_b;
    int nvar = 1;
    for (int j = 0; j < g.K; j++) nvar *= 4;
    const uint64_t total = dim * (uint64_t)nvar;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const int nkeep = 1 << g.keep_b_n;
    // weight of initialisation s_j for term t_j (0-based): rows of
    // {1,0,0,0}, {0,1,0,0}, {-1,-1,2,0}, {-1,-1,0,2}
    for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += stride) {
        const int s = (int)(t / dim);
        const uint64_t x = t % dim;
        const double p = down[s][x];
        if (p == 0.0) continue;
        const unsigned __int128 fx = fixed_of(p);
        const int xk = extract(x, g.keep_b, g.keep_b_n);
        int sd[kMaxCuts];
        int ss = s;
        for (int j = 0; j < g.K; j++) {
            sd[j] = ss & 3;
            ss >>= 2;
        }
        const int ncode = 1 << (2 * g.K);
        for (int code = 0; code < ncode; code++) {
            bool zero = false, neg = false;
            int shift = 0;
            for (int j = 0; j < g.K && !zero; j++) {
                const int term = (code >> (2 * j)) & 3;
                const int sj = sd[j];
                if (term == 0) zero = sj != 0;
                else if (term == 1) zero = sj != 1;
                else if (sj <= 1) neg = !neg;        // -1 for |0>, |1>
                else if (sj == term) shift++;        // +2 for |+> (term 3) or |+i> (term 4)
                else zero = true;
            }
            if (zero) continue;
            unsigned __int128 w = fx << shift;
            if (neg) w = ~w + 1;
            atomic_add_s128(bins + 2 * ((uint64_t)code * nkeep + xk), w);
        }
    }
}

__global__ void k_bins_s128_to_double(const unsigned long long* __restrict__ bins, uint64_t n, double* out) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        out[i] = s128_to_double(bins[2 * i], bins[2 * i + 1]);
}

// out[xb * na + xa] = 2^-K sum_c U[c][xa] * D[c][xb]
__global__ void k_cut_combine(const double* __restrict__ U, const double* __restrict__ Dn, int ncode, uint64_t na,
                              uint64_t nb, double scale, double* __restrict__ out) {
    const uint64_t total = na * nb;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += stride) {
        const uint64_t xa = t % na, xb = t / na;
        double acc = 0.0;
        for (int c = 0; c < ncode; c++) acc = fma(U[(uint64_t)c * na + xa], Dn[(uint64_t)c * nb + xb], acc);
        out[t] = scale * acc;
    }
}

__global__ void k_zero(unsigned long long* p, uint64_t n) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) p[i] = 0ull;
}

unsigned grid_of(uint64_t work, int sms) {
    uint64_t g = (work + 255) / 256;
    const uint64_t cap = (uint64_t)sms * 8;
    if (g > cap) g = cap;
    return (unsigned)(g < 1 ? 1 : g);
}

}  // namespace

extern "C" int sv_cut_reconstruct(const double* const* up_probs, const double* const* down_probs, int n_cuts,
                                  int width_a, const int32_t* cut_pos_a, int width_b, uint64_t keep_mask_a,
                                  uint64_t keep_mask_b, double* out, size_t out_len, int out_is_device) {
    if (!up_probs || !down_probs || !cut_pos_a || !out) return SV_ERR_ARG;
    if (n_cuts < 1 || n_cuts > kMaxCuts || width_a < n_cuts + 1 || width_a > 34 || width_b < 1 || width_b > 34)
        return SV_ERR_ARG;
    CutGeom g;
    std::memset(&g, 0, sizeof(g));
    g.K = n_cuts;
    g.width_a = width_a;
    g.width_b = width_b;
    uint64_t cutmask = 0;
    for (int j = 0; j < n_cuts; j++) {
        if (cut_pos_a[j] < 0 || cut_pos_a[j] >= width_a || ((cutmask >> cut_pos_a[j]) & 1)) return SV_ERR_QUBIT;
        cutmask |= 1ull << cut_pos_a[j];
        g.cut_pos[j] = (int8_t)cut_pos_a[j];
    }
    if ((keep_mask_a & cutmask) || (keep_mask_a >> width_a) || (keep_mask_b >> width_b)) return SV_ERR_QUBIT;
    for (int q = 0; q < width_a; q++)
        if ((keep_mask_a >> q) & 1) g.keep_a[g.keep_a_n++] = (int8_t)q;
    for (int q = 0; q < width_b; q++)
        if ((keep_mask_b >> q) & 1) g.keep_b[g.keep_b_n++] = (int8_t)q;
    if (g.keep_a_n + g.keep_b_n > 34) return SV_ERR_SIZE;
    const uint64_t na = 1ull << g.keep_a_n, nb = 1ull << g.keep_b_n;
    if (out_len != na * nb) return SV_ERR_SIZE;
    const int ncode = 1 << (2 * n_cuts);
    int nup = 1, ndown = 1;
    for (int j = 0; j < n_cuts; j++) {
        nup *= 3;
        ndown *= 4;
    }
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return SV_ERR_CUDA;
    // device scratch: pointer tables, 128-bit bins, float64 U and D, output staging
    const size_t ptr_bytes = (size_t)(nup + ndown) * sizeof(double*);
    const size_t ub = (size_t)ncode * na, db = (size_t)ncode * nb;
    const size_t bins_bytes = 2 * 8 * (ub + db);
    const size_t f_bytes = 8 * (ub + db);
    const size_t out_bytes = out_is_device ? 0 : 8 * na * nb;
    unsigned char* scratch = nullptr;
    const size_t total = ptr_bytes + 256 + bins_bytes + f_bytes + out_bytes + 256;
    cudaError_t e = cudaMalloc(&scratch, total);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? SV_ERR_OOM : SV_ERR_CUDA;
    }
    auto** d_ptrs = (const double**)scratch;
    auto* bins = (unsigned long long*)(scratch + ((ptr_bytes + 255) & ~(size_t)255));
    auto* Uf = (double*)(bins + 2 * (ub + db));
    double* Df = Uf + ub;
    double* d_out = out_is_device ? out : (Df + db);
    std::vector<const double*> hp(up_probs, up_probs + nup);
    hp.insert(hp.end(), down_probs, down_probs + ndown);
    int rc = SV_OK;
    cudaStream_t s = nullptr;
    if (cudaMemcpy(d_ptrs, hp.data(), ptr_bytes, cudaMemcpyHostToDevice) != cudaSuccess) rc = SV_ERR_CUDA;
    if (rc == SV_OK) {
        k_zero<<<grid_of(2 * (ub + db), sms), 256, 0, s>>>(bins, 2 * (ub + db));
        k_cut_up<<<grid_of((1ull << width_a) * nup, sms), 256, 0, s>>>(d_ptrs, g, bins);
        k_cut_down<<<grid_of((1ull << width_b) * ndown, sms), 256, 0, s>>>(d_ptrs + nup, g, bins + 2 * ub);
        k_bins_s128_to_double<<<grid_of(ub + db, sms), 256, 0, s>>>(bins, ub + db, Uf);
        k_cut_combine<<<grid_of(na * nb, sms), 256, 0, s>>>(Uf, Df, ncode, na, nb, 1.0 / (double)(1ull << n_cuts),
                                                           d_out);
        if (cudaGetLastError() != cudaSuccess) rc = SV_ERR_CUDA;
    }
    if (rc == SV_OK && !out_is_device &&
        cudaMemcpy(out, d_out, 8 * na * nb, cudaMemcpyDeviceToHost) != cudaSuccess)
        rc = SV_ERR_CUDA;
    if (rc == SV_OK && cudaDeviceSynchronize() != cudaSuccess) rc = SV_ERR_CUDA;
    cudaFree(scratch);
    return rc;
}

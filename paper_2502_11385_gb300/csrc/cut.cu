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
// Three steps, none with atomics:
//  1. k_marginal_var: every variant's distribution summed over the qubits
//     that are neither kept nor cut, one thread per (variant, bin), exactly
//     in 128-bit fixed point (units of 2^-112; a bin of a distribution is at
//     most 1) -- the one pass over all variant data, bound by HBM;
//  2. k_up_terms / k_down_terms: U_i and D_i as exact integer combinations
//     (weights 0, +-1, +-2 per cut) of those small marginals, in signed
//     128-bit fixed point (|U| <= 2^K, |D| <= 4^K), rounded once to float64
//     and split into float pairs (hi, lo: 48 significant bits);
//  3. k_combine: the [2^kb x 4^K] x [4^K x 2^ka] contraction, tiled through
//     shared memory, in compensated float-pair arithmetic on the FP32 units
//     (error-free TwoProd and TwoSum, Ogita, Rump and Oishi 2005): absolute
//     error about 2^-47 sum_i |U_i D_i| 2^-K per output.
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
    uint64_t mask_a;            // upstream marginal qubits: the kept ones, then the cut ones
    uint64_t mask_b;            // downstream marginal qubits: the kept ones
    int8_t mq_a[40];            // upstream marginal qubits in bin-bit order (kept ascending, then cut j)
    int8_t mq_b[40];            // downstream kept qubits, ascending
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

__device__ __forceinline__ double s128_to_double(unsigned __int128 v) {
    const bool neg = (unsigned long long)(v >> 64) >> 63;
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

__device__ __forceinline__ unsigned __int128 ld128(const unsigned long long* p, uint64_t i) {
    return ((unsigned __int128)p[2 * i + 1] << 64) | p[2 * i];
}
__device__ __forceinline__ void st128(unsigned long long* p, uint64_t i, unsigned __int128 v) {
    p[2 * i] = (unsigned long long)v;
    p[2 * i + 1] = (unsigned long long)(v >> 64);
}

// Step 1: out[v * nbins + b] = sum of p_v[i] over every i whose bits at the
// marginal qubits mq[0..nm) are b.  The other indices are walked in
// increasing order with ((r | M) + 1) & ~M.
__global__ void k_marginal_var(const double* const* __restrict__ var, int nvar, int width, uint64_t M,
                               const int8_t* __restrict__ mq_g, int nm, unsigned long long* __restrict__ out) {
    __shared__ int8_t mq[40];
    if (threadIdx.x < 40) mq[threadIdx.x] = threadIdx.x < nm ? mq_g[threadIdx.x] : 0;
    __syncthreads();
    const uint64_t nbins = 1ull << nm, total = nbins * (uint64_t)nvar;
    const uint64_t dim = 1ull << width;
    const uint64_t rest = dim >> nm;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += stride) {
        const uint64_t b = t % nbins;
        const double* p = var[t / nbins];
        uint64_t base = 0;
        for (int j = 0; j < nm; j++) base |= ((b >> j) & 1ull) << mq[j];
        unsigned __int128 acc = 0;
        uint64_t r = 0;
        for (uint64_t k = 0; k < rest; k++) {
            acc += fixed_of(p[base | r]);
            r = ((r | M) + 1) & ~M;
        }
        st128(out, t, acc);
    }
}

// Step 2, upstream: U_code(xk) = 2^(#terms 1, 2) sum over the outcomes y of
// the cuts with terms 3, 4 of (-1)^(their y) m_v(xk, y), the other cuts' y
// fixed by the term (term 1: y = 0, term 2: y = 1).
__global__ void k_up_terms(const unsigned long long* __restrict__ mup, int K, int ka,
                           float2* __restrict__ U, int ncode) {
    const uint64_t na = 1ull << ka, total = na * (uint64_t)ncode, nb_up = na << K;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += stride) {
        const int code = (int)(t / na);
        const uint64_t xk = t % na;
        int v = 0, p3 = 1, shift = 0, ybase = 0, freem = 0;
        for (int j = 0; j < K; j++) {
            const int term = (code >> (2 * j)) & 3;
            v += (term <= 1 ? 0 : term - 1) * p3;
            p3 *= 3;
            if (term <= 1) {
                shift++;
                ybase |= term << j;
            } else {
                freem |= 1 << j;
            }
        }
        unsigned __int128 acc = 0;
        // every assignment of the free cuts' outcomes: subsets of freem
        int y = 0;
        for (;;) {
            const unsigned __int128 m = ld128(mup, (uint64_t)v * nb_up + xk + ((uint64_t)(ybase | y) << ka));
            if (__popc(y) & 1) acc -= m;
            else acc += m;
            if (y == freem) break;
            y = ((y | ~freem) + 1) & freem;
        }
        const double d = s128_to_double(acc << shift);
        const float hi = (float)d;
        U[t] = make_float2(hi, (float)(d - (double)hi));
    }
}

// Step 2, downstream: D_code(xb) = sum over initialisations s of the product
// over cuts of w(term_j, s_j) m_s(xb), with w rows (1,0,0,0), (0,1,0,0),
// (-1,-1,2,0), (-1,-1,0,2).
__global__ void k_down_terms(const unsigned long long* __restrict__ mdn, int K, int kb,
                             float2* __restrict__ Dn, int ncode) {
    const uint64_t nb = 1ull << kb, total = nb * (uint64_t)ncode;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += stride) {
        const int code = (int)(t / nb);
        const uint64_t xb = t % nb;
        unsigned __int128 acc = 0;
        // enumerate s digit by digit: terms 1, 2 have one choice, terms 3, 4 three
        int choice[kMaxCuts], nchoice[kMaxCuts];
        for (int j = 0; j < K; j++) {
            choice[j] = 0;
            nchoice[j] = ((code >> (2 * j)) & 3) <= 1 ? 1 : 3;
        }
        for (;;) {
            int s = 0, p4 = 1, shift = 0;
            bool neg = false;
            for (int j = 0; j < K; j++) {
                const int term = (code >> (2 * j)) & 3;
                int sj;
                if (term <= 1) sj = term;
                else if (choice[j] < 2) {  // -|0>, -|1>
                    sj = choice[j];
                    neg = !neg;
                } else {  // +2 |+> (term 3) or +2 |+i> (term 4)
                    sj = term;
                    shift++;
                }
                s += sj * p4;
                p4 *= 4;
            }
            unsigned __int128 m = ld128(mdn, (uint64_t)s * nb + xb) << shift;
            if (neg) acc -= m;
            else acc += m;
            int j = 0;
            while (j < K && ++choice[j] == nchoice[j]) choice[j++] = 0;
            if (j == K) break;
        }
        const double d = s128_to_double(acc);
        const float hi = (float)d;
        Dn[t] = make_float2(hi, (float)(d - (double)hi));
    }
}

// Step 3: out[xb na + xa] = scale sum_c U[c][xa] D[c][xb], float-pair dot
// products.  A CTA of 256 threads computes a 64 x 64 tile (4 x 4 outputs a
// thread), 32 codes at a time through shared memory.
constexpr int kTile = 64, kCodes = 32;

__device__ __forceinline__ void dot2_add(float& s, float& c, float2 a, float2 b) {
    const float p = __fmul_rn(a.x, b.x);
    const float e = fmaf(a.x, b.x, -p);                      // a.hi b.hi = p + e exactly
    const float t = __fadd_rn(s, p), z = __fsub_rn(t, s);
    const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(p, z));  // s + p = t + err exactly
    s = t;
    c += err + e + fmaf(a.x, b.y, a.y * b.x);
}

__global__ void __launch_bounds__(256) k_combine(const float2* __restrict__ U, const float2* __restrict__ Dn,
                                                 int ncode, uint64_t na, uint64_t nb, double scale,
                                                 double* __restrict__ out) {
    __shared__ float2 su[kCodes][kTile], sd[kCodes][kTile];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const uint64_t ta = (uint64_t)blockIdx.x * kTile;
    const uint64_t ntb = (nb + kTile - 1) / kTile;
    for (uint64_t bt = blockIdx.y; bt < ntb; bt += gridDim.y) {  // output row tiles beyond the grid's y range
    const uint64_t tb = bt * kTile;
    float s[4][4], c[4][4];
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) s[i][j] = c[i][j] = 0.f;
    for (int c0 = 0; c0 < ncode; c0 += kCodes) {
        __syncthreads();
        for (int e = threadIdx.x; e < kCodes * kTile; e += 256) {
            const int cc = e / kTile, x = e % kTile;
            const bool live = c0 + cc < ncode;
            su[cc][x] = (live && ta + x < na) ? U[(uint64_t)(c0 + cc) * na + ta + x] : make_float2(0.f, 0.f);
            sd[cc][x] = (live && tb + x < nb) ? Dn[(uint64_t)(c0 + cc) * nb + tb + x] : make_float2(0.f, 0.f);
        }
        __syncthreads();
        for (int cc = 0; cc < kCodes; cc++) {
            float2 a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; i++) {
                a[i] = su[cc][tx + 16 * i];
                b[i] = sd[cc][ty + 16 * i];
            }
#pragma unroll
            for (int i = 0; i < 4; i++)
#pragma unroll
                for (int j = 0; j < 4; j++) dot2_add(s[i][j], c[i][j], a[i], b[j]);
        }
    }
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const uint64_t xa = ta + tx + 16 * i, xb = tb + ty + 16 * j;
            if (xa < na && xb < nb) out[xb * na + xa] = scale * ((double)s[i][j] + (double)c[i][j]);
        }
    }
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
    int nma = 0, nmb = 0;
    for (int q = 0; q < width_a; q++)
        if ((keep_mask_a >> q) & 1) g.mq_a[nma++] = (int8_t)q;
    g.keep_a_n = nma;
    for (int j = 0; j < n_cuts; j++) g.mq_a[nma++] = g.cut_pos[j];
    for (int q = 0; q < width_b; q++)
        if ((keep_mask_b >> q) & 1) g.mq_b[nmb++] = (int8_t)q;
    g.keep_b_n = nmb;
    g.mask_a = keep_mask_a | cutmask;
    g.mask_b = keep_mask_b;
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
    // device scratch: pointer tables, marginal qubit lists, 128-bit marginals,
    // float-pair term tables, output staging
    const size_t ptr_bytes = (size_t)(nup + ndown) * sizeof(double*);
    const uint64_t nbin_a = na << n_cuts;
    const size_t mup_bytes = 16 * (size_t)nup * nbin_a, mdn_bytes = 16 * (size_t)ndown * nb;
    const size_t u_bytes = 8 * (size_t)ncode * na, d_bytes = 8 * (size_t)ncode * nb;
    const size_t out_bytes = out_is_device ? 0 : 8 * na * nb;
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t o_mq = al(ptr_bytes), o_mup = o_mq + 256, o_mdn = o_mup + al(mup_bytes),
                 o_u = o_mdn + al(mdn_bytes), o_d = o_u + al(u_bytes), o_out = o_d + al(d_bytes);
    unsigned char* scratch = nullptr;
    cudaError_t e = cudaMalloc(&scratch, o_out + out_bytes + 256);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? SV_ERR_OOM : SV_ERR_CUDA;
    }
    auto** d_ptrs = (const double**)scratch;
    auto* d_mq = (int8_t*)(scratch + o_mq);  // mq_a at 0, mq_b at 64
    auto* mup = (unsigned long long*)(scratch + o_mup);
    auto* mdn = (unsigned long long*)(scratch + o_mdn);
    auto* Ut = (float2*)(scratch + o_u);
    auto* Dt = (float2*)(scratch + o_d);
    double* d_out = out_is_device ? out : (double*)(scratch + o_out);
    std::vector<const double*> hp(up_probs, up_probs + nup);
    hp.insert(hp.end(), down_probs, down_probs + ndown);
    int8_t mqs[128];
    std::memset(mqs, 0, sizeof(mqs));
    std::memcpy(mqs, g.mq_a, 40);
    std::memcpy(mqs + 64, g.mq_b, 40);
    int rc = SV_OK;
    cudaStream_t s = nullptr;
    if (cudaMemcpy(d_ptrs, hp.data(), ptr_bytes, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(d_mq, mqs, sizeof(mqs), cudaMemcpyHostToDevice) != cudaSuccess)
        rc = SV_ERR_CUDA;
    if (rc == SV_OK) {
        const int nm_a = g.keep_a_n + n_cuts;
        k_marginal_var<<<grid_of(nbin_a * nup, sms), 256, 0, s>>>(d_ptrs, nup, width_a, g.mask_a, d_mq, nm_a, mup);
        k_marginal_var<<<grid_of(nb * ndown, sms), 256, 0, s>>>(d_ptrs + nup, ndown, width_b, g.mask_b, d_mq + 64,
                                                              g.keep_b_n, mdn);
        k_up_terms<<<grid_of(na * ncode, sms), 256, 0, s>>>(mup, n_cuts, g.keep_a_n, Ut, ncode);
        k_down_terms<<<grid_of(nb * ncode, sms), 256, 0, s>>>(mdn, n_cuts, g.keep_b_n, Dt, ncode);
        const uint64_t gy = (nb + kTile - 1) / kTile;
        const dim3 grid((unsigned)((na + kTile - 1) / kTile), (unsigned)(gy < 65535 ? gy : 65535));
        k_combine<<<grid, 256, 0, s>>>(Ut, Dt, ncode, na, nb, 1.0 / (double)(1ull << n_cuts), d_out);
        if (cudaGetLastError() != cudaSuccess) rc = SV_ERR_CUDA;
    }
    if (rc == SV_OK && !out_is_device &&
        cudaMemcpy(out, d_out, 8 * na * nb, cudaMemcpyDeviceToHost) != cudaSuccess)
        rc = SV_ERR_CUDA;
    if (rc == SV_OK && cudaDeviceSynchronize() != cudaSuccess) rc = SV_ERR_CUDA;
    cudaFree(scratch);
    return rc;
}

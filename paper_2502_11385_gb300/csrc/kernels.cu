// sm_103a kernels of the statevector engine.
//
//   K1 k_init          amp := e_basis
//   K5 k_tile_pass     cache-blocked pass: gather a tile of 2^m amplitudes over
//                      the pass's local qubits into shared memory, apply the
//                      pass's fused blocks in order, write the tile back
//                      (the single-GPU counterpart of Aer's chunk blocking,
//                      Sec. III-B, Fig. 4)
//   K7 k_probs         p_i = |a_i|^2 (Listing 3's probabilities())
//      k_norm_*        sum_i p_i, exact 128-bit fixed-point accumulation
//      k_marginal      marginal distribution over chosen qubits (the
//                      Builder's partial reconstruction, Sec. IV-A)
//
// Amplitudes are interleaved complex; index bit q is qubit q.
#include <cuda_runtime.h>

#include <cuda_bf16.h>

#include <algorithm>

#include "kernels.cuh"
#include "sv.h"

namespace svk {

template <typename R>
struct alignas(2 * sizeof(R)) Cx {
    R re, im;
};

__device__ __forceinline__ float fmaT(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fmaT(double a, double b, double c) { return fma(a, b, c); }

// ---------------------------------------------------------------------------
// Shared-memory layout of a tile: 16-byte slots, XOR-swizzled so that warps
// gathering amplitudes at power-of-two strides spread over the banks.
// ---------------------------------------------------------------------------
// swz(j) = j ^ L(j) with L linear over GF(2) (shifts and XORs), so
// swz(a ^ b) = swz(a) ^ swz(b).
template <typename R>
__device__ __forceinline__ int swz(int j) {
    constexpr int VS = (sizeof(R) == 4) ? 1 : 0;  // log2(amplitudes per 16-byte slot); R = float or double
    int s = j >> VS;
    int h = (s >> 3) ^ (s >> 6) ^ (s >> 9) ^ (s >> 12);
    s ^= h & 7;
    return (s << VS) | (j & ((1 << VS) - 1));
}

// ---------------------------------------------------------------------------
// K1: initialise to a basis state.
// ---------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ int4 unit_vector16(int e);  // 16 bytes holding 1 at amplitude e, 0 elsewhere
template <>
__device__ __forceinline__ int4 unit_vector16<float>(int e) {
    const int one = __float_as_int(1.0f);
    return e == 0 ? make_int4(one, 0, 0, 0) : make_int4(0, 0, one, 0);
}
template <>
__device__ __forceinline__ int4 unit_vector16<double>(int) {
    const long long one = __double_as_longlong(1.0);
    return make_int4((int)(one & 0xffffffffll), (int)(one >> 32), 0, 0);
}

template <typename R>
__global__ void k_init(Cx<R>* __restrict__ a, uint64_t dim, uint64_t basis) {
    constexpr int PER = 16 / sizeof(Cx<R>);  // amplitudes per 16-byte store; dim is a multiple
    const uint64_t nvec = dim / PER;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < nvec; v += stride) {
        const int4 z = (basis / PER == v) ? unit_vector16<R>((int)(basis % PER)) : make_int4(0, 0, 0, 0);
        reinterpret_cast<int4*>(a)[v] = z;
    }
}

// ---------------------------------------------------------------------------
// K5: tile pass.
// ---------------------------------------------------------------------------
// Offset of matrix row/column b inside a group: bit j of b selects tile
// position pos[j] (pm[j] = 1 << pos[j]).
template <int K>
__device__ __forceinline__ int group_offset(int b, const int (&pm)[K]) {
    int off = 0;
#pragma unroll
    for (int j = 0; j < K; j++)
        if ((b >> j) & 1) off |= pm[j];
    return off;
}

// Groups a thread handles per step of a k-qubit dense op: each coefficient
// load then feeds G independent groups.
// (Native float64 is bound by the FP64 pipe, so it keeps one group per step.)
template <int K, typename R>
struct GroupsPerStep {
    static constexpr int value = sizeof(R) == 8 ? 1 : (K <= 2 ? 4 : (K == 3 ? 2 : 1));
};

template <int K>
__device__ __forceinline__ int insert_zero_bits(int g, const int (&pos)[K]) {
#pragma unroll
    for (int j = 0; j < K; j++) {
        const int p = pos[j];
        g = ((g >> p) << (p + 1)) | (g & ((1 << p) - 1));
    }
    return g;
}

template <int K, typename R>
__device__ __forceinline__ void op_dense(Cx<R>* sm, int m, const DevOp& op, const Cx<R>* __restrict__ M) {
    constexpr int D = 1 << K;
    constexpr int G = GroupsPerStep<K, R>::value;
    int pos[K], pm[K];
#pragma unroll
    for (int j = 0; j < K; j++) {
        pos[j] = op.pos[j];
        pm[j] = 1 << pos[j];
    }
    // the swizzle is linear over GF(2) and base / offset bits are disjoint:
    // swz(base | off) = swz(base) ^ swz(off)
    constexpr int DS = K <= 4 ? D : 1;  // 5-qubit blocks recompute offsets (registers)
    int soff[DS];
#pragma unroll
    for (int b = 0; b < DS; b++) soff[b] = swz<R>(group_offset<K>(b, pm));
    auto sofs = [&](int b) { return K <= 4 ? soff[b & (DS - 1)] : swz<R>(group_offset<K>(b, pm)); };
    const int ng = 1 << (m - K);
    for (int g0 = threadIdx.x; g0 < ng; g0 += blockDim.x * G) {
        int base[G];
        bool ok[G];
        Cx<R> a[G][D];
#pragma unroll
        for (int q = 0; q < G; q++) {
            const int g = g0 + q * blockDim.x;
            ok[q] = g < ng;
            base[q] = swz<R>(insert_zero_bits<K>(ok[q] ? g : 0, pos));
#pragma unroll
            for (int b = 0; b < D; b++) a[q][b] = sm[base[q] ^ sofs(b)];
        }
        // for blocks of up to 3 qubits the coefficient rows are
        // software-pipelined: row r + 1 is loaded while row r is multiplied
        constexpr bool kPipe = K <= 3 && sizeof(R) == 4;  // FP64 is bound by its pipe anyway
        constexpr int DP = kPipe ? D : 1;
        Cx<R> un[DP];
        if constexpr (kPipe) {
#pragma unroll
            for (int c = 0; c < D; c++) un[c] = M[c];
        }
#pragma unroll(K <= 2 ? D : 1)
        for (int r = 0; r < D; r++) {
            Cx<R> ur[DP];
            if constexpr (kPipe) {
#pragma unroll
                for (int c = 0; c < D; c++) ur[c] = un[c];
                if (r + 1 < D) {
#pragma unroll
                    for (int c = 0; c < D; c++) un[c] = M[(r + 1) * D + c];
                }
            }
            R re[G], im[G];
#pragma unroll
            for (int q = 0; q < G; q++) re[q] = im[q] = R(0);
#pragma unroll
            for (int c = 0; c < D; c++) {
                const Cx<R> u = kPipe ? ur[c % DP] : M[r * D + c];
#pragma unroll
                for (int q = 0; q < G; q++) {
                    re[q] = fmaT(u.re, a[q][c].re, re[q]);
                    re[q] = fmaT(-u.im, a[q][c].im, re[q]);
                    im[q] = fmaT(u.re, a[q][c].im, im[q]);
                    im[q] = fmaT(u.im, a[q][c].re, im[q]);
                }
            }
            const int off = sofs(r);
#pragma unroll
            for (int q = 0; q < G; q++)
                if (ok[q]) sm[base[q] ^ off] = Cx<R>{re[q], im[q]};
        }
    }
}

// Diagonal ops visit amplitude i = threadIdx.x + it * (CTA size).  The
// phase-table index takes bit j from tile position pos[j] (or, for a
// non-local qubit, from the tile's base index); the bits below log2 of the
// CTA size come from the thread id and are gathered once per op.
struct DiagIndex {
    int idx_t;  // table-index bits fixed for this thread
    int hp;     // 5 bits per table bit j: its tile position relative to the CTA size, or 31
    int sw_t;   // swizzle of the thread's part of i
};

template <typename SwzT, int LT = 8>  // LT = log2 of the CTA size
__device__ __forceinline__ DiagIndex diag_index(const DevOp& op, uint64_t tile_base) {
    DiagIndex d;
    d.idx_t = 0;
    d.hp = 0;
    const int t = threadIdx.x;
#pragma unroll
    for (int j = 0; j < 5; j++) {
        int h = 31;  // (it >> 31) & 1 = 0: the bit is not taken from it
        if (j < op.k) {
            const int p = op.pos[j];
            if (p < 0) d.idx_t |= (int)((tile_base >> op.qbit[j]) & 1) << j;
            else if (p < LT) d.idx_t |= ((t >> p) & 1) << j;
            else h = p - LT;
        }
        d.hp |= h << (5 * j);
    }
    d.sw_t = swz<SwzT>(t);
    return d;
}

template <typename SwzT, int LT = 8>
__device__ __forceinline__ void diag_at(const DiagIndex& d, int it, int& idx, int& sidx) {
    idx = d.idx_t;
#pragma unroll
    for (int j = 0; j < 5; j++) idx |= ((it >> ((d.hp >> (5 * j)) & 31)) & 1) << j;
    sidx = d.sw_t ^ swz<SwzT>(it << LT);
}

// Applies a <- f(u, a) to every amplitude of the tile (u its phase-table
// entry), U amplitudes of a thread at a time: their loads are all issued
// before their stores, so the U table and tile reads overlap.
template <int U, int LT, typename SwzT, typename T, typename E, typename F>
__device__ __forceinline__ void diag_sweep(T* sm, int m, const DiagIndex& d, const E* M, F f) {
    const int N = 1 << m;
    if (N >= (1 << LT)) {
        const int iters = N >> LT;
        int it = 0;
        for (; it + U <= iters; it += U) {
            int idx[U], si[U];
            E u[U];
            T a[U];
#pragma unroll
            for (int q = 0; q < U; q++) diag_at<SwzT, LT>(d, it + q, idx[q], si[q]);
#pragma unroll
            for (int q = 0; q < U; q++) {
                u[q] = M[idx[q]];
                a[q] = sm[si[q]];
            }
#pragma unroll
            for (int q = 0; q < U; q++) sm[si[q]] = f(u[q], a[q]);
        }
        for (; it < iters; it++) {
            int idx, si;
            diag_at<SwzT, LT>(d, it, idx, si);
            sm[si] = f(M[idx], sm[si]);
        }
    } else if ((int)threadIdx.x < N) {  // a tile smaller than the CTA: threads past N idle
        int idx, si;
        diag_at<SwzT, LT>(d, 0, idx, si);
        sm[si] = f(M[idx], sm[si]);
    }
}

template <typename R, int LT = 8>  // LT = log2 of the CTA size
__device__ __forceinline__ void op_diag(Cx<R>* sm, int m, const DevOp& op, const Cx<R>* __restrict__ M,
                                        uint64_t tile_base) {
    const DiagIndex d = diag_index<R, LT>(op, tile_base);
    constexpr int U = sizeof(R) == 4 ? 4 : 2;
    if (op.flags & OPF_SIGN_ONLY)
        diag_sweep<U, LT, R>(sm, m, d, M, [](Cx<R> u, Cx<R> a) { return u.re < R(0) ? Cx<R>{-a.re, -a.im} : a; });
    else
        diag_sweep<U, LT, R>(sm, m, d, M, [](Cx<R> u, Cx<R> a) {
            return Cx<R>{fmaT(u.re, a.re, -u.im * a.im), fmaT(u.re, a.im, u.im * a.re)};
        });
}

// ---------------------------------------------------------------------------
// Permutation blocks (X, Y, CX, SWAP with diagonal gates whose phases are
// powers of i): out[r] = i^code(r) in[src(r)] inside every group of 2^k
// amplitudes, moved along the permutation's cycles with one temporary (each
// amplitude read once and written once); i^code is a swap of the real and
// imaginary parts and sign changes, exact in every tile format.  The moves
// (dst | code << 5 | end-of-cycle << 7, in cycle order) are the op's
// coefficient elements, decoded by the caller's mv(t).
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T rot_i(T v, int code) {  // v * i^code for {re, im} pairs
    using E = decltype(v.re);
    const E re = v.re, im = v.im;
    if (code == 1) return T{-im, re};
    if (code == 2) return T{-re, -im};
    if (code == 3) return T{im, -re};
    return v;
}

// Groups of a k-qubit op: zero bits inserted at the op's tile positions.
__device__ __forceinline__ int group_base(int g, const int (&pos)[5], int k) {
#pragma unroll
    for (int j = 0; j < 5; j++)
        if (j < k) g = ((g >> pos[j]) << (pos[j] + 1)) | (g & ((1 << pos[j]) - 1));
    return g;
}

// s_mv: the op's moves in cycle order, s_src: per output row r, the row it
// takes its amplitude from and the phase code (src | code << 5); both staged
// in shared memory by the caller.  Blocks of up to 3 qubits move a group's
// 2^k amplitudes through registers (all reads, then all writes); larger
// blocks follow the cycles with one temporary.
template <int K, typename S, typename SwzT>
__device__ __forceinline__ void op_perm(S* sm, int m, const DevOp& op, const int* s_mv, const int* s_src, int tid,
                                        int nthreads, S (*rot)(S, int)) {
    constexpr int D = 1 << K;
    int sp[5], pos[5];
#pragma unroll
    for (int j = 0; j < 5; j++) {
        pos[j] = j < K ? op.pos[j] : 31;
        sp[j] = j < K ? swz<SwzT>(1 << op.pos[j]) : 0;
    }
    auto off = [&](int b) {
        int o = 0;
#pragma unroll
        for (int j = 0; j < K; j++)
            if ((b >> j) & 1) o ^= sp[j];
        return o;
    };
    const int ng = 1 << (m - K);
    for (int g = tid; g < ng; g += nthreads) {
        const int base = swz<SwzT>(group_base(g, pos, K));
        if constexpr (K <= 3) {
            S v[D];  // v[r] = the source of output row r (all reads before any write)
#pragma unroll
            for (int r = 0; r < D; r++) v[r] = sm[base ^ off(s_src[r] & 31)];
#pragma unroll
            for (int r = 0; r < D; r++) sm[base ^ off(r)] = rot(v[r], (s_src[r] >> 5) & 3);
        } else {
            for (int t = 0; t < D;) {
                int mv = s_mv[t];
                const S first = sm[base ^ off(mv & 31)];
                for (;;) {
                    const bool end = (mv & 128) != 0;
                    const int nx = end ? 0 : s_mv[t + 1];
                    const S a = end ? first : sm[base ^ off(nx & 31)];
                    sm[base ^ off(mv & 31)] = rot(a, (mv >> 5) & 3);
                    t++;
                    if (end) break;
                    mv = nx;
                }
            }
        }
    }
}

__device__ __forceinline__ Cx<float> rot_cf(Cx<float> v, int c) { return rot_i(v, c); }
__device__ __forceinline__ Cx<double> rot_cd(Cx<double> v, int c) { return rot_i(v, c); }

// ---------------------------------------------------------------------------
// K5-df: tile pass for complex128 states with double-float arithmetic.
//
// GB300's FP64 units run about 70x slower than its FP32 units, so complex128
// gates are computed on (hi, lo) float pairs instead (Dekker 1971): each
// float64 amplitude component is split once per pass, when the tile is
// loaded, into hi = its leading 24 significant bits and lo = the next 23
// (47 bits, |x - hi - lo| <= 2^-47 |x|), with integer bit operations so the
// FP64 pipe stays idle; block products use error-free TwoProd (FMA) and
// TwoSum transforms (the compensated dot product of Ogita, Rump and Oishi
// 2005, with double-float inputs); the tile is re-assembled into float64 on
// store, again with integer operations.
// ---------------------------------------------------------------------------
struct alignas(16) DF4 {
    float rh, rl, ih, il;  // re = rh + rl, im = ih + il
};
__device__ __forceinline__ DF4 rot_df(DF4 v, int c) {  // v * i^c
    if (c == 1) return DF4{-v.ih, -v.il, v.rh, v.rl};
    if (c == 2) return DF4{-v.rh, -v.rl, -v.ih, -v.il};
    if (c == 3) return DF4{v.ih, v.il, -v.rh, -v.rl};
    return v;
}

__device__ __forceinline__ void d2df(double x, float& h, float& l) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned hi32 = (unsigned)(b >> 32), lo32 = (unsigned)b;
    const unsigned sign = hi32 & 0x80000000u;
    const int e = (int)((hi32 >> 20) & 0x7ff);
    if (e < 897) {  // |x| < 2^-126 (or zero): below float's normal range, dropped
                    // (for 2^-126 <= |x| < 2^-103 only hi is kept: absolute error < 2^-126)
        h = 0.f;
        l = 0.f;
        return;
    }
    // amplitudes satisfy |x| <= 1 < 2^127, so e - 896 fits float's exponent field
    h = __uint_as_float(sign | ((unsigned)(e - 896) << 23) | ((hi32 & 0xFFFFFu) << 3) | (lo32 >> 29));
    const unsigned r = (lo32 >> 6) & 0x7FFFFFu;  // next 23 mantissa bits, weight 2^(e-1069)
    const int B = e - 919;                       // float exponent field with 2^(B-150) = 2^(e-1069)
    if (B < 1 || r == 0u) {
        l = 0.f;
        return;
    }
    const unsigned one = sign | ((unsigned)B << 23);
    l = __fadd_rn(__uint_as_float(one | r), -__uint_as_float(one));  // exact: (1 + r 2^-23) 2^(B-127) - 2^(B-127)
}

__device__ __forceinline__ double df2d(float h, float l) {
    const float s = __fadd_rn(h, l);  // Fast2Sum: |l| <= ulp(s)/2 afterwards
    l = __fadd_rn(l, -__fadd_rn(s, -h));
    h = s;
    const unsigned hb = __float_as_uint(h);
    const unsigned eh = (hb >> 23) & 0xffu;
    if (eh == 0u) return 0.0;  // zero or subnormal hi: below the amplitudes' range
    const unsigned long long D = ((unsigned long long)(hb & 0x80000000u) << 32) |
                                 ((unsigned long long)(eh + 896u) << 52) |
                                 ((unsigned long long)(hb & 0x7FFFFFu) << 29);
    const unsigned lb = __float_as_uint(l);
    if ((lb & 0x7FFFFFFFu) == 0u) return __longlong_as_double((long long)D);
    // l = ml * 2^(el - 150) (subnormal l: no implicit bit, el taken as 1)
    const unsigned el_raw = (lb >> 23) & 0xffu;
    const unsigned el = el_raw ? el_raw : 1u;
    const unsigned long long ml = (unsigned long long)((lb & 0x7FFFFFu) | (el_raw ? 0x800000u : 0u));
    // in units of ulp_double(h) = 2^(eh - 179): k = ml * 2^(el - eh + 29), el <= eh - 24
    const int sh = (int)el - (int)eh + 29;
    unsigned long long k = sh >= 0 ? (ml << sh) : (sh > -40 ? (ml >> (-sh)) : 0ull);
    unsigned long long mag = D & 0x7FFFFFFFFFFFFFFFull;
    if ((lb ^ hb) & 0x80000000u) {
        if ((hb & 0x7FFFFFu) == 0u) k <<= 1;  // hi is a power of two: the result lies in the lower binade
        mag -= k;
    } else {
        mag += k;  // no carry out of the mantissa: |l| <= 2^28 ulp_double(h)
    }
    return __longlong_as_double((long long)((D & 0x8000000000000000ull) | mag));
}

// (sh, sl) += x * y for double-floats x = (xh, xl), y = (yh, yl): TwoProd of the
// high parts, first-order cross terms, TwoSum into the running sum.  __fmul_rn
// and __fadd_rn keep the compiler from contracting the transforms into FMAs.
__device__ __forceinline__ void df_mac(float& sh, float& sl, float xh, float xl, float yh, float yl) {
    const float ph = __fmul_rn(xh, yh);
    const float pe = fmaf(xh, yh, -ph);
    const float pl = fmaf(xh, yl, fmaf(xl, yh, pe));
    const float s = __fadd_rn(sh, ph);
    const float bb = __fadd_rn(s, -sh);
    const float err = __fadd_rn(__fadd_rn(sh, -__fadd_rn(s, -bb)), __fadd_rn(ph, -bb));
    sh = s;
    sl = __fadd_rn(sl, __fadd_rn(err, pl));
}

__device__ __forceinline__ void df_norm(float& h, float& l) {
    const float s = __fadd_rn(h, l);
    l = __fadd_rn(l, -__fadd_rn(s, -h));
    h = s;
}

// (sh, sl) = x * y as an unnormalised double-float (TwoProd + cross terms).
__device__ __forceinline__ void df_mul(float& sh, float& sl, float xh, float xl, float yh, float yl) {
    sh = __fmul_rn(xh, yh);
    sl = fmaf(xh, yl, fmaf(xl, yh, fmaf(xh, yh, -sh)));
}

template <int K>
__device__ __forceinline__ void op_dense_df(DF4* sm, int m, const DevOp& op, const DF4* __restrict__ M) {
    constexpr int D = 1 << K;
    constexpr int G = K <= 3 ? 2 : 1;
    int pos[K], pm[K];
#pragma unroll
    for (int j = 0; j < K; j++) {
        pos[j] = op.pos[j];
        pm[j] = 1 << pos[j];
    }
    const int ng = 1 << (m - K);
    for (int g0 = threadIdx.x; g0 < ng; g0 += blockDim.x * G) {
        int base[G];
        bool ok[G];
        DF4 a[G][D];
#pragma unroll
        for (int q = 0; q < G; q++) {
            const int g = g0 + q * blockDim.x;
            ok[q] = g < ng;
            base[q] = swz<double>(insert_zero_bits<K>(ok[q] ? g : 0, pos));
#pragma unroll
            for (int b = 0; b < D; b++) a[q][b] = sm[base[q] ^ swz<double>(group_offset<K>(b, pm))];
        }
#pragma unroll(K <= 1 ? D : 1)
        for (int r = 0; r < D; r++) {
            const DF4* Mrow = M + r * D;
            float rh[G], rl[G], ih[G], il[G];
            {
                const DF4 u = Mrow[0];
#pragma unroll
                for (int q = 0; q < G; q++) {
                    df_mul(rh[q], rl[q], u.rh, u.rl, a[q][0].rh, a[q][0].rl);
                    df_mac(rh[q], rl[q], -u.ih, -u.il, a[q][0].ih, a[q][0].il);
                    df_mul(ih[q], il[q], u.rh, u.rl, a[q][0].ih, a[q][0].il);
                    df_mac(ih[q], il[q], u.ih, u.il, a[q][0].rh, a[q][0].rl);
                }
            }
#pragma unroll
            for (int c = 1; c < D; c++) {
                const DF4 u = Mrow[c];
#pragma unroll
                for (int q = 0; q < G; q++) {
                    df_mac(rh[q], rl[q], u.rh, u.rl, a[q][c].rh, a[q][c].rl);
                    df_mac(rh[q], rl[q], -u.ih, -u.il, a[q][c].ih, a[q][c].il);
                    df_mac(ih[q], il[q], u.rh, u.rl, a[q][c].ih, a[q][c].il);
                    df_mac(ih[q], il[q], u.ih, u.il, a[q][c].rh, a[q][c].rl);
                }
            }
            const int off = swz<double>(group_offset<K>(r, pm));
#pragma unroll
            for (int q = 0; q < G; q++) {
                df_norm(rh[q], rl[q]);
                df_norm(ih[q], il[q]);
                if (ok[q]) sm[base[q] ^ off] = DF4{rh[q], rl[q], ih[q], il[q]};
            }
        }
    }
}

__device__ __forceinline__ void op_diag_df(DF4* sm, int m, const DevOp& op, const DF4* __restrict__ M,
                                           uint64_t tile_base) {
    const DiagIndex d = diag_index<double>(op, tile_base);
    if (op.flags & OPF_SIGN_ONLY) {
        diag_sweep<2, 8, double>(sm, m, d, M, [](DF4 u, DF4 a) {
            return u.rh < 0.f ? DF4{-a.rh, -a.rl, -a.ih, -a.il} : a;
        });
    } else {
        diag_sweep<2, 8, double>(sm, m, d, M, [](DF4 u, DF4 a) {
            float rh, rl, ih, il;
            df_mul(rh, rl, u.rh, u.rl, a.rh, a.rl);
            df_mac(rh, rl, -u.ih, -u.il, a.ih, a.il);
            df_mul(ih, il, u.rh, u.rl, a.ih, a.il);
            df_mac(ih, il, u.ih, u.il, a.rh, a.rl);
            df_norm(rh, rl);
            df_norm(ih, il);
            return DF4{rh, rl, ih, il};
        });
    }
}

// ---------------------------------------------------------------------------
// K5-tc: complex128 block products on the tensor cores (exact digit split).
//
// In this mode a tile holds every amplitude component as a Q62 fixed-point
// int64 (x * 2^62; the components of a normalised state never exceed 1 in
// magnitude).  A k-qubit block (k = 3 or 4; smaller blocks are padded with
// identity qubits) y = U x is taken in real form (R = 2^(k+1) <= 32 rows and
// columns: real parts, then imaginary parts) and both operands are split into
// seven 8-bit digits, x = 2^6 sum_j X_j 2^(48 - 8j) (Q62 units; the top digit
// is signed with |X_0| <= 256, the others are bytes), likewise the matrix,
// whose digit fragments are prepared on the host.  Products of digits are
// exact in bfloat16 x bfloat16 -> float32 MMAs and the partial sums of each
// level L = i + j stay below 2^24 (at most 7 pairs x 32 terms x 2^16), so each
// level is accumulated exactly in float32.  Levels 0..6 are kept (28 digit
// pairs); y = sum_L Z_L 2^(46 - 8L) is re-assembled in int64 (the dropped
// levels contribute below 2^-50 in magnitude).
// ---------------------------------------------------------------------------
struct alignas(16) Q2 {
    long long re, im;
};
__device__ __forceinline__ Q2 rot_q(Q2 v, int c) { return rot_i(v, c); }  // exact: |re|, |im| < 2^63

// float64 -> fixed point with FB fraction bits (x * 2^FB truncated toward
// zero), for |x| < 2^(62 - FB) (components of a normalised state): the
// significand with its implicit bit is placed at bits 62..10 and shifted
// right by 1023 - exponent + 62 - FB; zero and subnormal inputs (shift
// clamped at 63) give 0.  Branch-free.
template <int FB = 62>
__device__ __forceinline__ long long d2q(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
    const int s = min(max(1023 + 62 - FB - (int)((hi >> 20) & 0x7FFu), 0), 63);
    const unsigned mh = (__funnelshift_l(lo, hi, 10) & 0x3FFFFFFFu) | 0x40000000u;
    const long long v = (long long)((((unsigned long long)mh << 32) | (unsigned long long)(lo << 10)) >> s);
    return (int)hi < 0 ? -v : v;
}

// Fixed point with FB fraction bits -> float64, truncated toward zero: |q|
// normalised by its leading-zero count, the 52 bits below the leading one
// form the fraction.
template <int FB = 62>
__device__ __forceinline__ double q2d(long long q) {
    const unsigned long long sign = (unsigned long long)q & 0x8000000000000000ull;
    const unsigned long long a = sign ? 0ull - (unsigned long long)q : (unsigned long long)q;
    const int lz = __clzll((long long)a);
    const unsigned long long n = a << (lz & 63);                      // leading one at bit 63 (a != 0)
    const unsigned long long E = (unsigned long long)(1086 - FB - lz);  // value = a * 2^-FB
    const unsigned long long bits = sign | (E << 52) | ((n >> 11) & ((1ull << 52) - 1));
    return __longlong_as_double(a ? (long long)bits : 0ll);
}

__device__ __forceinline__ void mma_bf16_16816(float (&c)[4], const uint4& a, unsigned b0, unsigned b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a.x), "r"(a.y), "r"(a.z), "r"(a.w), "r"(b0), "r"(b1));
}

// bfloat16 bits of byte k (0..3) of word w, as an exact integer in [0, 255]:
// 2^23 + b is assembled with one byte permute, then 2^23 is subtracted.
__device__ __forceinline__ unsigned bf16_byte_pair(unsigned w0, unsigned w1, unsigned sel) {
    const unsigned f0 = __byte_perm(w0, 0x4B000000u, sel);
    const unsigned f1 = __byte_perm(w1, 0x4B000000u, sel);
    const float g0 = __uint_as_float(f0) - 8388608.0f;
    const float g1 = __uint_as_float(f1) - 8388608.0f;
    return __byte_perm(__float_as_uint(g0), __float_as_uint(g1), 0x7632);  // high halves: bf16(g0) | bf16(g1) << 16
}

// Signed top digit d0 = v >> 48 of two values (|d0| <= 256), packed as bf16 x 2.
__device__ __forceinline__ unsigned bf16_top_pair(long long v0, long long v1) {
    const int d0 = (int)(v0 >> 48), d1 = (int)(v1 >> 48);
    const float g0 = __int_as_float(0x4B400000 + d0) - 12582912.0f;
    const float g1 = __int_as_float(0x4B400000 + d1) - 12582912.0f;
    return __byte_perm(__float_as_uint(g0), __float_as_uint(g1), 0x7632);
}

// Seven 8-bit digits of two Q62 values x0, x1 (v = x >> 6; digit 0 = v >> 48
// signed, digit j >= 1 = byte 6 - j of v), packed pairwise as bf16 x 2.
__device__ __forceinline__ void tc_digits_pair(long long x0, long long x1, unsigned (&out)[7]) {
    const long long v0 = x0 >> 6, v1 = x1 >> 6;
    const unsigned lo0 = (unsigned)v0, hi0 = (unsigned)((unsigned long long)v0 >> 32);
    const unsigned lo1 = (unsigned)v1, hi1 = (unsigned)((unsigned long long)v1 >> 32);
    out[0] = bf16_top_pair(v0, v1);
    out[1] = bf16_byte_pair(hi0, hi1, 0x7541);  // byte 5 of v = byte 1 of hi
    out[2] = bf16_byte_pair(hi0, hi1, 0x7540);  // byte 4 = byte 0 of hi
    out[3] = bf16_byte_pair(lo0, lo1, 0x7543);
    out[4] = bf16_byte_pair(lo0, lo1, 0x7542);
    out[5] = bf16_byte_pair(lo0, lo1, 0x7541);
    out[6] = bf16_byte_pair(lo0, lo1, 0x7540);
}

// Dense block of 3 or 4 qubits on the tensor cores (8-bit digits, levels 0..6).
// A fragments: Af[((i * MT + mt) * KT + ks) * 32 + lane] for digit i, m-tile mt,
// k-step ks.  Each warp takes n-tiles of 8 groups.  Real-form row / column k
// of a block is the real part of amplitude k (k < D) or the imaginary part of
// amplitude k - D.
template <int K>
__device__ __forceinline__ void op_dense_tc(Q2* sm, int m, const DevOp& op, const uint4* __restrict__ Af) {
    static_assert(K == 3 || K == 4, "tensor-core blocks have 3 or 4 qubits");
    constexpr int D = 1 << K, R = 2 * D, MT = R / 16, KT = R / 16;
    constexpr int ND = 7, NL = 7;
    int pos[K], pm[K];
#pragma unroll
    for (int j = 0; j < K; j++) {
        pos[j] = op.pos[j];
        pm[j] = 1 << pos[j];
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int g = lane >> 2, t = lane & 3;
    const int ng = 1 << (m - K), ntiles = ng >> 3;
    for (int nt = warp; nt < ntiles; nt += nwarps) {
        // B operand: this lane's column is group g of the n-tile; its rows in
        // k-step ks are ks*16 + {2t, 2t+1, 2t+8, 2t+9}.  Each amplitude it needs
        // is loaded once and both its real and imaginary digits are formed.
        const int bg = swz<double>(insert_zero_bits<K>(nt * 8 + g, pos));
        unsigned bf[KT][ND][2];
        if constexpr (K == 3) {
            // one k-step: rows 2t, 2t+1 = re of amplitudes 2t, 2t+1; rows 2t+8, 2t+9 = their im
            const Q2 a0 = sm[bg ^ swz<double>(group_offset<K>(2 * t, pm))];
            const Q2 a1 = sm[bg ^ swz<double>(group_offset<K>(2 * t + 1, pm))];
            unsigned dre[ND], dim_[ND];
            tc_digits_pair(a0.re, a1.re, dre);
            tc_digits_pair(a0.im, a1.im, dim_);
#pragma unroll
            for (int j = 0; j < ND; j++) {
                bf[0][j][0] = dre[j];
                bf[0][j][1] = dim_[j];
            }
        } else {
            // k-step 0: re of amplitudes {2t, 2t+1, 2t+8, 2t+9}; k-step 1: their im
            const Q2 a0 = sm[bg ^ swz<double>(group_offset<K>(2 * t, pm))];
            const Q2 a1 = sm[bg ^ swz<double>(group_offset<K>(2 * t + 1, pm))];
            const Q2 a2 = sm[bg ^ swz<double>(group_offset<K>(2 * t + 8, pm))];
            const Q2 a3 = sm[bg ^ swz<double>(group_offset<K>(2 * t + 9, pm))];
            unsigned d[ND];
            tc_digits_pair(a0.re, a1.re, d);
#pragma unroll
            for (int j = 0; j < ND; j++) bf[0][j][0] = d[j];
            tc_digits_pair(a2.re, a3.re, d);
#pragma unroll
            for (int j = 0; j < ND; j++) bf[0][j][1] = d[j];
            tc_digits_pair(a0.im, a1.im, d);
#pragma unroll
            for (int j = 0; j < ND; j++) bf[1][j][0] = d[j];
            tc_digits_pair(a2.im, a3.im, d);
#pragma unroll
            for (int j = 0; j < ND; j++) bf[1][j][1] = d[j];
        }
        // Every lane has built its B fragments before the first mma.sync (the
        // instruction is warp-wide), so each m-tile's outputs can be written as
        // soon as they are assembled.
        // A fragments are fetched one digit ahead so each load overlaps the
        // MMAs of the previous digit
        uint4 a_next = Af[lane];  // digit 0, m-tile 0, k-step 0
#pragma unroll 1
        for (int mt = 0; mt < MT; mt++) {
            float acc[NL][4];
#pragma unroll
            for (int L = 0; L < NL; L++) acc[L][0] = acc[L][1] = acc[L][2] = acc[L][3] = 0.f;
#pragma unroll
            for (int ks = 0; ks < KT; ks++) {
#pragma unroll
                for (int i = 0; i < ND; i++) {
                    const uint4 a = a_next;
                    // next (digit, k-step) of this m-tile, else digit 0 of the next m-tile
                    const int ni = i + 1 < ND ? i + 1 : 0;
                    const int nks = i + 1 < ND ? ks : ks + 1;
                    const int nmt = (i + 1 < ND || ks + 1 < KT) ? mt : mt + 1;
                    if (nmt < MT) a_next = Af[((ni * MT + nmt) * KT + (nks < KT ? nks : 0)) * 32 + lane];
#pragma unroll
                    for (int j = 0; j < ND; j++)
                        if (i + j < NL) mma_bf16_16816(acc[i + j], a, bf[ks][j][0], bf[ks][j][1]);
                }
            }
            __syncwarp();
#pragma unroll
            for (int e = 0; e < 4; e++) {
                // y = sum_L Z_L 2^(46 - 8L) in Q62 units = 2^6 (P01 2^32 + P23 2^16 +
                // P45) + Z_6 / 4 with P_ab = 256 Z_a + Z_b formed as 64-bit products
                // (|Z_L| <= (L+1) 2^21); two's-complement wrap of the sums is harmless
                long long z[NL];
#pragma unroll
                for (int L = 0; L < NL; L++) z[L] = __float2int_rn(acc[L][e]);
                const unsigned long long p01 = (unsigned long long)(z[0] * 256 + z[1]);
                const unsigned long long p23 = (unsigned long long)(z[2] * 256 + z[3]);
                const unsigned long long p45 = (unsigned long long)(z[4] * 256 + z[5]);
                unsigned long long v = (p01 << 32) + (p23 << 16) + p45;
                v = (v << 6) + (unsigned long long)((z[6] + 2) >> 2);
                const int row = mt * 16 + g + ((e >> 1) << 3);
                const int col = 2 * t + (e & 1);
                const int b = row & (D - 1);
                const int cg = swz<double>(insert_zero_bits<K>(nt * 8 + col, pos));
                Q2* dst = &sm[cg ^ swz<double>(group_offset<K>(b, pm))];
                if (row >> K) dst->im = (long long)v;
                else dst->re = (long long)v;
            }
        }
        __syncwarp();
    }
}

// (a * b) >> 62, floor: Q62 x Q62 -> Q62, or a Q62 phase times a Q56
// amplitude -> Q56
__device__ __forceinline__ long long qmul(long long a, long long b) {
    const long long hi = __mul64hi(a, b);
    const unsigned long long lo = (unsigned long long)(a * b);
    return (long long)(((unsigned long long)hi << 2) | (lo >> 62));
}

template <int LT = 8>  // log2 of the CTA size
__device__ __forceinline__ void op_diag_tc(Q2* sm, int m, const DevOp& op, const Q2* __restrict__ M,
                                           uint64_t tile_base) {
    const DiagIndex d = diag_index<double, LT>(op, tile_base);
    // one amplitude a thread at a time: two push the tcgen05 kernel past its 128 registers
    if (op.flags & OPF_SIGN_ONLY)
        diag_sweep<1, LT, double>(sm, m, d, M, [](Q2 u, Q2 a) { return u.re < 0 ? Q2{-a.re, -a.im} : a; });
    else
        diag_sweep<1, LT, double>(sm, m, d, M, [](Q2 u, Q2 a) {
            // three products instead of four (Gauss): k1 = c (x + y), k2 = x (d - c),
            // k3 = y (c + d) for u = c + i d, a = x + i y; re = k1 - k3, im = k1 + k2,
            // each off by less than two units after the floors, as the four-product
            // form is.  |x + y| <= sqrt(2) |a| and |d -/+ c| <= sqrt(2) 2^62 stay in range.
            const long long k1 = qmul(u.re, a.re + a.im);
            return Q2{k1 - qmul(a.im, u.re + u.im), k1 + qmul(a.re, u.im - u.re)};
        });
}

// ---------------------------------------------------------------------------
// K5-t05: the same digit products on the fifth-generation tensor cores
// (tcgen05.mma issued by one thread; amplitude digits and accumulators in
// tensor memory, block digits in shared memory).
//
// Here the tile holds Q56 (v = x * 2^56, the Q62 value >> 6: the digit
// split never used the low 6 bits) and digits are balanced:
// v = sum_j X_j 256^(6 - j) with
// |X_0| <= 256 and X_j in [-128, 127] for j >= 1 (bytes 0..5 of
// u = v + 2^56 + 0x808080808080, minus 128; its top 16 bits are X_0 + 256, in
// 0..512), and held as float16, exact for integers below 2^11: byte permutes
// place two such values b in the mantissas of 1024 + b, one packed half
// subtraction removes 1024 + 128 (1024 + 256 for X_0).  For a unitary block
// every level sum then stays below 2^21.5 (the host checks the bound 2^22 per
// block), so it is exact in float32, and with the accumulator started at
// 1.5 * 2^23 (below) its bits are 0x4B400000 + z: the level reads as an
// integer.  The digit work is bound by the SM's integer pipe, so the
// re-assembly keeps to multiply-adds.
//
// One round covers 128 groups (one M = 128 tile; 3-qubit blocks take two
// M-tiles per round):
//   A_i (tensor memory, 128 lanes x R/2 columns) = digit i of the groups'
//       R = 2^(k+1) real components, a column holding two fp16 K-elements;
//   B   (shared, 7R x R fp16, K-major core matrices of 8 rows x 16 bytes, no
//       swizzle): row j R + r' = digit j of real-form row r of the block
//       (r' = (amp >> 2) 8 + part 4 + (amp & 3) for output component part
//       (0 = re, 1 = im) of amplitude amp, so that one thread reads the re
//       and im outputs of 4 amplitudes from 8 adjacent columns);
//   D   (tensor memory, 128 lanes x 7R fp32 columns): column L R + r' =
//       level L of output r'.
// Amplitude digit i meets block digits j = 0..6-i in one MMA of
// N = (7 - i) R whose accumulator starts at column i R, so each level i + j
// collects in its own columns: 7 x R/16 MMAs per M-tile and round.  Two A
// buffers in tensor memory (one CTA per SM holds all 512 columns) let the
// threads split round r + 1 while the MMAs of round r run; the CTA has 512
// threads (16 warps) to hide the latency of the digit work.
// ---------------------------------------------------------------------------
namespace t05 {

constexpr int kThreads = 512;              // split / re-assembly threads: 16 warps, 4 per TMEM lane quarter
constexpr int kLogThreads = 9;
constexpr int kCtaThreads = kThreads + 32; // complex64 mode: plus one warp that only issues the MMAs
constexpr int kIssuer = kThreads;          // its first thread
constexpr int kBBytes = 14 * 32 * 32;      // 7R x R fp16 for R = 32
constexpr int kSmemBase = kBBytes;  // block digits; the amplitude tile follows (A lives in tensor memory)
constexpr int kSmemMin = 116 * 1024;       // one CTA per SM (it holds all 512 TMEM columns)
constexpr int kTmemCols = 512;             // the whole of an SM's tensor memory
constexpr unsigned kMagicBits = 0x4B400000u;  // bits of 1.5 * 2^23
// The accumulator starts every round at 1.5 * 2^23 = 3072 * 4096: one MMA of
// a constant A slice (TMEM columns kAConst.., K-element 0 = fp16 3072, the
// rest 0; free columns beside both A buffers) by a constant B slice (shared
// memory, K-row 0 = fp16 4096), so every level sum z lands as the float
// 1.5 * 2^23 + z, whose bits are 0x4B400000 + z: the level is read as an
// integer without a float add.  The host's per-block bound |z| <= 2^22
// holds for every partial sum too (it bounds the sum of the products'
// magnitudes), so each partial sum stays an integer in [2^23, 2^24].
constexpr uint32_t kAConst = 368;
constexpr unsigned kHalf3072 = 0x6A00u, kHalf4096 = 0x6C00u;
constexpr int kBiasRows = 7 * 32;  // N of the widest accumulator (7 R, R = 32)
constexpr unsigned long long kWaitNs = 1000000000ull;  // a bounded wait gives up after one second
constexpr unsigned kWaitPolls = 1u << 26;                 // and after this many polls in any case
constexpr unsigned kSuspendNs = 20000;                    // longest sleep of one poll

__device__ int g_fault;  // set when a bounded wait ran out (read and cleared by the host)

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor (K-major, no swizzle): start address, byte
// step between core matrices along K (lbo) and along M / N (sbo), version 1.
__device__ __forceinline__ uint64_t desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: f32 accumulator, f16 A and B, both
// K-major, M = 128, N = n.
__device__ __forceinline__ uint32_t idesc(int n) {
    return (1u << 4) | ((uint32_t)(n >> 3) << 17) | ((128u >> 4) << 24);
}

__device__ __forceinline__ void mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t id, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(id), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(mbar)
                 : "memory");
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t));
    return t;
}

// Waits for the phase of the given parity to complete; false after kWaitNs
// nanoseconds (or kWaitPolls polls), so the caller reports SV_ERR_TIMEOUT
// instead of hanging.
__device__ __forceinline__ bool wait(uint32_t mbar, uint32_t parity) {
    const unsigned long long t0 = global_ns();
    for (unsigned it = 0; it < kWaitPolls; it++) {
        uint32_t done;
        // the thread sleeps until the phase completes or kSuspendNs pass
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(mbar), "r"(parity), "n"(kSuspendNs)
            : "memory");
        if (done) return true;
        if ((it & 15) == 15 && global_ns() - t0 > kWaitNs) return false;
    }
    return false;
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

// 8 consecutive fp32 columns of this warp's 32 TMEM lanes
__device__ __forceinline__ void ld8(uint32_t taddr, uint32_t (&r)[8]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr)
                 : "memory");
}
__device__ __forceinline__ void ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory"); }

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

__device__ __forceinline__ unsigned sub_h2(unsigned a, unsigned b) {
    unsigned d;
    asm("sub.rn.f16x2 %0, %1, %2;\n" : "=r"(d) : "r"(a), "r"(b));
    return d;
}

__device__ __forceinline__ unsigned long long mad_wide(unsigned a, unsigned b, unsigned long long c) {
    unsigned long long d;
    asm("mad.wide.u32 %0, %1, %2, %3;\n" : "=l"(d) : "r"(a), "r"(b), "l"(c));
    return d;
}

// u = x + 2^56 + 0x808080808080 (mod 2^64) as one wide multiply-add.
__device__ __forceinline__ unsigned long long digit_bias(long long x) {
    const unsigned lo = (unsigned)x, hi = (unsigned)((unsigned long long)x >> 32);
    return mad_wide(lo, 1u, ((unsigned long long)(hi + 0x01008080u) << 32) | 0x80808080u);
}

// Two bytes b, b' (bytes 2k and 2k + 1 of m) as fp16 1024 + b, 1024 + b':
// the exponent bytes come from the constant.
template <int K>
__device__ __forceinline__ unsigned h2_pair(unsigned m) {
    return __byte_perm(m, 0x64646464u, K == 0 ? 0x4140 : 0x4342);
}

// The seven balanced digits of two Q56 values, packed pairwise as fp16 x 2.
__device__ __forceinline__ void bal_digits_pair(long long x0, long long x1, unsigned (&o)[7]) {
    const unsigned long long u0 = digit_bias(x0), u1 = digit_bias(x1);
    const unsigned lo0 = (unsigned)u0, hi0 = (unsigned)(u0 >> 32);
    const unsigned lo1 = (unsigned)u1, hi1 = (unsigned)(u1 >> 32);
    // top digit plus 256 (0..512): the top 16 bits of u, under the exponent of 1024
    o[0] = sub_h2(__byte_perm(hi0, hi1, 0x7632) | 0x64006400u, 0x65006500u);
    // bytes of the two values interleaved, then one permute per digit
    const unsigned mh = __byte_perm(hi0, hi1, 0x5140);  // bytes 4, 5
    const unsigned m1 = __byte_perm(lo0, lo1, 0x7362);  // bytes 2, 3
    const unsigned m0 = __byte_perm(lo0, lo1, 0x5140);  // bytes 0, 1
    o[1] = sub_h2(h2_pair<1>(mh), 0x64806480u);  // byte 5 of u
    o[2] = sub_h2(h2_pair<0>(mh), 0x64806480u);  // byte 4
    o[3] = sub_h2(h2_pair<1>(m1), 0x64806480u);
    o[4] = sub_h2(h2_pair<0>(m1), 0x64806480u);
    o[5] = sub_h2(h2_pair<1>(m0), 0x64806480u);
    o[6] = sub_h2(h2_pair<0>(m0), 0x64806480u);
}

// Level pair (2q, 2q + 1) of one output: 256 z_2q + z_2q+1 + 0x8B400000 from
// the accumulator bits w = 0x4B400000 + z (257 * 0x4B400000 = 0x8B400000
// mod 2^32); for |z| <= 2^22 the sum lies in [0, 2^32), so it needs no
// further offset before it is widened.
__device__ __forceinline__ unsigned level_pair(uint32_t w0, uint32_t w1) {
    unsigned d;
    asm("mad.lo.u32 %0, %1, 256, %2;\n" : "=r"(d) : "r"(w0), "r"(w1));
    return d;
}

// Level 6 of one output rounded to the output's unit: 0x4B400000 +
// floor((z + 128) / 256) from the accumulator 1.5 * 2^23 + z: one exact add
// (z + 128) and one multiply-add rounded down.
__device__ __forceinline__ unsigned level6(uint32_t a) {
    return __float_as_uint(__fmaf_rd(__uint_as_float(a) + (128.0f - 12582912.0f), 0.00390625f, 12582912.0f));
}

// 2^64 minus the offsets the three pairs (0x8B400000 each, at 2^32, 2^16 and
// 1) and level 6 (0x4B400000) carry.
constexpr unsigned kPairOffset = 257u * kMagicBits;  // 0x8B400000 (mod 2^32)
constexpr unsigned long long kLevelBias =
    0ull - (unsigned long long)kPairOffset * ((1ull << 32) + (1ull << 16) + 1ull) - kMagicBits;
static_assert(kPairOffset == 0x8B400000u && kLevelBias == 0x74BF74BF29800000ull, "level offsets");

// Per-op address table of a pass (ints, built once per CTA and pass): every
// tile of the pass applies the same ops, so the swizzled offsets a thread
// needs depend only on the op's qubit positions.  insert_zero_bits and swz
// are linear over XOR, so the base of group g splits into its lane bits
// (kTabLane + (g & 31)), its higher bits (kTabHi + (g >> 5)) and the round
// (kTabS + b for bit b of the round index).
constexpr int kTabOff = 0;    // [b] = swz(group_offset(b)), b < 2^k
constexpr int kTabS = 32;     // [b] = swz(insert_zero_bits(groups_per_round << b))
constexpr int kTabLane = 36;  // [l] = swz(insert_zero_bits(l)), l < 32
constexpr int kTabHi = 68;    // [h] = swz(insert_zero_bits(h << 5)), h < 8
constexpr int kTabInts = 80;

template <typename SwzT>
__device__ __forceinline__ int op_table_entry(const DevOp& op, int kt, int gpr, int t) {
    if (op.kind != OP_DENSE) return 0;
    int pos[5];
#pragma unroll
    for (int j = 0; j < 5; j++) pos[j] = j < kt ? op.pos[j] : 0;
    auto ins = [&](int g) {
#pragma unroll
        for (int j = 0; j < 5; j++)
            if (j < kt) g = ((g >> pos[j]) << (pos[j] + 1)) | (g & ((1 << pos[j]) - 1));
        return g;
    };
    if (t < kTabS) {
        int off = 0;
#pragma unroll
        for (int j = 0; j < 5; j++)
            if (j < kt && ((t >> j) & 1)) off |= 1 << pos[j];
        return swz<SwzT>(off);
    }
    if (t < kTabLane) return swz<SwzT>(ins(gpr << (t - kTabS)));
    if (t < kTabHi) return swz<SwzT>(ins(t - kTabLane));
    return swz<SwzT>(ins((t - kTabHi) << 5));
}

struct Ctx {
    unsigned char* b;  // block digits / parts in shared memory
    uint32_t b_addr, mbar, tmem;
    uint32_t bias_addr;  // complex128 digits: the constant B slice of the accumulator preload
    uint32_t phase;
    bool failed;
};

// Dense block of 3 or 4 qubits on tcgen05 (balanced 8-bit digits, levels 0..6),
// amplitude digits (the A operand) in tensor memory.
//
// TMEM (512 columns): accumulator at columns [0, 256) (7R columns per M-tile,
// M-tile mt at 128 mt), two A buffers at [256, 384) and [384, 512): digit
// plane i of M-tile mt at (mt 7 + i) R/2, column c holding the K-elements
// 2c (low half) and 2c + 1 of the lane's row.  K order: k' = 8 cg + 4 part + e
// for component part of amplitude 4 cg + e (the host writes B in the same
// order), so one thread stores its 4 amplitudes' digits as 4 adjacent
// columns and later reads their outputs from 8 adjacent accumulator columns.
// While the MMAs of round r run, the threads split round r + 1 into the other
// A buffer; the (single) accumulator is re-assembled after the MMAs finish.
template <int K>
__device__ __forceinline__ void op_dense(Q2* sm, int m, const DevOp& op, const uint4* __restrict__ Bg, Ctx& cx,
                                         const int* tab) {
    static_assert(K == 3 || K == 4, "tensor-core blocks have 3 or 4 qubits");
    constexpr int D = 1 << K, R = 2 * D;
    constexpr int SBO = 16 * R;              // B: bytes between 8-row core groups
    constexpr int GPR = K == 3 ? 256 : 128;  // groups per round
    constexpr uint32_t kABuf = 256;          // TMEM column of A buffer 0 (buffer 1 at +128)
    int pos[K], pm[K];
#pragma unroll
    for (int j = 0; j < K; j++) {
        pos[j] = op.pos[j];
        pm[j] = 1 << pos[j];
    }
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (int i = tid; i < 14 * R * R / 16; i += kThreads) cp_async16(cx.b_addr + 16 * i, Bg + i);
    const int ng = 1 << (m - K);
    // thread -> (TMEM lane quarter = row, M-tile, 4 amplitudes cg), for both the split and the re-assembly
    const int cg = K == 4 ? warp >> 2 : (warp >> 2) & 1;
    const int mt_t = K == 4 ? 0 : warp >> 3;
    const int row = (warp & 3) * 32 + lane;
    const uint32_t lane_bits = (uint32_t)((warp & 3) * 32) << 16;
    int off[4];
    const int loc = mt_t * 128 + row;
    int loc_sw;
    // insert_zero_bits and swz are linear over XOR and round g0 = r GPR has
    // no bit in common with loc, so the round's base is loc_sw XOR the
    // offsets S[b] of the set bits b of r (at most 4 rounds per tile here)
    int S[3];
    if (tab) {  // the pass's table (shared memory)
        const int4 o4 = *reinterpret_cast<const int4*>(tab + kTabOff + 4 * cg);
        off[0] = o4.x;
        off[1] = o4.y;
        off[2] = o4.z;
        off[3] = o4.w;
        loc_sw = tab[kTabLane + (loc & 31)] ^ tab[kTabHi + (loc >> 5)];
#pragma unroll
        for (int b = 0; b < 3; b++) S[b] = tab[kTabS + b];
    } else {
#pragma unroll
        for (int e = 0; e < 4; e++) off[e] = swz<double>(group_offset<K>(4 * cg + e, pm));
        loc_sw = swz<double>(insert_zero_bits<K>(loc, pos));
#pragma unroll
        for (int b = 0; b < 3; b++) S[b] = swz<double>(insert_zero_bits<K>(GPR << b, pos));
    }
    auto base_of = [&](int g0) {
        const int r = g0 / GPR;
        return loc_sw ^ ((r & 1) ? S[0] : 0) ^ ((r & 2) ? S[1] : 0) ^ ((r & 4) ? S[2] : 0);
    };
    auto n_mt_of = [&](int g0) { return (K == 3 && g0 + 128 < ng) ? 2 : 1; };
    // digits of the thread's 4 amplitudes of the round at g0 into A buffer ab
    auto split = [&](int g0, int ab) {
        if (mt_t >= n_mt_of(g0)) return;  // warp-uniform
        unsigned d[4][7];
        if (g0 + loc < ng) {
            const int bg = base_of(g0);
            Q2 v[4];
#pragma unroll
            for (int e = 0; e < 4; e++) v[e] = sm[bg ^ off[e]];
            bal_digits_pair(v[0].re, v[1].re, d[0]);
            bal_digits_pair(v[2].re, v[3].re, d[1]);
            bal_digits_pair(v[0].im, v[1].im, d[2]);
            bal_digits_pair(v[2].im, v[3].im, d[3]);
        } else {
#pragma unroll
            for (int i = 0; i < 7; i++) d[0][i] = d[1][i] = d[2][i] = d[3][i] = 0u;
        }
        const uint32_t a0 = cx.tmem + lane_bits + kABuf + (uint32_t)ab * 128 + (uint32_t)(mt_t * 7) * (R / 2) + 4 * cg;
#pragma unroll
        for (int i = 0; i < 7; i++)
            asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1,%2,%3,%4};\n" ::"r"(a0 + i * (R / 2)),
                         "r"(d[0][i]), "r"(d[1][i]), "r"(d[2][i]), "r"(d[3][i])
                         : "memory");
    };
    auto reassemble = [&](int r0) {
        fence_after();
        if (mt_t >= n_mt_of(r0)) return;  // warp-uniform
        const uint32_t t0 = cx.tmem + lane_bits + mt_t * 128 + 8 * cg;
        // out = P0 2^32 + P1 2^16 + P2 + level 6 (mod 2^64), the offsets removed by one constant
        unsigned long long y[8];
        uint32_t z[4][8];
        ld8(t0, z[0]);
        ld8(t0 + R, z[1]);
        ld8(t0 + 2 * R, z[2]);
        ld8(t0 + 3 * R, z[3]);
        ld_wait();
#pragma unroll
        for (int e = 0; e < 8; e++) {
            y[e] = ((unsigned long long)(level_pair(z[0][e], z[1][e]) + (unsigned)(kLevelBias >> 32)) << 32) |
                   (unsigned)kLevelBias;
            y[e] = mad_wide(level_pair(z[2][e], z[3][e]), 65536u, y[e]);
        }
        ld8(t0 + 4 * R, z[0]);
        ld8(t0 + 5 * R, z[1]);
        ld8(t0 + 6 * R, z[2]);
        ld_wait();
#pragma unroll
        for (int e = 0; e < 8; e++) {
            y[e] = mad_wide(level_pair(z[0][e], z[1][e]), 1u, y[e]);
            y[e] = mad_wide(level6(z[2][e]), 1u, y[e]);
        }
        if (r0 + loc < ng) {
            const int bg = base_of(r0);
#pragma unroll
            for (int e = 0; e < 4; e++) sm[bg ^ off[e]] = Q2{(long long)y[e], (long long)y[e + 4]};
        }
    };
    auto issue = [&](int g0, int ab) {
        // (OPF_TEST_NO_MMA, a test hook: nothing is issued, so the bounded wait runs out)
        if (tid != 0 || (op.flags & OPF_TEST_NO_MMA)) return;
        fence_after();
        const int n_mt = n_mt_of(g0);
        for (int mt = 0; mt < n_mt; mt++) {
            // accumulator <- 1.5 * 2^23 in all 7R columns, then every digit MMA accumulates
            asm volatile(
                "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}\n" ::"r"(cx.tmem + mt * 128),
                "r"(cx.tmem + kAConst), "l"(desc(cx.bias_addr, 128, 256)), "r"(idesc(7 * R)), "r"(0u)
                : "memory");
#pragma unroll
            for (int i = 0; i < 7; i++)
#pragma unroll
                for (int ks = 0; ks < R / 16; ks++) {
                    const uint32_t ta = cx.tmem + kABuf + (uint32_t)ab * 128 + (uint32_t)(mt * 7 + i) * (R / 2) + ks * 8;
                    const uint64_t db = desc(cx.b_addr + ks * 256, 128, SBO);
                    asm volatile(
                        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}\n" ::"r"(
                            cx.tmem + mt * 128 + i * R),
                        "r"(ta), "l"(db), "r"(idesc((7 - i) * R)), "r"(1u)
                        : "memory");
                }
        }
        commit(cx.mbar);
    };
    split(0, 0);
    asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory");
    cp_async_wait_all();  // the block digits
    fence_async_smem();
    fence_before();
    __syncthreads();
    issue(0, 0);
    int g0 = 0, ab = 0;
    for (;; g0 += GPR, ab ^= 1) {
        const int gn = g0 + GPR;
        if (gn < ng) split(gn, ab ^ 1);  // overlaps the MMAs of round g0
        const bool ok = wait(cx.mbar, cx.phase);
        cx.phase ^= 1;
        if (ok) reassemble(g0);
        asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory");
        fence_before();
        if (__syncthreads_or(!ok)) {
            if (tid == 0) atomicExch(&g_fault, 1);
            wait(cx.mbar, cx.phase ^ 1);  // give the MMAs in flight one more bounded wait
            cx.failed = true;
            return;
        }
        if (gn >= ng) break;
        issue(gn, ab ^ 1);
    }
}

}  // namespace t05

// ---------------------------------------------------------------------------
// K5-t32: complex64 block products on tcgen05 (bfloat16 triple split).
//
// Each float32 component x of the tile is split into three bfloat16 parts,
// x = h + m + l with h = bf16(x), m = bf16(x - h), l = bf16(x - h - m) (each
// residual is exact in float32; |x - h - m - l| <= 2^-24 |x|); the block's
// real form likewise, from its float64 entries.  The six products of parts
// (i, j) with i + j <= 2 carry float32 accuracy (the dropped ones are below
// 2^-24 relative): amplitude part i meets block parts 0..2-i in one MMA of
// N = (3 - i) R into TMEM columns [i R, 3R), so level L = i + j collects in
// columns [L R, (L+1) R) with float32 accumulation; the output is
// (Z_2 + Z_1) + Z_0.  No exact re-assembly is needed: complex64 only asks
// for float32 rounding.
//
// One round covers 128 groups (one M = 128 tile) for blocks of 3..5 qubits
// (smaller blocks are padded to 3): A_i (tensor memory, 128 lanes x R/2
// columns, two bf16 K-elements per column) = part i of the groups' real
// components, B (shared, 3R x R bf16, K-major core matrices of 8 rows x 16
// bytes: row j R + r' = part j of real-form row r, r' = (amp / P) 2P +
// part P + (amp mod P) with P = D / 4 amplitudes per thread, columns in the
// K order of A), D (tensor memory, 3R columns).  Two A buffers let the
// threads split round r + 1 while the MMAs of round r run, as in the
// complex128 mode.
// ---------------------------------------------------------------------------
namespace t32 {

constexpr int kBBytes = 6 * 64 * 64;  // 3R x R bf16 for R = 64
constexpr int kSmemBase = kBBytes;    // block parts; the amplitude tile follows (A lives in tensor memory)

__device__ __forceinline__ uint32_t idesc(int n) {  // kind::f16, f32 accumulator, bf16 A and B, M = 128
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((128u >> 4) << 24);
}

__device__ __forceinline__ unsigned bf16x2_rn(float lo, float hi) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const unsigned*>(&v);
}

// Three bfloat16 parts of two float32 values, packed pairwise (x0 low half).
__device__ __forceinline__ void bf3_pair(float x0, float x1, unsigned& h, unsigned& m, unsigned& l) {
    h = bf16x2_rn(x0, x1);
    const float r0 = x0 - __uint_as_float(h << 16), r1 = x1 - __uint_as_float(h & 0xFFFF0000u);
    m = bf16x2_rn(r0, r1);
    l = bf16x2_rn(r0 - __uint_as_float(m << 16), r1 - __uint_as_float(m & 0xFFFF0000u));
}

template <int N>
__device__ __forceinline__ void ldN(uint32_t taddr, uint32_t (&r)[N]);
template <>
__device__ __forceinline__ void ldN<4>(uint32_t taddr, uint32_t (&r)[4]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(taddr)
                 : "memory");
}
template <>
__device__ __forceinline__ void ldN<8>(uint32_t taddr, uint32_t (&r)[8]) {
    t05::ld8(taddr, r);
}
template <>
__device__ __forceinline__ void ldN<16>(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
}

// Dense block of 3..5 qubits on tcgen05 (bfloat16 triple split), the
// amplitude parts (A operand) in tensor memory: accumulator in columns
// [0, 3R), two A buffers at 256 and 384 (part plane i at i R/2, a column
// holding two bf16 K-elements); K order k' = 2P (amp / P) + P part +
// (amp mod P), so a thread's P amplitudes fill P adjacent columns per part.
// While the MMAs of round r run, the threads split round r + 1 into the other
// A buffer; the accumulator is re-assembled after the MMAs finish.
template <int K>
__device__ __forceinline__ void op_dense(Cx<float>* sm, int m, const DevOp& op, const uint4* __restrict__ Bg,
                                         t05::Ctx& cx, const int* tab) {
    static_assert(K >= 3 && K <= 5, "tensor-core blocks have 3 to 5 qubits");
    using namespace t05;
    constexpr int D = 1 << K, R = 2 * D;
    constexpr int SBO = 16 * R;  // B: bytes between 8-row core groups
    constexpr int P = D / 4;     // amplitudes per thread
    constexpr uint32_t kABuf = 256;
    int pos[K], pm[K];
#pragma unroll
    for (int j = 0; j < K; j++) {
        pos[j] = op.pos[j];
        pm[j] = 1 << pos[j];
    }
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool worker = tid < kThreads;  // warp-uniform; the last warp only issues the MMAs
    for (int i = tid; i < 6 * R * R / 16; i += kCtaThreads) cp_async16(cx.b_addr + 16 * i, Bg + i);
    const int ng = 1 << (m - K);
    const int cg = (warp & 15) >> 2;
    const int row = (warp & 3) * 32 + lane;
    const uint32_t lane_bits = (uint32_t)((warp & 3) * 32) << 16;
    int off[P];
    int row_sw;
    // round bases from per-op offsets, as in the complex128 digit op (rounds of
    // 128 groups, at most 16 per tile)
    int S[4];
    if (tab) {  // the pass's table (shared memory)
#pragma unroll
        for (int e = 0; e < P; e++) off[e] = tab[kTabOff + P * cg + e];
        row_sw = tab[kTabLane + lane] ^ tab[kTabHi + (warp & 3)];
#pragma unroll
        for (int b = 0; b < 4; b++) S[b] = tab[kTabS + b];
    } else {
#pragma unroll
        for (int e = 0; e < P; e++) off[e] = swz<float>(group_offset<K>(P * cg + e, pm));
        row_sw = swz<float>(insert_zero_bits<K>(row, pos));
#pragma unroll
        for (int b = 0; b < 4; b++) S[b] = swz<float>(insert_zero_bits<K>(128 << b, pos));
    }
    auto base_of = [&](int g0) {
        const int r = g0 >> 7;
        return row_sw ^ ((r & 1) ? S[0] : 0) ^ ((r & 2) ? S[1] : 0) ^ ((r & 4) ? S[2] : 0) ^ ((r & 8) ? S[3] : 0);
    };
    auto split = [&](int g0, int ab) {
        if (!worker) return;
        unsigned h[2][P / 2], mm[2][P / 2], l[2][P / 2];
        if (g0 + row < ng) {
            const int bg = base_of(g0);
            Cx<float> v[P];
#pragma unroll
            for (int e = 0; e < P; e++) v[e] = sm[bg ^ off[e]];
#pragma unroll
            for (int e = 0; e < P / 2; e++) {
                bf3_pair(v[2 * e].re, v[2 * e + 1].re, h[0][e], mm[0][e], l[0][e]);
                bf3_pair(v[2 * e].im, v[2 * e + 1].im, h[1][e], mm[1][e], l[1][e]);
            }
        } else {
#pragma unroll
            for (int e = 0; e < P / 2; e++) h[0][e] = h[1][e] = mm[0][e] = mm[1][e] = l[0][e] = l[1][e] = 0u;
        }
        const uint32_t a0 = cx.tmem + lane_bits + kABuf + (uint32_t)ab * 128 + P * cg;
        auto st = [&](uint32_t ta, const unsigned (&re)[P / 2], const unsigned (&im)[P / 2]) {
            if constexpr (P == 8)
                asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};\n" ::"r"(ta),
                             "r"(re[0]), "r"(re[1]), "r"(re[2]), "r"(re[3]), "r"(im[0]), "r"(im[1]), "r"(im[2]),
                             "r"(im[3])
                             : "memory");
            else if constexpr (P == 4)
                asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1,%2,%3,%4};\n" ::"r"(ta), "r"(re[0]),
                             "r"(re[1]), "r"(im[0]), "r"(im[1])
                             : "memory");
            else
                asm volatile("tcgen05.st.sync.aligned.32x32b.x2.b32 [%0], {%1,%2};\n" ::"r"(ta), "r"(re[0]), "r"(im[0])
                             : "memory");
        };
        st(a0, h[0], h[1]);
        st(a0 + R / 2, mm[0], mm[1]);
        st(a0 + R, l[0], l[1]);
    };
    auto reassemble = [&](int r0) {
        fence_after();
        if (!worker) return;
        const uint32_t t0 = cx.tmem + lane_bits + 2 * P * cg;
        uint32_t z0[2 * P], z1[2 * P], z2[2 * P];
        ldN<2 * P>(t0, z0);
        ldN<2 * P>(t0 + R, z1);
        ldN<2 * P>(t0 + 2 * R, z2);
        ld_wait();
        if (r0 + row < ng) {
            const int bg = base_of(r0);
            auto y = [&](int c) {
                return (__uint_as_float(z2[c]) + __uint_as_float(z1[c])) + __uint_as_float(z0[c]);
            };
#pragma unroll
            for (int e = 0; e < P; e++) sm[bg ^ off[e]] = Cx<float>{y(e), y(P + e)};
        }
    };
    auto issue = [&](int ab) {
        if (tid != kIssuer || (op.flags & OPF_TEST_NO_MMA)) return;
        fence_after();
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int ks = 0; ks < R / 16; ks++) {
                const uint32_t ta = cx.tmem + kABuf + (uint32_t)ab * 128 + i * (R / 2) + ks * 8;
                const uint64_t db = desc(cx.b_addr + ks * 256, 128, SBO);
                asm volatile(
                    "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}\n" ::"r"(cx.tmem + i * R),
                    "r"(ta), "l"(db), "r"(idesc((3 - i) * R)), "r"((uint32_t)((i | ks) != 0))
                    : "memory");
            }
        commit(cx.mbar);
    };
    split(0, 0);
    asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory");
    cp_async_wait_all();
    fence_async_smem();
    fence_before();
    __syncthreads();
    issue(0);
    int g0 = 0, ab = 0;
    for (;; g0 += 128, ab ^= 1) {
        const int gn = g0 + 128;
        if (gn < ng) split(gn, ab ^ 1);  // overlaps the MMAs of round g0
        const bool ok = worker ? wait(cx.mbar, cx.phase) : true;
        cx.phase ^= 1;
        if (ok) reassemble(g0);
        asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory");
        fence_before();
        if (__syncthreads_or(!ok)) {
            if (tid == 0) atomicExch(&g_fault, 1);
            wait(cx.mbar, cx.phase ^ 1);  // give the MMAs in flight one more bounded wait
            cx.failed = true;
            return;
        }
        if (gn >= ng) break;
        issue(ab ^ 1);
    }
}

}  // namespace t32

// ---------------------------------------------------------------------------
// K5: the tile-pass kernel, shared by the arithmetic modes.
// ---------------------------------------------------------------------------
enum TileMode { MODE_F32 = 0, MODE_F64 = 1, MODE_DF = 2, MODE_TC = 3, MODE_T05 = 4, MODE_T32 = 5 };
__host__ __device__ constexpr bool uses_tmem(int mode) { return mode == MODE_T05 || mode == MODE_T32; }
__host__ __device__ constexpr int tile_threads(int mode) {
    return mode == MODE_T32 ? t05::kCtaThreads : (mode == MODE_T05 ? t05::kThreads : kTileThreads);
}

template <int MODE>
struct TileTraits;
// Bytes of one diagonal entry in a mode's coefficient array: Q56 / Q62 pairs
// (tensor-core complex128), double-float quadruples, complex128 or complex64.
__host__ __device__ constexpr int diag_entry_bytes(int mode) { return mode == MODE_F32 || mode == MODE_T32 ? 8 : 16; }
template <>
struct TileTraits<MODE_F32> {
    using Store = Cx<float>;
    using Smem = Cx<float>;
    using Coef = Cx<float>;
    using SwzT = float;
};
template <>
struct TileTraits<MODE_F64> {
    using Store = Cx<double>;
    using Smem = Cx<double>;
    using Coef = Cx<double>;
    using SwzT = double;
};
template <>
struct TileTraits<MODE_DF> {
    using Store = Cx<double>;
    using Smem = DF4;
    using Coef = DF4;
    using SwzT = double;
};
template <>
struct TileTraits<MODE_TC> {
    using Store = Cx<double>;
    using Smem = Q2;
    using Coef = uint4;  // dense: MMA fragments; diagonal: Q2 entries
    using SwzT = double;
};
template <>
struct TileTraits<MODE_T05> {
    using Store = Cx<double>;
    using Smem = Q2;
    using Coef = uint4;  // dense: block digits in their shared-memory image; diagonal: Q2 entries
    using SwzT = double;
};
template <>
struct TileTraits<MODE_T32> {
    using Store = Cx<float>;
    using Smem = Cx<float>;
    using Coef = uint4;  // dense: block parts in their shared-memory image; diagonal: Cx<float> entries
    using SwzT = float;
};

// The move of a permutation op's row t, from its coefficient element.
__device__ __forceinline__ int perm_move(const Cx<float>* M, int t) { return (int)M[t].re; }
__device__ __forceinline__ int perm_move(const Cx<double>* M, int t) { return (int)M[t].re; }
__device__ __forceinline__ int perm_move(const DF4* M, int t) { return (int)M[t].rh; }
__device__ __forceinline__ int perm_move(const uint4* M, int t) { return (int)M[t].x; }
__device__ __forceinline__ Cx<float> perm_rot(Cx<float> v, int c) { return rot_cf(v, c); }
__device__ __forceinline__ Cx<double> perm_rot(Cx<double> v, int c) { return rot_cd(v, c); }
__device__ __forceinline__ DF4 perm_rot(DF4 v, int c) { return rot_df(v, c); }
__device__ __forceinline__ Q2 perm_rot(Q2 v, int c) { return rot_q(v, c); }

// Stages a permutation op's moves in shared memory (every thread of the CTA
// takes part: it holds two CTA barriers) and applies it.
template <typename S, typename SwzT, typename C>
__device__ __forceinline__ void apply_perm(S* sm, int m, const DevOp& op, const C* __restrict__ M) {
    __shared__ int s_mv[32], s_src[32];
    const int D = 1 << op.k, t = threadIdx.x;
    __syncthreads();  // the previous op's reads of the tables are done
    if (t < D) s_mv[t] = perm_move(M, t);
    __syncthreads();
    if (t < D) {  // row a_t takes its amplitude from the next row of its cycle
        const int v = s_mv[t];
        int nx;
        if (v & 128) {  // last of its cycle: from the cycle's first row
            int u = t;
            while (u > 0 && !(s_mv[u - 1] & 128)) u--;
            nx = s_mv[u];
        } else {
            nx = s_mv[t + 1];
        }
        s_src[v & 31] = (nx & 31) | (v & 0x60);
    }
    __syncthreads();
    auto rot = static_cast<S (*)(S, int)>(perm_rot);
    switch (op.k) {
        case 1: op_perm<1, S, SwzT>(sm, m, op, s_mv, s_src, t, blockDim.x, rot); break;
        case 2: op_perm<2, S, SwzT>(sm, m, op, s_mv, s_src, t, blockDim.x, rot); break;
        case 3: op_perm<3, S, SwzT>(sm, m, op, s_mv, s_src, t, blockDim.x, rot); break;
        case 4: op_perm<4, S, SwzT>(sm, m, op, s_mv, s_src, t, blockDim.x, rot); break;
        default: op_perm<5, S, SwzT>(sm, m, op, s_mv, s_src, t, blockDim.x, rot); break;
    }
}

template <int MODE, int KMAX>
__device__ __forceinline__ void apply_op(typename TileTraits<MODE>::Smem* sm, int m, const DevOp& op,
                                         const typename TileTraits<MODE>::Coef* __restrict__ M, uint64_t base) {
    if (op.kind == OP_PERM) {
        apply_perm<typename TileTraits<MODE>::Smem, typename TileTraits<MODE>::SwzT>(sm, m, op, M);
        return;
    }
    if constexpr (MODE == MODE_TC) {
        if (op.kind == OP_DIAG) {
            op_diag_tc(sm, m, op, reinterpret_cast<const Q2*>(M), base);
        } else if (op.k <= 3) {
            op_dense_tc<3>(sm, m, op, M);
        } else {
            op_dense_tc<(KMAX >= 4 ? 4 : 3)>(sm, m, op, M);  // the planner caps these blocks at 4 qubits
        }
    } else if constexpr (MODE == MODE_DF) {
        if (op.kind == OP_DIAG) {
            op_diag_df(sm, m, op, M, base);
        } else if (op.k == 1) {
            op_dense_df<1>(sm, m, op, M);
        } else if (op.k == 2) {
            op_dense_df<(KMAX >= 2 ? 2 : 1)>(sm, m, op, M);
        } else if (op.k == 3) {
            op_dense_df<(KMAX >= 3 ? 3 : 1)>(sm, m, op, M);
        } else if (op.k == 4) {
            op_dense_df<(KMAX >= 4 ? 4 : 1)>(sm, m, op, M);
        } else {
            op_dense_df<(KMAX >= 5 ? 5 : 1)>(sm, m, op, M);
        }
    } else {
        using R = typename TileTraits<MODE>::SwzT;
        if (op.kind == OP_DIAG) {
            op_diag<R>(sm, m, op, M, base);
        } else if (op.k == 1) {
            op_dense<1, R>(sm, m, op, M);
        } else if (op.k == 2) {
            op_dense<(KMAX >= 2 ? 2 : 1), R>(sm, m, op, M);
        } else if (op.k == 3) {
            op_dense<(KMAX >= 3 ? 3 : 1), R>(sm, m, op, M);
        } else if (op.k == 4) {
            op_dense<(KMAX >= 4 ? 4 : 1), R>(sm, m, op, M);
        } else {
            op_dense<(KMAX >= 5 ? 5 : 1), R>(sm, m, op, M);
        }
    }
}

// Sweeps the tiles of every (state, pass) entry: gather the tile's 2^m
// amplitudes (runs of 2^c contiguous ones, 16-byte loads) into shared memory,
// apply the pass's ops in order, scatter the tile back.  Persistent: each CTA
// strides over the flattened tile space of all entries.
template <int MODE, int KMAX>
__global__ void __launch_bounds__(tile_threads(MODE), MODE == MODE_TC ? 2 : 1)
    k_tile_pass(const BatchEntry* __restrict__ E, int n_entries, uint64_t total_tiles, const DevOp* __restrict__ ops,
                const typename TileTraits<MODE>::Coef* __restrict__ coef) {
    using Tr = TileTraits<MODE>;
    using Store = typename Tr::Store;
    using Smem = typename Tr::Smem;
    using SwzT = typename Tr::SwzT;
    extern __shared__ __align__(1024) unsigned char smraw[];
    // tcgen05 modes: block digits / parts first, the tile after them
    Smem* sm = reinterpret_cast<Smem*>(
        smraw + (MODE == MODE_T05 ? t05::kSmemBase : (MODE == MODE_T32 ? t32::kSmemBase : 0)));
    __shared__ uint64_t dep[2][32];  // deposit tables for the tile's high local bits
    __shared__ __align__(16) DevPass P;
    __shared__ uint64_t s_state, s_begin, s_next_base;
    __shared__ __align__(8) uint64_t t05_mbar;
    __shared__ uint32_t t05_tmem;
    constexpr int kOpCache = 48;  // the pass's op descriptors, read once per pass
    __shared__ DevOp s_ops[kOpCache];
    __shared__ __align__(16) uint4 s_diag[32];  // the current diagonal op's entries (at most 32 x 16 bytes)
    __shared__ __align__(16) int s_tab[uses_tmem(MODE) ? kOpCache * t05::kTabInts : 4];
    // complex128 digits: the constant B slice of the accumulator preload (7R x 16 fp16, K-major
    // core matrices: 8-row groups 256 bytes apart, the two 8-element K halves 128 bytes apart)
    __shared__ __align__(128) unsigned s_bias_b[MODE == MODE_T05 ? t05::kBiasRows * 8 : 1];
    t05::Ctx cx{};
    if constexpr (uses_tmem(MODE)) {
        if (threadIdx.x < 32) {  // warp 0 owns the tensor-memory allocation
            asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                             t05::smem_addr(&t05_tmem)),
                         "r"(t05::kTmemCols)
                         : "memory");
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
        }
        if (threadIdx.x == 0) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(t05::smem_addr(&t05_mbar)) : "memory");
            asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        }
        t05::fence_before();
        __syncthreads();
        t05::fence_after();
        cx.b = smraw;
        cx.b_addr = t05::smem_addr(cx.b);
        cx.mbar = t05::smem_addr(&t05_mbar);
        cx.tmem = t05_tmem;
        cx.bias_addr = t05::smem_addr(s_bias_b);
        cx.phase = 0;
        cx.failed = false;
        if constexpr (MODE == MODE_T05) {
            // K-element 0 of every row: B = 4096 (first word of each 16-byte row of the low K half)
            for (int w = threadIdx.x; w < t05::kBiasRows * 8; w += blockDim.x)
                s_bias_b[w] = ((w & 3) == 0 && (w & 63) < 32) ? t05::kHalf4096 : 0u;
            if (threadIdx.x < 128) {  // A = 3072 at K-element 0 of every TMEM lane, one lane quarter per warp
                const uint32_t ta = t05_tmem + ((uint32_t)(threadIdx.x & ~31) << 16) + t05::kAConst;
                asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%2,%2,%2,%2,%2,%2};\n" ::"r"(ta),
                             "r"(t05::kHalf3072), "r"(0u)
                             : "memory");
                asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory");
            }
            t05::fence_async_smem();
            t05::fence_before();
            __syncthreads();
            t05::fence_after();
        }
    }
    int cur = -1;
    // tensor-memory modes: this tile's cp.async loads were issued during the
    // previous tile's store phase (same entry, Q56 / float32 in HBM)
    bool preloaded = false;
    for (uint64_t t = blockIdx.x; t < total_tiles; t += gridDim.x) {
        int lo = 0, hi = n_entries - 1;  // entry owning tile t (uniform across the CTA)
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (E[mid].tile_begin <= t) lo = mid;
            else hi = mid - 1;
        }
        if (lo != cur) {
            __syncthreads();
            const unsigned* src = reinterpret_cast<const unsigned*>(&E[lo].p);
            unsigned* dst = reinterpret_cast<unsigned*>(&P);
            for (int i = threadIdx.x; i < (int)(sizeof(DevPass) / 4); i += blockDim.x) dst[i] = src[i];
            if (threadIdx.x == 0) {
                s_state = E[lo].state;
                s_begin = E[lo].tile_begin;
            }
            __syncthreads();
            if (P.n_ops <= kOpCache) {
                const int4* osrc = reinterpret_cast<const int4*>(ops + P.op0);
                int4* odst = reinterpret_cast<int4*>(s_ops);
                for (int i = threadIdx.x; i < P.n_ops * (int)(sizeof(DevOp) / 16); i += blockDim.x) odst[i] = osrc[i];
                if constexpr (uses_tmem(MODE)) {  // the pass's address tables, from the global descriptors
                    for (int i = threadIdx.x; i < P.n_ops * t05::kTabInts; i += blockDim.x) {
                        const int o = i / t05::kTabInts, t = i - o * t05::kTabInts;
                        const DevOp& op = ops[P.op0 + o];
                        // the block size each op is dispatched with below
                        if constexpr (MODE == MODE_T05) {
                            const int kt = op.k <= 3 ? 3 : (KMAX >= 4 ? 4 : 3);
                            s_tab[i] = t05::op_table_entry<double>(op, kt, kt == 3 ? 256 : 128, t);
                        } else {
                            const int kt = op.k <= 3 ? 3 : (op.k == 4 ? (KMAX >= 4 ? 4 : 3) : (KMAX >= 5 ? 5 : 3));
                            s_tab[i] = t05::op_table_entry<float>(op, kt, 128, t);
                        }
                    }
                }
            }
            if (threadIdx.x < 64) {
                const int w = threadIdx.x >> 5, v = threadIdx.x & 31, hb = P.m - P.c;
                uint64_t d = 0;
                for (int b = 0; b < 5; b++) {
                    const int bit = w * 5 + b;
                    if (bit < hb && ((v >> b) & 1)) d |= 1ull << P.L[P.c + bit];
                }
                dep[w][v] = d;
            }
            __syncthreads();
            cur = lo;
        }
        Store* st = reinterpret_cast<Store*>(s_state);
        const int m = P.m, c = P.c;
        const int cmask = (1 << c) - 1;
        const uint64_t tl = t - s_begin;
        uint64_t base = 0;
        for (int b = 0; b < P.n - m; b++)
            if ((tl >> b) & 1) base |= 1ull << P.NL[b];
        if (threadIdx.x == 0) {  // base of the CTA's next tile (same entry), for the L2 prefetch
            const uint64_t tn = t + gridDim.x;
            uint64_t bn = ~0ull;
            if (tn < total_tiles && tn - s_begin < P.tile_count) {
                const uint64_t tln = tn - s_begin;
                bn = 0;
                for (int b = 0; b < P.n - m; b++)
                    if ((tln >> b) & 1) bn |= 1ull << P.NL[b];
            }
            s_next_base = bn;
        }
        if constexpr (MODE == MODE_DF) {
            const int N = 1 << m;
            for (int j = threadIdx.x; j < N; j += blockDim.x) {
                const int r = j >> c;
                const uint64_t gidx = base | dep[0][r & 31] | dep[1][(r >> 5) & 31] | (uint64_t)(j & cmask);
                const Cx<double> a = st[gidx];
                DF4 v;
                d2df(a.re, v.rh, v.rl);
                d2df(a.im, v.ih, v.il);
                sm[swz<double>(j)] = v;
            }
        } else if constexpr (MODE == MODE_TC || MODE == MODE_T05) {
            // fixed-point tile: Q62 (mma.sync mode), Q56 (tcgen05 mode, whose digits are those of x >> 6)
            constexpr int kTileFB = MODE == MODE_T05 ? 56 : 62;
            // loads in flight per thread before the conversions
            constexpr int U = MODE == MODE_T05 ? 8 : 4;
            const int N = 1 << m, nt = blockDim.x;
            auto load = [&](auto conv) {
                for (int j0 = threadIdx.x; j0 < N; j0 += U * nt) {
                    Cx<double> a[U];
#pragma unroll
                    for (int u = 0; u < U; u++) {
                        const int j = j0 + u * nt, r = j >> c;
                        if (j < N) a[u] = st[base | dep[0][r & 31] | dep[1][(r >> 5) & 31] | (uint64_t)(j & cmask)];
                    }
#pragma unroll
                    for (int u = 0; u < U; u++) {
                        const int j = j0 + u * nt;
                        if (j < N) sm[swz<double>(j)] = Q2{conv(a[u].re), conv(a[u].im)};
                    }
                }
            };
            if (MODE == MODE_T05 && preloaded) {
                t05::cp_async_wait_all();
            } else if (MODE == MODE_T05 && (P.io & IO_LOAD_Q56)) {
                // uniform: the previous pass left Q56, a plain copy: every 16-byte
                // slot of the tile in flight at once, global to shared memory
                const uint32_t sbase = t05::smem_addr(sm);
                for (int j = threadIdx.x; j < N; j += nt) {
                    const int r = j >> c;
                    t05::cp_async16(sbase + 16u * (uint32_t)swz<double>(j),
                                    st + (base | dep[0][r & 31] | dep[1][(r >> 5) & 31] | (uint64_t)(j & cmask)));
                }
                t05::cp_async_wait_all();
            } else {
                load([](double v) { return d2q<kTileFB>(v); });
            }
        } else {
            constexpr int PER = 16 / sizeof(Store);  // amplitudes per 16-byte vector
            // the one-CTA-per-SM tensor-memory mode has no other CTA to hide
            // the loads: it copies with cp.async, the whole tile in flight
            const int nvec = (1 << m) / PER, nt = blockDim.x;
            if constexpr (uses_tmem(MODE)) {
                if (!preloaded) {
                    const uint32_t sbase = t05::smem_addr(sm);
                    for (int v = threadIdx.x; v < nvec; v += nt) {
                        const int j = v * PER, r = j >> c;
                        t05::cp_async16(sbase + (uint32_t)(sizeof(Smem) * swz<SwzT>(j)),
                                        st + (base | dep[0][r & 31] | dep[1][(r >> 5) & 31] | (uint64_t)(j & cmask)));
                    }
                }
                t05::cp_async_wait_all();
            } else {
                for (int v = threadIdx.x; v < nvec; v += nt) {
                    const int j = v * PER, r = j >> c;
                    *reinterpret_cast<int4*>(sm + swz<SwzT>(j)) = *reinterpret_cast<const int4*>(
                        st + (base | dep[0][r & 31] | dep[1][(r >> 5) & 31] | (uint64_t)(j & cmask)));
                }
            }
        }
        __syncthreads();
        {
            // Prefetch the CTA's next tile (same entry) into L2 while this one
            // is computed: one bulk prefetch per run of 2^c contiguous
            // amplitudes (256 bytes), so the next load phase reads from L2.
            // The next tile's base comes from thread 0 (computed before the
            // load phase), so a thread adds one address and one instruction.
            const int runs = 1 << (m - c);
            const uint64_t bn = s_next_base;
            if (bn != ~0ull && (int)threadIdx.x < runs) {
                const int r = threadIdx.x;
                const Store* src = st + (bn | dep[0][r & 31] | dep[1][(r >> 5) & 31]);
                asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(src), "r"((int)(sizeof(Store) << c))
                             : "memory");
            }
        }
        const int n_ops = P.n_ops, op0 = P.op0;
        for (int o = 0; o < n_ops; o++) {
            const DevOp op = n_ops <= kOpCache ? s_ops[o] : ops[op0 + o];
            // a diagonal op's 2^k entries (at most 32) are staged in shared
            // memory by every thread, so each amplitude reads its phase there
            // (the previous op ended with a barrier)
            const typename Tr::Coef* opc = coef + op.coeff;
            if (op.kind == OP_DIAG) {
                constexpr int kEB = diag_entry_bytes(MODE);
                const unsigned* src = reinterpret_cast<const unsigned*>(opc);
                unsigned* dst = reinterpret_cast<unsigned*>(s_diag);
                for (int i = threadIdx.x; i < (kEB / 4) << op.k; i += blockDim.x) dst[i] = src[i];
                __syncthreads();
                opc = reinterpret_cast<const typename Tr::Coef*>(s_diag);
            }
            if constexpr (MODE == MODE_T05) {
                if (op.kind == OP_PERM)
                    apply_perm<Q2, double>(sm, m, op, coef + op.coeff);
                else if (op.kind == OP_DIAG)
                    op_diag_tc<t05::kLogThreads>(sm, m, op, reinterpret_cast<const Q2*>(opc), base);
                else {
                    const int* tab = n_ops <= kOpCache ? s_tab + o * t05::kTabInts : nullptr;
                    if (op.k <= 3) t05::op_dense<3>(sm, m, op, coef + op.coeff, cx, tab);
                    else t05::op_dense<(KMAX >= 4 ? 4 : 3)>(sm, m, op, coef + op.coeff, cx, tab);  // capped at 4 qubits
                }
                if (cx.failed) break;  // uniform: decided by a block-wide vote
            } else if constexpr (MODE == MODE_T32) {
                if (op.kind == OP_PERM) {
                    apply_perm<Cx<float>, float>(sm, m, op, coef + op.coeff);
                } else if (op.kind == OP_DIAG) {
                    if (threadIdx.x < t05::kThreads)  // the issuing warp sits out the 512-thread sweep
                        op_diag<float, t05::kLogThreads>(sm, m, op, reinterpret_cast<const Cx<float>*>(opc), base);
                }
                else {
                    const int* tab = n_ops <= kOpCache ? s_tab + o * t05::kTabInts : nullptr;
                    if (op.k <= 3) t32::op_dense<3>(sm, m, op, coef + op.coeff, cx, tab);  // smaller blocks are padded
                    else if (op.k == 4) t32::op_dense<(KMAX >= 4 ? 4 : 3)>(sm, m, op, coef + op.coeff, cx, tab);
                    else t32::op_dense<(KMAX >= 5 ? 5 : 3)>(sm, m, op, coef + op.coeff, cx, tab);
                }
                if (cx.failed) break;
            } else {
                apply_op<MODE, KMAX>(sm, m, op, opc, base);
            }
            __syncthreads();
        }
        if constexpr (uses_tmem(MODE)) {
            if (cx.failed) break;  // the state is left undefined; the host reports SV_ERR_TIMEOUT
        }
        if constexpr (MODE == MODE_DF) {
            const int N = 1 << m;
            for (int j = threadIdx.x; j < N; j += blockDim.x) {
                const int r = j >> c;
                const uint64_t gidx = base | dep[0][r & 31] | dep[1][(r >> 5) & 31] | (uint64_t)(j & cmask);
                const DF4 v = sm[swz<double>(j)];
                st[gidx] = Cx<double>{df2d(v.rh, v.rl), df2d(v.ih, v.il)};
            }
        } else if constexpr (MODE == MODE_TC || MODE == MODE_T05) {
            constexpr int kTileFB = MODE == MODE_T05 ? 56 : 62;
            const int N = 1 << m;
            // the CTA's next tile (same entry) reads Q56: each thread refills its
            // slots with it by cp.async as soon as it has stored them
            const uint64_t bn = s_next_base;
            const bool fuse = MODE == MODE_T05 && bn != ~0ull && (P.io & IO_LOAD_Q56);
            const uint32_t sbase = t05::smem_addr(sm);
            auto store = [&](auto conv) {
                for (int j = threadIdx.x; j < N; j += blockDim.x) {
                    const int r = j >> c;
                    const uint64_t dj = dep[0][r & 31] | dep[1][(r >> 5) & 31] | (uint64_t)(j & cmask);
                    const Q2 v = sm[swz<double>(j)];
                    st[base | dj] = Cx<double>{conv(v.re), conv(v.im)};
                    if (fuse) t05::cp_async16(sbase + 16u * (uint32_t)swz<double>(j), st + (bn | dj));
                }
            };
            preloaded = fuse;
            if (MODE == MODE_T05 && (P.io & IO_STORE_Q56))  // uniform: the next pass reads Q56
                store([](long long q) { return __longlong_as_double(q); });
            else
                store([](long long q) { return q2d<kTileFB>(q); });
        } else {
            constexpr int PER = 16 / sizeof(Store);
            const int nvec = (1 << m) / PER;
            // tensor-memory mode: refill each stored slot with the CTA's next tile (same entry) by cp.async
            const uint64_t bn = s_next_base;
            const bool fuse = uses_tmem(MODE) && bn != ~0ull;
            const uint32_t sbase = t05::smem_addr(sm);
            for (int v = threadIdx.x; v < nvec; v += blockDim.x) {
                const int j = v * PER;
                const int r = j >> c;
                const uint64_t dj = dep[0][r & 31] | dep[1][(r >> 5) & 31] | (uint64_t)(j & cmask);
                *reinterpret_cast<int4*>(st + (base | dj)) = *reinterpret_cast<const int4*>(sm + swz<SwzT>(j));
                if (fuse) t05::cp_async16(sbase + (uint32_t)(sizeof(Smem) * swz<SwzT>(j)), st + (bn | dj));
            }
            preloaded = fuse;
        }
        __syncthreads();
    }
    if constexpr (uses_tmem(MODE)) {
        t05::fence_before();
        __syncthreads();
        if (threadIdx.x < 32) {
            t05::fence_after();
            asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(cx.tmem),
                         "r"(t05::kTmemCols)
                         : "memory");
        }
    }
}

// ---------------------------------------------------------------------------
// K7: probabilities, exact norm, marginals.
// ---------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ double prob_of(Cx<R> v) {
    const double re = (double)v.re, im = (double)v.im;
    return fma(re, re, im * im);  // exact products for float inputs, one rounding
}

// x 2^-down (x >= 0, x 2^-down < 16) as an unsigned 128-bit fixed-point
// number in units of 2^-124.
__device__ __forceinline__ unsigned __int128 to_fixed(double x, int down = 0) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int e = (int)((b >> 52) & 0x7ff);
    if (e == 0) return 0;  // zero or subnormal (below 2^-1022): below the grid
    const unsigned long long mant = (b & ((1ull << 52) - 1)) | (1ull << 52);
    const int sh = e - 1075 + 124 - down;
    if (sh >= 0) return (unsigned __int128)mant << sh;
    if (sh <= -53) return 0;
    return (unsigned __int128)(mant >> (-sh));
}

__device__ __forceinline__ double fixed_to_double(unsigned __int128 v) {
    if (v == 0) return 0.0;
    const unsigned long long hi = (unsigned long long)(v >> 64), lo = (unsigned long long)v;
    const int lz = hi ? __clzll(hi) : 64 + __clzll(lo);
    const unsigned __int128 nv = v << lz;
    unsigned long long top = (unsigned long long)(nv >> 64);
    top |= ((unsigned long long)nv != 0ull) ? 1ull : 0ull;  // sticky bit
    return ldexp(__ull2double_rn(top), 64 - lz - 124);
}

__device__ __forceinline__ unsigned __int128 warp_sum128(unsigned __int128 v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long lo = (unsigned long long)v, hi = (unsigned long long)(v >> 64);
        const unsigned long long lo2 = __shfl_down_sync(0xffffffffu, lo, o);
        const unsigned long long hi2 = __shfl_down_sync(0xffffffffu, hi, o);
        v += ((unsigned __int128)hi2 << 64) | lo2;
    }
    return v;
}

__device__ __forceinline__ unsigned __int128 block_sum128(unsigned __int128 v) {
    __shared__ unsigned long long red[2][32];
    v = warp_sum128(v);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) {
        red[0][w] = (unsigned long long)v;
        red[1][w] = (unsigned long long)(v >> 64);
    }
    __syncthreads();
    unsigned __int128 r = 0;
    if (w == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        if (lane < nw) r = ((unsigned __int128)red[1][lane] << 64) | red[0][lane];
        r = warp_sum128(r);
    }
    return r;  // valid in thread 0
}

template <typename R>
__global__ void k_probs(const Cx<R>* __restrict__ a, uint64_t i0, uint64_t len, double* __restrict__ p) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += stride)
        p[i] = prob_of<R>(a[i0 + i]);
}

template <typename R>
__global__ void k_norm_partial(const Cx<R>* __restrict__ a, uint64_t dim, unsigned long long* __restrict__ part,
                               int down) {
    unsigned __int128 acc = 0;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < dim; i += stride)
        acc += to_fixed(prob_of<R>(a[i]), down);
    acc = block_sum128(acc);
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = (unsigned long long)acc;
        part[2 * blockIdx.x + 1] = (unsigned long long)(acc >> 64);
    }
}

__global__ void k_norm_final(const unsigned long long* __restrict__ part, int nparts, double* out) {
    unsigned __int128 acc = 0;
    for (int i = threadIdx.x; i < nparts; i += blockDim.x)
        acc += ((unsigned __int128)part[2 * i + 1] << 64) | part[2 * i];
    acc = block_sum128(acc);
    if (threadIdx.x == 0) *out = fixed_to_double(acc);
}

struct MaskInfo {
    int32_t nq;
    int8_t q[kMaxQ];
};

__device__ __forceinline__ void atomic_add128(unsigned long long* bin, unsigned __int128 v) {
    const unsigned long long lo = (unsigned long long)v;
    unsigned long long hi = (unsigned long long)(v >> 64);
    const unsigned long long old = atomicAdd(bin, lo);
    if (old + lo < old) hi += 1ull;  // carry out of the low word
    if (hi) atomicAdd(bin + 1, hi);
}

template <typename R>
__global__ void k_marginal(const Cx<R>* __restrict__ a, uint64_t dim, const MaskInfo mi,
                           unsigned long long* __restrict__ gbins, int nbins, int use_smem) {
    extern __shared__ unsigned long long sbins[];
    if (use_smem) {
        for (int b = threadIdx.x; b < 2 * nbins; b += blockDim.x) sbins[b] = 0ull;
        __syncthreads();
    }
    unsigned long long* bins = use_smem ? sbins : gbins;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < dim; i += stride) {
        int k = 0;
        for (int j = 0; j < mi.nq; j++) k |= (int)((i >> mi.q[j]) & 1) << j;
        const unsigned __int128 fx = to_fixed(prob_of<R>(a[i]));
        if (fx) atomic_add128(bins + 2 * k, fx);
    }
    if (use_smem) {
        __syncthreads();
        for (int b = threadIdx.x; b < nbins; b += blockDim.x) {
            const unsigned __int128 v = ((unsigned __int128)sbins[2 * b + 1] << 64) | sbins[2 * b];
            if (v) atomic_add128(gbins + 2 * b, v);
        }
    }
}

__global__ void k_bins_to_double(const unsigned long long* __restrict__ bins, uint64_t nbins, double* out) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t b = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; b < nbins; b += stride)
        out[b] = fixed_to_double(((unsigned __int128)bins[2 * b + 1] << 64) | bins[2 * b]);
}

// Largest |component| of a state, as the bit pattern of a non-negative
// double (such patterns order like the values): atomicMax into *out.
__global__ void k_max_abs(const double* __restrict__ a, uint64_t n, unsigned long long* out) {
    unsigned long long m = 0;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const unsigned long long b = (unsigned long long)__double_as_longlong(a[i]) & 0x7FFFFFFFFFFFFFFFull;
        m = b > m ? b : m;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long x = __shfl_down_sync(0xffffffffu, m, o);
        m = x > m ? x : m;
    }
    if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

__global__ void k_zero_u64(unsigned long long* p, uint64_t n) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) p[i] = 0ull;
}

// ---------------------------------------------------------------------------
// Multi-state init and probabilities (batched form): each CTA walks the
// entries in order and grid-strides over each entry's elements.
// ---------------------------------------------------------------------------
template <typename R>
__global__ void k_init_multi(const StateEntry* __restrict__ E, int n_entries) {
    constexpr int PER = 16 / sizeof(Cx<R>);
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (int e = 0; e < n_entries; e++) {
        Cx<R>* a = reinterpret_cast<Cx<R>*>(E[e].state);
        const uint64_t nvec = (1ull << E[e].n) / PER;
        for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < nvec; v += stride)
            reinterpret_cast<int4*>(a)[v] = (v == 0) ? unit_vector16<R>(0) : make_int4(0, 0, 0, 0);
    }
}

template <typename R>
__global__ void k_probs_multi(const StateEntry* __restrict__ E, int n_entries) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (int e = 0; e < n_entries; e++) {
        const Cx<R>* a = reinterpret_cast<const Cx<R>*>(E[e].state);
        double* p = reinterpret_cast<double*>(E[e].probs);
        const uint64_t dim = 1ull << E[e].n;
        for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < dim; i += stride)
            p[i] = prob_of<R>(a[i]);
    }
}

// ---------------------------------------------------------------------------
// Launchers.
// ---------------------------------------------------------------------------
static unsigned grid_for(uint64_t work, int threads, const DevInfo& di, int per_sm = 8) {
    uint64_t g = (work + threads - 1) / threads;
    const uint64_t cap = (uint64_t)di.sms * per_sm;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (unsigned)g;
}

cudaError_t launch_init(int dt, void* amp, int n, uint64_t basis, cudaStream_t s, const DevInfo& di) {
    const uint64_t dim = 1ull << n;
    if (dt == SV_C64)
        k_init<float><<<grid_for(dim / 2, 256, di), 256, 0, s>>>((Cx<float>*)amp, dim, basis);
    else
        k_init<double><<<grid_for(dim, 256, di), 256, 0, s>>>((Cx<double>*)amp, dim, basis);
    return cudaGetLastError();
}

template <int MODE, int KMAX>
static cudaError_t tile_pass_impl(const BatchEntry* d_entries, int n_entries, uint64_t total_tiles, int max_m,
                                  const DevOp* d_ops, const void* d_coef, cudaStream_t s, const DevInfo& di) {
    using Tr = TileTraits<MODE>;
    size_t smem = ((size_t)1 << max_m) * sizeof(typename Tr::Smem);
    if (MODE == MODE_T05) smem = std::max<size_t>(smem + t05::kSmemBase, t05::kSmemMin);
    if (MODE == MODE_T32) smem = std::max<size_t>(smem + t32::kSmemBase, t05::kSmemMin);
    static int configured_dev = -1;
    static size_t dyn_max = 0;
    if (configured_dev != di.device) {
        cudaFuncAttributes fa{};
        cudaError_t e = cudaFuncGetAttributes(&fa, k_tile_pass<MODE, KMAX>);
        if (e != cudaSuccess) return e;
        dyn_max = di.smem_optin - fa.sharedSizeBytes;  // opt-in limit minus the kernel's static shared memory
        e = cudaFuncSetAttribute(k_tile_pass<MODE, KMAX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn_max);
        if (e != cudaSuccess) return e;
        configured_dev = di.device;
    }
    if (smem > dyn_max) return cudaErrorInvalidValue;
    const int threads = tile_threads(MODE);
    int per_sm = 1;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tile_pass<MODE, KMAX>, threads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    uint64_t grid = (uint64_t)di.sms * per_sm;
    if (grid > total_tiles) grid = total_tiles;
    k_tile_pass<MODE, KMAX><<<(unsigned)grid, threads, smem, s>>>(
        d_entries, n_entries, total_tiles, d_ops, (const typename Tr::Coef*)d_coef);
    return cudaGetLastError();
}

template <int MODE>
static cudaError_t tile_pass_mode(int kmax, const BatchEntry* d_entries, int n_entries, uint64_t total_tiles,
                                  int max_m, const DevOp* d_ops, const void* d_coef, cudaStream_t s,
                                  const DevInfo& di) {
    switch (kmax) {
        case 1: return tile_pass_impl<MODE, 1>(d_entries, n_entries, total_tiles, max_m, d_ops, d_coef, s, di);
        case 2: return tile_pass_impl<MODE, 2>(d_entries, n_entries, total_tiles, max_m, d_ops, d_coef, s, di);
        case 3: return tile_pass_impl<MODE, 3>(d_entries, n_entries, total_tiles, max_m, d_ops, d_coef, s, di);
        case 4: return tile_pass_impl<MODE, 4>(d_entries, n_entries, total_tiles, max_m, d_ops, d_coef, s, di);
        default: return tile_pass_impl<MODE, 5>(d_entries, n_entries, total_tiles, max_m, d_ops, d_coef, s, di);
    }
}

cudaError_t launch_tile_pass(int dt, int arith, const BatchEntry* d_entries, int n_entries, uint64_t total_tiles,
                             int max_m, int kmax, const DevOp* d_ops, const void* d_coef, cudaStream_t s,
                             const DevInfo& di) {
    if (n_entries <= 0 || total_tiles == 0) return cudaSuccess;
    if (dt == SV_C64 && arith == SV_ARITH_TC)
        return tile_pass_mode<MODE_T32>(kmax, d_entries, n_entries, total_tiles, max_m, d_ops, d_coef, s, di);
    if (dt == SV_C64)
        return tile_pass_mode<MODE_F32>(kmax, d_entries, n_entries, total_tiles, max_m, d_ops, d_coef, s, di);
    if (arith == SV_ARITH_DF64)
        return tile_pass_mode<MODE_DF>(kmax, d_entries, n_entries, total_tiles, max_m, d_ops, d_coef, s, di);
    if (arith == SV_ARITH_TC)
        return tile_pass_mode<MODE_T05>(kmax, d_entries, n_entries, total_tiles, max_m, d_ops, d_coef, s, di);
    if (arith == SV_ARITH_TC_SYNC)
        return tile_pass_mode<MODE_TC>(kmax, d_entries, n_entries, total_tiles, max_m, d_ops, d_coef, s, di);
    return tile_pass_mode<MODE_F64>(kmax, d_entries, n_entries, total_tiles, max_m, d_ops, d_coef, s, di);
}

cudaError_t launch_init_multi(int dt, const StateEntry* d_entries, int n_entries, uint64_t total_amps,
                              cudaStream_t s, const DevInfo& di) {
    if (n_entries <= 0) return cudaSuccess;
    const unsigned grid = grid_for(total_amps / 2 + 1, 256, di, 8);
    if (dt == SV_C64) k_init_multi<float><<<grid, 256, 0, s>>>(d_entries, n_entries);
    else k_init_multi<double><<<grid, 256, 0, s>>>(d_entries, n_entries);
    return cudaGetLastError();
}

cudaError_t launch_probs_multi(int dt, const StateEntry* d_entries, int n_entries, uint64_t total_amps,
                               cudaStream_t s, const DevInfo& di) {
    if (n_entries <= 0) return cudaSuccess;
    const unsigned grid = grid_for(total_amps, 256, di, 8);
    if (dt == SV_C64) k_probs_multi<float><<<grid, 256, 0, s>>>(d_entries, n_entries);
    else k_probs_multi<double><<<grid, 256, 0, s>>>(d_entries, n_entries);
    return cudaGetLastError();
}

cudaError_t tc_fault_take(int* fault) {
    int zero = 0;
    cudaError_t e = cudaMemcpyFromSymbol(fault, t05::g_fault, sizeof(int));
    if (e == cudaSuccess && *fault) e = cudaMemcpyToSymbol(t05::g_fault, &zero, sizeof(int));
    return e;
}

cudaError_t launch_max_abs_c128(const void* amp, int n, unsigned long long* d_out, cudaStream_t s,
                               const DevInfo& di) {
    const uint64_t count = 2ull << n;  // re and im of 2^n amplitudes
    k_zero_u64<<<1, 32, 0, s>>>(d_out, 1);
    k_max_abs<<<grid_for(count, 256, di), 256, 0, s>>>((const double*)amp, count, d_out);
    return cudaGetLastError();
}

cudaError_t launch_probs(int dt, const void* amp, uint64_t i0, uint64_t len, double* p, cudaStream_t s,
                         const DevInfo& di) {
    if (dt == SV_C64)
        k_probs<float><<<grid_for(len, 256, di), 256, 0, s>>>((const Cx<float>*)amp, i0, len, p);
    else
        k_probs<double><<<grid_for(len, 256, di), 256, 0, s>>>((const Cx<double>*)amp, i0, len, p);
    return cudaGetLastError();
}

static constexpr int kNormThreads = 256;
size_t norm_scratch_bytes(const DevInfo& di) { return (size_t)di.sms * 8 * 2 * sizeof(unsigned long long); }

cudaError_t launch_norm(int dt, const void* amp, int n, void* d_scratch, double* d_out, cudaStream_t s,
                        const DevInfo& di, int down) {
    const uint64_t dim = 1ull << n;
    const unsigned grid = grid_for(dim, kNormThreads, di, 8);
    auto* part = (unsigned long long*)d_scratch;
    if (dt == SV_C64)
        k_norm_partial<float><<<grid, kNormThreads, 0, s>>>((const Cx<float>*)amp, dim, part, down);
    else
        k_norm_partial<double><<<grid, kNormThreads, 0, s>>>((const Cx<double>*)amp, dim, part, down);
    k_norm_final<<<1, 1024, 0, s>>>(part, (int)grid, d_out);
    return cudaGetLastError();
}

cudaError_t launch_marginal(int dt, const void* amp, int n, uint64_t qubit_mask, void* d_bins, double* d_out,
                            cudaStream_t s, const DevInfo& di) {
    MaskInfo mi{};
    for (int q = 0; q < n; q++)
        if ((qubit_mask >> q) & 1) mi.q[mi.nq++] = (int8_t)q;
    const uint64_t nbins = 1ull << mi.nq, dim = 1ull << n;
    auto* bins = (unsigned long long*)d_bins;
    k_zero_u64<<<grid_for(2 * nbins, 256, di), 256, 0, s>>>(bins, 2 * nbins);
    const int use_smem = nbins <= 2048 ? 1 : 0;
    const size_t smem = use_smem ? 2 * nbins * sizeof(unsigned long long) : 0;
    const unsigned grid = grid_for(dim, 256, di, 4);
    if (dt == SV_C64)
        k_marginal<float><<<grid, 256, smem, s>>>((const Cx<float>*)amp, dim, mi, bins, (int)nbins, use_smem);
    else
        k_marginal<double><<<grid, 256, smem, s>>>((const Cx<double>*)amp, dim, mi, bins, (int)nbins, use_smem);
    k_bins_to_double<<<grid_for(nbins, 256, di), 256, 0, s>>>(bins, nbins, d_out);
    return cudaGetLastError();
}

}  // namespace svk

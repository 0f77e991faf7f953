// C-ABI of the statevector engine (include/sv.h, include/sv_plan.h).
//
// Each call validates its arguments, runs the host planner where needed,
// uploads the launch descriptors and block coefficients, launches the sm_103a
// kernels on the handle's stream and waits for them.  No C++ exception
// crosses the boundary.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstdint>
#include <chrono>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <utility>
#include <vector>

#include "device_types.hpp"
#include "kernels.cuh"
#include "plan.hpp"
#include "sv.h"
#include "sv_plan.h"

using svk::DevOp;
using svk::DevPass;

struct sv_state {
    int n = 0, dt = 0;
    size_t bytes = 0;
    void* amp = nullptr;
    bool owned = false;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    svk::DevInfo di;
    // device workspace: launch descriptors and block coefficients
    void* d_ws = nullptr;
    size_t d_ws_cap = 0;
    void* h_ws = nullptr;  // pinned staging of the same
    size_t h_ws_cap = 0;
    void* d_red = nullptr;  // reduction scratch
    size_t d_red_cap = 0;
    sv_apply_stats last{};
    bool failed = false;
    // contents came from the caller (sv_set_amplitudes, sv_create_on): the
    // tensor-core mode checks their magnitude once before relying on it
    bool foreign = false;
    std::vector<cudaEvent_t> events;  // timing events, reused across calls
};

struct sv_plan {
    svp::Plan plan;
    int dt = 0;
};

namespace {

#define SV_TRY(expr)                                   \
    do {                                               \
        cudaError_t _e = (expr);                       \
        if (_e != cudaSuccess) return fail_cuda(s, _e); \
    } while (0)

int fail_cuda(sv_state* s, cudaError_t e) {
    if (s) s->failed = true;
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return SV_ERR_OOM;
    }
    return SV_ERR_CUDA;
}

int amp_bytes(int dt) { return dt == SV_C64 ? 8 : 16; }
bool dt_ok(int dt) { return dt == SV_C64 || dt == SV_C128; }

std::mutex g_di_mu;
svk::DevInfo g_di[64];
bool g_di_ok[64] = {false};

cudaError_t device_info(svk::DevInfo* out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(g_di_mu);
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!g_di_ok[dev]) {
        svk::DevInfo d;
        d.device = dev;
        e = cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        int smem = 0;
        e = cudaDeviceGetAttribute(&smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        if (e != cudaSuccess) return e;
        d.smem_optin = (size_t)smem;
        g_di[dev] = d;
        g_di_ok[dev] = true;
    }
    *out = g_di[dev];
    return cudaSuccess;
}

// Tile shape per dtype: 2^m amplitudes in shared memory, the lowest c qubits
// always in the tile (runs of 2^c contiguous amplitudes = 256 bytes).  The
// tensor-memory mode takes 128 KiB tiles (one CTA per SM, 16 warps).
int default_tile(int dt, int arith = SV_ARITH_NATIVE) {
    if (dt == SV_C64) return arith == SV_ARITH_TC ? 14 : 13;
    return arith == SV_ARITH_TC ? 13 : 12;
}
constexpr int kGateDown = 36;   // pre-scale of the norm that gates caller-supplied states
int coalesce_of(int dt) { return dt == SV_C64 ? 5 : 4; }
int max_tile(int dt, const svk::DevInfo& di) {
    int m = dt == SV_C64 ? 14 : 13;
    while (m > 6 && ((size_t)1 << m) * amp_bytes(dt) > di.smem_optin - 2048) m--;
    return m;
}

// complex128 arithmetic.  SV_ARITH_AUTO takes the tensor-memory digit mode
// from kAutoTcQubits qubits on (measured crossover on GB300: below it the
// state is at most 64 tiles, fewer than the SMs, and the double-float pass,
// with less work per op, is faster: 19 q 1.50 ms vs 1.90 ms per circuit,
// 20 q 2.46 ms vs 2.00 ms) and double-float arithmetic below; explicit
// tensor-core modes need tiles of at least 8 qubits and fall back to
// double-float below.
constexpr int kAutoTcQubits = 20;
// complex64: the float32 FMA pass wins up to 22 qubits (measured: 22 q
// 2.52 ms vs 2.71 ms per circuit, 23 q 4.26 ms vs 3.40 ms)
constexpr int kAutoTc32Qubits = 23;

int resolve_arith(int dt, const sv_run_opts* o, int n = 34) {
    const int a = o ? o->arith : 0;
    if (dt == SV_C64) {  // float32 FMAs, or the bfloat16 triple split on the tensor cores
        if (n < 8 || (a != SV_ARITH_TC && a != SV_ARITH_AUTO)) return SV_ARITH_NATIVE;
        return (a == SV_ARITH_TC || n >= kAutoTc32Qubits) ? SV_ARITH_TC : SV_ARITH_NATIVE;
    }
    if (a == SV_ARITH_NATIVE) return SV_ARITH_NATIVE;
    if (a == SV_ARITH_DF64 || n < 8) return SV_ARITH_DF64;
    if (a == SV_ARITH_TC_SYNC) return SV_ARITH_TC_SYNC;
    if (a == SV_ARITH_TC) return SV_ARITH_TC;
    return n >= kAutoTcQubits ? SV_ARITH_TC : SV_ARITH_DF64;
}

bool is_tc(int arith) { return arith == SV_ARITH_TC || arith == SV_ARITH_TC_SYNC; }

// Device-measured cost tables (sv_calibrate / sv_set_costs), per (dtype,
// resolved arithmetic); the planner's cost model when one is installed.
std::mutex g_costs_mu;
std::map<std::pair<int, int>, sv_costs> g_costs;

bool measured_costs(int dt, int arith, sv_costs* out) {
    std::lock_guard<std::mutex> lk(g_costs_mu);
    auto it = g_costs.find({dt, arith});
    if (it == g_costs.end()) return false;
    *out = it->second;
    return true;
}

svp::Plan plan_for(int n, int dt, const sv_gate* g, size_t ng, const sv_run_opts* o, int smem_max_m) {
    int k = o ? o->max_fuse_k : 0;
    if (k < 0) k = 0;
    if (k > svp::kMaxFuse) k = svp::kMaxFuse;
    const int c = coalesce_of(dt);
    const int arith = resolve_arith(dt, o, n);
    int m = (o && o->tile_qubits > 0) ? o->tile_qubits : default_tile(dt, arith);
    m = std::min(m, smem_max_m);
    m = std::min(m, c + 10);
    m = std::max(m, c + svp::kMaxFuse);
    svp::Machine mc;
    sv_costs measured;
    if (measured_costs(dt, arith, &measured)) mc.measured = &measured;
    int ak = arith == SV_ARITH_TC ? svp::AK_TC32 : svp::AK_FP32;
    if (dt == SV_C128) ak = arith == SV_ARITH_DF64 ? svp::AK_DF64 : (is_tc(arith) ? svp::AK_TC : svp::AK_FP64);
    return svp::make_plan(n, g, ng, k, m, c, amp_bytes(dt), ak, mc);
}

// Serialises a plan into descriptors (passes by value, ops and coefficients
// into one contiguous upload).
struct Word16 {
    uint32_t w[4];
};

struct Lowered {
    std::vector<DevPass> passes;
    std::vector<DevOp> ops;
    std::vector<svp::cd> coef;   // complex coefficients (FP32 / FP64 / df64 modes)
    std::vector<Word16> tc;      // tensor-core modes: block digits and Q62 phases
    bool is_tc = false;
    bool tc_ok = true;           // every block's digit sums stay in the exact float32 range
};

// ---- tensor-core lowering ------------------------------------------------
int64_t q62_of(double x) {
    const double v = std::ldexp(x, 62);
    if (v >= 9.2233720368547758e18) return INT64_MAX;
    if (v <= -9.2233720368547758e18) return -INT64_MAX;
    return (int64_t)std::llround(v);
}

uint32_t bf16_of_digit(int d) {
    float f = (float)d;
    uint32_t u;
    std::memcpy(&u, &f, 4);
    return u >> 16;  // exact: |d| <= 256
}

// Digit j of a Q62 value: 8-bit digits for blocks of up to 4 qubits (seven
// digits), 7-bit digits for 5-qubit blocks (eight digits); the same split the
// tensor-core kernel applies to the amplitudes.
int tc_digit(int64_t q, int j, int db) {
    const int top = 56 - db;
    int64_t v = q >> 6;
    if (db == 7) v >>= 1;
    return j == 0 ? (int)(v >> top) : (int)((v >> (top - db * j)) & ((1 << db) - 1));
}

// Embeds a block of k < 3 qubits at tile positions pos[] into a 3-qubit block
// (identity on the added positions); returns the new positions and matrix.
void extend_to3(int k, const int* pos, const std::vector<svp::cd>& M, uint64_t local_pos_mask_avail, int* pos3,
                std::vector<svp::cd>& M3) {
    uint64_t used = 0;
    for (int j = 0; j < k; j++) used |= 1ull << pos[j];
    uint64_t all = used;
    for (int p = 0; p < 64 && __builtin_popcountll(all) < 3; p++)
        if (((local_pos_mask_avail >> p) & 1) && !((all >> p) & 1)) all |= 1ull << p;
    int n3 = 0;
    int src_bit[3] = {-1, -1, -1};  // matrix bit of the original block for new bit b, or -1
    for (int p = 0; p < 64; p++)
        if ((all >> p) & 1) {
            for (int j = 0; j < k; j++)
                if (pos[j] == p) src_bit[n3] = j;
            pos3[n3++] = p;
        }
    const int D = 1 << k;
    M3.assign(64, svp::cd(0, 0));
    for (int r = 0; r < 8; r++)
        for (int c = 0; c < 8; c++) {
            bool same_extra = true;
            int rr = 0, cc = 0;
            for (int b = 0; b < 3; b++) {
                const int rb = (r >> b) & 1, cb = (c >> b) & 1;
                if (src_bit[b] < 0) same_extra = same_extra && rb == cb;
                else {
                    rr |= rb << src_bit[b];
                    cc |= cb << src_bit[b];
                }
            }
            if (same_extra) M3[r * 8 + c] = M[(size_t)rr * D + cc];
        }
}

// Digit fragments of a complex D x D matrix in mma.m16n8k16 A-operand order.
void tc_fragments(int k, const std::vector<svp::cd>& M, std::vector<Word16>& out) {
    const int D = 1 << k, R = 2 * D, MT = R / 16, KT = R / 16;
    std::vector<int64_t> q((size_t)R * R);
    for (int r = 0; r < R; r++)
        for (int c = 0; c < R; c++) {
            const svp::cd u = M[(size_t)(r % D) * D + (c % D)];
            double v;
            if (r < D) v = c < D ? u.real() : -u.imag();
            else v = c < D ? u.imag() : u.real();
            q[(size_t)r * R + c] = q62_of(v);
        }
    const int db = 8, nd = 7;  // tensor-core blocks have at most 4 qubits
    auto A = [&](int i, int row, int col) { return bf16_of_digit(tc_digit(q[(size_t)row * R + col], i, db)); };
    for (int i = 0; i < nd; i++)
        for (int mt = 0; mt < MT; mt++)
            for (int ks = 0; ks < KT; ks++)
                for (int lane = 0; lane < 32; lane++) {
                    const int g = lane >> 2, t = lane & 3, r0 = mt * 16 + g, c0 = ks * 16 + 2 * t;
                    Word16 w;
                    w.w[0] = A(i, r0, c0) | (A(i, r0, c0 + 1) << 16);
                    w.w[1] = A(i, r0 + 8, c0) | (A(i, r0 + 8, c0 + 1) << 16);
                    w.w[2] = A(i, r0, c0 + 8) | (A(i, r0, c0 + 9) << 16);
                    w.w[3] = A(i, r0 + 8, c0 + 8) | (A(i, r0 + 8, c0 + 9) << 16);
                    out.push_back(w);
                }
}

// Balanced digits of a Q62 value for the tensor-memory kernel: v = q >> 6 =
// sum_j d_j 256^(6 - j), d_0 = (v + 0x808080808080) >> 48, d_j = byte 6 - j
// of v + 0x808080808080 minus 128 (so |d_0| <= 256, d_j in [-128, 127]).
void balanced_digits(int64_t q, int (&d)[7]) {
    const int64_t u = (q >> 6) + 0x808080808080ll;
    d[0] = (int)(u >> 48);
    for (int j = 1; j < 7; j++) d[j] = (int)((u >> (8 * (6 - j))) & 255) - 128;
}

// float16 bits of an integer |d| < 2^11 (exact).
uint16_t f16_of_int(int d) {
    if (d == 0) return 0;
    const unsigned a = (unsigned)(d < 0 ? -d : d);
    int e = 31 - __builtin_clz(a);  // 2^e <= a < 2^(e+1)
    const unsigned mant = (a << (10 - e)) & 0x3FFu;
    return (uint16_t)((d < 0 ? 0x8000u : 0u) | ((unsigned)(e + 15) << 10) | mant);
}

// Block digits in the shared-memory image the tcgen05 kernel copies: B is
// 7R x R fp16, row j R + r' = digit j of real-form row r (r' = (amp >> 2) 8 +
// part 4 + (amp & 3) for output part 0 = re / 1 = im of amplitude amp); the
// K position of real-form column c = cp D + ca is k' = 8 (ca >> 2) + 4 cp +
// (ca & 3), the order in which the kernel stores amplitude digits in tensor
// memory; K-major core matrices of 8 rows x 16 bytes (128 bytes between core
// matrices along K, 16 R bytes along N).  Returns
// false if some level sum could exceed 2^22 in magnitude (amplitude digits
// bounded by 256 for the top digit and 128 for the others).
bool t05_block_image(int k, const std::vector<svp::cd>& M, std::vector<Word16>& out) {
    const int D = 1 << k, R = 2 * D, SBO = 16 * R;
    std::vector<uint16_t> img((size_t)7 * R * R, 0);
    bool ok = true;
    for (int r = 0; r < R; r++) {
        const int part = r / D, amp = r % D;
        const int rp = (amp >> 2) * 8 + part * 4 + (amp & 3);
        int64_t S[7] = {0, 0, 0, 0, 0, 0, 0};
        for (int c = 0; c < R; c++) {
            const svp::cd u = M[(size_t)amp * D + (c % D)];
            double v;
            if (part == 0) v = c < D ? u.real() : -u.imag();
            else v = c < D ? u.imag() : u.real();
            int d[7];
            balanced_digits(q62_of(v), d);
            // K position of real-form column c (component cp of amplitude ca):
            // k' = 8 (ca >> 2) + 4 cp + (ca & 3)
            const int cp = c / D, ca = c % D;
            const int kq = 8 * (ca >> 2) + 4 * cp + (ca & 3);
            for (int j = 0; j < 7; j++) {
                S[j] += d[j] < 0 ? -d[j] : d[j];
                const int n = j * R + rp;
                const size_t off = (size_t)(n >> 3) * SBO + (size_t)(kq >> 3) * 128 + (n & 7) * 16 + (kq & 7) * 2;
                img[off / 2] = f16_of_int(d[j]);
            }
        }
        for (int L = 0; L < 7; L++) {
            int64_t b = 0;
            for (int i = 0; i <= L; i++) b += (i == 0 ? 256 : 128) * S[L - i];
            if (b > (1ll << 22)) ok = false;
        }
    }
    const size_t words = img.size() * 2 / sizeof(Word16);
    const size_t at = out.size();
    out.resize(at + words);
    std::memcpy(out.data() + at, img.data(), img.size() * 2);
    return ok;
}

// inject_stall (tests only): the first dense tensor-memory block issues no
// MMAs, so its bounded wait runs out (OPF_TEST_NO_MMA).
// Block parts for the complex64 tensor-core kernel: B is 3R x R bf16, row
// j R + r' = part j of real-form row r (x = h + m + l, h = bf16(x),
// m = bf16(x - h), l = bf16(x - h - m), from the float64 entry), with
// r' = (amp / P) 2P + part P + (amp mod P), P = D / 4; real-form column
// c = cp D + ca sits at K position k' = 2P (ca / P) + P cp + (ca mod P), the
// order in which the kernel stores amplitude parts in tensor memory; K-major
// core matrices of 8 rows x 16 bytes (128 bytes between core matrices along
// K, 16 R bytes along N).
uint16_t bf16_rn(double x) {
    float f = (float)x;  // float64 -> float32 -> bfloat16, both to nearest (the parts below
    uint32_t u;          // absorb the double rounding: x - h is formed from x itself)
    std::memcpy(&u, &f, 4);
    u += 0x7FFFu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}
double bf16_value(uint16_t b) {
    const uint32_t u = (uint32_t)b << 16;
    float f;
    std::memcpy(&f, &u, 4);
    return (double)f;
}
void t32_block_image(int k, const std::vector<svp::cd>& M, std::vector<Word16>& out) {
    const int D = 1 << k, R = 2 * D, SBO = 16 * R, Pq = D / 4;
    std::vector<uint16_t> img((size_t)3 * R * R, 0);
    for (int r = 0; r < R; r++) {
        const int part = r / D, amp = r % D;
        const int rp = (amp / Pq) * 2 * Pq + part * Pq + (amp % Pq);
        for (int c = 0; c < R; c++) {
            const svp::cd u = M[(size_t)amp * D + (c % D)];
            double v;
            if (part == 0) v = c < D ? u.real() : -u.imag();
            else v = c < D ? u.imag() : u.real();
            const uint16_t h = bf16_rn(v);
            const double r1 = v - bf16_value(h);
            const uint16_t m = bf16_rn(r1);
            const uint16_t l = bf16_rn(r1 - bf16_value(m));
            const uint16_t parts[3] = {h, m, l};
            for (int j = 0; j < 3; j++) {
                const int n = j * R + rp;
                const int cp = c / D, ca = c % D;
                const int kq = 2 * Pq * (ca / Pq) + Pq * cp + (ca % Pq);  // K order of the amplitude parts in TMEM
                img[((size_t)(n >> 3) * SBO + (size_t)(kq >> 3) * 128 + (n & 7) * 16 + (kq & 7) * 2) / 2] = parts[j];
            }
        }
    }
    const size_t at = out.size();
    out.resize(at + img.size() * 2 / sizeof(Word16));
    std::memcpy(out.data() + at, img.data(), img.size() * 2);
}

void lower(const svp::Plan& P, Lowered& L, int arith = SV_ARITH_NATIVE, bool inject_stall = false,
           int dt = SV_C128) {
    L.passes.clear();
    L.ops.clear();
    L.coef.clear();
    L.tc.clear();
    L.is_tc = is_tc(arith);
    L.tc_ok = true;
    const bool t05 = arith == SV_ARITH_TC;  // tcgen05 (complex128 digits or complex64 triple split)
    const bool c64 = dt == SV_C64;
    auto block_digits = [&](int k, const std::vector<svp::cd>& M) {
        if (c64) t32_block_image(k, M, L.tc);
        else if (t05) L.tc_ok = t05_block_image(k, M, L.tc) && L.tc_ok;
        else tc_fragments(k, M, L.tc);
    };
    for (const auto& ps : P.passes) {
        DevPass dp;
        std::memset(&dp, 0, sizeof(dp));
        dp.n = P.n;
        dp.m = ps.m;
        dp.c = std::min(P.coalesce, ps.m);
        dp.tile_count = 1ull << (P.n - ps.m);
        int pos_of[64];
        int nl = 0, li = 0;
        for (int q = 0; q < P.n; q++) {
            if ((ps.local_mask >> q) & 1) {
                pos_of[q] = li;
                dp.L[li++] = (int8_t)q;
            } else {
                pos_of[q] = -1;
                dp.NL[nl++] = (int8_t)q;
            }
        }
        dp.op0 = (int32_t)L.ops.size();
        // one op per block; a permutation block with other than quarter phases
        // adds a diagonal op after it, and a Kronecker block outside the
        // tensor-core modes becomes one butterfly per qubit
        auto emit_diag = [&](DevOp op, const std::vector<svp::cd>& d, bool sign_only) {
            op.kind = svk::OP_DIAG;
            op.flags = sign_only ? svk::OPF_SIGN_ONLY : 0;
            if (L.is_tc) {
                op.coeff = (int32_t)L.tc.size();
                if (c64) {  // float pairs, two entries per 16 bytes
                    for (size_t e = 0; e < d.size(); e += 2) {
                        float f[4] = {(float)d[e].real(), (float)d[e].imag(), 0.f, 0.f};
                        if (e + 1 < d.size()) {
                            f[2] = (float)d[e + 1].real();
                            f[3] = (float)d[e + 1].imag();
                        }
                        Word16 w;
                        std::memcpy(&w, f, 16);
                        L.tc.push_back(w);
                    }
                } else {
                    for (const auto& u : d) {
                        const int64_t re = q62_of(u.real()), im = q62_of(u.imag());
                        Word16 w;
                        std::memcpy(&w.w[0], &re, 8);
                        std::memcpy(&w.w[2], &im, 8);
                        L.tc.push_back(w);
                    }
                }
            } else {
                op.coeff = (int32_t)L.coef.size();
                L.coef.insert(L.coef.end(), d.begin(), d.end());
            }
            L.ops.push_back(op);
        };
        auto emit_dense = [&](DevOp op, int k, const std::vector<svp::cd>& M) {
            op.kind = svk::OP_DENSE;
            op.k = k;
            op.flags = 0;
            if (L.is_tc) {
                op.coeff = (int32_t)L.tc.size();
                if (k < 3) {
                    int pos3[3];
                    std::vector<svp::cd> M3;
                    const uint64_t avail = ((1ull << ps.m) - 1);
                    extend_to3(k, op.pos, M, avail, pos3, M3);
                    op.k = 3;
                    for (int j = 0; j < 3; j++) op.pos[j] = pos3[j];
                    block_digits(3, M3);
                } else {
                    block_digits(k, M);
                }
            } else {
                op.coeff = (int32_t)L.coef.size();
                L.coef.insert(L.coef.end(), M.begin(), M.end());
            }
            if (inject_stall && t05) {
                op.flags |= svk::OPF_TEST_NO_MMA;
                inject_stall = false;
            }
            L.ops.push_back(op);
            dp.kmax = std::max(dp.kmax, (int32_t)op.k);
        };
        // permutation: the rows in cycle order, one coefficient element each
        // holding dst | quarter-phase code << 5 | end-of-cycle << 7 (an exact
        // small integer in every coefficient format)
        auto emit_perm = [&](DevOp op, const svp::Block& b) {
            op.kind = svk::OP_PERM;
            op.flags = 0;
            const int D = 1 << b.k;
            std::vector<int> moves;
            std::vector<char> seen(D, 0);
            for (int a0 = 0; a0 < D; a0++) {
                if (seen[a0]) continue;
                int a = a0;
                for (;;) {
                    seen[a] = 1;
                    const int nx = b.src[a];
                    int code = 0;
                    if (b.quarter) {
                        const svp::cd v = b.phase[a];
                        code = v.real() == 1.0 ? 0 : v.imag() == 1.0 ? 1 : v.real() == -1.0 ? 2 : 3;
                    }
                    moves.push_back(a | (code << 5) | (nx == a0 ? 128 : 0));
                    if (nx == a0) break;
                    a = nx;
                }
            }
            if (L.is_tc) {
                op.coeff = (int32_t)L.tc.size();
                for (int v : moves) L.tc.push_back(Word16{{(uint32_t)v, 0u, 0u, 0u}});
            } else {
                op.coeff = (int32_t)L.coef.size();
                for (int v : moves) L.coef.push_back(svp::cd((double)v, 0.0));
            }
            L.ops.push_back(op);
            if (!b.quarter) emit_diag(op, b.phase, false);
        };
        for (int bi : ps.blocks) {
            const svp::Block& b = P.blocks[bi];
            DevOp op;
            std::memset(&op, 0, sizeof(op));
            op.k = b.k;
            for (int j = 0; j < b.k; j++) {
                op.pos[j] = pos_of[b.qubits[j]];
                op.qbit[j] = b.qubits[j];
            }
            if (b.kind == svp::BK_DIAG) {
                emit_diag(op, b.mat, b.sign_only);
            } else if (b.kind == svp::BK_PERM) {
                emit_perm(op, b);
            } else if (b.kind == svp::BK_KRON && !L.is_tc) {
                for (int j = 0; j < b.k; j++) {
                    DevOp o1;
                    std::memset(&o1, 0, sizeof(o1));
                    o1.pos[0] = pos_of[b.qubits[j]];
                    o1.qbit[0] = b.qubits[j];
                    emit_dense(o1, 1, std::vector<svp::cd>(b.factors.begin() + 4 * j, b.factors.begin() + 4 * j + 4));
                }
            } else {
                emit_dense(op, b.k, b.mat);
            }
        }
        if (dp.kmax < 1) dp.kmax = 1;
        dp.n_ops = (int32_t)(L.ops.size() - dp.op0);
        L.passes.push_back(dp);
    }
    if (t05 && !c64) {  // complex128 digits: the state stays in Q56 between the circuit's passes
        const size_t np = L.passes.size();
        for (size_t i = 0; i < np; i++)
            L.passes[i].io = (i > 0 ? svk::IO_LOAD_Q56 : 0) | (i + 1 < np ? svk::IO_STORE_Q56 : 0);
    }
}

cudaError_t ensure(void** p, size_t* cap, size_t need, bool pinned) {
    if (*cap >= need && *p) return cudaSuccess;
    size_t ncap = std::max(need, (size_t)1 << 16);
    if (*p) {
        if (pinned) cudaFreeHost(*p);
        else cudaFree(*p);
        *p = nullptr;
        *cap = 0;
    }
    cudaError_t e = pinned ? cudaMallocHost(p, ncap) : cudaMalloc(p, ncap);
    if (e == cudaSuccess) *cap = ncap;
    return e;
}

double now_ms() {
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

// Writes block coefficients in the kernel's format: complex64 -> float pairs,
// complex128 native -> double pairs, complex128 df64 -> (hi, lo) float pairs.
size_t coef_elem_bytes(int dt) { return dt == SV_C64 ? 8 : 16; }

void write_coefs(const std::vector<svp::cd>& coef, int dt, int arith, unsigned char* dst) {
    if (dt == SV_C64) {
        auto* c = (float*)dst;
        for (size_t i = 0; i < coef.size(); i++) {
            c[2 * i] = (float)coef[i].real();
            c[2 * i + 1] = (float)coef[i].imag();
        }
    } else if (arith == SV_ARITH_DF64) {
        auto* c = (float*)dst;  // hi = float(x), lo = float(x - hi)
        for (size_t i = 0; i < coef.size(); i++) {
            const double re = coef[i].real(), im = coef[i].imag();
            const float rh = (float)re, ih = (float)im;
            c[4 * i] = rh;
            c[4 * i + 1] = (float)(re - (double)rh);
            c[4 * i + 2] = ih;
            c[4 * i + 3] = (float)(im - (double)ih);
        }
    } else {
        auto* c = (double*)dst;
        for (size_t i = 0; i < coef.size(); i++) {
            c[2 * i] = coef[i].real();
            c[2 * i + 1] = coef[i].imag();
        }
    }
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

size_t coef_bytes(const Lowered& L, int dt) {
    return L.is_tc ? L.tc.size() * sizeof(Word16) : L.coef.size() * coef_elem_bytes(dt);
}

// Internal status: a tensor-core block failed the exact-range check (the
// caller re-plans in double-float arithmetic).
constexpr int kRetryDF64 = 1;

int apply_plan(sv_state* s, const svp::Plan& P, int arith, bool timing, bool inject_stall = false) {
    Lowered L;
    lower(P, L, arith, inject_stall, s->dt);
    if (!L.tc_ok) return kRetryDF64;
    const size_t ops_bytes = L.ops.size() * sizeof(DevOp);
    const size_t coef_off = align256(ops_bytes);
    const size_t ent_off = align256(coef_off + coef_bytes(L, s->dt));
    const size_t total = ent_off + L.passes.size() * sizeof(svk::BatchEntry);
    SV_TRY(ensure(&s->d_ws, &s->d_ws_cap, total, false));
    SV_TRY(ensure(&s->h_ws, &s->h_ws_cap, total, true));
    auto* h = (unsigned char*)s->h_ws;
    if (ops_bytes) std::memcpy(h, L.ops.data(), ops_bytes);
    if (L.is_tc) {
        if (!L.tc.empty()) std::memcpy(h + coef_off, L.tc.data(), L.tc.size() * sizeof(Word16));
    } else {
        write_coefs(L.coef, s->dt, arith, h + coef_off);
    }
    auto* ent = (svk::BatchEntry*)(h + ent_off);
    for (size_t i = 0; i < L.passes.size(); i++) {
        ent[i].state = (uint64_t)(uintptr_t)s->amp;
        ent[i].tile_begin = 0;
        ent[i].p = L.passes[i];
    }
    SV_TRY(cudaMemcpyAsync(s->d_ws, s->h_ws, total, cudaMemcpyHostToDevice, s->stream));
    s->last.upload_bytes = (double)total;
    const auto* d_ops = (const DevOp*)s->d_ws;
    const void* d_coef = (const unsigned char*)s->d_ws + coef_off;
    const auto* d_ent = (const svk::BatchEntry*)((const unsigned char*)s->d_ws + ent_off);
    int launches = 0;
    if (timing) {
        while (s->events.size() < L.passes.size() + 1) {
            cudaEvent_t e;
            SV_TRY(cudaEventCreate(&e));
            s->events.push_back(e);
        }
        SV_TRY(cudaEventRecord(s->events[0], s->stream));
    }
    for (size_t i = 0; i < L.passes.size(); i++) {
        const DevPass& dp = L.passes[i];
        SV_TRY(svk::launch_tile_pass(s->dt, arith, d_ent + i, 1, dp.tile_count, dp.m, dp.kmax, d_ops, d_coef,
                                     s->stream, s->di));
        launches++;
        if (timing) SV_TRY(cudaEventRecord(s->events[launches], s->stream));
    }
    SV_TRY(cudaStreamSynchronize(s->stream));
    if (arith == SV_ARITH_TC) {
        int fault = 0;
        SV_TRY(svk::tc_fault_take(&fault));
        if (fault) {
            s->failed = true;
            return SV_ERR_TIMEOUT;
        }
    }
    s->last.n_launches = launches;
    s->last.kernel_ms = 0;
    s->last.max_kernel_ms = 0;
    for (int i = 0; timing && i < launches; i++) {
        float ms = 0;
        SV_TRY(cudaEventElapsedTime(&ms, s->events[i], s->events[i + 1]));
        s->last.kernel_ms += ms;
        s->last.max_kernel_ms = std::max(s->last.max_kernel_ms, (double)ms);
    }
    return SV_OK;
}

}  // namespace

extern "C" {

size_t sv_state_bytes(int n, int dt) {
    if (n < 1 || n > svp::kMaxQubits || !dt_ok(dt)) return 0;
    return ((size_t)1 << n) * (size_t)amp_bytes(dt);
}

static int create_common(int n, int dt, sv_state** out, sv_state** made) {
    if (!out || n < 1 || n > svp::kMaxQubits || !dt_ok(dt)) return SV_ERR_ARG;
    sv_state* s = new (std::nothrow) sv_state();
    if (!s) return SV_ERR_OOM;
    s->n = n;
    s->dt = dt;
    s->bytes = sv_state_bytes(n, dt);
    cudaError_t e = device_info(&s->di);
    if (e != cudaSuccess) {
        delete s;
        return SV_ERR_CUDA;
    }
    *made = s;
    return SV_OK;
}

int sv_create(int n, int dt, sv_state** out) {
    sv_state* s = nullptr;
    int rc = create_common(n, dt, out, &s);
    if (rc) return rc;
    size_t fr = 0, to = 0;
    if (cudaMemGetInfo(&fr, &to) == cudaSuccess && s->bytes > fr) {
        delete s;
        return SV_ERR_OOM;
    }
    cudaError_t e = cudaMalloc(&s->amp, s->bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete s;
        return e == cudaErrorMemoryAllocation ? SV_ERR_OOM : SV_ERR_CUDA;
    }
    s->owned = true;
    e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        cudaFree(s->amp);
        delete s;
        return SV_ERR_CUDA;
    }
    s->own_stream = true;
    rc = sv_reset(s, 0);
    if (rc) {
        sv_destroy(s);
        return rc;
    }
    *out = s;
    return SV_OK;
}

int sv_create_on(void* dev_ptr, size_t bytes, int n, int dt, void* stream, sv_state** out) {
    if (!dev_ptr || ((uintptr_t)dev_ptr & 15)) return SV_ERR_ARG;
    if (bytes != sv_state_bytes(n, dt)) return SV_ERR_SIZE;
    sv_state* s = nullptr;
    int rc = create_common(n, dt, out, &s);
    if (rc) return rc;
    s->amp = dev_ptr;
    s->owned = false;
    s->stream = (cudaStream_t)stream;
    s->own_stream = false;
    s->foreign = true;
    *out = s;
    return SV_OK;
}

int sv_rebind(sv_state* s, void* dev_ptr, size_t bytes, int n, int dt) {
    if (!s || s->owned || !dev_ptr || ((uintptr_t)dev_ptr & 15)) return SV_ERR_ARG;
    if (n < 1 || n > svp::kMaxQubits || !dt_ok(dt)) return SV_ERR_ARG;
    if (bytes != sv_state_bytes(n, dt)) return SV_ERR_SIZE;
    if (s->stream) SV_TRY(cudaStreamSynchronize(s->stream));
    s->amp = dev_ptr;
    s->n = n;
    s->dt = dt;
    s->bytes = bytes;
    s->failed = false;
    s->foreign = true;
    s->last = sv_apply_stats{};
    return SV_OK;
}

void sv_destroy(sv_state* s) {
    if (!s) return;
    if (s->stream) cudaStreamSynchronize(s->stream);
    if (s->owned && s->amp) cudaFree(s->amp);
    if (s->d_ws) cudaFree(s->d_ws);
    if (s->h_ws) cudaFreeHost(s->h_ws);
    if (s->d_red) cudaFree(s->d_red);
    for (cudaEvent_t e : s->events) cudaEventDestroy(e);
    if (s->own_stream && s->stream) cudaStreamDestroy(s->stream);
    delete s;
}

int sv_num_qubits(const sv_state* s) { return s ? s->n : SV_ERR_ARG; }
int sv_dtype_of(const sv_state* s) { return s ? s->dt : SV_ERR_ARG; }
void* sv_device_ptr(const sv_state* s) { return s ? s->amp : nullptr; }

int sv_reset(sv_state* s, uint64_t basis) {
    if (!s) return SV_ERR_ARG;
    if (basis >> s->n) return SV_ERR_ARG;
    SV_TRY(svk::launch_init(s->dt, s->amp, s->n, basis, s->stream, s->di));
    SV_TRY(cudaStreamSynchronize(s->stream));
    s->failed = false;
    s->foreign = false;
    return SV_OK;
}

int sv_apply_circuit(sv_state* s, const sv_gate* g, size_t ng, const sv_run_opts* o) {
    if (!s) return SV_ERR_ARG;
    if (s->failed) return SV_ERR_STATE;
    int rc = svp::validate(s->n, g, ng);
    if (rc) return rc;
    if (ng == 0) return SV_OK;
    const double t0 = now_ms();
    svp::Plan P = plan_for(s->n, s->dt, g, ng, o, max_tile(s->dt, s->di));
    if (o && (o->debug_checks & 1) && svp::check_plan(P, ng, g) != 0) return SV_ERR_STATE;
    const double t1 = now_ms();
    int arith = resolve_arith(s->dt, o, s->n);
    if (s->dt == SV_C128 && is_tc(arith) && s->foreign) {
        // caller-supplied amplitudes: the fixed-point tile needs every component
        // of every state the circuit passes through to stay within [-1, 1].  A
        // norm of at most 1 guarantees it (the blocks are unitary, so the norm
        // is kept and bounds every component); a bound on the components alone
        // does not (one Hadamard takes (1, 1) to (sqrt 2, 0)).  The max-abs pass
        // comes first so that the exact fixed-point norm, pre-scaled by 2^-36,
        // cannot overflow (at most 2^34 terms of at most 2 each).
        SV_TRY(ensure(&s->d_red, &s->d_red_cap, svk::norm_scratch_bytes(s->di) + 256, false));
        SV_TRY(svk::launch_max_abs_c128(s->amp, s->n, (unsigned long long*)s->d_red, s->stream, s->di));
        unsigned long long bits = 0;
        SV_TRY(cudaMemcpyAsync(&bits, s->d_red, 8, cudaMemcpyDeviceToHost, s->stream));
        SV_TRY(cudaStreamSynchronize(s->stream));
        double mx;
        std::memcpy(&mx, &bits, 8);
        bool ok = mx <= 1.0;
        if (ok) {
            const size_t scratch = svk::norm_scratch_bytes(s->di);
            double* d_out = (double*)((unsigned char*)s->d_red + scratch);
            double nrm = 0;
            SV_TRY(svk::launch_norm(s->dt, s->amp, s->n, s->d_red, d_out, s->stream, s->di, kGateDown));
            SV_TRY(cudaMemcpyAsync(&nrm, d_out, sizeof(double), cudaMemcpyDeviceToHost, s->stream));
            SV_TRY(cudaStreamSynchronize(s->stream));
            // a float64-normalised state may exceed 1 by rounding; 2^-40 of slack
            // keeps components below 1 + 2^-41, far inside the digits' range
            ok = std::ldexp(nrm, kGateDown) <= 1.0 + std::ldexp(1.0, -40);
        }
        if (ok) s->foreign = false;  // evolution by unitaries keeps the norm
        else arith = SV_ARITH_DF64;
    }
    if (arith != resolve_arith(s->dt, o, s->n)) {  // re-plan for double-float arithmetic
        sv_run_opts df = o ? *o : sv_run_opts{};
        df.arith = SV_ARITH_DF64;
        P = plan_for(s->n, s->dt, g, ng, &df, max_tile(s->dt, s->di));
    }
    rc = apply_plan(s, P, arith, o && o->timing, o && (o->debug_checks & 2));
    if (rc == kRetryDF64) {  // a block outside the digit scheme's exact range
        sv_run_opts df = o ? *o : sv_run_opts{};
        df.arith = SV_ARITH_DF64;
        arith = SV_ARITH_DF64;
        P = plan_for(s->n, s->dt, g, ng, &df, max_tile(s->dt, s->di));
        rc = apply_plan(s, P, arith, o && o->timing);
    }
    s->last.n_blocks = (int32_t)P.blocks.size();
    s->last.n_passes = (int32_t)P.passes.size();
    s->last.fuse_k = P.fuse_k;
    s->last.tile_qubits = P.tile_m;
    s->last.arith = arith;
    s->last.flops = P.flops;
    s->last.alu_ops = P.alu_ops;
    s->last.tensor_flops = is_tc(arith) ? P.mma_flops : 0.0;
    s->last.hbm_bytes = 2.0 * (double)s->bytes * (double)P.passes.size();
    s->last.plan_ms = t1 - t0;
    return rc;
}

int sv_last_stats(const sv_state* s, sv_apply_stats* out) {
    if (!s || !out) return SV_ERR_ARG;
    *out = s->last;
    return SV_OK;
}

int sv_probabilities(sv_state* s, double* out, size_t out_len, int out_is_device) {
    if (!s || !out) return SV_ERR_ARG;
    if (s->failed) return SV_ERR_STATE;
    const uint64_t dim = 1ull << s->n;
    if (out_len != dim) return SV_ERR_SIZE;
    if (out_is_device) {
        SV_TRY(svk::launch_probs(s->dt, s->amp, 0, dim, out, s->stream, s->di));
        SV_TRY(cudaStreamSynchronize(s->stream));
        return SV_OK;
    }
    // page-locked host output mapped into the device's address space: the kernel
    // stores into it directly over the host link, no staging copy
    cudaPointerAttributes pa{};
    if (cudaPointerGetAttributes(&pa, out) == cudaSuccess && pa.type == cudaMemoryTypeHost && pa.devicePointer) {
        SV_TRY(svk::launch_probs(s->dt, s->amp, 0, dim, (double*)pa.devicePointer, s->stream, s->di));
        SV_TRY(cudaStreamSynchronize(s->stream));
        return SV_OK;
    }
    (void)cudaGetLastError();
    // pageable host output: through a bounded device staging buffer, chunk by chunk
    const uint64_t chunk = std::min<uint64_t>(dim, 1ull << 24);
    SV_TRY(ensure(&s->d_red, &s->d_red_cap, chunk * sizeof(double), false));
    for (uint64_t i0 = 0; i0 < dim; i0 += chunk) {
        const uint64_t len = std::min(chunk, dim - i0);
        SV_TRY(svk::launch_probs(s->dt, s->amp, i0, len, (double*)s->d_red, s->stream, s->di));
        SV_TRY(cudaMemcpyAsync(out + i0, s->d_red, len * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
        SV_TRY(cudaStreamSynchronize(s->stream));
    }
    return SV_OK;
}

int sv_marginal_probabilities(sv_state* s, uint64_t mask, double* out, size_t out_len, int out_is_device) {
    if (!s || !out) return SV_ERR_ARG;
    if (s->failed) return SV_ERR_STATE;
    if (s->n < 64 && (mask >> s->n)) return SV_ERR_QUBIT;
    const int k = __builtin_popcountll(mask);
    const uint64_t nbins = 1ull << k;
    if (out_len != nbins) return SV_ERR_SIZE;
    const size_t bins_bytes = 2 * 8 * nbins;
    const size_t need = bins_bytes + (out_is_device ? 0 : nbins * sizeof(double));
    SV_TRY(ensure(&s->d_red, &s->d_red_cap, need, false));
    double* d_out = out_is_device ? out : (double*)((unsigned char*)s->d_red + bins_bytes);
    SV_TRY(svk::launch_marginal(s->dt, s->amp, s->n, mask, s->d_red, d_out, s->stream, s->di));
    if (!out_is_device)
        SV_TRY(cudaMemcpyAsync(out, d_out, nbins * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    SV_TRY(cudaStreamSynchronize(s->stream));
    return SV_OK;
}

int sv_amplitudes(sv_state* s, void* out, size_t bytes, int out_is_device) {
    if (!s || !out) return SV_ERR_ARG;
    if (bytes != s->bytes) return SV_ERR_SIZE;
    SV_TRY(cudaMemcpyAsync(out, s->amp, bytes, out_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                           s->stream));
    SV_TRY(cudaStreamSynchronize(s->stream));
    return SV_OK;
}

int sv_set_amplitudes(sv_state* s, const void* in, size_t bytes, int in_is_device) {
    if (!s || !in) return SV_ERR_ARG;
    if (bytes != s->bytes) return SV_ERR_SIZE;
    SV_TRY(cudaMemcpyAsync(s->amp, in, bytes, in_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                           s->stream));
    SV_TRY(cudaStreamSynchronize(s->stream));
    s->failed = false;
    s->foreign = true;
    return SV_OK;
}

// ---- measured autotuner ---------------------------------------------------
namespace {

// A block of the given class on `qubits`, its matrix formed by the planner
// from a short gate list: dense = U3 on every qubit, a CZ chain, U3 again;
// diag = RZZ + RZ (general phases); sign = CZ; perm = a CX chain, a SWAP, X
// and Y (quarter phases).
svp::Block calibration_block(int kind, const std::vector<int>& q) {
    const int k = (int)q.size();
    std::vector<sv_gate> g;
    auto add = [&](int op, int q0, int q1, double t, double ph, double la) { g.push_back(sv_gate{op, q0, q1, t, ph, la}); };
    int bk = svp::BK_DENSE;
    if (kind == 0) {
        for (int j = 0; j < k; j++) add(SV_U3, q[j], -1, 0.4 + 0.3 * j, 0.7, -0.2 * j);
        for (int j = 0; j + 1 < k; j++) add(SV_CZ, q[j], q[j + 1], 0, 0, 0);
        for (int j = 0; j < k; j++) add(SV_U3, q[j], -1, 1.1 - 0.2 * j, -0.3, 0.5);
    } else if (kind == 1) {
        add(SV_RZZ, q[0], q[1], 0.37, 0, 0);
        add(SV_RZ, q[0], -1, 0.11, 0, 0);
        bk = svp::BK_DIAG;
    } else if (kind == 2) {
        add(SV_CZ, q[0], q[1], 0, 0, 0);
        bk = svp::BK_DIAG;
    } else {
        for (int j = 0; j + 1 < k; j++) add(SV_CX, q[j], q[j + 1], 0, 0, 0);
        if (k > 1) add(SV_SWAP, q[0], q[k - 1], 0, 0, 0);
        add(SV_X, q[0], -1, 0, 0, 0);
        if (k > 1) add(SV_Y, q[1], -1, 0, 0, 0);
        bk = svp::BK_PERM;
    }
    svp::Block b;
    b.kind = bk;
    for (int x : q) b.mask |= 1ull << x;
    b.k = 0;
    for (int x = 0; x < 64; x++)
        if ((b.mask >> x) & 1) b.qubits[b.k++] = x;
    for (size_t t = 0; t < g.size(); t++) b.gates.push_back((int)t);
    std::vector<svp::Block> v{b};
    svp::finalize(v, g.data());
    return v[0];
}

}  // namespace

extern "C" {

int sv_calibrate(int dt, int arith_req, sv_costs* out) {
    if (!out || !dt_ok(dt)) return SV_ERR_ARG;
    const int n = dt == SV_C64 ? 25 : 24;  // 256 MiB: above the L2
    sv_run_opts o{};
    o.arith = arith_req;
    const int arith = resolve_arith(dt, &o, n);
    sv_state* s = nullptr;
    int rc = sv_create(n, dt, &s);
    if (rc) return rc;
    const int m = std::min(default_tile(dt, arith), max_tile(dt, s->di));
    const int c = coalesce_of(dt);
    const double dim = std::ldexp(1.0, n);
    constexpr int kReps = 8;
    // kernel time of np passes over the tile qubits 0..m-1, the middle one
    // applying `mid`; the fastest of three runs
    auto time_plan = [&](int np, const std::vector<svp::Block>& mid, double* ms) -> int {
        svp::Plan P;
        P.n = n;
        P.fuse_k = svp::kMaxFuse;
        P.tile_m = m;
        P.coalesce = c;
        P.blocks = mid;
        for (int i = 0; i < np; i++) {
            svp::Pass ps;
            ps.local_mask = (1ull << m) - 1;
            ps.m = m;
            if (i == np / 2)
                for (size_t b = 0; b < mid.size(); b++) ps.blocks.push_back((int)b);
            P.passes.push_back(ps);
        }
        double best = 1e300;
        for (int rep = 0; rep < 3; rep++) {
            int r = sv_reset(s, 0);
            if (r == SV_OK) r = apply_plan(s, P, arith, true);
            if (r != SV_OK) return r;
            best = std::min(best, s->last.kernel_ms);
        }
        *ms = best;
        return SV_OK;
    };
    auto reps_of = [&](int kind, int k) {
        std::vector<svp::Block> v;
        for (int r = 0; r < kReps; r++) {  // alternately on the lowest and the highest tile qubits
            std::vector<int> q;
            for (int j = 0; j < k; j++) q.push_back((r & 1) ? m - k + j : j);
            v.push_back(calibration_block(kind, q));
        }
        return v;
    };
    sv_costs C;
    std::memset(&C, 0, sizeof(C));
    C.dt = dt;
    C.arith = arith;
    C.n_qubits = n;
    C.tile_qubits = m;
    double t2 = 0, t3 = 0, t = 0;
    const std::vector<svp::Block> none;
    const double ps_per_ms = 1e9 / dim;  // ms over the whole state -> ps per amplitude
    auto per_op = [&](double tm) { return std::max(0.0, (tm - t3) * ps_per_ms / kReps); };
    rc = time_plan(2, none, &t2);
    if (rc == SV_OK) rc = time_plan(3, none, &t3);
    if (rc == SV_OK) C.pass_ps = std::max(0.0, (t3 - t2) * ps_per_ms);
    const int kmax = (dt == SV_C128 && arith == SV_ARITH_TC) ? 4 : 5;
    for (int k = 1; k <= 5 && rc == SV_OK; k++) {
        if (k <= kmax) {
            rc = time_plan(3, reps_of(0, k), &t);
            if (rc == SV_OK) C.dense_ps[k] = per_op(t);
        }
        if (rc == SV_OK) rc = time_plan(3, reps_of(3, k), &t);
        if (rc == SV_OK) C.perm_ps[k] = per_op(t);
    }
    if (rc == SV_OK) rc = time_plan(3, reps_of(1, 2), &t);
    if (rc == SV_OK) C.diag_ps = per_op(t);
    if (rc == SV_OK) rc = time_plan(3, reps_of(2, 2), &t);
    if (rc == SV_OK) C.sign_ps = per_op(t);
    sv_destroy(s);
    if (rc == SV_OK) *out = C;
    return rc;
}

int sv_set_costs(int dt, int arith, const sv_costs* costs) {
    if (!dt_ok(dt)) return SV_ERR_ARG;
    if (arith != SV_ARITH_NATIVE && arith != SV_ARITH_DF64 && arith != SV_ARITH_TC && arith != SV_ARITH_TC_SYNC)
        return SV_ERR_ARG;
    std::lock_guard<std::mutex> lk(g_costs_mu);
    if (!costs) {
        g_costs.erase({dt, arith});
        return SV_OK;
    }
    if (!(costs->pass_ps >= 0)) return SV_ERR_ARG;
    g_costs[{dt, arith}] = *costs;
    return SV_OK;
}

}  // extern "C"

int sv_norm(sv_state* s, double* out) {
    if (!s || !out) return SV_ERR_ARG;
    if (s->failed) return SV_ERR_STATE;
    const size_t scratch = svk::norm_scratch_bytes(s->di);
    SV_TRY(ensure(&s->d_red, &s->d_red_cap, scratch + 256, false));
    double* d_out = (double*)((unsigned char*)s->d_red + scratch);
    SV_TRY(svk::launch_norm(s->dt, s->amp, s->n, s->d_red, d_out, s->stream, s->di));
    SV_TRY(cudaMemcpyAsync(out, d_out, sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    SV_TRY(cudaStreamSynchronize(s->stream));
    return SV_OK;
}

}  // extern "C"

struct sv_batch {
    svk::DevInfo di;
    cudaStream_t stream = nullptr;
    void* arena = nullptr;      // states, device-side probabilities, descriptors
    size_t arena_bytes = 0;
    bool own_arena = true;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    int n_items = 0, n_launches = 0;
    double last_ms = 0;
    struct HostCopy {
        double* dst;
        size_t off, bytes;
    };
    std::vector<HostCopy> host_copies;
};

namespace {

struct BatchItemPlan {
    int idx, n, dt, arith;
    svp::Plan plan;
    Lowered low;
    size_t state_off = 0, probs_off = 0;  // in the arena
    bool host_out = false;
};

void batch_free(sv_batch* b) {
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->arena && b->own_arena) cudaFree(b->arena);
    for (auto& e : b->ev)
        if (e) cudaEventDestroy(e);
    if (b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

}  // namespace

extern "C" {

// Builds a batch; with ext_arena == nullptr it allocates its own arena, with
// size_only it only reports the arena size in *size_out.
static int batch_build(const sv_batch_item* items, size_t n_items, const sv_run_opts* opts, int* item_status,
                       void* ext_arena, size_t ext_bytes, bool size_only, size_t* size_out, sv_batch** out) {
    if ((!out && !size_only) || (n_items && !items)) return SV_ERR_ARG;
    sv_batch* b = new (std::nothrow) sv_batch();
    if (!b) return SV_ERR_OOM;
    sv_state* s = nullptr;  // for SV_TRY
    auto fail = [&](int rc) {
        batch_free(b);
        return rc;
    };
    if (device_info(&b->di) != cudaSuccess) return fail(SV_ERR_CUDA);
    // plan every item on its own
    std::vector<BatchItemPlan> P;
    P.reserve(n_items);
    for (size_t i = 0; i < n_items; i++) {
        const sv_batch_item& it = items[i];
        int rc = SV_OK;
        if (it.n_qubits < 1 || it.n_qubits > svp::kMaxQubits || !dt_ok(it.dt) || !it.probs_out) rc = SV_ERR_ARG;
        if (rc == SV_OK) rc = svp::validate(it.n_qubits, it.gates, it.n_gates);
        if (item_status) item_status[i] = rc;
        if (rc != SV_OK) continue;
        BatchItemPlan bp;
        bp.idx = (int)i;
        bp.n = it.n_qubits;
        bp.dt = it.dt;
        bp.arith = resolve_arith(it.dt, opts, it.n_qubits);
        bp.plan = plan_for(it.n_qubits, it.dt, it.gates, it.n_gates, opts, max_tile(it.dt, b->di));
        lower(bp.plan, bp.low, bp.arith, false, bp.dt);
        if (!bp.low.tc_ok) {  // a block outside the digit scheme's exact range: double-float
            sv_run_opts df = opts ? *opts : sv_run_opts{};
            df.arith = SV_ARITH_DF64;
            bp.arith = SV_ARITH_DF64;
            bp.plan = plan_for(it.n_qubits, it.dt, it.gates, it.n_gates, &df, max_tile(it.dt, b->di));
            lower(bp.plan, bp.low, bp.arith, false, bp.dt);
        }
        bp.host_out = !it.probs_on_device;
        P.push_back(std::move(bp));
    }
    b->n_items = (int)P.size();
    // arena layout: states | device-side probabilities (host outputs) | ops | coefs | entries
    size_t off = 0;
    for (auto& bp : P) {
        bp.state_off = off;
        off += align256(sv_state_bytes(bp.n, bp.dt));
    }
    for (auto& bp : P) {
        if (!bp.host_out) continue;
        bp.probs_off = off;
        off += align256(((size_t)8) << bp.n);
    }
    // group by kernel mode (dtype, arithmetic): kBatchModes values of mode_of
    constexpr int kBatchModes = 6;
    auto mode_of = [](const BatchItemPlan& bp) {
        if (bp.dt == SV_C64) return bp.arith == SV_ARITH_TC ? 5 : 0;
        if (bp.arith == SV_ARITH_DF64) return 2;
        if (bp.arith == SV_ARITH_TC) return 3;
        return bp.arith == SV_ARITH_TC_SYNC ? 4 : 1;
    };
    std::vector<DevOp> ops;
    std::vector<unsigned char> coefs;  // per-mode coefficient blobs, concatenated
    struct Launch {
        int mode, dt, arith, n_ent, max_m, kmax;
        size_t ent_index;
        uint64_t tiles;
    };
    std::vector<Launch> launches;
    std::vector<svk::BatchEntry> entries;
    std::vector<svk::StateEntry> sentries;
    struct SLaunch {
        int dt;
        size_t first;
        int count;
        uint64_t amps;
    };
    std::vector<SLaunch> slaunch;
    std::vector<size_t> coef_base(P.size(), 0), op_base(P.size(), 0);
    for (size_t i = 0; i < P.size(); i++) {
        auto& bp = P[i];
        op_base[i] = ops.size();
        for (auto op : bp.low.ops) ops.push_back(op);
        // coefficient offsets are in elements; keep each item's blob aligned to its element size
        const size_t esz = bp.low.is_tc ? sizeof(Word16) : coef_elem_bytes(bp.dt);  // unit of op.coeff
        size_t cb = (coefs.size() + esz - 1) / esz * esz;
        coefs.resize(cb + coef_bytes(bp.low, bp.dt));
        if (bp.low.is_tc) {
            if (!bp.low.tc.empty()) std::memcpy(coefs.data() + cb, bp.low.tc.data(), bp.low.tc.size() * sizeof(Word16));
        } else {
            write_coefs(bp.low.coef, bp.dt, bp.arith, coefs.data() + cb);
        }
        coef_base[i] = cb;
    }
    const size_t ops_off = off;
    off += align256(ops.size() * sizeof(DevOp) + 16);
    const size_t coef_off = off;
    off += align256(coefs.size() + 16);
    // multi-state launches per (mode, pass index); the op/coef offsets inside each
    // entry's pass point at the item's ops; coefficient offsets are rebased below
    for (int mode = 0; mode < kBatchModes; mode++) {
        size_t max_passes = 0;
        std::vector<size_t> members;
        for (size_t i = 0; i < P.size(); i++)
            if (mode_of(P[i]) == mode) {
                members.push_back(i);
                max_passes = std::max(max_passes, P[i].low.passes.size());
            }
        if (members.empty()) continue;
        SLaunch sl{P[members[0]].dt, sentries.size(), 0, 0};
        for (size_t i : members) {
            svk::StateEntry se{};
            se.n = P[i].n;
            sentries.push_back(se);  // addresses filled once the arena exists
            sl.count++;
            sl.amps += 1ull << P[i].n;
        }
        slaunch.push_back(sl);
        for (size_t p = 0; p < max_passes; p++) {
            Launch L{mode, P[members[0]].dt, P[members[0]].arith, 0, 1, 1, entries.size(), 0};
            for (size_t i : members) {
                if (p >= P[i].low.passes.size()) continue;
                svk::BatchEntry e{};
                e.tile_begin = L.tiles;
                e.p = P[i].low.passes[p];
                e.p.op0 += (int32_t)op_base[i];
                e.state = (uint64_t)i;  // patched to an address below
                entries.push_back(e);
                L.n_ent++;
                L.tiles += e.p.tile_count;
                L.max_m = std::max(L.max_m, (int)e.p.m);
                L.kmax = std::max(L.kmax, (int)e.p.kmax);
            }
            launches.push_back(L);
        }
    }
    // rebase each op's coefficient offset: element offset inside its item's blob
    for (size_t i = 0; i < P.size(); i++) {
        const size_t esz = P[i].low.is_tc ? sizeof(Word16) : coef_elem_bytes(P[i].dt);
        for (size_t o = 0; o < P[i].low.ops.size(); o++) ops[op_base[i] + o].coeff += (int32_t)(coef_base[i] / esz);
    }
    const size_t ent_off = off;
    off += align256(entries.size() * sizeof(svk::BatchEntry) + 16);
    const size_t sent_off = off;
    off += align256(sentries.size() * sizeof(svk::StateEntry) + 16);
    b->arena_bytes = off;
    if (size_only) {
        *size_out = off;
        return fail(SV_OK);
    }
    if (ext_arena) {
        if (ext_bytes < off || ((uintptr_t)ext_arena & 255)) return fail(SV_ERR_SIZE);
        b->arena = ext_arena;
        b->own_arena = false;
    } else {
        size_t fr = 0, to = 0;
        if (cudaMemGetInfo(&fr, &to) == cudaSuccess && off > fr) return fail(SV_ERR_OOM);
        cudaError_t e = cudaMalloc(&b->arena, off);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(e == cudaErrorMemoryAllocation ? SV_ERR_OOM : SV_ERR_CUDA);
        }
    }
    auto* A = (unsigned char*)b->arena;
    for (auto& en : entries) en.state = (uint64_t)(uintptr_t)(A + P[(size_t)en.state].state_off);
    {
        size_t k = 0;
        for (int mode = 0; mode < kBatchModes; mode++)
            for (size_t i = 0; i < P.size(); i++) {
                if (mode_of(P[i]) != mode) continue;
                sentries[k].state = (uint64_t)(uintptr_t)(A + P[i].state_off);
                sentries[k].probs = P[i].host_out ? (uint64_t)(uintptr_t)(A + P[i].probs_off)
                                                  : (uint64_t)(uintptr_t)items[P[i].idx].probs_out;
                k++;
            }
        if (k != sentries.size()) return fail(SV_ERR_STATE);  // every state entry has its addresses
    }
    for (auto& bp : P)
        if (bp.host_out)
            b->host_copies.push_back({items[bp.idx].probs_out, bp.probs_off, ((size_t)8) << bp.n});
    // upload descriptors (synchronous copies from host vectors)
    if (cudaMemcpy(A + ops_off, ops.data(), ops.size() * sizeof(DevOp), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(A + coef_off, coefs.data(), coefs.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(A + ent_off, entries.data(), entries.size() * sizeof(svk::BatchEntry), cudaMemcpyHostToDevice) !=
            cudaSuccess ||
        cudaMemcpy(A + sent_off, sentries.data(), sentries.size() * sizeof(svk::StateEntry), cudaMemcpyHostToDevice) !=
            cudaSuccess)
        return fail(SV_ERR_CUDA);
    // highest stream priority: a batch of small circuits is scheduled ahead of
    // pending launches of long single-circuit passes on other streams
    int prio_lo = 0, prio_hi = 0;
    if (cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi) != cudaSuccess ||
        cudaStreamCreateWithPriority(&b->stream, cudaStreamNonBlocking, prio_hi) != cudaSuccess)
        return fail(SV_ERR_CUDA);
    if (cudaEventCreate(&b->ev[0]) != cudaSuccess || cudaEventCreate(&b->ev[1]) != cudaSuccess)
        return fail(SV_ERR_CUDA);
    // capture: init (per mode) -> passes -> probabilities (per mode)
    if (cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return fail(SV_ERR_CUDA);
    cudaError_t ce = cudaSuccess;
    const auto* d_ops = (const DevOp*)(A + ops_off);
    const auto* d_ent = (const svk::BatchEntry*)(A + ent_off);
    const auto* d_sent = (const svk::StateEntry*)(A + sent_off);
    for (const auto& sl : slaunch)
        if (ce == cudaSuccess) {
            ce = svk::launch_init_multi(sl.dt, d_sent + sl.first, sl.count, sl.amps, b->stream, b->di);
            b->n_launches++;
        }
    for (const auto& L : launches)
        if (ce == cudaSuccess && L.n_ent > 0) {
            ce = svk::launch_tile_pass(L.dt, L.arith, d_ent + L.ent_index, L.n_ent, L.tiles, L.max_m, L.kmax, d_ops,
                                       A + coef_off, b->stream, b->di);
            b->n_launches++;
        }
    for (const auto& sl : slaunch)
        if (ce == cudaSuccess) {
            ce = svk::launch_probs_multi(sl.dt, d_sent + sl.first, sl.count, sl.amps, b->stream, b->di);
            b->n_launches++;
        }
    cudaGraph_t g = nullptr;
    cudaError_t ee = cudaStreamEndCapture(b->stream, &g);
    if (ce != cudaSuccess || ee != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return fail(SV_ERR_CUDA);
    }
    b->graph = g;
    if (cudaGraphInstantiate(&b->exec, g, 0) != cudaSuccess) return fail(SV_ERR_CUDA);
    (void)s;
    *out = b;
    return SV_OK;
}

int sv_batch_create(const sv_batch_item* items, size_t n_items, const sv_run_opts* opts, int* item_status,
                    sv_batch** out) {
    return batch_build(items, n_items, opts, item_status, nullptr, 0, false, nullptr, out);
}

int sv_batch_arena_bytes(const sv_batch_item* items, size_t n_items, const sv_run_opts* opts, size_t* bytes) {
    if (!bytes) return SV_ERR_ARG;
    return batch_build(items, n_items, opts, nullptr, nullptr, 0, true, bytes, nullptr);
}

int sv_batch_create_in(const sv_batch_item* items, size_t n_items, const sv_run_opts* opts, int* item_status,
                       void* arena, size_t arena_bytes, sv_batch** out) {
    if (!arena) return SV_ERR_ARG;
    return batch_build(items, n_items, opts, item_status, arena, arena_bytes, false, nullptr, out);
}

int sv_batch_execute(sv_batch* b) {
    if (!b || !b->exec) return SV_ERR_ARG;
    if (cudaEventRecord(b->ev[0], b->stream) != cudaSuccess) return SV_ERR_CUDA;
    if (cudaGraphLaunch(b->exec, b->stream) != cudaSuccess) return SV_ERR_CUDA;
    if (cudaEventRecord(b->ev[1], b->stream) != cudaSuccess) return SV_ERR_CUDA;
    for (const auto& hc : b->host_copies)
        if (cudaMemcpyAsync(hc.dst, (unsigned char*)b->arena + hc.off, hc.bytes, cudaMemcpyDeviceToHost, b->stream) !=
            cudaSuccess)
            return SV_ERR_CUDA;
    if (cudaStreamSynchronize(b->stream) != cudaSuccess) return SV_ERR_CUDA;
    int fault = 0;
    if (svk::tc_fault_take(&fault) != cudaSuccess) return SV_ERR_CUDA;
    if (fault) return SV_ERR_TIMEOUT;
    float ms = 0;
    if (cudaEventElapsedTime(&ms, b->ev[0], b->ev[1]) == cudaSuccess) b->last_ms = ms;
    return SV_OK;
}

void sv_batch_destroy(sv_batch* b) {
    if (b && b->stream) cudaStreamSynchronize(b->stream);
    batch_free(b);
}

int sv_batch_stats(const sv_batch* b, sv_batch_info* out) {
    if (!b || !out) return SV_ERR_ARG;
    out->n_items = b->n_items;
    out->n_launches = b->n_launches;
    out->arena_bytes = (double)b->arena_bytes;
    out->last_ms = b->last_ms;
    return SV_OK;
}

int sv_batch_run(const sv_batch_item* items, size_t n_items, const sv_run_opts* opts, int* item_status) {
    sv_batch* b = nullptr;
    int rc = sv_batch_create(items, n_items, opts, item_status, &b);
    if (rc != SV_OK) return rc;
    rc = sv_batch_execute(b);
    sv_batch_destroy(b);
    if (rc == SV_OK && item_status)
        for (size_t i = 0; i < n_items; i++)
            if (item_status[i] != SV_OK) rc = item_status[i];
    return rc;
}

const char* sv_status_str(int st) {
    switch (st) {
        case SV_OK: return "ok";
        case SV_ERR_ARG: return "invalid argument";
        case SV_ERR_QUBIT: return "qubit index out of range or repeated";
        case SV_ERR_OOM: return "out of device memory";
        case SV_ERR_SIZE: return "size mismatch";
        case SV_ERR_CUDA: return "CUDA runtime error";
        case SV_ERR_TIMEOUT: return "device-side wait timed out";
        case SV_ERR_STATE: return "state unusable after an earlier failure";
        default: return "unknown status";
    }
}

const char* sv_version(void) { return "libsv 0.1 (sm_103a)"; }

// ---------------------------------------------------------------------------
// Plan introspection (host only).
// ---------------------------------------------------------------------------
int sv_plan_build(int n, int dt, const sv_gate* g, size_t ng, const sv_run_opts* o, sv_plan** out) {
    if (!out || n < 1 || n > svp::kMaxQubits || !dt_ok(dt)) return SV_ERR_ARG;
    int rc = svp::validate(n, g, ng);
    if (rc) return rc;
    sv_plan* p = new (std::nothrow) sv_plan();
    if (!p) return SV_ERR_OOM;
    p->dt = dt;
    const int smem_max_m = dt == SV_C64 ? 14 : 13;  // GB300: 227 KiB per CTA
    p->plan = plan_for(n, dt, g, ng, o, smem_max_m);
    *out = p;
    return SV_OK;
}

void sv_plan_free(sv_plan* p) { delete p; }

int sv_plan_summary_get(const sv_plan* p, sv_plan_summary* out) {
    if (!p || !out) return SV_ERR_ARG;
    out->n_blocks = (int32_t)p->plan.blocks.size();
    out->n_passes = (int32_t)p->plan.passes.size();
    out->fuse_k = p->plan.fuse_k;
    out->tile_qubits = p->plan.tile_m;
    out->flops = p->plan.flops;
    out->model_ms = p->plan.model_s * 1e3;
    return SV_OK;
}

int sv_plan_block(const sv_plan* p, int b, int* kind, int* k, int* qubits, int* n_gates, int* gate_ids,
                  size_t cap_gates, double* mat, size_t cap_mat) {
    if (!p || b < 0 || b >= (int)p->plan.blocks.size()) return SV_ERR_ARG;
    const svp::Block& B = p->plan.blocks[b];
    if (kind) *kind = B.kind;
    if (k) *k = B.k;
    if (qubits)
        for (int j = 0; j < B.k; j++) qubits[j] = B.qubits[j];
    if (n_gates) *n_gates = (int)B.gates.size();
    if (gate_ids)
        for (size_t i = 0; i < B.gates.size() && i < cap_gates; i++) gate_ids[i] = B.gates[i];
    if (mat)
        for (size_t i = 0; i < B.mat.size() && 2 * i + 1 < cap_mat; i++) {
            mat[2 * i] = B.mat[i].real();
            mat[2 * i + 1] = B.mat[i].imag();
        }
    return SV_OK;
}

int sv_plan_pass(const sv_plan* p, int i, uint64_t* local_mask, int* n_blocks, int* block_ids, size_t cap) {
    if (!p || i < 0 || i >= (int)p->plan.passes.size()) return SV_ERR_ARG;
    const svp::Pass& P = p->plan.passes[i];
    if (local_mask) *local_mask = P.local_mask;
    if (n_blocks) *n_blocks = (int)P.blocks.size();
    if (block_ids)
        for (size_t j = 0; j < P.blocks.size() && j < cap; j++) block_ids[j] = P.blocks[j];
    return SV_OK;
}

int sv_plan_check(const sv_plan* p, const sv_gate* g, size_t ng) {
    if (!p) return SV_ERR_ARG;
    return svp::check_plan(p->plan, ng, g) == 0 ? SV_OK : SV_ERR_STATE;
}

}  // extern "C"

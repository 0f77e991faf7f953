// C-ABI of the statevector engine (include/sv.h, include/sv_plan.h).
//
// Each call validates its arguments, runs the host planner where needed,
// uploads the launch descriptors and block coefficients, launches the sm_103a
// kernels on the handle's stream and waits for them.  No C++ exception
// crosses the boundary.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
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
// always in the tile (runs of 2^c contiguous amplitudes = 256 bytes).
int default_tile(int dt) { return dt == SV_C64 ? 13 : 12; }
int coalesce_of(int dt) { return dt == SV_C64 ? 5 : 4; }
int max_tile(int dt, const svk::DevInfo& di) {
    int m = dt == SV_C64 ? 14 : 13;
    while (m > 6 && ((size_t)1 << m) * amp_bytes(dt) > di.smem_optin - 2048) m--;
    return m;
}

int resolve_arith(int dt, const sv_run_opts* o) {
    if (dt == SV_C64) return SV_ARITH_NATIVE;
    int a = o ? o->arith : 0;
    if (a == SV_ARITH_DF64) return SV_ARITH_DF64;
    return SV_ARITH_NATIVE;
}

svp::Plan plan_for(int n, int dt, const sv_gate* g, size_t ng, const sv_run_opts* o, int smem_max_m) {
    int k = o ? o->max_fuse_k : 0;
    if (k < 0) k = 0;
    if (k > svp::kMaxFuse) k = svp::kMaxFuse;
    const int c = coalesce_of(dt);
    int m = (o && o->tile_qubits > 0) ? o->tile_qubits : default_tile(dt);
    m = std::min(m, smem_max_m);
    m = std::min(m, c + 10);
    m = std::max(m, c + svp::kMaxFuse);
    svp::Machine mc;
    int ak = svp::AK_FP32;
    if (dt == SV_C128) ak = resolve_arith(dt, o) == SV_ARITH_DF64 ? svp::AK_DF64 : svp::AK_FP64;
    return svp::make_plan(n, g, ng, k, m, c, amp_bytes(dt), ak, mc);
}

// Serialises a plan into descriptors (passes by value, ops and coefficients
// into one contiguous upload).
struct Lowered {
    std::vector<DevPass> passes;
    std::vector<DevOp> ops;
    std::vector<svp::cd> coef;
};

void lower(const svp::Plan& P, Lowered& L) {
    L.passes.clear();
    L.ops.clear();
    L.coef.clear();
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
        for (int bi : ps.blocks) {
            const svp::Block& b = P.blocks[bi];
            DevOp op;
            std::memset(&op, 0, sizeof(op));
            op.kind = b.kind == svp::BK_DIAG ? svk::OP_DIAG : svk::OP_DENSE;
            op.k = b.k;
            op.coeff = (int32_t)L.coef.size();
            op.flags = (b.kind == svp::BK_DIAG && b.sign_only) ? svk::OPF_SIGN_ONLY : 0;
            for (int j = 0; j < b.k; j++) {
                op.pos[j] = pos_of[b.qubits[j]];
                op.qbit[j] = b.qubits[j];
            }
            L.coef.insert(L.coef.end(), b.mat.begin(), b.mat.end());
            L.ops.push_back(op);
            if (op.kind == svk::OP_DENSE) dp.kmax = std::max(dp.kmax, (int32_t)b.k);
        }
        if (dp.kmax < 1) dp.kmax = 1;
        dp.n_ops = (int32_t)(L.ops.size() - dp.op0);
        L.passes.push_back(dp);
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

int apply_plan(sv_state* s, const svp::Plan& P, int arith, bool timing) {
    Lowered L;
    lower(P, L);
    const size_t ops_bytes = L.ops.size() * sizeof(DevOp);
    const size_t esz = amp_bytes(s->dt);
    const size_t coef_off = (ops_bytes + 255) & ~(size_t)255;
    const size_t total = coef_off + L.coef.size() * esz + 256;
    SV_TRY(ensure(&s->d_ws, &s->d_ws_cap, total, false));
    SV_TRY(ensure(&s->h_ws, &s->h_ws_cap, total, true));
    auto* h = (unsigned char*)s->h_ws;
    if (ops_bytes) std::memcpy(h, L.ops.data(), ops_bytes);
    if (s->dt == SV_C64) {
        auto* c = (float*)(h + coef_off);
        for (size_t i = 0; i < L.coef.size(); i++) {
            c[2 * i] = (float)L.coef[i].real();
            c[2 * i + 1] = (float)L.coef[i].imag();
        }
    } else if (arith == SV_ARITH_DF64) {
        // (hi, lo) float pairs: hi = float(x), lo = float(x - hi)
        auto* c = (float*)(h + coef_off);
        for (size_t i = 0; i < L.coef.size(); i++) {
            const double re = L.coef[i].real(), im = L.coef[i].imag();
            const float rh = (float)re, ih = (float)im;
            c[4 * i] = rh;
            c[4 * i + 1] = (float)(re - (double)rh);
            c[4 * i + 2] = ih;
            c[4 * i + 3] = (float)(im - (double)ih);
        }
    } else {
        auto* c = (double*)(h + coef_off);
        for (size_t i = 0; i < L.coef.size(); i++) {
            c[2 * i] = L.coef[i].real();
            c[2 * i + 1] = L.coef[i].imag();
        }
    }
    SV_TRY(cudaMemcpyAsync(s->d_ws, s->h_ws, total, cudaMemcpyHostToDevice, s->stream));
    s->last.upload_bytes = (double)total;
    const auto* d_ops = (const DevOp*)s->d_ws;
    const void* d_coef = (const unsigned char*)s->d_ws + coef_off;
    int launches = 0;
    if (timing) {
        while (s->events.size() < L.passes.size() + 1) {
            cudaEvent_t e;
            SV_TRY(cudaEventCreate(&e));
            s->events.push_back(e);
        }
        SV_TRY(cudaEventRecord(s->events[0], s->stream));
    }
    for (const auto& dp : L.passes) {
        SV_TRY(svk::launch_tile_pass(s->dt, arith, s->amp, dp, d_ops, d_coef, s->stream, s->di));
        launches++;
        if (timing) SV_TRY(cudaEventRecord(s->events[launches], s->stream));
    }
    SV_TRY(cudaStreamSynchronize(s->stream));
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
    *out = s;
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
    if (o && o->debug_checks && svp::check_plan(P, ng, g) != 0) return SV_ERR_STATE;
    const double t1 = now_ms();
    const int arith = resolve_arith(s->dt, o);
    rc = apply_plan(s, P, arith, o && o->timing);
    s->last.n_blocks = (int32_t)P.blocks.size();
    s->last.n_passes = (int32_t)P.passes.size();
    s->last.fuse_k = P.fuse_k;
    s->last.tile_qubits = P.tile_m;
    s->last.arith = arith;
    s->last.flops = P.flops;
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
    // host output: through a bounded device staging buffer, chunk by chunk
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
    return SV_OK;
}

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

int sv_batch_run(const sv_batch_item* items, size_t n_items, const sv_run_opts* opts, int* item_status) {
    if (n_items && !items) return SV_ERR_ARG;
    int worst = SV_OK;
    for (size_t i = 0; i < n_items; i++) {
        const sv_batch_item& it = items[i];
        sv_state* s = nullptr;
        int rc = sv_create(it.n_qubits, it.dt, &s);
        if (rc == SV_OK) rc = sv_apply_circuit(s, it.gates, it.n_gates, opts);
        if (rc == SV_OK) rc = sv_probabilities(s, it.probs_out, (size_t)1 << it.n_qubits, it.probs_on_device);
        if (s) sv_destroy(s);
        if (item_status) item_status[i] = rc;
        if (rc != SV_OK && worst == SV_OK) worst = rc;
    }
    return worst;
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

// Cut-subcircuit variants with shared work (the CutQC Evaluator's instances,
// Sec. IV-A, Fig. 1; three measurement bases per cut output and four
// initialisations per cut input, Eqs. 3.2-3.6).
//
// Upstream: every variant is the same body followed by a basis-change suffix
// on the cut qubits, so the body is simulated once and each variant applies
// only its suffix to a copy.
// Downstream: every variant is the same body applied to a product state of the
// cut qubits, each in |0>, |1>, |+> or |+i>.  The body U is linear, so
//   U (x)_j |s_j> |0..> = sum_b prod_j c_{s_j}(b_j) U|b>,
// c_0 = (1, 0), c_1 = (0, 1), c_+ = (1, 1)/sqrt2, c_{+i} = (1, i)/sqrt2:
// the body runs once per computational basis state b of the cut qubits
// (2^K runs) and each variant is a linear combination of those states.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <vector>

#include "sv.h"

namespace {

constexpr int kMaxTerms = 64;  // 2^K for K <= 6

struct LinTerms {
    int32_t n_terms;
    uint64_t src[kMaxTerms];
    double cre[kMaxTerms], cim[kMaxTerms];
};

// complex64: float arithmetic
__global__ void k_lincomb_f32(float2* __restrict__ out, uint64_t dim, const LinTerms T) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < dim; i += stride) {
        float re = 0.f, im = 0.f;
        for (int t = 0; t < T.n_terms; t++) {
            const float2 a = reinterpret_cast<const float2*>(T.src[t])[i];
            const float cr = (float)T.cre[t], ci = (float)T.cim[t];
            re = fmaf(cr, a.x, fmaf(-ci, a.y, re));
            im = fmaf(cr, a.y, fmaf(ci, a.x, im));
        }
        out[i] = make_float2(re, im);
    }
}

// complex128: float64 arithmetic (a handful of multiply-adds per amplitude:
// small next to the body simulations it replaces)
__global__ void k_lincomb_f64(double2* __restrict__ out, uint64_t dim, const LinTerms T) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < dim; i += stride) {
        double re = 0.0, im = 0.0;
        for (int t = 0; t < T.n_terms; t++) {
            const double2 a = reinterpret_cast<const double2*>(T.src[t])[i];
            re = fma(T.cre[t], a.x, fma(-T.cim[t], a.y, re));
            im = fma(T.cre[t], a.y, fma(T.cim[t], a.x, im));
        }
        out[i] = make_double2(re, im);
    }
}

int lincomb(sv_state* out, const LinTerms& T) {
    const int n = sv_num_qubits(out), dt = sv_dtype_of(out);
    const uint64_t dim = 1ull << n;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return SV_ERR_CUDA;
    uint64_t grid = (dim + 255) / 256;
    if (grid > (uint64_t)sms * 8) grid = (uint64_t)sms * 8;
    if (dt == SV_C64)
        k_lincomb_f32<<<(unsigned)grid, 256>>>((float2*)sv_device_ptr(out), dim, T);
    else
        k_lincomb_f64<<<(unsigned)grid, 256>>>((double2*)sv_device_ptr(out), dim, T);
    if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) return SV_ERR_CUDA;
    return SV_OK;
}

struct Owned {
    std::vector<sv_state*> v;
    ~Owned() {
        for (auto* s : v) sv_destroy(s);
    }
};

}  // namespace

extern "C" int sv_cut_variants(int dt, const sv_gate* body_a, size_t n_a, int width_a, const int32_t* cut_pos_a,
                               const sv_gate* body_b, size_t n_b, int width_b, const int32_t* cut_pos_b, int n_cuts,
                               double* const* up_out, double* const* down_out, int outs_on_device,
                               const sv_run_opts* opts) {
    if (n_cuts < 1 || n_cuts > 6 || !cut_pos_a || !cut_pos_b || !up_out || !down_out) return SV_ERR_ARG;
    for (int j = 0; j < n_cuts; j++)
        if (cut_pos_a[j] < 0 || cut_pos_a[j] >= width_a || cut_pos_b[j] < 0 || cut_pos_b[j] >= width_b)
            return SV_ERR_QUBIT;
    int nup = 1, ndown = 1, nbasis = 1 << n_cuts;
    for (int j = 0; j < n_cuts; j++) {
        nup *= 3;
        ndown *= 4;
    }
    Owned own;
    // ---- upstream: body once, suffix per variant on a copy ----
    sv_state *body = nullptr, *work = nullptr;
    int rc = sv_create(width_a, dt, &body);
    if (rc) return rc;
    own.v.push_back(body);
    if ((rc = sv_create(width_a, dt, &work))) return rc;
    own.v.push_back(work);
    if ((rc = sv_apply_circuit(body, body_a, n_a, opts))) return rc;
    const size_t bytes_a = sv_state_bytes(width_a, dt);
    const double pi = 3.14159265358979323846;
    for (int v = 0; v < nup; v++) {
        std::vector<sv_gate> suffix;
        int vv = v;
        for (int j = 0; j < n_cuts; j++) {
            const int m = vv % 3;
            vv /= 3;
            const int q = cut_pos_a[j];
            if (m == 1) suffix.push_back(sv_gate{SV_H, q, -1, 0, 0, 0});
            if (m == 2) {
                suffix.push_back(sv_gate{SV_U3, q, -1, 0.0, 0.0, -pi / 2});  // S^dagger
                suffix.push_back(sv_gate{SV_H, q, -1, 0, 0, 0});
            }
        }
        sv_state* src = body;
        if (!suffix.empty()) {
            if ((rc = sv_set_amplitudes(work, sv_device_ptr(body), bytes_a, 1))) return rc;
            if ((rc = sv_apply_circuit(work, suffix.data(), suffix.size(), opts))) return rc;
            src = work;
        }
        if ((rc = sv_probabilities(src, up_out[v], (size_t)1 << width_a, outs_on_device))) return rc;
    }
    // ---- downstream: body on the 2^K basis states of the cut qubits ----
    std::vector<sv_state*> basis(nbasis, nullptr);
    for (int b = 0; b < nbasis; b++) {
        if ((rc = sv_create(width_b, dt, &basis[b]))) return rc;
        own.v.push_back(basis[b]);
        uint64_t idx = 0;
        for (int j = 0; j < n_cuts; j++)
            if ((b >> j) & 1) idx |= 1ull << cut_pos_b[j];
        if ((rc = sv_reset(basis[b], idx))) return rc;
        if ((rc = sv_apply_circuit(basis[b], body_b, n_b, opts))) return rc;
    }
    sv_state* comb = nullptr;
    if ((rc = sv_create(width_b, dt, &comb))) return rc;
    own.v.push_back(comb);
    const double r2 = 1.0 / std::sqrt(2.0);
    for (int s = 0; s < ndown; s++) {
        LinTerms T{};
        for (int b = 0; b < nbasis; b++) {
            double cr = 1.0, ci = 0.0;  // prod_j c_{s_j}(b_j)
            int ss = s;
            for (int j = 0; j < n_cuts; j++) {
                const int sj = ss & 3, bj = (b >> j) & 1;
                ss >>= 2;
                double fr, fi;
                if (sj == 0) { fr = bj ? 0.0 : 1.0; fi = 0.0; }
                else if (sj == 1) { fr = bj ? 1.0 : 0.0; fi = 0.0; }
                else if (sj == 2) { fr = r2; fi = 0.0; }
                else { fr = bj ? 0.0 : r2; fi = bj ? r2 : 0.0; }  // (1, i)/sqrt2
                const double nr = cr * fr - ci * fi, ni = cr * fi + ci * fr;
                cr = nr;
                ci = ni;
            }
            if (cr == 0.0 && ci == 0.0) continue;
            T.src[T.n_terms] = (uint64_t)(uintptr_t)sv_device_ptr(basis[b]);
            T.cre[T.n_terms] = cr;
            T.cim[T.n_terms] = ci;
            T.n_terms++;
        }
        if ((rc = lincomb(comb, T))) return rc;
        if ((rc = sv_probabilities(comb, down_out[s], (size_t)1 << width_b, outs_on_device))) return rc;
    }
    return SV_OK;
}

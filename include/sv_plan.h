/*
 * libsv plan introspection -- host-only entry points (no GPU needed).
 *
 * They expose the planner that sv_apply_circuit runs before launching: the
 * fusion of the gate list into blocks of at most k qubits and the grouping of
 * the blocks into tile passes (the single-GPU form of the cache blocking of
 * Sec. III-B, Fig. 4: every block of a pass acts on qubits held in the pass's
 * shared-memory tile, so one HBM sweep applies them all).  Tests use them to
 * check the plan on a machine without a GPU; none of them touches device
 * memory.  Status codes and ownership rules are those of sv.h.
 */
#ifndef LIBSV_SV_PLAN_H
#define LIBSV_SV_PLAN_H

#include "sv.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sv_plan sv_plan;

/* Plans gates for an n-qubit state of dtype dt with the given options (the
 * same plan sv_apply_circuit would use).  Validation errors as in
 * sv_apply_circuit.  The plan is freed with sv_plan_free. */
int sv_plan_build(int n, int dt, const sv_gate* gates, size_t n_gates,
                  const sv_run_opts* opts, sv_plan** out);
void sv_plan_free(sv_plan* p);

/* Counts and model of the plan: fused blocks, passes, the fusion width and
 * tile qubits chosen, modelled real flops and modelled time (ms). */
typedef struct {
    int32_t n_blocks, n_passes, fuse_k, tile_qubits;
    double flops, model_ms;
} sv_plan_summary;
int sv_plan_summary_get(const sv_plan* p, sv_plan_summary* out);

/* Block b: kind (0 dense, 1 diagonal, 2 permutation -- one nonzero per row,
 * applied by moving amplitudes -- or 3 Kronecker -- a tensor product of
 * one-qubit matrices, applied as one butterfly per qubit outside the
 * tensor-core modes), k, its qubits (ascending; matrix bit j is qubits[j]),
 * the input-gate indices it holds (up to cap_gates written, *n_gates =
 * total), and its matrix as interleaved (re, im) float64 -- 2^k entries for
 * diagonal, (2^k)^2 row-major for the other kinds (up to cap_mat doubles
 * written).  The classes are those of the fusion step's block analysis (the
 * transpile phase Aer runs before simulating, Sec. III-B). */
int sv_plan_block(const sv_plan* p, int b, int* kind, int* k, int* qubits,
                  int* n_gates, int* gate_ids, size_t cap_gates,
                  double* mat, size_t cap_mat);

/* Pass i: tile qubit mask and its block indices in application order. */
int sv_plan_pass(const sv_plan* p, int i, uint64_t* local_mask, int* n_blocks,
                 int* block_ids, size_t cap);

/* Plan invariants: every gate exactly once, per-qubit gate order kept,
 * 1 <= k <= 5, dense blocks local to their pass.  SV_OK when they hold. */
int sv_plan_check(const sv_plan* p, const sv_gate* gates, size_t n_gates);

#ifdef __cplusplus
}
#endif
#endif /* LIBSV_SV_PLAN_H */

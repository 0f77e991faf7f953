// Host planner of the statevector engine: gate IR -> fused blocks -> tile passes.
//
// The paper hands gate application to Qiskit Aer, whose transpiler blocks the
// gates so that runs of them act on a set of "local" qubits held in one chunk
// (qubit reordering and noiseless swap insertion, Sec. III-B, Fig. 4).  On one
// GB300 the chunk becomes a shared-memory tile: a pass streams every tile of
// the state through shared memory once and applies, per tile, every block
// whose qubits are all held in the tile.  Any qubit set can be the tile's, so
// no swap gates are needed: a pass simply gathers a different set.
#pragma once
#include <complex>
#include <cstddef>
#include <cstdint>
#include <vector>

#include "sv.h"

namespace svp {

using cd = std::complex<double>;

constexpr int kMaxFuse = 5;        // largest fused block (qubits)
constexpr int kMaxQubits = 34;

int gate_arity(int op);            // 1, 2, or 0 for an unknown opcode
bool gate_is_diagonal(int op);     // Z, S, T, RZ, CZ, RZZ
bool gate_is_monomial(int op);     // one nonzero per row: the diagonal gates and X, Y, CX, SWAP
// Row-major 2x2 or 4x4 matrix (two-qubit local index b(q0) + 2 b(q1)),
// computed in float64 with the host libm.
void gate_matrix(const sv_gate& g, cd* m);

// Validates a gate list for an n-qubit register; SV_OK or the sv_status.
int validate(int n, const sv_gate* g, size_t ng);

// Block classes (the fused block's matrix structure decides how a tile
// applies it):
//   BK_DENSE  any unitary: a 2^k x 2^k product per group of amplitudes;
//   BK_DIAG   diagonal: a phase per amplitude, from the amplitude's index;
//   BK_PERM   monomial (one nonzero per row: X, Y, CX, SWAP with diagonal
//             gates): out[r] = phase[r] in[src[r]], a move of amplitudes
//             inside each group, no products;
//   BK_KRON   a tensor product of one-qubit matrices (only one-qubit gates):
//             k butterflies instead of one 2^k product where arithmetic,
//             not the tensor cores, applies the blocks.
enum BlockKind { BK_DENSE = 0, BK_DIAG = 1, BK_PERM = 2, BK_KRON = 3 };

struct Block {
    int kind = BK_DENSE;
    int k = 0;
    int qubits[kMaxFuse] = {0, 0, 0, 0, 0};  // ascending; matrix bit j <-> qubits[j]
    uint64_t mask = 0;
    std::vector<int> gates;                  // input indices, application order
    std::vector<cd> mat;                     // dense / perm / kron: (2^k)^2 row-major; diag: 2^k
    bool sign_only = false;                  // diag entries all +1 / -1
    std::vector<int> src;                    // perm: source row of each output row
    std::vector<cd> phase;                   // perm: the nonzero of each row
    bool quarter = false;                    // perm: every phase is 1, i, -1 or -i
    std::vector<cd> factors;                 // kron: 2x2 of qubits[0], qubits[1], ... (row-major)
};

struct Pass {
    uint64_t local_mask = 0;                 // qubits held in the tile
    int m = 0;                               // popcount(local_mask)
    std::vector<int> blocks;                 // application order
};

struct Plan {
    int n = 0, fuse_k = 0, tile_m = 0, coalesce = 0;
    std::vector<Block> blocks;
    std::vector<Pass> passes;
    double flops = 0;      // modelled real flops (FMA = 2)
    double alu_ops = 0;    // modelled ALU lane operations (FP32 for df64/complex64, FP64 native)
    double mma_flops = 0;  // tensor-core mode: bfloat16 MMA flops of the digit products
    double model_s = 0;    // modelled time
};

// Arithmetic of the tile kernels: float32 (complex64), native float64, or
// double-float pairs on the FP32 units (complex128).
// AK_TC: complex128 digit products on the tensor cores; AK_TC32: complex64
// bfloat16 triple split on the tensor cores.
enum ArithKind { AK_FP32 = 0, AK_FP64 = 1, AK_DF64 = 2, AK_TC = 3, AK_TC32 = 4 };

struct Machine {           // throughput model used by the autotuner (measured on GB300)
    double hbm_Bps = 6.6e12;
    double fp32_ips = 3.2e13;   // FP32 lane instructions per second (FFMA / FADD / FMUL)
    double fp64_ips = 4.6e11;   // FP64 lane instructions per second
    double smem_Bps = 3.5e13;
    double mma_flops = 5.8e14;  // bfloat16 mma.sync, dense
    double tc05_flops = 1.2e15; // tcgen05 16-bit MMAs as issued by the tile pass (about 60 % of peak)
    double launch_s = 4e-6;
    const sv_costs* measured = nullptr;  // device-measured costs (sv_calibrate), replacing the model above
};

// Greedy fusion: each gate joins the latest block among those holding its
// qubits when the union stays within fuse_k qubits; otherwise it opens a new
// block.  fuse_k = 1 keeps every gate on its own.  keep_monomial = 1: a gate
// that is not monomial does not join a block made of monomial gates only (it
// opens a new block), so runs of X / CX / SWAP / diagonal gates stay
// permutation blocks; 2: a monomial gate does not join a block holding other
// gates either.  With pack, a gate that cannot join the latest block holding
// its qubits may join any later block with room (the one it overlaps most
// among the last 64), so gates on disjoint qubits share blocks (a layer of
// one-qubit gates becomes Kronecker blocks).  make_plan tries every variant.
std::vector<Block> fuse(int n, const sv_gate* g, size_t ng, int fuse_k, int keep_monomial = 0,
                        bool pack = false);

// Fills Block::mat / kind / sign_only (and src / phase / quarter for
// permutation blocks, factors for Kronecker blocks) from the gates (float64
// products).
void finalize(std::vector<Block>& blocks, const sv_gate* g);

// Groups blocks into tile passes of tile_m qubits whose lowest `coalesce`
// qubits are always local (contiguous runs for coalesced loads).
std::vector<Pass> schedule(int n, const std::vector<Block>& blocks, int tile_m, int coalesce);

// Modelled cost of a plan (seconds) for a state of `amp_bytes` per amplitude;
// *flops receives the real flops of the block products (FMA = 2).
double model_cost(const Plan& p, int amp_bytes, int arith, const Machine& mc, double* flops,
                  double* alu_ops = nullptr, double* mma_flops = nullptr);

// Full planning with optional autotuning over fuse_k (0 = auto).
Plan make_plan(int n, const sv_gate* g, size_t ng, int fuse_k, int tile_m, int coalesce,
               int amp_bytes, int arith, const Machine& mc);

// Checks plan invariants: every gate exactly once, per-qubit order kept,
// block sizes, locality of dense blocks.  Returns 0 when valid.
int check_plan(const Plan& p, size_t ng, const sv_gate* g);

}  // namespace svp

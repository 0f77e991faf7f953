// Descriptors shared by the host launcher and the sm_103a kernels.
#pragma once
#include <cstdint>

namespace svk {

constexpr int kMaxQ = 40;

// OP_PERM: out[r] = i^code(r) in[src(r)] inside every group of 2^k amplitudes;
// its coefficient elements list the rows in cycle order (dst | code << 5 |
// end-of-cycle << 7, exact small integers in every coefficient format).
enum OpKind : int32_t { OP_DENSE = 0, OP_DIAG = 1, OP_PERM = 2 };
// OPF_TEST_NO_MMA (tensor-memory mode, tests only): the op issues no MMAs,
// so its bounded wait runs out and the call reports SV_ERR_TIMEOUT.
enum OpFlags : int32_t { OPF_SIGN_ONLY = 1, OPF_TEST_NO_MMA = 2 };

// One fused block inside a tile pass (64 bytes).
struct alignas(16) DevOp {
    int32_t kind;     // OpKind
    int32_t k;        // qubits of the block (1..5)
    int32_t coeff;    // offset of its coefficients (complex elements)
    int32_t flags;    // OpFlags
    int32_t pos[5];   // dense / perm: tile positions, ascending; diag: tile position or -1
    int32_t qbit[5];  // diag: global qubit of matrix bit j
    int32_t pad[2];
};

// How a complex128 tcgen05 pass reads and writes the state: between the
// passes of one circuit the state stays in the kernel's Q56 fixed point
// (two int64 per amplitude, the same 16 bytes), so only the first pass
// converts from float64 and only the last converts back.
enum PassIo : int32_t { IO_LOAD_Q56 = 1, IO_STORE_Q56 = 2 };

// One tile pass: the tile holds the qubits L[0..m) (ascending, L[j] = j for
// j < c), the other n - m qubits NL[] index the tiles.
struct DevPass {
    int32_t n, m, c, n_ops;
    int32_t op0, kmax;    // first op; largest dense block of the pass
    int32_t io, pad;      // PassIo bits (0: float64 in and out)
    uint64_t tile_count;  // 2^(n-m)
    int8_t L[kMaxQ];
    int8_t NL[kMaxQ];
};

// One (state, pass) pair of a tile-pass launch.  A launch sweeps the tiles of
// all its entries as one flattened index space: entry e owns tiles
// [tile_begin, tile_begin + p.tile_count).
struct alignas(16) BatchEntry {
    uint64_t state;       // device address of the state's amplitudes
    uint64_t tile_begin;  // first flattened tile of this entry
    DevPass p;
};

// One state of a multi-state init / probabilities launch.
struct alignas(16) StateEntry {
    uint64_t state;  // device address of the amplitudes
    uint64_t probs;  // device address of its 2^n float64 probabilities
    int32_t n, pad[3];
};

}  // namespace svk

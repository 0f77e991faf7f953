// Host planner: gate matrices, fusion, tile-pass scheduling, cost model.
#include "plan.hpp"

#include <algorithm>
#include <cmath>
#include <cstring>

namespace svp {

namespace {
inline int popc(uint64_t x) { return __builtin_popcountll(x); }
const double kPi = 3.14159265358979323846264338327950288;
}  // namespace

int gate_arity(int op) {
    if (op < 0 || op >= SV_NUM_OPS) return 0;
    return op >= SV_CX ? 2 : 1;
}

bool gate_is_diagonal(int op) {
    return op == SV_Z || op == SV_S || op == SV_T || op == SV_RZ || op == SV_CZ || op == SV_RZZ;
}

bool gate_is_monomial(int op) {
    return gate_is_diagonal(op) || op == SV_X || op == SV_Y || op == SV_CX || op == SV_SWAP;
}

void gate_matrix(const sv_gate& g, cd* m) {
    const cd I(0, 1);
    const int d = 1 << gate_arity(g.op);
    for (int i = 0; i < d * d; i++) m[i] = 0;
    const double c = std::cos(g.theta / 2), s = std::sin(g.theta / 2);
    const double r2 = 1.0 / std::sqrt(2.0);
    auto ph = [](double a) { return cd(std::cos(a), std::sin(a)); };
    switch (g.op) {
        case SV_H: m[0] = r2; m[1] = r2; m[2] = r2; m[3] = -r2; break;
        case SV_X: m[1] = 1; m[2] = 1; break;
        case SV_Y: m[1] = -I; m[2] = I; break;
        case SV_Z: m[0] = 1; m[3] = -1; break;
        case SV_S: m[0] = 1; m[3] = I; break;
        case SV_T: m[0] = 1; m[3] = ph(kPi / 4); break;
        case SV_RX: m[0] = c; m[1] = -I * s; m[2] = -I * s; m[3] = c; break;
        case SV_RY: m[0] = c; m[1] = -s; m[2] = s; m[3] = c; break;
        case SV_RZ: m[0] = ph(-g.theta / 2); m[3] = ph(g.theta / 2); break;
        case SV_U3:
            m[0] = c;
            m[1] = -ph(g.lambda) * s;
            m[2] = ph(g.phi) * s;
            m[3] = ph(g.phi + g.lambda) * c;
            break;
        case SV_CX:  // local index b(q0) + 2 b(q1); flips b(q1) when b(q0) = 1
            for (int a = 0; a < 4; a++) {
                int b0 = a & 1, b1 = a >> 1;
                m[(b0 | ((b1 ^ b0) << 1)) * 4 + a] = 1;
            }
            break;
        case SV_CZ: m[0] = 1; m[5] = 1; m[10] = 1; m[15] = -1; break;
        case SV_RZZ: {
            cd a = ph(-g.theta / 2), b = ph(g.theta / 2);
            m[0] = a; m[5] = b; m[10] = b; m[15] = a;
            break;
        }
        case SV_SWAP:
            for (int a = 0; a < 4; a++) {
                int b0 = a & 1, b1 = a >> 1;
                m[(b1 | (b0 << 1)) * 4 + a] = 1;
            }
            break;
        default: break;
    }
}

int validate(int n, const sv_gate* g, size_t ng) {
    if (ng && !g) return SV_ERR_ARG;
    for (size_t t = 0; t < ng; t++) {
        int k = gate_arity(g[t].op);
        if (k == 0) return SV_ERR_ARG;
        if (!std::isfinite(g[t].theta) || !std::isfinite(g[t].phi) || !std::isfinite(g[t].lambda))
            return SV_ERR_ARG;
        if (g[t].q0 < 0 || g[t].q0 >= n) return SV_ERR_QUBIT;
        if (k == 2 && (g[t].q1 < 0 || g[t].q1 >= n || g[t].q1 == g[t].q0)) return SV_ERR_QUBIT;
    }
    return SV_OK;
}

static uint64_t gate_mask(const sv_gate& g) {
    uint64_t m = 1ull << g.q0;
    if (gate_arity(g.op) == 2) m |= 1ull << g.q1;
    return m;
}

static void set_qubits(Block& b) {
    b.k = 0;
    for (int q = 0; q < 64; q++)
        if ((b.mask >> q) & 1) b.qubits[b.k++] = q;
}

std::vector<Block> fuse(int n, const sv_gate* g, size_t ng, int fuse_k, int keep_monomial, bool pack) {
    std::vector<Block> blocks;
    std::vector<char> monomial;   // per block: every gate so far is monomial
    std::vector<int> cur(n, -1);  // latest block holding each qubit
    for (size_t t = 0; t < ng; t++) {
        const uint64_t gm = gate_mask(g[t]);
        const bool mono = gate_is_monomial(g[t].op);
        int bstar = -1;
        for (int q = 0; q < n; q++)
            if ((gm >> q) & 1) bstar = std::max(bstar, cur[q]);
        // keep_monomial 1: a non-monomial gate stays out of a monomial block;
        // 2: and a monomial gate out of a block holding another kind
        auto fits = [&](int b) {
            return popc(blocks[b].mask | gm) <= fuse_k && !(keep_monomial >= 1 && !mono && monomial[b]) &&
                   !(keep_monomial >= 2 && mono && !monomial[b]);
        };
        int target = -1;
        if (fuse_k > 1 && bstar >= 0 && fits(bstar)) target = bstar;
        if (fuse_k > 1 && target < 0 && pack) {
            // any block at or after bstar may take the gate: every block holding
            // its qubits comes no later, and none after it holds them; the most
            // overlapping of the last few blocks wins
            int best = 1 << 30;
            for (int b = (int)blocks.size() - 1; b >= std::max(bstar, 0) && b >= (int)blocks.size() - 64; b--) {
                if (!fits(b)) continue;
                const int u = popc(blocks[b].mask | gm);
                if (u < best) {
                    best = u;
                    target = b;
                }
            }
        }
        if (target >= 0) {
            blocks[target].mask |= gm;
            blocks[target].gates.push_back((int)t);
            monomial[target] = monomial[target] && mono;
        } else {
            Block b;
            b.mask = gm;
            b.gates.push_back((int)t);
            blocks.push_back(b);
            monomial.push_back(mono);
            target = (int)blocks.size() - 1;
        }
        for (int q = 0; q < n; q++)
            if ((gm >> q) & 1) cur[q] = target;
    }
    for (auto& b : blocks) {
        set_qubits(b);
        bool diag = true, mono = true, oneq = true;
        for (int t : b.gates) {
            diag = diag && gate_is_diagonal(g[t].op);
            mono = mono && gate_is_monomial(g[t].op);
            oneq = oneq && gate_arity(g[t].op) == 1;
        }
        b.kind = diag ? BK_DIAG : (mono ? BK_PERM : ((oneq && b.k > 1) ? BK_KRON : BK_DENSE));
    }
    return blocks;
}

// Embeds gate g (acting on its own local index) into the block's 2^k space and
// left-multiplies: M <- G_emb * M.
static void left_multiply(Block& b, const sv_gate& g, std::vector<cd>& M) {
    const int k = b.k, D = 1 << k;
    cd gm[16];
    gate_matrix(g, gm);
    const int ga = gate_arity(g.op);
    int gp[2] = {0, 0};  // block-local bit of the gate's qubits
    for (int j = 0; j < k; j++) {
        if (b.qubits[j] == g.q0) gp[0] = j;
        if (ga == 2 && b.qubits[j] == g.q1) gp[1] = j;
    }
    const int gd = 1 << ga;
    std::vector<cd> out((size_t)D * D, cd(0, 0));
    for (int r = 0; r < D; r++) {
        // row r of G_emb: nonzero only at columns c equal to r outside the gate bits
        int lr = 0;
        for (int a = 0; a < ga; a++) lr |= ((r >> gp[a]) & 1) << a;
        int rbase = r;
        for (int a = 0; a < ga; a++) rbase &= ~(1 << gp[a]);
        for (int lc = 0; lc < gd; lc++) {
            cd coef = gm[lr * gd + lc];
            if (coef == cd(0, 0)) continue;
            int c = rbase;
            for (int a = 0; a < ga; a++) c |= ((lc >> a) & 1) << gp[a];
            for (int col = 0; col < D; col++) out[(size_t)r * D + col] += coef * M[(size_t)c * D + col];
        }
    }
    M.swap(out);
}

void finalize(std::vector<Block>& blocks, const sv_gate* g) {
    for (auto& b : blocks) {
        const int D = 1 << b.k;
        std::vector<cd> M((size_t)D * D, cd(0, 0));
        for (int i = 0; i < D; i++) M[(size_t)i * D + i] = 1;
        for (int t : b.gates) left_multiply(b, g[t], M);
        if (b.kind == BK_DIAG) {
            b.mat.resize(D);
            bool sign = true;
            for (int i = 0; i < D; i++) {
                b.mat[i] = M[(size_t)i * D + i];
                sign = sign && b.mat[i].imag() == 0.0 && std::fabs(b.mat[i].real()) == 1.0;
            }
            b.sign_only = sign;
            continue;
        }
        if (b.kind == BK_PERM) {
            // a product of monomial gates keeps one nonzero per row (exact zeros:
            // every factor's other entries are exact zeros)
            b.src.assign(D, -1);
            b.phase.assign(D, cd(0, 0));
            b.quarter = true;
            for (int r = 0; r < D; r++) {
                for (int c = 0; c < D; c++) {
                    const cd v = M[(size_t)r * D + c];
                    if (v == cd(0, 0)) continue;
                    b.src[r] = c;
                    b.phase[r] = v;
                }
                const cd v = b.phase[r];
                const bool q = (v.imag() == 0.0 && std::fabs(v.real()) == 1.0) ||
                               (v.real() == 0.0 && std::fabs(v.imag()) == 1.0);
                b.quarter = b.quarter && q;
            }
        }
        if (b.kind == BK_KRON) {
            // per qubit, the product of its one-qubit gates in order
            b.factors.assign((size_t)4 * b.k, cd(0, 0));
            for (int j = 0; j < b.k; j++) {
                cd f[4] = {1, 0, 0, 1};
                for (int t : b.gates) {
                    if (g[t].q0 != b.qubits[j]) continue;
                    cd u[4];
                    gate_matrix(g[t], u);
                    const cd r[4] = {u[0] * f[0] + u[1] * f[2], u[0] * f[1] + u[1] * f[3],
                                     u[2] * f[0] + u[3] * f[2], u[2] * f[1] + u[3] * f[3]};
                    for (int e = 0; e < 4; e++) f[e] = r[e];
                }
                for (int e = 0; e < 4; e++) b.factors[(size_t)4 * j + e] = f[e];
            }
        }
        b.mat.swap(M);
    }
}

// The blocks (in list order) that can run in one pass whose tile holds the
// qubits of `local`: a dense block joins when its qubits are local, a
// diagonal block always; a block that cannot join blocks its qubits for
// every later block of the pass.  Returns the dense work joined (sum of 2^k).
static double pass_with(const std::vector<Block>& blocks, const std::vector<char>& done, size_t first,
                        uint64_t local, std::vector<int>* out) {
    uint64_t blocked = 0;
    double work = 0;
    for (size_t b = first; b < blocks.size(); b++) {
        if (done[b]) continue;
        const Block& B = blocks[b];
        if (B.mask & blocked) {
            blocked |= B.mask;
            continue;
        }
        if (B.kind == BK_DIAG || (B.mask & ~local) == 0) {
            if (out) out->push_back((int)b);
            if (B.kind != BK_DIAG) work += (double)(1 << B.k);
        } else {
            blocked |= B.mask;
        }
    }
    return work;
}

std::vector<Pass> schedule(int n, const std::vector<Block>& blocks, int tile_m, int coalesce) {
    std::vector<Pass> passes;
    const size_t nb = blocks.size();
    std::vector<char> done(nb, 0);
    size_t first = 0;  // first block not yet done
    const uint64_t all = (n >= 64) ? ~0ull : ((1ull << n) - 1);
    if (tile_m >= n) {
        Pass p;
        p.local_mask = all;
        p.m = n;
        for (size_t b = 0; b < nb; b++) p.blocks.push_back((int)b);
        if (nb) passes.push_back(p);
        return passes;
    }
    const int c = std::min(coalesce, n);
    const uint64_t low = (1ull << c) - 1;
    auto fill = [&](uint64_t local) {  // up to tile_m qubits with the lowest unused ones
        for (int q = 0; q < n && popc(local) < tile_m; q++) local |= 1ull << q;
        return local;
    };
    while (first < nb) {
        // candidate 1: greedy, the tile grows with the blocks in list order
        uint64_t local = low, blocked = 0;
        for (size_t b = first; b < nb; b++) {
            if (done[b]) continue;
            const Block& B = blocks[b];
            if (B.mask & blocked) {
                blocked |= B.mask;
                continue;
            }
            if (B.kind == BK_DIAG) continue;
            const uint64_t need = local | B.mask;
            if (popc(need) <= tile_m) local = need;
            else blocked |= B.mask;
        }
        uint64_t best = fill(local);
        double best_work = pass_with(blocks, done, first, best, nullptr);
        // candidates 2: the low qubits plus a contiguous window of the others
        const int w = tile_m - c;
        for (int s = c; w > 0 && s + w <= n; s++) {
            const uint64_t cand = low | (((1ull << w) - 1) << s);
            const double work = pass_with(blocks, done, first, cand, nullptr);
            if (work > best_work) {
                best_work = work;
                best = cand;
            }
        }
        Pass p;
        pass_with(blocks, done, first, best, &p.blocks);
        for (int b : p.blocks) done[b] = 1;
        p.local_mask = best;
        p.m = popc(best);
        passes.push_back(p);
        while (first < nb && done[first]) first++;
    }
    return passes;
}

static bool tc_arith(int arith) { return arith == AK_TC || arith == AK_TC32; }

static double block_flops(const Block& b, double dim, int arith) {
    // real flops (FMA = 2) of the block applied to the whole 2^n state
    if (b.kind == BK_DIAG) return b.sign_only ? 0.0 : 6.0 * dim;
    if (b.kind == BK_PERM) return b.quarter ? 0.0 : 6.0 * dim;  // moves, then a phase pass if not quarter
    if (b.kind == BK_KRON && !tc_arith(arith)) return 16.0 * (double)b.k * dim;  // k butterflies
    return 8.0 * (double)(1 << b.k) * dim;
}

// ALU lane instructions per amplitude for one block.
static double block_instr(const Block& b, int arith) {
    const double D = (double)(1 << b.k);
    const double cmac = arith == AK_DF64 ? 44.0 : 4.0;  // one complex multiply-add
    if (b.kind == BK_DIAG) {
        if (b.sign_only) return 1.0;
        return cmac;
    }
    if (b.kind == BK_PERM) return 2.0 + (b.quarter ? 0.0 : cmac);
    // complex multiply-add: 4 real FMAs; double-float: 4 x (TwoProd + cross
    // terms + TwoSum) = 44 FP32 instructions; a Kronecker block is k one-qubit
    // butterflies (2 multiply-adds per amplitude each)
    if (b.kind == BK_KRON) return cmac * 2.0 * b.k;
    return cmac * D;
}

// Tensor-core modes: 16-bit MMA flops per amplitude of a dense block (digit
// pairs of a real 2D x 2D product: 28 for complex128, 6 for the complex64
// triple split; blocks of fewer than 3 qubits padded to 3) and CUDA-core
// operations per amplitude (digit split, re-assembly).
static double tc_mma_flops(const Block& b, int arith) {
    if (b.kind == BK_DIAG || b.kind == BK_PERM) return 0.0;
    const int k = std::max(3, b.k);
    return (arith == AK_TC32 ? 6.0 : 28.0) * 8.0 * (double)(1 << k);
}
static double tc_alu(const Block& b, int arith) {
    if (b.kind == BK_DIAG) return b.sign_only ? 2.0 : (arith == AK_TC32 ? 4.0 : 40.0);
    if (b.kind == BK_PERM) return 4.0 + (b.quarter ? 0.0 : (arith == AK_TC32 ? 4.0 : 40.0));
    return arith == AK_TC32 ? 30.0 : 150.0;
}

// Measured cost of one block, picoseconds per amplitude (sv_costs).
static double measured_ps(const Block& b, int arith, const sv_costs& c) {
    const bool tc = tc_arith(arith);
    const int kd = tc ? std::max(3, b.k) : b.k;
    switch (b.kind) {
        case BK_DIAG: return b.sign_only ? c.sign_ps : c.diag_ps;
        case BK_PERM: return c.perm_ps[b.k] + (b.quarter ? 0.0 : c.diag_ps);
        case BK_KRON: return tc ? c.dense_ps[kd] : b.k * c.dense_ps[1];
        default: return c.dense_ps[kd];
    }
}

// Time of one block over the whole state, without the pass it joins: the
// measured table, else the analytic terms of model_cost for the block alone.
static double block_cost(const Block& b, int arith, const Machine& mc, double dim, int amp_bytes) {
    if (mc.measured) return measured_ps(b, arith, *mc.measured) * 1e-12 * dim;
    const double rate = arith == AK_FP64 ? mc.fp64_ips : mc.fp32_ips;
    if (tc_arith(arith))
        return tc_alu(b, arith) * dim / rate +
               tc_mma_flops(b, arith) * dim / (arith == AK_TC32 ? mc.tc05_flops : mc.mma_flops);
    return std::max(block_instr(b, arith) * dim / rate, 2.0 * dim * amp_bytes / mc.smem_Bps);
}

double model_cost(const Plan& p, int amp_bytes, int arith, const Machine& mc, double* flops, double* alu_ops,
                  double* mma_flops) {
    const double dim = std::ldexp(1.0, p.n);
    const double state = dim * amp_bytes;
    const double rate = arith == AK_FP64 ? mc.fp64_ips : mc.fp32_ips;
    double total = 0, fl_all = 0, ops_all = 0, mma_all = 0;
    for (const auto& ps : p.passes) {
        double fl = 0, instr = 0, smem = 0, mma = 0;
        for (int bi : ps.blocks) {
            fl += block_flops(p.blocks[bi], dim, arith);
            if (arith == AK_TC || arith == AK_TC32) {
                instr += tc_alu(p.blocks[bi], arith) * dim;
                mma += tc_mma_flops(p.blocks[bi], arith) * dim;
            } else {
                instr += block_instr(p.blocks[bi], arith) * dim;
            }
            smem += 2.0 * state;
        }
        if (arith == AK_DF64 || arith == AK_TC) instr += 60.0 * dim;  // float64 conversions per pass
        fl_all += fl;
        ops_all += instr;
        mma_all += mma;
        if (mc.measured) {  // a pass's measured time: its tile traffic plus each op's
            double t_ps = mc.measured->pass_ps;
            for (int bi : ps.blocks) t_ps += measured_ps(p.blocks[bi], arith, *mc.measured);
            total += t_ps * 1e-12 * dim + mc.launch_s;
            continue;
        }
        const double alu = instr / rate + mma / (arith == AK_TC32 ? mc.tc05_flops : mc.mma_flops);
        const double hbm = 2.0 * state / mc.hbm_Bps;
        const double sm = smem / mc.smem_Bps;
        total += std::max(std::max(alu, hbm), sm) + mc.launch_s;
    }
    if (flops) *flops = fl_all;
    if (alu_ops) *alu_ops = ops_all;
    if (mma_flops) *mma_flops = mma_all;
    return total;
}

Plan make_plan(int n, const sv_gate* g, size_t ng, int fuse_k, int tile_m, int coalesce,
               int amp_bytes, int arith, const Machine& mc) {
    Plan best;
    best.model_s = 1e300;
    int k_lo = fuse_k > 0 ? fuse_k : 1, k_hi = fuse_k > 0 ? fuse_k : kMaxFuse;
    if (arith == AK_TC) {  // tensor-core blocks have at most 4 qubits
        k_hi = std::min(k_hi, 4);
        k_lo = std::min(k_lo, k_hi);
    }
    // the tensor-core modes pad blocks below 3 qubits to 3, so narrower
    // fusion only adds blocks: the autotuner starts at 3 there
    if (fuse_k == 0 && tc_arith(arith)) k_lo = std::min(3, k_hi);
    // the autotuner: every fusion width, with and without keeping runs of
    // monomial gates as permutation blocks, with and without packing gates
    // on disjoint qubits into one block.  The variants of a width are scored
    // by their blocks' cost alone and only the cheapest is scheduled into
    // passes (scheduling is most of the planning time), then the widths are
    // compared by the full cost model.
    const double dim = std::ldexp(1.0, n);
    for (int k = k_lo; k <= k_hi; k++) {
        std::vector<Block> chosen;
        double chosen_cost = 1e300;
        for (int variant = 0; variant < (k > 1 ? 6 : 1); variant++) {
            const int keep = variant % 3;
            const bool pack = variant >= 3;
            std::vector<Block> blocks = fuse(n, g, ng, k, keep, pack);
            // known before the matrices are formed: diagonal blocks made of CZ / Z
            // gates only are sign flips; permutation blocks without T / RZ / RZZ
            // have quarter phases
            for (auto& b : blocks) {
                bool sign = true, quarter = true;
                for (int t : b.gates) {
                    sign = sign && (g[t].op == SV_CZ || g[t].op == SV_Z);
                    quarter = quarter && g[t].op != SV_T && g[t].op != SV_RZ && g[t].op != SV_RZZ;
                }
                if (b.kind == BK_DIAG) b.sign_only = sign;
                if (b.kind == BK_PERM) b.quarter = quarter;
            }
            double cost = 0;
            for (const auto& b : blocks) cost += block_cost(b, arith, mc, dim, amp_bytes);
            if (cost < chosen_cost) {
                chosen_cost = cost;
                chosen.swap(blocks);
            }
        }
        Plan p;
        p.n = n;
        p.fuse_k = k;
        p.tile_m = std::min(tile_m, n);
        p.coalesce = std::min(coalesce, n);
        p.blocks.swap(chosen);
        p.passes = schedule(n, p.blocks, p.tile_m, p.coalesce);
        double fl = 0;
        p.model_s = model_cost(p, amp_bytes, arith, mc, &fl);
        p.flops = fl;
        if (p.model_s < best.model_s) best = std::move(p);
    }
    finalize(best.blocks, g);
    double fl = 0, ops = 0, mma = 0;
    best.model_s = model_cost(best, amp_bytes, arith, mc, &fl, &ops, &mma);
    best.flops = fl;
    best.alu_ops = ops;
    best.mma_flops = mma;
    return best;
}

int check_plan(const Plan& p, size_t ng, const sv_gate* g) {
    std::vector<int> seen(ng, 0);
    std::vector<int> last(p.n, -1);  // last gate index applied per qubit
    std::vector<char> used(p.blocks.size(), 0);
    for (const auto& ps : p.passes) {
        if (popc(ps.local_mask) != ps.m) return 1;
        for (int bi : ps.blocks) {
            if (bi < 0 || bi >= (int)p.blocks.size() || used[bi]) return 2;
            used[bi] = 1;
            const Block& b = p.blocks[bi];
            if (b.k < 1 || b.k > kMaxFuse) return 3;
            if (b.kind != BK_DIAG && (b.mask & ~ps.local_mask)) return 4;
            for (int t : b.gates) {
                if (t < 0 || (size_t)t >= ng || seen[t]) return 5;
                seen[t] = 1;
                uint64_t gm = gate_mask(g[t]);
                if (gm & ~b.mask) return 6;
                for (int q = 0; q < p.n; q++) {
                    if (!((gm >> q) & 1)) continue;
                    if (last[q] > t) return 7;  // per-qubit order broken
                    last[q] = t;
                }
            }
        }
    }
    for (size_t t = 0; t < ng; t++)
        if (!seen[t]) return 8;
    return 0;
}

}  // namespace svp

// Host planner of the streaming path: turns one circuit into the list of passes (tile programs),
// Pauli-sum launches and reductions that a QNG step needs. The schedule depends only on the gate
// list, never on theta, so it is built once per context and uploaded with the workspace.
//
// Segments, in launch order:
//   forward  psi <- U_{P-1} ... U_0 |0>                                   (Sec. 2, psi_k)
//   energy   b <- W psi; a <- H b (Pauli kernel); <E> = <b|a>; a <- W^dag a  (Eq. 2's <E>)
//   adjoint  for i = P-1..0: dE_i = -Im <psi|sigma_i|a>, then psi, a <- U_i^dag  (reverse sweep)
//   metric   for every column j: a <- psi, b <- F_j^dag sigma_j F_j psi, <sigma_j> = <F psi|sigma|F psi>,
//            psi <- U_j psi; then for i = j-1..0: L_ij = (1/4) Re <a|sigma_i|b>, a, b <- U_i^dag
//            (Algorithm 1's inner loop with phi = b and lambda = a, each step one adjoint gate on both)
//   metric (complex)  the same with Im <a|sigma_i|b> as well (the complex-metric call's segment)
// Consecutive steps of a segment share a pass while the qubits their non-diagonal operations act on
// fit in the tile window and their inner products fit in the slot budget.
#include <algorithm>
#include <cstdint>
#include <set>

#include "qng_large.h"

namespace qng {
namespace large {

namespace {

bool rot_kind(int k) { return k == QNG_GATE_RX || k == QNG_GATE_RY || k == QNG_GATE_RZ; }
int axis_of(int k) { return k == QNG_GATE_RX ? kAxisX : (k == QNG_GATE_RY ? kAxisY : kAxisZ); }

struct Group {
    std::vector<PassOp> ops;
    std::vector<RedSpec> reds; // inner products of the group; an op's slot indexes this list
};

PassOp mk(int kind) {
    PassOp o = {};
    o.kind = kind;
    o.r0 = o.r1 = -1;
    o.q0 = o.q1 = -1;
    o.axis = -1;
    o.param = -1;
    o.slot = -1;
    return o;
}

// reads / writes of an op, per register (bit r)
void access(const PassOp &o, int &rd, int &wr) {
    rd = wr = 0;
    switch (o.kind) {
    case kOpCopy: rd = 1 << o.r0; wr = 1 << o.r1; break;
    case kOpZero: wr = 1 << o.r0; break;
    case kOpRot:
    case kOpFixed: rd = wr = o.regs; break;
    case kOpSigma: rd = wr = 1 << o.r0; break;
    case kOpIp: rd = (1 << o.r0) | (1 << o.r1); break;
    case kOpStep: rd = (1 << o.r0) | (1 << o.r1); wr = o.param >= 0 ? rd : 0; break;
    case kOpStep2: rd = (1 << kRegA) | (1 << kRegB) | (1 << kRegB2); wr = o.param >= 0 ? rd : 0; break;
    default: break;
    }
}

// Local bit of qubit q in a pass's tile (low qubits, then the window), or -1 outside the tile.
int local_bit(const PassDesc &pd, int q) {
    if (q < 0) return -1;
    if (q < pd.low) return q;
    for (int k = 0; k < pd.win; ++k)
        if (pd.wq[k] == q) return pd.low + k;
    return -1;
}

// The qubit whose amplitude pairs an operation mixes (-1 when it is diagonal or touches no qubit).
int pair_target(const PassOp &o) {
    switch (o.kind) {
    case kOpRot:
    case kOpSigma:
    case kOpIp:
    case kOpStep:
    case kOpStep2: return (o.axis == kAxisX || o.axis == kAxisY) ? o.q0 : -1;
    case kOpFixed:
        if (o.fixed_kind == QNG_GATE_CNOT) return o.q1;
        if (o.fixed_kind == QNG_GATE_CZ || o.fixed_kind == QNG_GATE_Z) return -1;
        return o.q0;
    default: return -1;
    }
}

// Bank classes of the register-phase tile layout: the 16-byte chunk index c = l >> 1 is stored at
// c ^ ((c >> 3 ^ c >> 6 ^ c >> 9) & 7), so local bit b >= 1 moves the chunk's bank group along bit
// (b - 1) % 3 and local bit 0 picks the 8-byte half of the chunk. Threads of a half-warp (8-byte
// accesses) or quarter-warp (16-byte accesses) hit distinct banks when their thread-index bits are
// one local bit of each class.
int bank_class(int b) { return b == 0 ? 3 : (b - 1) % 3; }

// The straight-line form of operations [i, j) of a phase (PassPhase::macro), or 0.
int32_t macro_form(const std::vector<PassOp> &ops, size_t i, size_t j) {
    const int m = (int)(j - i);
    if (m < 1 || m > 4) return 0;
    bool steps = true, steps2 = true, fwd = true, rev = true, cnots = true;
    const int ax = ops[i].axis, regs = ops[i].regs;
    const int ab = (1 << kRegA) | (1 << kRegB), abb = ab | (1 << kRegB2);
    for (int k = 0; k < m; ++k) {
        const PassOp &o = ops[i + k];
        const bool xy = o.adjoint == 0 && o.axis == ax && (ax == kAxisX || ax == kAxisY);
        steps = steps && o.kind == kOpStep && o.r0 == kRegA && o.r1 == kRegB && xy;
        steps2 = steps2 && o.kind == kOpStep2 && xy;
        fwd = fwd && o.kt == k;
        rev = rev && o.kt == m - 1 - k;
        cnots = cnots && o.kind == kOpFixed && o.fixed_kind == QNG_GATE_CNOT && (regs == ab || regs == abb) &&
                o.regs == regs && o.kt == k && (k < m - 1 ? o.dk0 == k + 1 : o.dk0 < 0);
    }
    if ((steps || steps2) && (fwd || rev))
        return (steps ? kMacroSteps : kMacroSteps2) | (fwd ? 0 : kMacroRev) | (ax << 4) | m;
    if (cnots) return kMacroCnot | (regs == abb ? 1 << 4 : 0) | m;
    return 0;
}

// Diagonal operations on a and b: 1 a Z-axis step taking Re, 2 one taking Re and Im, 3 a CZ or Z
// gate; on a, b and b2 (two columns): 4, 5, 6 the same; 0 anything else.
int diag_kind(const PassOp &o) {
    const int ab = (1 << kRegA) | (1 << kRegB), abb = ab | (1 << kRegB2);
    const bool zs = o.axis == kAxisZ && (o.adjoint == 0 || o.adjoint == 2);
    if (o.kind == kOpStep && zs && o.r0 == kRegA && o.r1 == kRegB) return o.adjoint == 0 ? 1 : 2;
    if (o.kind == kOpStep2 && zs) return o.adjoint == 0 ? 4 : 5;
    if (o.kind == kOpFixed && (o.fixed_kind == QNG_GATE_CZ || o.fixed_kind == QNG_GATE_Z))
        return o.regs == ab ? 3 : (o.regs == abb ? 6 : 0);
    return 0;
}

// Mark the runs of diagonal operations among ops [i, j) of a phase (PassOp::zrun). Diagonal
// operators commute with one another, so within such a run every step's inner product
// <a|sigma_z|b> is the one on the run's starting registers, and the rotations and signs of the run
// compose into one phase factor per amplitude: the kernel applies them once, after the run's inner
// products.
void mark_zruns(std::vector<PassOp> &ops, size_t i, size_t j) {
    size_t o = i;
    while (o < j) {
        if (!diag_kind(ops[o])) {
            ++o;
            continue;
        }
        size_t e = o;
        const int fam = diag_kind(ops[o]) >= 4 ? 3 : 0;  // the run's register family: (a, b) or (a, b, b2)
        int im = 0, steps = 0;
        while (e < j && e - o < (size_t)kMaxZrun) {
            const int k = diag_kind(ops[e]);
            if (!k || (k > 3 ? 3 : 0) != fam) break;
            if (k - fam != 3) {
                if (im && k - fam != im) break;
                im = k - fam;
                ++steps;
            }
            ++e;
        }
        if (steps >= 2) {
            ops[o].zrun = (int8_t)((int)(e - o) | (im == 2 ? kZrunIm : 0) | (fam ? kZrunDual : 0));
            for (size_t x = o + 1; x < e; ++x) ops[x].zrun = -1;
        }
        o = e;
    }
}

// Split a pass's operations into register phases (see PassPhase): a phase takes operations while
// their pair targets fit in four register bits. ops are annotated with their register positions.
// Returns false when the pass needs more than kMaxPhases phases.
bool make_phases(const PassDesc &pd, std::vector<PassOp> &ops, std::vector<PassPhase> &out, size_t *fit_ops) {
    std::vector<PassPhase> ph;
    size_t i = 0;
    while (i < ops.size() || (ops.empty() && ph.empty())) {
        std::vector<int> R;
        size_t j = i;
        for (; j < ops.size(); ++j) {
            const int lb = local_bit(pd, pair_target(ops[j]));
            if (pair_target(ops[j]) < 0 || std::count(R.begin(), R.end(), lb)) continue;
            if (R.size() == 4) break;
            R.push_back(lb);
        }
        // fill to four register bits from the top, keeping a thread bit in every bank class
        auto left_in_class = [&](int cls) {
            int c = 0;
            for (int b = 0; b < kPhaseTile; ++b)
                if (bank_class(b) == cls && !std::count(R.begin(), R.end(), b)) ++c;
            return c;
        };
        for (int pass = 0; pass < 2 && R.size() < 4; ++pass)
            for (int b = kPhaseTile - 1; b >= 0 && R.size() < 4; --b) {
                if (std::count(R.begin(), R.end(), b)) continue;
                if (pass == 0 && (b == 0 || left_in_class(bank_class(b)) <= 1)) continue;
                R.push_back(b);
            }
        // local bit 0, when held, is register position 0 (16-byte accesses of amplitude pairs)
        auto z = std::find(R.begin(), R.end(), 0);
        if (z != R.end()) std::iter_swap(R.begin(), z);
        PassPhase p = {};
        p.op_begin = (int32_t)i;
        p.op_end = (int32_t)j;
        for (int k = 0; k < 4; ++k) p.rbit[k] = (int8_t)R[k];
        // thread bits: first one local bit of each bank class (16-byte mode: the three chunk
        // classes; 8-byte mode: the half bit too), then the rest in increasing order
        std::vector<int> T;
        const bool vmode = R[0] == 0;
        const int want[4] = {3, 0, 1, 2};
        for (int w = vmode ? 1 : 0; w < 4; ++w)
            for (int b = 0; b < kPhaseTile; ++b)
                if (bank_class(b) == want[w] && !std::count(R.begin(), R.end(), b) && !std::count(T.begin(), T.end(), b)) {
                    T.push_back(b);
                    break;
                }
        for (int b = 0; b < kPhaseTile; ++b)
            if (!std::count(R.begin(), R.end(), b) && !std::count(T.begin(), T.end(), b)) T.push_back(b);
        for (int k = 0; k < 8; ++k) p.tbit[k] = (int8_t)T[k];
        int rm = 0, wm = 0;
        for (size_t o = i; o < j; ++o) {
            PassOp &op = ops[o];
            auto pos = [&](int q) -> int8_t {
                const int lb = local_bit(pd, q);
                for (int k = 0; k < 4; ++k)
                    if (lb >= 0 && R[k] == lb) return (int8_t)k;
                return (int8_t)-1;
            };
            op.kt = pair_target(op) >= 0 ? pos(pair_target(op)) : (int8_t)-1;
            op.dk0 = pos(op.q0);
            op.dk1 = pos(op.q1);
            op.zrun = 0;
            int rd, wr;
            access(op, rd, wr);
            rm |= rd | wr;
            wm |= wr;
        }
        p.rmask = rm;
        p.wmask = wm;
        // the longest suffix of the phase's operations with a straight-line form; runs of diagonal
        // operations among the rest
        p.macro = 0;
        size_t mstart = j;
        for (size_t k = j >= 4 ? std::max(i, j - 4) : i; k < j && !p.macro; ++k) {
            p.macro = macro_form(ops, k, j);
            if (p.macro) mstart = k;
        }
        mark_zruns(ops, i, mstart);
        ph.push_back(p);
        if ((int)ph.size() > kMaxPhases) {
            *fit_ops = (size_t)ph[kMaxPhases].op_begin;
            return false;
        }
        if (ops.empty()) break;
        i = j;
    }
    out.insert(out.end(), ph.begin(), ph.end());
    return true;
}

struct Builder {
    int n, P, low, t, win;
    const std::vector<qng_gate> &gates;
    std::vector<int> rot_at;                 // gate index of rotation k
    std::vector<std::vector<int>> fixed_of;  // fixed gates of U_k (circuit order)
    std::vector<int> trailing;               // W
    Schedule &S;
    int parity = 0;

    Builder(const std::vector<qng_gate> &g, int n_, int P_, Schedule &s) : n(n_), P(P_), gates(g), S(s) {
        std::vector<int> pend;
        for (int k = 0; k < (int)g.size(); ++k) {
            if (rot_kind(g[k].kind)) {
                rot_at.push_back(k);
                fixed_of.push_back(pend);
                pend.clear();
            } else {
                pend.push_back(k);
            }
        }
        trailing = pend;
    }


    void add_fixed(Group &gr, int gi, int regs) {
        const qng_gate &g = gates[gi];
        PassOp o = mk(kOpFixed);
        o.regs = regs;
        o.fixed_kind = g.kind;
        o.q0 = g.q0;
        o.q1 = g.q1;
        gr.ops.push_back(o);
    }
    void add_rot(Group &gr, int k, bool adjoint, int regs) {
        const qng_gate &g = gates[rot_at[k]];
        PassOp o = mk(kOpRot);
        o.regs = regs;
        o.param = k;
        o.adjoint = adjoint;
        o.axis = axis_of(g.kind);
        o.q0 = g.q0;
        gr.ops.push_back(o);
    }
    // one recurrence step: inner product of (r0, r1) with sigma_k, then R_k^dag on both when rot;
    // im = 2 takes both parts, the imaginary one into kRegionLim at the same index
    void add_step(Group &gr, int k, int r0, int r1, int im, bool rot, double mul, int region, int64_t index) {
        const qng_gate &g = gates[rot_at[k]];
        PassOp o = mk(kOpStep);
        o.r0 = r0;
        o.r1 = r1;
        o.regs = (1 << r0) | (1 << r1);
        o.adjoint = im;
        o.axis = axis_of(g.kind);
        o.q0 = g.q0;
        o.param = rot ? k : -1;
        o.slot = (int)gr.reds.size();
        gr.ops.push_back(o);
        gr.reds.push_back(RedSpec{o.slot, mul, region, index});
        if (im == 2) gr.reds.push_back(RedSpec{o.slot + 1, mul, kRegionLim, index});
    }
    // the step of two columns that share a (kOpStep2): column index_b's entry from <a|sigma_k|b>,
    // column index_b2's from <a|sigma_k|b2>, then R_k^dag on a, b and b2 when rot
    void add_step2(Group &gr, int k, int im, bool rot, int64_t index_b, int64_t index_b2) {
        const qng_gate &g = gates[rot_at[k]];
        PassOp o = mk(kOpStep2);
        o.r0 = kRegA;
        o.r1 = kRegB;
        o.regs = (1 << kRegA) | (1 << kRegB) | (1 << kRegB2);
        o.adjoint = im;
        o.axis = axis_of(g.kind);
        o.q0 = g.q0;
        o.param = rot ? k : -1;
        o.slot = (int)gr.reds.size();
        gr.ops.push_back(o);
        if (im == 2) {
            gr.reds.push_back(RedSpec{o.slot, 0.25, kRegionL, index_b});
            gr.reds.push_back(RedSpec{o.slot + 1, 0.25, kRegionLim, index_b});
            gr.reds.push_back(RedSpec{o.slot + 2, 0.25, kRegionL, index_b2});
            gr.reds.push_back(RedSpec{o.slot + 3, 0.25, kRegionLim, index_b2});
        } else {
            gr.reds.push_back(RedSpec{o.slot, 0.25, kRegionL, index_b});
            gr.reds.push_back(RedSpec{o.slot + 1, 0.25, kRegionL, index_b2});
        }
    }
    // b <- F_k^dag sigma_k F_k src and <sigma_k> = <F_k src|sigma_k|F_k src> into kRegionSigma[k]: the
    // start of column k (src = psi or a, both Psi[k] there); also_src applies F_k to src as well
    void add_column_start(Group &gr, int k, int src, int b, bool also_src) {
        PassOp c = mk(kOpCopy);
        c.r0 = src;
        c.r1 = b;
        gr.ops.push_back(c);
        for (int gi : fixed_of[k]) add_fixed(gr, gi, (1 << b) | (also_src ? 1 << src : 0));
        add_ip(gr, k, b, b, 0, 1.0, kRegionSigma, k);
        const qng_gate &g = gates[rot_at[k]];
        PassOp sg = mk(kOpSigma);
        sg.r0 = b;
        sg.axis = axis_of(g.kind);
        sg.q0 = g.q0;
        gr.ops.push_back(sg);
        for (int f = (int)fixed_of[k].size() - 1; f >= 0; --f) add_fixed(gr, fixed_of[k][f], 1 << b);
    }
    void add_ip(Group &gr, int k_axis_param, int r0, int r1, int im, double mul, int region, int64_t index, bool sigma = true) {
        PassOp o = mk(kOpIp);
        o.r0 = r0;
        o.r1 = r1;
        o.adjoint = im;
        if (sigma) {
            const qng_gate &g = gates[rot_at[k_axis_param]];
            o.axis = axis_of(g.kind);
            o.q0 = g.q0;
        }
        o.slot = (int)gr.reds.size();
        gr.ops.push_back(o);
        gr.reds.push_back(RedSpec{o.slot, mul, region, index});
    }

    // Pack the segment's operations, in order, into passes: a pass takes operations while the
    // qubits their non-diagonal parts act on fit in the tile window and its inner products fit in
    // the slot budget (a step may span several passes). Then launch the segment's reduction.
    void emit(std::vector<Group> &groups, int segment, int dead_at_end) {
        struct Item { PassOp op; int need; int nred; int regs; RedSpec red[4]; };
        std::vector<Item> items;
        for (Group &g : groups) {
            for (const PassOp &o : g.ops) {
                Item it;
                it.op = o;
                it.need = -1;
                if (o.kind == kOpRot || o.kind == kOpSigma || o.kind == kOpIp || o.kind == kOpStep || o.kind == kOpStep2) {
                    if (o.axis == kAxisX || o.axis == kAxisY) it.need = o.q0;
                } else if (o.kind == kOpFixed) {
                    if (o.fixed_kind == QNG_GATE_CNOT) it.need = o.q1;
                    else if (o.fixed_kind != QNG_GATE_CZ && o.fixed_kind != QNG_GATE_Z) it.need = o.q0;
                }
                if (it.need >= 0 && it.need < low) it.need = -1;
                it.nred = (o.kind == kOpIp || o.kind == kOpStep) ? (o.kind == kOpStep && o.adjoint == 2 ? 2 : 1)
                        : (o.kind == kOpStep2 ? (o.adjoint == 2 ? 4 : 2) : 0);
                int rd, wr;
                access(o, rd, wr);
                it.regs = rd | wr;
                for (int r = 0; r < it.nred; ++r) it.red[r] = g.reds[o.slot + r];
                items.push_back(it);
            }
        }
        size_t i0 = 0;
        int slot_base = 0;
        const int red_begin = (int)S.reds.size();
        size_t limit = SIZE_MAX;  // operations of the next pass at most (register-phase limits)
        while (i0 < items.size()) {
            std::set<int> win_set;
            std::vector<PassOp> ops;
            std::vector<RedSpec> reds;
            int regs_used = 0;
            size_t i1 = i0;
            while (i1 < items.size()) {
                const Item &it = items[i1];
                const bool new_q = it.need >= 0 && !win_set.count(it.need);
                if (i1 > i0 && ((new_q && (int)win_set.size() >= win) || ((int)reds.size() + it.nred > kMaxSlots))) break;
                // at most three registers in a pass: the register-phase kernel holds three slots (psi and b2
                // share one), and the tile-program kernel keeps two CTAs per SM
                if (i1 > i0 && (S.phased || S.pairs) && __builtin_popcount(regs_used | it.regs) > 3) break;
                regs_used |= it.regs;
                if (i1 > i0 && (i1 - i0 >= limit || (S.phased && i1 - i0 >= (size_t)kMaxPhaseOps))) break;
                if (new_q) win_set.insert(it.need);
                PassOp o = it.op;
                if (it.nred) o.slot = (int)reds.size();
                for (int r = 0; r < it.nred; ++r) {
                    RedSpec rs = it.red[r];
                    rs.slot = o.slot + r;
                    reds.push_back(rs);
                }
                ops.push_back(o);
                ++i1;
            }
            PassDesc pd = {};
            pd.n = n;
            pd.low = low;
            std::vector<int> wq(win_set.begin(), win_set.end());
            for (int q = low; q < n && (int)wq.size() < win; ++q)
                if (!std::count(wq.begin(), wq.end(), q)) wq.push_back(q);
            std::sort(wq.begin(), wq.end());
            pd.win = (int)wq.size();
            for (int k = 0; k < kMaxWin; ++k) pd.wq[k] = k < pd.win ? wq[k] : -1;
            pd.t = low + pd.win;
            int first_read = 0, written = 0, touched = 0;
            for (const PassOp &o : ops) {
                int rd, wr;
                access(o, rd, wr);
                first_read |= rd & ~touched;  // the first access of these registers is a read: load them
                touched |= rd | wr;
                written |= wr;
            }
            pd.regmask = touched;
            pd.loadmask = first_read;
            pd.storemask = written;
            if (i1 == items.size()) pd.storemask &= ~dead_at_end;
            pd.phase_begin = (int)S.phases.size();
            pd.nphases = 0;
            if (S.phased) {
                size_t fit = 0;
                if (!make_phases(pd, ops, S.phases, &fit)) {
                    limit = fit;  // form this pass again with the operations its phases can take
                    continue;
                }
                pd.nphases = (int)S.phases.size() - pd.phase_begin;
            }
            limit = SIZE_MAX;
            pd.op_begin = (int)S.ops.size();
            pd.nops = (int)ops.size();
            pd.nslots = (int)reds.size();
            pd.slot_base = slot_base;
            pd.parity = parity++;
            S.ops.insert(S.ops.end(), ops.begin(), ops.end());
            for (RedSpec r : reds) {
                r.slot += slot_base;
                S.reds.push_back(r);
            }
            slot_base += (int)reds.size();
            S.max_slots = std::max(S.max_slots, slot_base);
            Launch L;
            L.kind = Launch::Pass;
            L.pass = (int)S.passes.size();
            L.segment = segment;
            S.passes.push_back(pd);
            S.launches.push_back(L);
            i0 = i1;
        }
        const int nred = (int)S.reds.size() - red_begin;
        if (nred > 0) {
            Launch L;
            L.kind = Launch::Reduce;
            L.item_begin = red_begin;
            L.nitems = nred;
            L.use_fac = 1;
            L.segment = segment;
            S.launches.push_back(L);
        }
    }
};

}  // namespace

void build_schedule(const std::vector<qng_gate> &gates, int n, int P, int precision, Schedule &S,
                    const std::vector<uint8_t> *want) {
    Builder B(gates, n, P, S);
    B.low = std::min(n, precision == QNG_C128 ? 4 : 5);
    B.win = std::min(kMaxWin, n - B.low);
    B.t = B.low + B.win;
    S.n = n;
    S.low = B.low;
    S.t = B.t;
    S.phased = precision == QNG_C64 && B.t == kPhaseTile;
    S.pairs = true;
    const int PSI = 1 << kRegPsi, A = 1 << kRegA, Bm = 1 << kRegB;

    // forward: psi <- U_{P-1} ... U_0 |0>
    {
        std::vector<Group> gs(std::max(P, 1));
        PassOp z = mk(kOpZero);
        z.r0 = kRegPsi;
        gs[0].ops.push_back(z);
        for (int k = 0; k < P; ++k) {
            for (int gi : B.fixed_of[k]) B.add_fixed(gs[k], gi, PSI);
            B.add_rot(gs[k], k, false, PSI);
        }
        B.emit(gs, kSegForward, 0);
    }
    // energy: b <- W psi, record scale(b)^2 at slot 0, scale(a) <- scale(b); Pauli kernel; a <- W^dag a
    {
        std::vector<Group> gs(1);
        PassOp c = mk(kOpCopy);
        c.r0 = kRegPsi;
        c.r1 = kRegB;
        gs[0].ops.push_back(c);
        for (int gi : B.trailing) B.add_fixed(gs[0], gi, Bm);
        PassOp rf = mk(kOpRecordFac);
        rf.r0 = rf.r1 = kRegB;
        rf.slot = 0;
        gs[0].ops.push_back(rf);
        PassOp ss = mk(kOpSetScale);
        ss.r0 = kRegB;
        ss.r1 = kRegA;
        gs[0].ops.push_back(ss);
        B.emit(gs, kSegEnergy, 0);
        S.passes.back().nslots = 0;  // slot 0 is filled by the Pauli kernel
        Launch h;
        h.kind = Launch::Hpsi;
        h.segment = kSegEnergy;
        S.launches.push_back(h);
        Launch r;
        r.kind = Launch::Reduce;
        r.item_begin = (int)S.reds.size();
        r.nitems = 1;
        r.use_fac = 1;
        r.segment = kSegEnergy;
        S.reds.push_back(RedSpec{0, 1.0, kRegionEnergy, 0});
        S.launches.push_back(r);
        std::vector<Group> gw(1);
        for (int f = (int)B.trailing.size() - 1; f >= 0; --f) B.add_fixed(gw[0], B.trailing[f], A);
        if (!gw[0].ops.empty()) B.emit(gw, kSegEnergy, 0);
    }
    // adjoint sweep over (psi, a = eta)
    if (P > 0) {
        std::vector<Group> gs(P);
        for (int s = 0; s < P; ++s) {
            const int i = P - 1 - s;
            B.add_step(gs[s], i, kRegPsi, kRegA, 1, i > 0, -1.0, kRegionGrad, i);
            if (i > 0)
                for (int f = (int)B.fixed_of[i].size() - 1; f >= 0; --f) B.add_fixed(gs[s], B.fixed_of[i][f], PSI | A);
        }
        B.emit(gs, kSegAdjoint, PSI | A);
    }
    // metric columns (segment kSegMetric, Re L), then the same with Im L (kSegMetricIm)
    for (const int im : {0, 2}) {
    B.parity = 0;
    // columns another rank computes: psi only advances through U_j (runs of them share passes)
    std::vector<Group> skipped;
    auto flush_skipped = [&]() {
        if (!skipped.empty()) B.emit(skipped, im ? kSegMetricIm : kSegMetric, 0);
        skipped.clear();
    };
    for (int j = 0; j < P; ++j) {
        if (want && !(*want)[j]) {
            skipped.emplace_back();
            Group &g = skipped.back();
            if (j == 0) {
                PassOp z = mk(kOpZero);
                z.r0 = kRegPsi;
                g.ops.push_back(z);
            }
            for (int gi : B.fixed_of[j]) B.add_fixed(g, gi, PSI);
            B.add_rot(g, j, false, PSI);
            continue;
        }
        flush_skipped();
        if (S.pairs && (j & 1) && j + 1 < P && (!want || (*want)[j + 1])) {
            // columns u = j + 1 and l = j together, for odd j only, so that a column subset pairs
            // exactly as the whole instance does (psi = Psi[l] here): psi advances through U_l and
            // column u starts from it; u's first step (i = l) takes a to Psi[l], from which column l
            // starts in b2; then for i = l - 1 .. 0 one step serves both columns, a rotated once
            const int l = j, u = j + 1;
            const int AB = A | Bm, AB2 = A | Bm | (1 << kRegB2);
            std::vector<Group> gs(l + 2);
            Group &g0 = gs[0];
            for (int gi : B.fixed_of[l]) B.add_fixed(g0, gi, PSI);
            B.add_rot(g0, l, false, PSI);
            PassOp ca = mk(kOpCopy);
            ca.r0 = kRegPsi;
            ca.r1 = kRegA;
            g0.ops.push_back(ca);
            B.add_column_start(g0, u, kRegPsi, kRegB, true);
            B.add_rot(g0, u, false, PSI);
            B.add_step(gs[1], l, kRegA, kRegB, im, true, 0.25, kRegionL, (int64_t)l * P + u);
            for (int f = (int)B.fixed_of[l].size() - 1; f >= 0; --f) B.add_fixed(gs[1], B.fixed_of[l][f], AB);
            B.add_column_start(gs[1], l, kRegA, kRegB2, false);
            for (int s = 1; s <= l; ++s) {
                const int i = l - s;
                Group &g = gs[1 + s];
                B.add_step2(g, i, im, i > 0, (int64_t)i * P + u, (int64_t)i * P + l);
                if (i > 0)
                    for (int f = (int)B.fixed_of[i].size() - 1; f >= 0; --f) B.add_fixed(g, B.fixed_of[i][f], AB2);
            }
            B.emit(gs, im ? kSegMetricIm : kSegMetric, AB2);
            ++j;
            continue;
        }
        std::vector<Group> gs(j + 1);
        Group &g0 = gs[0];
        if (j == 0) {
            PassOp z = mk(kOpZero);
            z.r0 = kRegPsi;
            g0.ops.push_back(z);
        }
        PassOp c1 = mk(kOpCopy);
        c1.r0 = kRegPsi;
        c1.r1 = kRegA;
        g0.ops.push_back(c1);
        PassOp c2 = mk(kOpCopy);
        c2.r0 = kRegPsi;
        c2.r1 = kRegB;
        g0.ops.push_back(c2);
        for (int gi : B.fixed_of[j]) B.add_fixed(g0, gi, PSI | Bm);
        B.add_ip(g0, j, kRegB, kRegB, 0, 1.0, kRegionSigma, j);
        {
            const qng_gate &g = gates[B.rot_at[j]];
            PassOp sg = mk(kOpSigma);
            sg.r0 = kRegB;
            sg.axis = axis_of(g.kind);
            sg.q0 = g.q0;
            g0.ops.push_back(sg);
        }
        for (int f = (int)B.fixed_of[j].size() - 1; f >= 0; --f) B.add_fixed(g0, B.fixed_of[j][f], Bm);
        B.add_rot(g0, j, false, PSI);
        for (int s = 1; s <= j; ++s) {
            const int i = j - s;
            Group &g = gs[s];
            B.add_step(g, i, kRegA, kRegB, im, i > 0, 0.25, kRegionL, (int64_t)i * P + j);
            if (i > 0)
                for (int f = (int)B.fixed_of[i].size() - 1; f >= 0; --f) B.add_fixed(g, B.fixed_of[i][f], A | Bm);
        }
        B.emit(gs, im ? kSegMetricIm : kSegMetric, A | Bm);
    }
    flush_skipped();
    }
}

}  // namespace large
}  // namespace qng

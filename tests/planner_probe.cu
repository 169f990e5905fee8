// Host-only probe of the streaming planner (qng_large_plan.cu), built and run by
// tests/test_planner_host.py: reads a circuit, builds the schedule for complex64 (register-phase
// passes) or complex128 (tile-program passes), optionally for a column subset, checks the
// schedule's structural invariants and prints what the test compares:
//   red <segment> <region> <index>   one line per inner-product destination
//   step <segment> <kind> <rot>       one line per recurrence step (kOpStep 8 / kOpStep2 9; rot 1 if it
//                                     rotates its registers)
//   ok                                every invariant held (else a line "bad <what>" and exit 1)
// Input (stdin): n P G precision nwant, then G lines "kind q0 q1 param", then nwant column indices.
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "qng_large.h"

using namespace qng;
using namespace qng::large;

static int bad(const char *what, long a, long b) {
    std::printf("bad %s %ld %ld\n", what, a, b);
    return 1;
}

static bool diagonal_op(const PassOp &o) {
    if ((o.kind == kOpStep || o.kind == kOpStep2) && o.axis == kAxisZ) return true;
    return o.kind == kOpFixed && (o.fixed_kind == QNG_GATE_CZ || o.fixed_kind == QNG_GATE_Z);
}

int main() {
    int n, P, G, prec, nwant;
    if (std::scanf("%d %d %d %d %d", &n, &P, &G, &prec, &nwant) != 5) return 2;
    std::vector<qng_gate> gates(G);
    for (qng_gate &g : gates)
        if (std::scanf("%d %d %d %d", &g.kind, &g.q0, &g.q1, &g.param) != 4) return 2;
    std::vector<uint8_t> want;
    if (nwant >= 0) {
        want.assign(P, 0);
        for (int k = 0; k < nwant; ++k) {
            int j;
            if (std::scanf("%d", &j) != 1) return 2;
            want[j] = 1;
        }
    }
    Schedule S;
    build_schedule(gates, n, P, prec, S, nwant >= 0 ? &want : nullptr);
    // the reduction that follows each pass (its slots index that reduction's items)
    std::vector<int> red_of(S.launches.size(), -1);
    for (int l = (int)S.launches.size() - 1, cur = -1; l >= 0; --l) {
        if (S.launches[l].kind == Launch::Reduce) cur = l;
        red_of[l] = cur;
    }
    for (size_t li = 0; li < S.launches.size(); ++li) {
        const Launch &L = S.launches[li];
        if (L.kind == Launch::Reduce) {
            for (int k = 0; k < L.nitems; ++k) {
                const RedSpec &r = S.reds[L.item_begin + k];
                std::printf("red %d %d %lld\n", L.segment, r.region, (long long)r.index);
            }
            continue;
        }
        if (L.kind != Launch::Pass) continue;
        const PassDesc &pd = S.passes[L.pass];
        // at most three registers a pass, psi and b2 never together
        if (S.pairs && __builtin_popcount(pd.regmask) > 3) return bad("registers", L.pass, pd.regmask);
        if ((pd.regmask & 9) == 9) return bad("psi_b2", L.pass, pd.regmask);
        if (pd.nslots > kMaxSlots) return bad("slots", L.pass, pd.nslots);
        for (int o = 0; o < pd.nops; ++o) {
            const PassOp &op = S.ops[pd.op_begin + o];
            if (op.kind == kOpStep || op.kind == kOpStep2)
                std::printf("step %d %d %d\n", L.segment, op.kind, op.param >= 0 ? 1 : 0);
            if (op.kind == kOpStep2) {
                // a paired step serves columns u = l + 1 and l, l odd: its two L destinations
                const int nv = op.adjoint == 2 ? 2 : 1;
                const RedSpec *r0 = nullptr, *r1 = nullptr;
                if (red_of[li] < 0) return bad("no_reduce", L.pass, o);
                const Launch &R = S.launches[red_of[li]];
                for (int k = 0; k < R.nitems; ++k) {
                    const RedSpec &r = S.reds[R.item_begin + k];
                    if (r.slot == pd.slot_base + op.slot) r0 = &r;
                    else if (r.slot == pd.slot_base + op.slot + nv) r1 = &r;
                }
                if (!r0 || !r1) return bad("step2_slots", L.pass, o);
                const long u = r0->index % P, l = r1->index % P;
                if (u != l + 1 || (l & 1) == 0 || r0->index / P != r1->index / P) return bad("pair", u, l);
            }
        }
        if (!S.phased) continue;
        if (pd.nphases < 1) return bad("nphases", L.pass, pd.nphases);
        for (int p = 0; p < pd.nphases; ++p) {
            const PassPhase &ph = S.phases[pd.phase_begin + p];
            for (int o = ph.op_begin; o < ph.op_end; ++o) {
                const PassOp &op = S.ops[pd.op_begin + o];
                // a non-diagonal target is one of the phase's register bits
                bool pairs_qubit = (op.kind == kOpRot || op.kind == kOpSigma || op.kind == kOpIp || op.kind == kOpStep ||
                                    op.kind == kOpStep2) && (op.axis == kAxisX || op.axis == kAxisY);
                if (op.kind == kOpFixed && op.fixed_kind != QNG_GATE_CZ && op.fixed_kind != QNG_GATE_Z) pairs_qubit = true;
                if (pairs_qubit && (op.kt < 0 || op.kt > 3)) return bad("target_not_register", L.pass, o);
                // a marked diagonal run: inside the phase, diagonal, at least two steps
                if (op.zrun > 0) {
                    const int len = op.zrun & kMaxZrun;
                    if (o + len > ph.op_end) return bad("zrun_span", L.pass, o);
                    int steps = 0;
                    for (int x = o; x < o + len; ++x) {
                        const PassOp &d = S.ops[pd.op_begin + x];
                        if (!diagonal_op(d)) return bad("zrun_member", L.pass, x);
                        if (x > o && d.zrun != -1) return bad("zrun_mark", L.pass, x);
                        steps += d.kind != kOpFixed;
                    }
                    if (steps < 2) return bad("zrun_steps", L.pass, o);
                }
            }
            if (ph.macro) {
                // a straight-line block: the phase's last m operations, steps in register-bit order
                const int m = ph.macro & 15, kind = ph.macro & ~0xFF;
                if (m < 1 || m > 4 || m > ph.op_end - ph.op_begin) return bad("macro_len", L.pass, p);
                const bool rev = (ph.macro & kMacroRev) != 0;
                for (int k = 0; k < m; ++k) {
                    const PassOp &op = S.ops[pd.op_begin + ph.op_end - m + k];
                    const int bit = rev ? m - 1 - k : k;
                    if (kind == kMacroCnot) {
                        if (op.kind != kOpFixed || op.fixed_kind != QNG_GATE_CNOT || op.kt != k) return bad("macro_cnot", L.pass, k);
                    } else {
                        const int want_kind = kind == kMacroSteps2 ? kOpStep2 : kOpStep;
                        if (op.kind != want_kind || op.kt != bit || op.axis != ((ph.macro >> 4) & 7) || op.zrun != 0)
                            return bad("macro_step", L.pass, k);
                    }
                }
            }
        }
    }
    std::printf("ok\n");
    return 0;
}

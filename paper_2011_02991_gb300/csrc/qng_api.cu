// Host side of the C ABI declared in include/qng.h: argument validation, the device tables,
// the workspace layout, launch grouping and the entry points.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "qng_internal.h"
#include "qng_large.h"

using namespace qng;

namespace qng {

cudaError_t raise_smem_limit(const void *fn, size_t bytes) {
    static std::mutex mu;  // read, compare and set as one step across host threads
    std::lock_guard<std::mutex> lock(mu);
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, fn);
    if (e != cudaSuccess) return e;
    if ((size_t)fa.maxDynamicSharedSizeBytes >= bytes) return cudaSuccess;
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace qng

namespace {

struct HostInst {
    int n = 0, P = 0;
    bool general = false;          // has generalised rotations (CRX..CRP)
    std::vector<qng_gate> gates;
    std::vector<uint64_t> masks;   // (xmask, zmask) per gate
    std::vector<qng_pauli> terms;
};

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

bool is_gen(int k) { return k >= QNG_GATE_CRX && k <= QNG_GATE_CRP; }
bool is_rot(int k) { return k == QNG_GATE_RX || k == QNG_GATE_RY || k == QNG_GATE_RZ || is_gen(k); }
bool is_fixed(int k) { return k >= QNG_GATE_CZ && k <= QNG_GATE_H; }
bool is_two_qubit(int k) { return k == QNG_GATE_CZ || k == QNG_GATE_CNOT; }

qng_status validate(int n, const qng_gate *gates, int n_gates, const uint64_t *masks, const qng_pauli *terms,
                    int n_terms, HostInst &out) {
    if (n < 1 || n > kMaxQubits || n_gates < 0 || n_terms < 0) return QNG_ERR_ARG;
    if ((n_gates > 0 && !gates) || (n_terms > 0 && !terms)) return QNG_ERR_ARG;
    const uint64_t full = (n == 64) ? ~0ull : ((1ull << n) - 1);
    out.n = n;
    out.P = 0;
    out.general = false;
    out.masks.assign(2 * (size_t)n_gates, 0);
    for (int g = 0; g < n_gates; ++g) {
        const qng_gate &x = gates[g];
        const bool string = x.kind == QNG_GATE_RP || x.kind == QNG_GATE_CRP;
        if (x.kind == QNG_GATE_RP ? x.q0 != -1 : (x.q0 < 0 || x.q0 >= n)) return QNG_ERR_ARG;
        if (string) {
            if (!masks) return QNG_ERR_ARG;
            const uint64_t xm = masks[2 * g], zm = masks[2 * g + 1];
            if ((xm & ~full) || (zm & ~full)) return QNG_ERR_ARG;
            if (x.kind == QNG_GATE_CRP && ((xm | zm) >> x.q0) & 1) return QNG_ERR_ARG;  // S must leave the control
            out.masks[2 * g] = xm;
            out.masks[2 * g + 1] = zm;
        }
        if (x.kind >= QNG_GATE_CRX && x.kind <= QNG_GATE_CRZ && (x.q1 < 0 || x.q1 >= n || x.q1 == x.q0))
            return QNG_ERR_ARG;
        if (is_rot(x.kind)) {
            if (x.param != out.P) return QNG_ERR_ARG;  // one unique parameter per gate, in circuit order
            out.P++;
            out.general = out.general || is_gen(x.kind);
        } else if (is_fixed(x.kind)) {
            if (x.param != -1) return QNG_ERR_ARG;
            if (is_two_qubit(x.kind) && (x.q1 < 0 || x.q1 >= n || x.q1 == x.q0)) return QNG_ERR_ARG;
        } else {
            return QNG_ERR_ARG;
        }
    }
    for (int t = 0; t < n_terms; ++t) {
        if (!std::isfinite(terms[t].coeff)) return QNG_ERR_ARG;
        if ((terms[t].xmask & ~full) || (terms[t].zmask & ~full)) return QNG_ERR_ARG;
    }
    out.gates.assign(gates, gates + n_gates);
    out.terms.assign(terms, terms + n_terms);
    return QNG_OK;
}

}  // namespace

constexpr int kPipeMax = 8;      // chunks of a pipelined sweep at most
constexpr int kPipeMinP = 64;    // automatic pipelining from this many parameters
constexpr int kPipeDefault = 3;  // chunks when automatic

struct qng_ctx {
    int precision = QNG_C128;
    int count = 0;
    std::vector<HostInst> inst;
    // device-table images (host copies, uploaded by qng_set_workspace)
    std::vector<DevInst> t_inst;
    std::vector<DevParam> t_param;
    std::vector<DevGen> t_gen;  // one per parameter, like t_param
    std::vector<DevFixed> t_fixed;
    std::vector<DevDiag> t_diag;
    std::vector<DevTerm> t_term;
    std::vector<DevWork> t_work;
    std::vector<int32_t> t_group_inst;
    std::vector<Group> groups;
    int64_t total_params = 0, total_metric = 0;
    int max_P = 0;
    std::vector<int64_t> param_off, metric_off;
    // workspace layout (byte offsets)
    size_t o_status = 0, o_inst = 0, o_param = 0, o_fixed = 0, o_diag = 0, o_term = 0, o_work = 0, o_ginst = 0;
    size_t o_pctrl = 0, o_gen = 0;
    size_t o_coef = 0, o_sigma = 0, o_scale = 0, o_L = 0, o_grad = 0, o_energy = 0, o_chol = 0, o_ckpt = 0, o_eta = 0;
    size_t o_io_theta = 0, o_io_dtheta = 0, o_io_g = 0, o_io_grad = 0, o_io_energy = 0;
    size_t ws_bytes = 0;      // bytes the current plan needs
    size_t ws_cap = 0;        // bytes of the workspace the caller set
    unsigned char *ws = nullptr;
    cudaStream_t stream = nullptr;
    bool prepared = false;
    // tuning
    int tune_min_qubits = 0, tune_cl = -1, tune_threads = 0;
    int path = 0;             // 0 automatic, 1 on-chip, 2 streaming
    std::vector<uint8_t> col_want;  // column subset of a single instance (empty: every column)
    std::vector<int> group_order;   // launch groups by decreasing work
    // streaming path (one instance, registers in HBM)
    bool streaming = false;
    large::Schedule sched;
    int l_grid = 0;
    size_t o_reg[large::kRegs] = {0, 0, 0, 0};
    size_t o_regscale = 0, o_partial = 0, o_slotfac = 0, o_pdesc = 0, o_pops = 0, o_red = 0, o_phases = 0;
    size_t o_queue = 0;
    // mixed-precision solve: cluster size (0 = not used: P < 48 or its float32 matrix does not fit)
    int ir_C = 0;
    size_t o_irflag = 0;
    // block solve (one instance whose P is beyond the cluster solve's shared memory)
    bool bsolve = false;
    int bs_C = 1;
    size_t o_srhs = 0, o_sy = 0, o_sdinv = 0;
    // CUDA graph of one captured qng_step
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    // per-qubit-count launch shapes chosen by the autotuner (-1: default)
    int tuned_cl[kMaxQubits + 1];
    int tuned_threads[kMaxQubits + 1];
    int tuned_fwd[kMaxQubits + 1];
    int tuned_fcl[kMaxQubits + 1];  // cluster size (log2) of the checkpoint sweep (-1: the column kernel's)
    int64_t last_launches = 0;
    int last_solve = QNG_SOLVE_NONE;  // which solve the last step launched
    // pipelined sweep (one on-chip instance): the checkpoint sweep in chunks on a high-priority
    // stream; the columns each chunk makes ready run on a stream of their own meanwhile
    int pipe_req = 0;  // qng_set_pipeline: 0 automatic, 1 off, 2..kPipeMax chunks
    bool pipe_ready = false;
    cudaStream_t pipe_fwd = nullptr;
    cudaStream_t pipe_col[kPipeMax] = {};
    cudaEvent_t pipe_ev0 = nullptr;
    cudaEvent_t pipe_evf[kPipeMax] = {}, pipe_evc[kPipeMax] = {};
    // kernel timing (qng_profile)
    bool profiling = false;
    struct Mark { int cls; cudaEvent_t a, b; };
    std::vector<Mark> marks;
    std::vector<cudaEvent_t> spare;
    double prof_ms[QNG_KERNEL_CLASSES] = {};
    int64_t prof_n[QNG_KERNEL_CLASSES] = {};

    qng_ctx() {
        for (int k = 0; k <= kMaxQubits; ++k) { tuned_cl[k] = -1; tuned_threads[k] = 0; tuned_fwd[k] = 0; tuned_fcl[k] = -1; }
    }
    ~qng_ctx() {
        if (graph_exec) cudaGraphExecDestroy(graph_exec);
        if (graph) cudaGraphDestroy(graph);
        if (pipe_fwd) cudaStreamDestroy(pipe_fwd);
        for (int k = 0; k < kPipeMax; ++k) {
            if (pipe_col[k]) cudaStreamDestroy(pipe_col[k]);
            if (pipe_evf[k]) cudaEventDestroy(pipe_evf[k]);
            if (pipe_evc[k]) cudaEventDestroy(pipe_evc[k]);
        }
        if (pipe_ev0) cudaEventDestroy(pipe_ev0);
        for (auto &m : marks) { cudaEventDestroy(m.a); cudaEventDestroy(m.b); }
        for (auto e : spare) cudaEventDestroy(e);
    }
    cudaEvent_t take_event() {
        if (!spare.empty()) { cudaEvent_t e = spare.back(); spare.pop_back(); return e; }
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        return e;
    }

    Work work() const {
        Work w;
        w.status = reinterpret_cast<int32_t *>(ws + o_status);
        w.inst = reinterpret_cast<const DevInst *>(ws + o_inst);
        w.param = reinterpret_cast<const DevParam *>(ws + o_param);
        w.gen = reinterpret_cast<const DevGen *>(ws + o_gen);
        w.fixed = reinterpret_cast<const DevFixed *>(ws + o_fixed);
        w.diag = reinterpret_cast<const DevDiag *>(ws + o_diag);
        w.term = reinterpret_cast<const DevTerm *>(ws + o_term);
        w.work = reinterpret_cast<const DevWork *>(ws + o_work);
        w.group_inst = reinterpret_cast<const int32_t *>(ws + o_ginst);
        w.coef = reinterpret_cast<DevCoef *>(ws + o_coef);
        w.sigma = reinterpret_cast<double *>(ws + o_sigma);
        w.pctrl = reinterpret_cast<double *>(ws + o_pctrl);
        w.scale = reinterpret_cast<double *>(ws + o_scale);
        w.L = reinterpret_cast<double *>(ws + o_L);
        w.gradraw = reinterpret_cast<double *>(ws + o_grad);
        w.energy = reinterpret_cast<double *>(ws + o_energy);
        w.chol = reinterpret_cast<double *>(ws + o_chol);
        w.Lim = w.chol;
        w.srhs = reinterpret_cast<double *>(ws + o_srhs);
        w.sy = reinterpret_cast<double *>(ws + o_sy);
        w.sdinv = reinterpret_cast<double *>(ws + o_sdinv);
        w.irflag = reinterpret_cast<int32_t *>(ws + o_irflag);
        w.ckpt = ws + o_ckpt;
        w.eta = ws + o_eta;
        return w;
    }
};

namespace {

size_t amp_bytes(int precision) { return precision == QNG_C128 ? 16 : 8; }

int solve_cluster_log2(int max_P);

int default_cl(int n, int precision) {
    const int base = 9;  // measured best for both precisions at 12 qubits: 8 CTAs of 512 amplitudes
    return std::max(0, std::min(kMaxClusterLog2, n - base));
}

// The checkpoint sweep has one barrier per parameter and little work between barriers: two
// amplitudes per thread (64..512 threads) hide more float64 latency than the column kernel's shape.
int default_fwd_threads(int nl) {
    return std::max(64, std::min(512, (1 << nl) / 2));
}

// Cluster size (log2) of the checkpoint sweep for n qubits. The sweep is one sequential chain per
// instance, so a single instance takes twice the column kernel's CTAs (up to 16) while each keeps
// at least 256 amplitudes (measured at 12 qubits, c128: sweep 0.257 -> 0.206 ms); batches keep
// the column kernel's size (their sweeps already run side by side).
int fwd_cluster(const qng_ctx *c, int n, int cl) {
    int f = cl;
    if (c->tuned_fcl[n] >= 0) f = c->tuned_fcl[n];
    else if (c->count == 1 && cl + 1 <= kMaxFwdClusterLog2 && n - (cl + 1) >= 8) f = cl + 1;
    return std::max(0, std::min(f, std::min(kMaxFwdClusterLog2, n - 1)));
}

// CTA size of the checkpoint sweep: as set, else half the column kernel's amplitudes per CTA but
// no more threads than the sweep's own amplitudes per CTA (at least 64).
int fwd_threads_for(const qng_ctx *c, int n, int cl, int fcl) {
    if (c->tuned_fwd[n] > 0) return c->tuned_fwd[n];
    return std::min(default_fwd_threads(n - cl), std::max(64, 1 << std::min(n - fcl, 20)));
}

int default_threads(int nl) {
    const uint32_t Nl = 1u << nl;
    if (Nl <= 256) return 64;
    if (Nl <= 1024) return 128;
    return 256;
}

// Block-solve scratch (right-hand side, y, inverse diagonal blocks), empty without the block solve.
template <class Take> void take_block_solve(qng_ctx *c, Take &take) {
    c->o_irflag = take(sizeof(int32_t) * c->count);
    const int P = c->bsolve ? c->inst[0].P : 0;
    const int nblk = (P + kSolveBlock - 1) / kSolveBlock;
    c->o_srhs = take(sizeof(double) * P);
    c->o_sy = take(sizeof(double) * P);
    c->o_sdinv = take(sizeof(double) * nblk * kSolveBlock * kSolveBlock);
}

// Streaming path: schedule of passes and the workspace layout (no checkpoints).
qng_status plan_streaming(qng_ctx *c, int64_t scale_n) {
    const HostInst &h = c->inst[0];
    const size_t ab = amp_bytes(c->precision);
    c->sched = large::Schedule();
    large::build_schedule(h.gates, h.n, h.P, c->precision, c->sched, c->col_want.empty() ? nullptr : &c->col_want);
    const int64_t ntiles = 1ll << (h.n - c->sched.t);
    // k_pass: two CTAs per SM; the register-phase kernel: one persistent CTA per SM (152 on GB300)
    c->l_grid = (int)std::min<int64_t>(ntiles, c->sched.phased ? 152 : 152 * 2);
    c->t_inst[0].cl = 0;
    size_t off = 0;
    auto take = [&](size_t bytes) { const size_t o = align256(off); off = o + std::max<size_t>(bytes, 1); return o; };
    c->o_status = take(256);
    c->o_inst = take(sizeof(DevInst) * c->t_inst.size());
    c->o_param = take(sizeof(DevParam) * std::max<size_t>(c->t_param.size(), 1));
    c->o_gen = take(sizeof(DevGen) * std::max<size_t>(c->t_gen.size(), 1));
    c->o_fixed = take(sizeof(DevFixed) * std::max<size_t>(c->t_fixed.size(), 1));
    c->o_diag = take(sizeof(DevDiag) * std::max<size_t>(c->t_diag.size(), 1));
    c->o_term = take(sizeof(DevTerm) * std::max<size_t>(c->t_term.size(), 1));
    c->o_work = take(8);
    c->o_ginst = take(8);
    c->o_coef = take(sizeof(DevCoef) * c->total_params);
    c->o_sigma = take(sizeof(double) * c->total_params);
    c->o_pctrl = take(sizeof(double) * c->total_params);
    c->o_scale = take(sizeof(double) * scale_n);
    c->o_L = take(sizeof(double) * c->total_metric);
    c->o_grad = take(sizeof(double) * c->total_params);
    c->o_energy = take(sizeof(double) * c->count);
    c->o_chol = take(sizeof(double) * c->total_metric);
    c->o_io_theta = take(sizeof(double) * c->total_params);
    c->o_io_dtheta = take(sizeof(double) * c->total_params);
    c->o_io_g = take(sizeof(double) * c->total_metric);
    c->o_io_grad = take(sizeof(double) * c->total_params);
    c->o_io_energy = take(sizeof(double) * c->count);
    take_block_solve(c, take);
    c->o_regscale = take(sizeof(double) * 2 * large::kRegs);
    c->o_partial = take(sizeof(double) * (size_t)c->sched.max_slots * c->l_grid);
    c->o_slotfac = take(sizeof(double) * (size_t)c->sched.max_slots);
    c->o_pdesc = take(sizeof(large::PassDesc) * std::max<size_t>(c->sched.passes.size(), 1));
    c->o_pops = take(sizeof(large::PassOp) * std::max<size_t>(c->sched.ops.size(), 1));
    c->o_phases = take(sizeof(large::PassPhase) * std::max<size_t>(c->sched.phases.size(), 1));
    c->o_red = take(sizeof(large::ReduceItem) * std::max<size_t>(c->sched.reds.size(), 1));
    // b2 only for a schedule whose metric columns walk in pairs
    for (int r = 0; r < large::kRegs; ++r) c->o_reg[r] = (r != large::kRegB2 || c->sched.pairs) ? take(ab << h.n) : 0;
    c->o_ckpt = c->o_eta = 0;
    c->ws_bytes = align256(off);
    c->groups.clear();
    c->prepared = false;
    return QNG_OK;
}

// Build the device-table images, the launch groups and the workspace layout.
qng_status plan(qng_ctx *c) {
    c->t_inst.clear(); c->t_param.clear(); c->t_gen.clear(); c->t_fixed.clear(); c->t_diag.clear(); c->t_term.clear();
    c->t_work.clear(); c->t_group_inst.clear(); c->groups.clear();
    c->param_off.assign(c->count + 1, 0);
    c->metric_off.assign(c->count + 1, 0);
    const size_t ab = amp_bytes(c->precision);
    int64_t ckpt_amps = 0, eta_amps = 0, scale_n = 0;
    c->max_P = 0;
    for (int b = 0; b < c->count; ++b) {
        const HostInst &h = c->inst[b];
        DevInst d = {};
        d.n = h.n;
        d.P = h.P;
        d.nterms = (int32_t)h.terms.size();
        d.param_off = c->param_off[b];
        d.metric_off = c->metric_off[b];
        c->param_off[b + 1] = c->param_off[b] + h.P;
        c->metric_off[b + 1] = c->metric_off[b] + (int64_t)h.P * h.P;
        d.ckpt_off = ckpt_amps;
        ckpt_amps += (int64_t)(h.P + 1) << h.n;
        d.eta_off = eta_amps;
        eta_amps += 1ll << h.n;
        d.scale_off = scale_n;
        scale_n += h.P + 2;
        d.param_tab = (int32_t)c->t_param.size();
        d.term_off = (int32_t)c->t_term.size();
        c->max_P = std::max(c->max_P, h.P);
        // parameters with their preceding fixed gates
        std::vector<const qng_gate *> pending;
        auto flush_into = [&](DevParam &p) {
            p.fix_begin = (int32_t)c->t_fixed.size();
            p.fix_count = (int32_t)pending.size();
            bool all_diag = true;
            for (const qng_gate *g : pending) {
                c->t_fixed.push_back(DevFixed{g->kind, g->q0, g->q1, 0});
                if (g->kind != QNG_GATE_CZ && g->kind != QNG_GATE_Z) all_diag = false;
            }
            p.zmask = 0;
            if (all_diag) {
                uint64_t shift_mask[64] = {0};
                for (const qng_gate *g : pending) {
                    if (g->kind == QNG_GATE_Z) {
                        p.zmask ^= 1ull << g->q0;
                    } else {
                        const int u = std::min(g->q0, g->q1), v = std::max(g->q0, g->q1);
                        shift_mask[v - u] ^= 1ull << u;
                    }
                }
                p.diag_begin = (int32_t)c->t_diag.size();
                for (int s = 1; s < 64; ++s)
                    if (shift_mask[s]) c->t_diag.push_back(DevDiag{s, 0, shift_mask[s]});
                p.diag_count = (int32_t)c->t_diag.size() - p.diag_begin;
            } else {
                p.diag_begin = 0;
                p.diag_count = -1;
            }
            pending.clear();
        };
        for (size_t gi = 0; gi < h.gates.size(); ++gi) {
            const qng_gate &g = h.gates[gi];
            if (is_rot(g.kind)) {
                DevParam p = {};
                DevGen gg = {};
                if (is_gen(g.kind)) {
                    // K = C (x) S: a Pauli on the target (CRX..CRZ) or the gate's string (RP, CRP)
                    p.axis = kAxisGen;
                    p.q = 0;
                    if (g.kind == QNG_GATE_RP || g.kind == QNG_GATE_CRP) {
                        gg.gx = h.masks[2 * gi];
                        gg.gz = h.masks[2 * gi + 1];
                    } else {
                        const uint64_t t = 1ull << g.q1;
                        gg.gx = g.kind == QNG_GATE_CRZ ? 0 : t;
                        gg.gz = g.kind == QNG_GATE_CRX ? 0 : t;
                    }
                    gg.gctrl = g.kind == QNG_GATE_RP ? 0 : 1ull << g.q0;
                    gg.gny = __builtin_popcountll(gg.gx & gg.gz) & 3;
                } else {
                    p.axis = g.kind == QNG_GATE_RX ? kAxisX : (g.kind == QNG_GATE_RY ? kAxisY : kAxisZ);
                    p.q = g.q0;
                }
                flush_into(p);
                c->t_param.push_back(p);
                c->t_gen.push_back(gg);
            } else {
                pending.push_back(&g);
            }
        }
        set_zruns(c->t_param.data() + d.param_tab, h.P);
        d.w_begin = (int32_t)c->t_fixed.size();
        d.w_count = (int32_t)pending.size();
        for (const qng_gate *g : pending) c->t_fixed.push_back(DevFixed{g->kind, g->q0, g->q1, 0});
        // terms grouped by X mask (stable): H psi gathers psi[m ^ x] once per distinct mask
        const size_t tfirst = c->t_term.size();
        for (const qng_pauli &t : h.terms) {
            DevTerm dt = {};
            dt.coeff = t.coeff;
            dt.x = t.xmask;
            dt.z = t.zmask;
            dt.ny = __builtin_popcountll(t.xmask & t.zmask) & 3;
            c->t_term.push_back(dt);
        }
        std::stable_sort(c->t_term.begin() + tfirst, c->t_term.end(),
                         [](const DevTerm &a, const DevTerm &b) { return a.x < b.x; });
        c->t_inst.push_back(d);
    }
    c->total_params = c->param_off[c->count];
    c->total_metric = c->metric_off[c->count];
    c->streaming = c->count == 1 && (c->path == 2 || (c->path == 0 && c->inst[0].n > kMaxQubitsSmall));
    if (c->streaming && c->inst[0].general) return QNG_ERR_UNSUPPORTED;  // generalised rotations: on-chip only
    // mixed-precision solve where the cluster solve is there to take over
    c->ir_C = 0;
    if (c->max_P >= kBlockSolveMinP && solve_cluster_log2(c->max_P) >= 0) {
        const int C = c->max_P >= 128 ? 8 : 4;
        if (solve_ir_smem_bytes(c->max_P, C) <= kMaxSmem) c->ir_C = C;
    }
    // the block solve takes over where the cluster solve's rows no longer fit in shared memory
    c->bsolve = false;
    if (c->count == 1 && c->inst[0].P >= kBlockSolveMinP && solve_cluster_log2(c->inst[0].P) < 0 &&
        sblock_smem_bytes(c->inst[0].P, 8) <= kMaxSmem) {
        c->bsolve = true;
        c->bs_C = 8;
    }
    if (c->streaming) return plan_streaming(c, scale_n);

    // groups: instances sharing (cluster size, column CTA size, sweep cluster size, sweep CTA size)
    std::vector<std::array<int, 4>> shape(c->count);
    for (int b = 0; b < c->count; ++b) {
        const int n = c->inst[b].n;
        int cl = default_cl(n, c->precision);
        if (c->tuned_cl[n] >= 0) cl = c->tuned_cl[n];
        if (c->tune_cl >= 0 && n >= c->tune_min_qubits) cl = c->tune_cl;
        cl = std::max(0, std::min(cl, std::min(kMaxClusterLog2, n - 1)));
        int th = default_threads(n - cl);
        if (c->tuned_threads[n] > 0) th = c->tuned_threads[n];
        if (c->tune_threads > 0 && n >= c->tune_min_qubits) th = c->tune_threads;
        const int fcl = fwd_cluster(c, n, cl);
        const int fth = fwd_threads_for(c, n, cl, fcl);
        shape[b] = {cl, th, fcl, fth};
        c->t_inst[b].cl = cl;
    }
    std::vector<std::array<int, 4>> keys(shape);
    std::sort(keys.begin(), keys.end());
    keys.erase(std::unique(keys.begin(), keys.end()), keys.end());
    for (const auto &key : keys) {
        Group g;
        g.cl = key[0];
        g.threads = key[1];
        g.fwd_cl = key[2];
        g.fwd_threads = key[3];
        g.first_inst = (int)c->t_group_inst.size();
        std::vector<DevWork> items;
        for (int b = 0; b < c->count; ++b) {
            if (shape[b] != key) continue;
            c->t_group_inst.push_back(b);
            g.general = g.general || c->inst[b].general;
            g.max_n = std::max(g.max_n, c->inst[b].n);
            g.max_P = std::max(g.max_P, c->inst[b].P);
            if (c->inst[b].P > 0)
                for (int j = 0; j <= c->inst[b].P; ++j)
                    if (j == c->inst[b].P || c->col_want.empty() || c->col_want[j]) items.push_back(DevWork{b, j});
        }
        g.num_inst = (int)c->t_group_inst.size() - g.first_inst;
        // longest first: steps x amplitudes (column j has j steps, the gradient column P)
        auto cost = [&](const DevWork &w) { return (double)std::max(w.col, 1) * (double)(1ll << c->inst[w.inst].n); };
        std::stable_sort(items.begin(), items.end(), [&](const DevWork &a, const DevWork &b) { return cost(a) > cost(b); });
        g.first_work = (int)c->t_work.size();
        c->t_work.insert(c->t_work.end(), items.begin(), items.end());
        g.num_work = (int)items.size();
        g.first_grad = (int)c->t_work.size();
        for (const DevWork &w : items) if (w.col == c->inst[w.inst].P) c->t_work.push_back(w);
        g.num_grad = (int)c->t_work.size() - g.first_grad;
        g.first_met = (int)c->t_work.size();
        for (const DevWork &w : items) if (w.col < c->inst[w.inst].P) c->t_work.push_back(w);
        g.num_met = (int)c->t_work.size() - g.first_met;
        const size_t Nl = size_t(1) << (g.max_n - g.cl);
        const int nw = g.threads / 32;
        const size_t state = Nl * ab * (g.cl ? 3 : 1);
        g.smem_fwd = (size_t(1) << (g.max_n - g.fwd_cl)) * ab * (g.fwd_cl ? 3 : 1) + 64 * sizeof(double);
        g.smem_col = state + (size_t)(g.max_P + 1) * nw * sizeof(double) + (size_t)(g.max_P + 1) * sizeof(double);
        g.smem_col_im = g.smem_col + (size_t)(g.max_P + 1) * nw * sizeof(double);
        if (g.smem_col > kMaxSmem || g.smem_fwd > kMaxSmem) return QNG_ERR_UNSUPPORTED;
        c->groups.push_back(g);
    }

    // workspace layout
    size_t off = 0;
    auto take = [&](size_t bytes) { const size_t o = align256(off); off = o + std::max<size_t>(bytes, 1); return o; };
    c->o_status = take(256);
    c->o_inst = take(sizeof(DevInst) * c->t_inst.size());
    c->o_param = take(sizeof(DevParam) * c->t_param.size());
    c->o_gen = take(sizeof(DevGen) * c->t_gen.size());
    c->o_fixed = take(sizeof(DevFixed) * c->t_fixed.size());
    c->o_diag = take(sizeof(DevDiag) * c->t_diag.size());
    c->o_term = take(sizeof(DevTerm) * c->t_term.size());
    c->o_work = take(sizeof(DevWork) * c->t_work.size());
    c->o_ginst = take(sizeof(int32_t) * c->t_group_inst.size());
    c->o_coef = take(sizeof(DevCoef) * c->total_params);
    c->o_sigma = take(sizeof(double) * c->total_params);
    c->o_pctrl = take(sizeof(double) * c->total_params);
    c->o_scale = take(sizeof(double) * scale_n);
    c->o_L = take(sizeof(double) * c->total_metric);
    c->o_grad = take(sizeof(double) * c->total_params);
    c->o_energy = take(sizeof(double) * c->count);
    c->o_chol = take(sizeof(double) * c->total_metric);
    c->o_io_theta = take(sizeof(double) * c->total_params);
    c->o_io_dtheta = take(sizeof(double) * c->total_params);
    c->o_io_g = take(sizeof(double) * c->total_metric);
    c->o_io_grad = take(sizeof(double) * c->total_params);
    c->o_io_energy = take(sizeof(double) * c->count);
    c->o_queue = take(256 * std::max<size_t>(c->groups.size(), 1));
    take_block_solve(c, take);
    c->o_ckpt = take(ab * (size_t)ckpt_amps);
    c->o_eta = take(ab * (size_t)eta_amps);
    c->ws_bytes = align256(off);
    c->prepared = false;
    return QNG_OK;
}

// cluster size of the distributed solve (-1: the single-CTA finish kernel is used)
int solve_cluster_log2(int max_P) {
    if (max_P < 48) return -1;
    for (int cl = 3; cl >= 0; --cl)
        if (solve_smem_bytes(max_P, cl) <= 200 * 1024) return cl;
    return -1;
}

qng_status cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return QNG_OK;
    std::fprintf(stderr, "libqng: CUDA error %s\n", cudaGetErrorString(e));
    return QNG_ERR_CUDA;
}

qng_status upload(qng_ctx *c) {
    auto put = [&](size_t o, const void *src, size_t bytes) -> cudaError_t {
        if (bytes == 0) return cudaSuccess;
        return cudaMemcpyAsync(c->ws + o, src, bytes, cudaMemcpyHostToDevice, c->stream);
    };
    cudaError_t e;
    if ((e = cudaMemsetAsync(c->ws + c->o_status, 0, 256, c->stream)) != cudaSuccess) return cuda_status(e);
    if ((e = put(c->o_inst, c->t_inst.data(), sizeof(DevInst) * c->t_inst.size())) != cudaSuccess) return cuda_status(e);
    if ((e = put(c->o_param, c->t_param.data(), sizeof(DevParam) * c->t_param.size())) != cudaSuccess) return cuda_status(e);
    if ((e = put(c->o_gen, c->t_gen.data(), sizeof(DevGen) * c->t_gen.size())) != cudaSuccess) return cuda_status(e);
    if ((e = put(c->o_fixed, c->t_fixed.data(), sizeof(DevFixed) * c->t_fixed.size())) != cudaSuccess) return cuda_status(e);
    if ((e = put(c->o_diag, c->t_diag.data(), sizeof(DevDiag) * c->t_diag.size())) != cudaSuccess) return cuda_status(e);
    if ((e = put(c->o_term, c->t_term.data(), sizeof(DevTerm) * c->t_term.size())) != cudaSuccess) return cuda_status(e);
    if ((e = put(c->o_work, c->t_work.data(), sizeof(DevWork) * c->t_work.size())) != cudaSuccess) return cuda_status(e);
    if ((e = put(c->o_ginst, c->t_group_inst.data(), sizeof(int32_t) * c->t_group_inst.size())) != cudaSuccess)
        return cuda_status(e);
    // host tables must stay valid until the copies ran: pageable-memory copies are staged
    // synchronously with respect to the host, so returning here is safe
    if (c->streaming) {
        const large::Schedule &S = c->sched;
        if ((e = put(c->o_pdesc, S.passes.data(), sizeof(large::PassDesc) * S.passes.size())) != cudaSuccess) return cuda_status(e);
        if ((e = put(c->o_pops, S.ops.data(), sizeof(large::PassOp) * S.ops.size())) != cudaSuccess) return cuda_status(e);
        if ((e = put(c->o_phases, S.phases.data(), sizeof(large::PassPhase) * S.phases.size())) != cudaSuccess)
            return cuda_status(e);
        std::vector<large::ReduceItem> items(S.reds.size());
        for (size_t k = 0; k < S.reds.size(); ++k) {
            const large::RedSpec &r = S.reds[k];
            size_t region = r.region == large::kRegionSigma ? c->o_sigma
                          : r.region == large::kRegionL ? c->o_L
                          : r.region == large::kRegionGrad ? c->o_grad
                          : r.region == large::kRegionLim ? c->o_chol : c->o_energy;
            items[k].slot = r.slot;
            items[k].pad = 0;
            items[k].mul = r.mul;
            items[k].dst = reinterpret_cast<double *>(c->ws + region) + r.index;
        }
        if ((e = put(c->o_red, items.data(), sizeof(large::ReduceItem) * items.size())) != cudaSuccess) return cuda_status(e);
        static const double ones[2 * large::kRegs] = {1, 1, 1, 1, 1, 1, 1, 1};
        if ((e = put(c->o_regscale, ones, sizeof(ones))) != cudaSuccess) return cuda_status(e);
        size_t pass_smem = 0;
        for (const large::PassDesc &pd : S.passes)
            pass_smem = std::max(pass_smem, (size_t)__builtin_popcount(pd.regmask) * (amp_bytes(c->precision) << pd.t));
        if ((e = large::prepare_pass(c->precision, std::max<size_t>(pass_smem, 1))) != cudaSuccess) return cuda_status(e);
        if (S.phased && (e = large::prepare_pass_phased()) != cudaSuccess) return cuda_status(e);
        const int scl = solve_cluster_log2(c->max_P);
        if (scl >= 0 && (e = prepare_solve(solve_smem_bytes(c->max_P, scl))) != cudaSuccess) return cuda_status(e);
        if (c->bsolve && (e = prepare_sblock(c->inst[0].P, c->bs_C)) != cudaSuccess) return cuda_status(e);
        if (c->ir_C > 0 && (e = prepare_solve_ir(c->max_P, c->ir_C)) != cudaSuccess) return cuda_status(e);
        c->prepared = true;
        return QNG_OK;
    }
    size_t sf = 0, sc = 0, sci = 0;
    for (const Group &g : c->groups) {
        sf = std::max(sf, g.smem_fwd);
        sc = std::max(sc, g.smem_col);
        sci = std::max(sci, std::min(g.smem_col_im, kMaxSmem));
    }
    if ((e = prepare_kernels(c->precision, sf, sc, sci)) != cudaSuccess) return cuda_status(e);
    const int scl = solve_cluster_log2(c->max_P);
    if (scl >= 0 && (e = prepare_solve(solve_smem_bytes(c->max_P, scl))) != cudaSuccess) return cuda_status(e);
    if (c->bsolve && (e = prepare_sblock(c->inst[0].P, c->bs_C)) != cudaSuccess) return cuda_status(e);
    if (c->ir_C > 0 && (e = prepare_solve_ir(c->max_P, c->ir_C)) != cudaSuccess) return cuda_status(e);
    // streams and events of the pipelined sweep (single instance) and of the launch groups side by
    // side (batches), made here so that no stream is created inside a graph capture
    if (!c->pipe_ready) {
        int lo = 0, hi = 0;
        if ((e = cudaDeviceGetStreamPriorityRange(&lo, &hi)) != cudaSuccess) return cuda_status(e);
        if ((e = cudaStreamCreateWithPriority(&c->pipe_fwd, cudaStreamNonBlocking, hi)) != cudaSuccess) return cuda_status(e);
        if ((e = cudaEventCreateWithFlags(&c->pipe_ev0, cudaEventDisableTiming)) != cudaSuccess) return cuda_status(e);
        for (int k = 0; k < kPipeMax; ++k) {
            if ((e = cudaStreamCreateWithPriority(&c->pipe_col[k], cudaStreamNonBlocking, lo)) != cudaSuccess ||
                (e = cudaEventCreateWithFlags(&c->pipe_evf[k], cudaEventDisableTiming)) != cudaSuccess ||
                (e = cudaEventCreateWithFlags(&c->pipe_evc[k], cudaEventDisableTiming)) != cudaSuccess)
                return cuda_status(e);
        }
        c->pipe_ready = true;
    }
    // launch groups, most work first (they run side by side on their own streams)
    c->group_order.resize(c->groups.size());
    for (size_t k = 0; k < c->groups.size(); ++k) c->group_order[k] = (int)k;
    {
        std::vector<double> work(c->groups.size(), 0.0);
        for (size_t k = 0; k < c->groups.size(); ++k) {
            const Group &g = c->groups[k];
            for (int t = 0; t < g.num_inst; ++t) {
                const HostInst &h = c->inst[c->t_group_inst[g.first_inst + t]];
                work[k] += (double)h.P * h.P * (double)(1ll << h.n);
            }
        }
        std::stable_sort(c->group_order.begin(), c->group_order.end(), [&](int a, int b) { return work[a] > work[b]; });
    }
    // batched contexts: persistent column launches fed by a device work counter per group
    for (size_t k = 0; k < c->groups.size(); ++k) {
        Group &g = c->groups[k];
        g.queue = nullptr;
        g.resident_clusters = 0;
        if (c->count > 1) {
            g.queue = reinterpret_cast<int *>(c->ws + c->o_queue + 256 * k);
            g.resident_clusters = resident_clusters(g, c->precision);
        }
    }
    c->prepared = true;
    return QNG_OK;
}

// Record events around a launch when profiling (class cls), on the stream it is launched on.
template <class F> cudaError_t timed_on(qng_ctx *c, int cls, cudaStream_t st, F &&launch) {
    if (!c->profiling) return launch();
    cudaEvent_t a = c->take_event(), b = c->take_event();
    if (!a || !b) return cudaErrorMemoryAllocation;
    cudaError_t e = cudaEventRecord(a, st);
    if (e == cudaSuccess) e = launch();
    if (e == cudaSuccess) e = cudaEventRecord(b, st);
    if (e != cudaSuccess) { c->spare.push_back(a); c->spare.push_back(b); return e; }
    c->marks.push_back({cls, a, b});
    return cudaSuccess;
}
template <class F> cudaError_t timed(qng_ctx *c, int cls, F &&launch) { return timed_on(c, cls, c->stream, launch); }

// Chunks of the pipelined sweep for this call (0: one sweep, then one column launch).
int pipe_chunks(const qng_ctx *c) {
    if (!c->pipe_ready || c->streaming || c->count != 1 || c->groups.size() != 1 || !c->col_want.empty()) return 0;
    const int P = c->inst[0].P;
    // automatic: only for circuits with generalised rotations (measured faster there; with plain
    // rotations the column phase ends on the latency of its longest items, which cannot start
    // before the sweep has ended, and chunking only adds launches)
    const bool auto_on = P >= kPipeMinP && c->groups[0].general;
    int S = c->pipe_req == 0 ? (auto_on ? kPipeDefault : 0) : (c->pipe_req == 1 ? 0 : c->pipe_req);
    S = std::min(S, P / 2);
    return S >= 2 ? S : 0;
}

// Work-list ranges of the columns each chunk of the sweep makes ready. Chunk s covers parameters
// [K_s, K_s+1) and writes checkpoints up to K_s+1; column j reads checkpoints 0..j, so chunk 0
// readies columns 0..K_1 and chunk s columns K_s + 1..K_s+1 (the last chunk also the gradient
// column, P, which needs eta). False if a chunk's items are not contiguous in the list.
bool pipe_ranges(const qng_ctx *c, const Group &g, int wm, int wg, int S, const std::vector<int> &K,
                 std::vector<std::array<int, 2>> &rng) {
    const int first = wm && wg ? g.first_work : (wm ? g.first_met : g.first_grad);
    const int num = wm && wg ? g.num_work : (wm ? g.num_met : g.num_grad);
    rng.assign(S, {INT32_MAX, -1});
    std::vector<int> cnt(S, 0);
    for (int t = first; t < first + num; ++t) {
        const int j = c->t_work[t].col;
        int s = 0;
        while (s + 1 < S && j > K[s + 1]) ++s;
        rng[s][0] = std::min(rng[s][0], t);
        rng[s][1] = std::max(rng[s][1], t);
        ++cnt[s];
    }
    for (int s = 0; s < S; ++s) {
        if (cnt[s] == 0) { rng[s] = {first, 0}; continue; }
        if (rng[s][1] - rng[s][0] + 1 != cnt[s]) return false;
        rng[s][1] = cnt[s];  // (first item, count)
    }
    return true;
}

// Kernel class (qng_profile_read) of a launch of the streaming schedule.
int stream_class(const large::Launch &L) {
    if (L.kind == large::Launch::Hpsi) return 5;
    if (L.kind == large::Launch::Reduce) return 7;
    switch (L.segment) {
    case large::kSegForward: return 1;
    case large::kSegEnergy: return 4;
    case large::kSegAdjoint: return 6;
    default: return 2;
    }
}

// The streaming schedule's launches for the requested jobs.
qng_status run_streaming(qng_ctx *c, int jobs, int64_t &launches) {
    const large::Schedule &S = c->sched;
    const HostInst &h = c->inst[0];
    const bool energy = jobs & (kJobEnergy | kJobGradient | kJobSolve);
    const bool grad = jobs & (kJobGradient | kJobSolve);
    const bool metric = jobs & (kJobMetric | kJobSolve);
    large::PassArgs pa = {};
    pa.ops = reinterpret_cast<const large::PassOp *>(c->ws + c->o_pops);
    pa.coef = reinterpret_cast<const DevCoef *>(c->ws + c->o_coef);
    for (int r = 0; r < large::kRegs; ++r) pa.reg[r] = (r != large::kRegB2 || S.pairs) ? c->ws + c->o_reg[r] : nullptr;
    pa.regscale = reinterpret_cast<double *>(c->ws + c->o_regscale);
    pa.partial = reinterpret_cast<double *>(c->ws + c->o_partial);
    pa.slotfac = reinterpret_cast<double *>(c->ws + c->o_slotfac);
    pa.phases = reinterpret_cast<const large::PassPhase *>(c->ws + c->o_phases);
    pa.status = reinterpret_cast<int32_t *>(c->ws + c->o_status);
    const large::PassDesc *descs = reinterpret_cast<const large::PassDesc *>(c->ws + c->o_pdesc);
    const large::ReduceItem *items = reinterpret_cast<const large::ReduceItem *>(c->ws + c->o_red);
    const size_t ab = amp_bytes(c->precision);
    for (const large::Launch &L : S.launches) {
        const bool metric_im = jobs & kJobMetricIm;
        const bool want = (L.segment == large::kSegForward || L.segment == large::kSegEnergy) ? energy
                        : L.segment == large::kSegAdjoint ? grad
                        : L.segment == large::kSegMetric ? metric && !metric_im
                                                         : metric && metric_im;
        const int cls = stream_class(L);
        if (!want) continue;
        cudaError_t e = cudaSuccess;
        if (L.kind == large::Launch::Pass) {
            const large::PassDesc &pd = S.passes[L.pass];
            pa.desc = descs + L.pass;
            const size_t smem = (size_t)__builtin_popcount(pd.regmask) * (ab << pd.t);
            const int mim = L.segment == large::kSegMetricIm ? 1 : 0;
            if (S.phased)
                e = timed(c, cls, [&] {
                    return large::launch_pass_phased(pa, pd.regmask, c->l_grid, mim, c->stream);
                });
            else
                e = timed(c, cls, [&] { return large::launch_pass(pa, c->precision, c->l_grid, 256, smem, mim, c->stream); });
        } else if (L.kind == large::Launch::Hpsi) {
            e = timed(c, cls, [&] {
                return large::launch_hpsi(c->ws + c->o_reg[large::kRegB], c->ws + c->o_reg[large::kRegA],
                                          reinterpret_cast<const DevTerm *>(c->ws + c->o_term), (int)h.terms.size(), h.n,
                                          c->precision, pa.partial, c->l_grid, c->stream);
            });
        } else {
            e = timed(c, cls, [&] {
                return large::launch_reduce(pa.partial, pa.slotfac, c->l_grid, items + L.item_begin, L.nitems, L.use_fac,
                                            c->stream);
            });
        }
        if (e != cudaSuccess) return cuda_status(e);
        ++launches;
    }
    return QNG_OK;
}

qng_status run(qng_ctx *c, int jobs, const LaunchArgs &args) {
    if (!c) return QNG_ERR_ARG;
    if (!c->ws || !c->prepared) return QNG_ERR_WORKSPACE;
    if (!args.theta && c->total_params > 0) return QNG_ERR_ARG;
    // with a column subset only the partial metric (kJobParts) and the step from gathered parts run
    if (!c->col_want.empty() && (jobs & (kJobMetric | kJobSolve | kJobMetricIm)) && !(jobs & (kJobParts | kJobFromParts)))
        return QNG_ERR_UNSUPPORTED;
    const Work w = c->work();
    int64_t launches = 0;
    cudaError_t e = cudaSuccess;
    if (c->total_params > 0) {
        e = timed(c, 0, [&] { return launch_coef(w, args.theta, c->total_params, c->stream); });
        if (e != cudaSuccess) return cuda_status(e);
        launches += 1;
    }
    if (jobs & kJobFromParts) {
        // the metric columns, sigma and the gradient were computed apart (column partition) and
        // gathered: place them where the assembly and the solve read them, then solve
        const HostInst &h = c->inst[0];
        const size_t PP = sizeof(double) * (size_t)h.P * h.P, P1 = sizeof(double) * (size_t)h.P;
        if ((e = cudaMemcpyAsync(w.L, args.parts_L, PP, cudaMemcpyDeviceToDevice, c->stream)) != cudaSuccess ||
            (e = cudaMemcpyAsync(w.sigma, args.parts_sigma, P1, cudaMemcpyDeviceToDevice, c->stream)) != cudaSuccess ||
            (e = cudaMemcpyAsync(w.gradraw, args.parts_grad, P1, cudaMemcpyDeviceToDevice, c->stream)) != cudaSuccess)
            return cuda_status(e);
    }
    const bool need_cols = !(jobs & kJobFromParts) && (jobs & (kJobMetric | kJobGradient | kJobSolve));
    const bool want_eta = jobs & (kJobGradient | kJobSolve);
    if (c->streaming && !(jobs & kJobFromParts)) {
        qng_status st = run_streaming(c, jobs, launches);
        if (st != QNG_OK) return st;
    }
    const int wm = (jobs & (kJobMetric | kJobSolve)) ? 1 : 0;
    const int wg = (jobs & (kJobGradient | kJobSolve)) ? 1 : 0;
    const int wim = (jobs & kJobMetricIm) ? 1 : 0;
    int S = (wm && !(jobs & kJobFromParts)) ? pipe_chunks(c) : 0;
    std::vector<int> K;
    std::vector<std::array<int, 2>> rng;
    if (S) {
        const int P = c->inst[0].P;
        for (int s = 0; s <= S; ++s) K.push_back((int)((int64_t)s * P / S));
        if (!pipe_ranges(c, c->groups[0], wm, wg, S, K, rng)) S = 0;
    }
    if (S) {
        // fork: the sweep's stream follows the coefficients; chunk s's columns follow chunk s;
        // join: the main stream waits for every column chunk (the last follows the whole sweep)
        const Group &g = c->groups[0];
        if ((e = cudaEventRecord(c->pipe_ev0, c->stream)) != cudaSuccess) return cuda_status(e);
        if ((e = cudaStreamWaitEvent(c->pipe_fwd, c->pipe_ev0, 0)) != cudaSuccess) return cuda_status(e);
        for (int s = 0; s < S; ++s) {
            e = timed_on(c, 1, c->pipe_fwd, [&] {
                return launch_forward(w, g, c->precision, want_eta, c->pipe_fwd, K[s], K[s + 1], s == S - 1);
            });
            if (e != cudaSuccess) return cuda_status(e);
            if ((e = cudaEventRecord(c->pipe_evf[s], c->pipe_fwd)) != cudaSuccess) return cuda_status(e);
            cudaStream_t cs = c->pipe_col[s];
            if ((e = cudaStreamWaitEvent(cs, c->pipe_evf[s], 0)) != cudaSuccess) return cuda_status(e);
            if (rng[s][1] > 0) {
                e = timed_on(c, 2, cs, [&] {
                    return launch_columns_range(w, g, c->precision, wim, rng[s][0], rng[s][1], false, cs);
                });
                if (e != cudaSuccess) return cuda_status(e);
                launches += 1;
            }
            if ((e = cudaEventRecord(c->pipe_evc[s], cs)) != cudaSuccess) return cuda_status(e);
            if ((e = cudaStreamWaitEvent(c->stream, c->pipe_evc[s], 0)) != cudaSuccess) return cuda_status(e);
            launches += 1;
        }
    }
    // batches: each launch group's sweep and columns on a stream of its own, most work first, so that
    // the groups fill one another's tails; joined before the solve. Automatic for complex128, whose
    // float64-bound groups leave the SMs room (batch256: 198 -> 172 ms per step); complex64 runs the
    // groups in turn, which measured as fast or faster (47.2 against 49.1 ms). qng_set_pipeline(ctx, 1)
    // runs them in turn, 2..8 side by side.
    const bool side_by_side = !S && !(jobs & kJobFromParts) && !c->streaming && c->count > 1 && c->pipe_ready &&
                              c->groups.size() > 1 && c->groups.size() <= (size_t)kPipeMax &&
                              (c->pipe_req >= 2 || (c->pipe_req == 0 && c->precision == QNG_C128));
    if (side_by_side) {
        if ((e = cudaEventRecord(c->pipe_ev0, c->stream)) != cudaSuccess) return cuda_status(e);
        for (size_t idx = 0; idx < c->group_order.size(); ++idx) {
            const Group &g = c->groups[c->group_order[idx]];
            if (g.num_inst == 0) continue;
            cudaStream_t gs = idx == 0 ? c->stream : c->pipe_col[idx];
            if (idx > 0 && (e = cudaStreamWaitEvent(gs, c->pipe_ev0, 0)) != cudaSuccess) return cuda_status(e);
            e = timed_on(c, 1, gs, [&] { return launch_forward(w, g, c->precision, want_eta, gs); });
            if (e != cudaSuccess) return cuda_status(e);
            launches += 1;
            if (need_cols && (wm && wg ? g.num_work : (wm ? g.num_met : g.num_grad)) > 0) {
                e = timed_on(c, 2, gs, [&] { return launch_columns(w, g, c->precision, wm, wg, wim, gs); });
                if (e != cudaSuccess) return cuda_status(e);
                launches += 1;
            }
            if (idx > 0) {
                if ((e = cudaEventRecord(c->pipe_evc[idx], gs)) != cudaSuccess) return cuda_status(e);
                if ((e = cudaStreamWaitEvent(c->stream, c->pipe_evc[idx], 0)) != cudaSuccess) return cuda_status(e);
            }
        }
    } else if (!S && !(jobs & kJobFromParts)) {
        for (const Group &g : c->groups) {
            if (g.num_inst == 0) continue;
            e = timed(c, 1, [&] { return launch_forward(w, g, c->precision, want_eta, c->stream); });
            if (e != cudaSuccess) return cuda_status(e);
            launches += 1;
        }
    }
    LaunchArgs a = args;
    a.jobs = jobs;
    if (need_cols && !S && !side_by_side) {
        for (const Group &g : c->groups) {
            if ((wm && wg ? g.num_work : (wm ? g.num_met : g.num_grad)) == 0) continue;
            e = timed(c, 2, [&] { return launch_columns(w, g, c->precision, wm, wg, wim, c->stream); });
            if (e != cudaSuccess) return cuda_status(e);
            launches += 1;
        }
    }
    if (jobs & kJobParts) {  // partial metric of a column subset: the raw parts go out, no assembly
        const HostInst &h = c->inst[0];
        const size_t PP = sizeof(double) * (size_t)h.P * h.P, P1 = sizeof(double) * (size_t)h.P;
        if ((args.parts_L && (e = cudaMemcpyAsync(args.parts_L, w.L, PP, cudaMemcpyDeviceToDevice, c->stream)) != cudaSuccess) ||
            (args.parts_sigma && (e = cudaMemcpyAsync(args.parts_sigma, w.sigma, P1, cudaMemcpyDeviceToDevice, c->stream)) != cudaSuccess) ||
            (args.grad_out && (e = cudaMemcpyAsync(args.grad_out, w.gradraw, P1, cudaMemcpyDeviceToDevice, c->stream)) != cudaSuccess) ||
            (args.energy_out && (e = cudaMemcpyAsync(args.energy_out, w.energy, sizeof(double), cudaMemcpyDeviceToDevice, c->stream)) != cudaSuccess))
            return cuda_status(e);
        c->last_launches = launches;
        return QNG_OK;
    }
    const int scl = solve_cluster_log2(c->max_P);
    if (jobs & kJobSolve)
        c->last_solve = c->bsolve ? QNG_SOLVE_BLOCK
                      : scl < 0   ? QNG_SOLVE_SINGLE
                      : c->ir_C > 0 ? QNG_SOLVE_MIXED : QNG_SOLVE_CLUSTER;
    if ((jobs & kJobSolve) && c->bsolve) {
        const int P = c->inst[0].P, nblk = (P + kSolveBlock - 1) / kSolveBlock;
        e = timed(c, 3, [&] {
            cudaError_t r = cudaSuccess;
            for (int K = 0; K < nblk && r == cudaSuccess; ++K) r = launch_sblock(w, a, P, c->bs_C, K, c->stream);
            return r == cudaSuccess ? launch_sback(w, a, P, c->stream) : r;
        });
        launches += nblk + 1;
    } else if ((jobs & kJobSolve) && scl >= 0 && c->ir_C > 0) {
        // mixed precision first; the float64 cluster solve takes any instance it hands over
        e = timed(c, 3, [&] {
            cudaError_t r = launch_solve_ir(w, c->count, c->max_P, c->ir_C, a, c->stream);
            if (r != cudaSuccess) return r;
            LaunchArgs ag = a;
            ag.ir_gate = 1;
            return launch_solve(w, c->count, c->max_P, scl, ag, c->stream);
        });
        launches += 2;
    } else if ((jobs & kJobSolve) && scl >= 0) {
        e = timed(c, 3, [&] { return launch_solve(w, c->count, c->max_P, scl, a, c->stream); });
        launches += 1;
    } else {
        e = timed(c, 3, [&] { return launch_finish(w, c->count, c->max_P, a, c->stream); });
        launches += 1;
    }
    if (e != cudaSuccess) return cuda_status(e);
    c->last_launches = launches;
    return QNG_OK;
}

}  // namespace

extern "C" {

qng_status qng_create(int n_qubits, const qng_gate *gates, int n_gates, const qng_pauli *terms, int n_terms,
                      int precision, qng_ctx **out) {
    const int32_t nq = n_qubits, ng = n_gates, nt = n_terms;
    return qng_create_batch_ex(1, &nq, gates, &ng, nullptr, terms, &nt, precision, out);
}

qng_status qng_create_ex(int n_qubits, const qng_gate *gates, int n_gates, const uint64_t *gate_masks,
                         const qng_pauli *terms, int n_terms, int precision, qng_ctx **out) {
    const int32_t nq = n_qubits, ng = n_gates, nt = n_terms;
    return qng_create_batch_ex(1, &nq, gates, &ng, gate_masks, terms, &nt, precision, out);
}

qng_status qng_create_batch(int count, const int32_t *n_qubits, const qng_gate *gates, const int32_t *n_gates,
                            const qng_pauli *terms, const int32_t *n_terms, int precision, qng_ctx **out) {
    return qng_create_batch_ex(count, n_qubits, gates, n_gates, nullptr, terms, n_terms, precision, out);
}

qng_status qng_create_batch_ex(int count, const int32_t *n_qubits, const qng_gate *gates, const int32_t *n_gates,
                               const uint64_t *gate_masks, const qng_pauli *terms, const int32_t *n_terms,
                               int precision, qng_ctx **out) {
    if (!out) return QNG_ERR_ARG;
    *out = nullptr;
    if (count < 1 || !n_qubits || !n_gates || !n_terms) return QNG_ERR_ARG;
    if (precision != QNG_C64 && precision != QNG_C128) return QNG_ERR_ARG;
    qng_ctx *c = new (std::nothrow) qng_ctx;
    if (!c) return QNG_ERR_OOM;
    c->precision = precision;
    c->count = count;
    try {
        c->inst.resize(count);
    } catch (...) {
        delete c;
        return QNG_ERR_OOM;
    }
    int64_t go = 0, to = 0;
    for (int b = 0; b < count; ++b) {
        qng_status s = validate(n_qubits[b], gates ? gates + go : nullptr, n_gates[b],
                                gate_masks ? gate_masks + 2 * go : nullptr, terms ? terms + to : nullptr, n_terms[b],
                                c->inst[b]);
        if (s != QNG_OK) { delete c; return s; }
        go += n_gates[b];
        to += n_terms[b];
        if (c->inst[b].n > kMaxQubitsSmall && count > 1) { delete c; return QNG_ERR_UNSUPPORTED; }
    }
    qng_status s = plan(c);
    if (s != QNG_OK) { delete c; return s; }
    *out = c;
    return QNG_OK;
}

qng_status qng_get_sizes(const qng_ctx *c, int32_t *count, int64_t *total_params, int64_t *total_metric) {
    if (!c) return QNG_ERR_ARG;
    if (count) *count = c->count;
    if (total_params) *total_params = c->total_params;
    if (total_metric) *total_metric = c->total_metric;
    return QNG_OK;
}

qng_status qng_get_offsets(const qng_ctx *c, int64_t *param_offset, int64_t *metric_offset) {
    if (!c) return QNG_ERR_ARG;
    if (param_offset) std::copy(c->param_off.begin(), c->param_off.end(), param_offset);
    if (metric_offset) std::copy(c->metric_off.begin(), c->metric_off.end(), metric_offset);
    return QNG_OK;
}

qng_status qng_workspace_size(const qng_ctx *c, size_t *bytes) {
    if (!c || !bytes) return QNG_ERR_ARG;
    *bytes = c->ws_bytes;
    return QNG_OK;
}

qng_status qng_set_workspace(qng_ctx *c, void *workspace, size_t bytes, void *stream) {
    if (!c) return QNG_ERR_ARG;
    if (!workspace || bytes < c->ws_bytes || (reinterpret_cast<uintptr_t>(workspace) & 255)) return QNG_ERR_WORKSPACE;
    c->ws = static_cast<unsigned char *>(workspace);
    c->ws_cap = bytes;
    c->stream = static_cast<cudaStream_t>(stream);
    return upload(c);
}

qng_status qng_set_stream(qng_ctx *c, void *stream) {
    if (!c) return QNG_ERR_ARG;
    c->stream = static_cast<cudaStream_t>(stream);
    return QNG_OK;
}

qng_status qng_set_tuning(qng_ctx *c, int min_qubits, int cluster_log2, int threads) {
    if (!c) return QNG_ERR_ARG;
    if (cluster_log2 < -1 || cluster_log2 > kMaxClusterLog2) return QNG_ERR_ARG;
    if (threads != 0 && (threads < 64 || threads > 256 || threads % 32)) return QNG_ERR_ARG;
    const int old_min = c->tune_min_qubits, old_cl = c->tune_cl, old_th = c->tune_threads;
    c->tune_min_qubits = min_qubits;
    c->tune_cl = cluster_log2 == 0 && threads == 0 && min_qubits == 0 ? -1 : cluster_log2;
    c->tune_threads = threads;
    qng_status s = plan(c);
    if (s != QNG_OK || (c->ws && c->ws_bytes > c->ws_cap)) {
        c->tune_min_qubits = old_min; c->tune_cl = old_cl; c->tune_threads = old_th;
        plan(c);
        if (c->ws) upload(c);
        return s != QNG_OK ? s : QNG_ERR_WORKSPACE;
    }
    if (c->ws) return upload(c);
    return QNG_OK;
}

qng_status qng_metric(qng_ctx *c, const double *theta, double *g, double *sigma_opt) {
    if (!c || !g) return QNG_ERR_ARG;
    LaunchArgs a = {};
    a.theta = theta;
    a.g_out = g;
    a.sigma_out = sigma_opt;
    return run(c, kJobMetric, a);
}

qng_status qng_metric_complex(qng_ctx *c, const double *theta, double *g, double *g_im, double *sigma_opt) {
    if (!c || !g || !g_im) return QNG_ERR_ARG;
    for (const Group &grp : c->groups)
        if (grp.smem_col_im > kMaxSmem) return QNG_ERR_UNSUPPORTED;
    LaunchArgs a = {};
    a.theta = theta;
    a.g_out = g;
    a.gim_out = g_im;
    a.sigma_out = sigma_opt;
    return run(c, kJobMetric | kJobMetricIm, a);
}

qng_status qng_gradient(qng_ctx *c, const double *theta, double *grad, double *energy) {
    if (!c || !grad) return QNG_ERR_ARG;
    LaunchArgs a = {};
    a.theta = theta;
    a.grad_out = grad;
    a.energy_out = energy;
    return run(c, kJobGradient | kJobEnergy, a);
}

qng_status qng_energy(qng_ctx *c, const double *theta, double *energy) {
    if (!c || !energy) return QNG_ERR_ARG;
    LaunchArgs a = {};
    a.theta = theta;
    a.energy_out = energy;
    return run(c, kJobEnergy, a);
}

qng_status qng_energy_backward(qng_ctx *c, const double *theta, const double *grad_out, double *grad_theta) {
    if (!c || !grad_out || !grad_theta) return QNG_ERR_ARG;
    LaunchArgs a = {};
    a.theta = theta;
    a.grad_out = grad_theta;
    a.grad_scale = grad_out;
    return run(c, kJobGradient, a);
}

qng_status qng_step(qng_ctx *c, const double *theta, double dt, double lambda, double *dtheta, double *g_opt,
                    double *grad_opt, double *energy_opt) {
    if (!c || !dtheta) return QNG_ERR_ARG;
    if (!std::isfinite(dt) || !std::isfinite(lambda) || lambda < 0) return QNG_ERR_ARG;
    LaunchArgs a = {};
    a.theta = theta;
    a.dtheta_out = dtheta;
    a.g_out = g_opt;
    a.grad_out = grad_opt;
    a.energy_out = energy_opt;
    a.dt = dt;
    a.lambda = lambda;
    return run(c, kJobSolve | kJobGradient | kJobEnergy | kJobMetric, a);
}

qng_status qng_optimize(qng_ctx *c, double *theta, double dt, double lambda, int iters, double *energies) {
    if (!c || iters < 0 || (!theta && c->total_params > 0)) return QNG_ERR_ARG;
    if (!std::isfinite(dt) || !std::isfinite(lambda) || lambda < 0) return QNG_ERR_ARG;
    if (!c->ws || !c->prepared) return QNG_ERR_WORKSPACE;
    double *dth = reinterpret_cast<double *>(c->ws + c->o_io_dtheta);
    int64_t launches = 0;
    for (int t = 0; t < iters; ++t) {
        LaunchArgs a = {};
        a.theta = theta;
        a.dtheta_out = dth;
        a.energy_out = energies ? energies + (int64_t)t * c->count : nullptr;
        a.dt = dt;
        a.lambda = lambda;
        const qng_status s = run(c, kJobSolve | kJobGradient | kJobEnergy | kJobMetric, a);
        if (s != QNG_OK) return s;
        launches += c->last_launches + 1;
        const cudaError_t e = timed(c, 0, [&] { return launch_theta_update(c->work(), theta, dth, c->total_params, c->stream); });
        if (e != cudaSuccess) return cuda_status(e);
    }
    c->last_launches = launches;
    return QNG_OK;
}

qng_status qng_step_host(qng_ctx *c, const double *theta_host, double dt, double lambda, double *dtheta_host,
                         double *g_host, double *grad_host, double *energy_host) {
    if (!c || !dtheta_host || (!theta_host && c->total_params > 0)) return QNG_ERR_ARG;
    if (!c->ws || !c->prepared) return QNG_ERR_WORKSPACE;
    double *th = reinterpret_cast<double *>(c->ws + c->o_io_theta);
    double *dth = reinterpret_cast<double *>(c->ws + c->o_io_dtheta);
    double *g = reinterpret_cast<double *>(c->ws + c->o_io_g);
    double *gr = reinterpret_cast<double *>(c->ws + c->o_io_grad);
    double *en = reinterpret_cast<double *>(c->ws + c->o_io_energy);
    const size_t pb = sizeof(double) * c->total_params, mb = sizeof(double) * c->total_metric;
    cudaError_t e;
    if (pb && (e = cudaMemcpyAsync(th, theta_host, pb, cudaMemcpyHostToDevice, c->stream)) != cudaSuccess)
        return cuda_status(e);
    qng_status s = qng_step(c, th, dt, lambda, dth, g_host ? g : nullptr, grad_host ? gr : nullptr,
                            energy_host ? en : nullptr);
    if (s != QNG_OK) return s;
    if (pb && (e = cudaMemcpyAsync(dtheta_host, dth, pb, cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess)
        return cuda_status(e);
    if (g_host && mb && (e = cudaMemcpyAsync(g_host, g, mb, cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess)
        return cuda_status(e);
    if (grad_host && pb && (e = cudaMemcpyAsync(grad_host, gr, pb, cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess)
        return cuda_status(e);
    if (energy_host &&
        (e = cudaMemcpyAsync(energy_host, en, sizeof(double) * c->count, cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess)
        return cuda_status(e);
    return qng_sync(c);
}

qng_status qng_sync(qng_ctx *c) {
    if (!c) return QNG_ERR_ARG;
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_status(e);
    if (!c->ws) return QNG_OK;
    int32_t st = 0;
    if ((e = cudaMemcpyAsync(&st, c->ws + c->o_status, sizeof(st), cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess)
        return cuda_status(e);
    if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return cuda_status(e);
    if (st != 0) {
        if ((e = cudaMemsetAsync(c->ws + c->o_status, 0, sizeof(int32_t), c->stream)) != cudaSuccess) return cuda_status(e);
        if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return cuda_status(e);
        return static_cast<qng_status>(st);
    }
    return QNG_OK;
}

qng_status qng_set_path(qng_ctx *c, int path) {
    if (!c || path < 0 || path > 2) return QNG_ERR_ARG;
    if (path == 1 && c->count == 1 && c->inst[0].n > kMaxQubitsSmall) return QNG_ERR_UNSUPPORTED;
    if (path == 2 && c->count != 1) return QNG_ERR_UNSUPPORTED;
    const int old = c->path;
    c->path = path;
    qng_status s = plan(c);
    if (s != QNG_OK || (c->ws && c->ws_bytes > c->ws_cap)) {
        c->path = old;
        plan(c);
        if (c->ws) upload(c);
        return s != QNG_OK ? s : QNG_ERR_WORKSPACE;
    }
    if (c->ws) return upload(c);
    return QNG_OK;
}

qng_status qng_column_partition(int P, int ranks, int rank, int32_t *cols, int *ncols) {
    if (P < 0 || ranks < 1 || rank < 0 || rank >= ranks || !ncols || (P > 0 && !cols)) return QNG_ERR_ARG;
    // Units: the adjacent pairs (l, l + 1), l odd, whose walks share register a on the streaming
    // complex64 path (a rank holding both columns of a unit pairs them exactly as the whole
    // instance does), column 0 and, for even P, column P - 1 alone. Column j has j recurrence steps.
    // Groups: the units t and T - 1 - t together (2(P - 1) steps for even P: two pairs {k, P-1-k});
    // the middle unit of an odd count; columns 0 and P - 1 together. Groups go, largest first, to
    // the rank with the fewest steps so far (ties: the lowest rank), the same on every rank.
    std::vector<std::pair<int, int>> U;
    for (int l = 1; l + 1 < P; l += 2) U.push_back({l, l + 1});
    std::vector<std::vector<int32_t>> groups;
    if (P > 0) groups.push_back((P % 2 == 0 && P >= 2) ? std::vector<int32_t>{0, P - 1} : std::vector<int32_t>{0});
    const int T = (int)U.size();
    for (int t = 0; t < T / 2; ++t)
        groups.push_back({U[t].first, U[t].second, U[T - 1 - t].first, U[T - 1 - t].second});
    if (T & 1) groups.push_back({U[T / 2].first, U[T / 2].second});
    auto steps = [](const std::vector<int32_t> &g) {
        int64_t s = 0;
        for (int32_t j : g) s += j;
        return s;
    };
    std::stable_sort(groups.begin(), groups.end(), [&](const std::vector<int32_t> &a, const std::vector<int32_t> &b) {
        return steps(a) > steps(b);
    });
    std::vector<int64_t> load(ranks, 0);
    std::vector<int32_t> mine;
    for (const std::vector<int32_t> &g : groups) {
        const int r = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        load[r] += steps(g);
        if (r == rank) mine.insert(mine.end(), g.begin(), g.end());
    }
    std::sort(mine.begin(), mine.end());
    int m = 0;
    for (int32_t j : mine) cols[m++] = j;
    *ncols = m;
    return QNG_OK;
}

qng_status qng_set_column_subset(qng_ctx *c, const int32_t *cols, int ncols) {
    if (!c) return QNG_ERR_ARG;
    if (c->count != 1) return QNG_ERR_UNSUPPORTED;
    if (c->inst[0].general) return QNG_ERR_UNSUPPORTED;
    const int P = c->inst[0].P;
    std::vector<uint8_t> want;
    if (cols && ncols >= 0) {
        want.assign(std::max(P, 1), 0);
        for (int k = 0; k < ncols; ++k) {
            if (cols[k] < 0 || cols[k] >= P || want[cols[k]]) return QNG_ERR_ARG;
            want[cols[k]] = 1;
        }
    }
    std::vector<uint8_t> old = c->col_want;
    c->col_want = want;
    qng_status s = plan(c);
    if (s != QNG_OK || (c->ws && c->ws_bytes > c->ws_cap)) {
        c->col_want = old;
        plan(c);
        if (c->ws) upload(c);
        return s != QNG_OK ? s : QNG_ERR_WORKSPACE;
    }
    if (c->ws) return upload(c);
    return QNG_OK;
}

qng_status qng_metric_columns(qng_ctx *c, const double *theta, double *L, double *sigma, double *grad, double *energy) {
    if (!c || !L || !sigma) return QNG_ERR_ARG;
    if (c->count != 1) return QNG_ERR_UNSUPPORTED;
    LaunchArgs a = {};
    a.theta = theta;
    a.parts_L = L;
    a.parts_sigma = sigma;
    a.grad_out = grad;
    a.energy_out = energy;
    return run(c, kJobMetric | kJobGradient | kJobParts, a);
}

qng_status qng_step_from_parts(qng_ctx *c, const double *theta, const double *L, const double *sigma,
                               const double *grad, double dt, double lambda, double *dtheta, double *g_opt) {
    if (!c || !L || !sigma || !grad || !dtheta || !(lambda >= 0.0) || !std::isfinite(dt)) return QNG_ERR_ARG;
    if (c->count != 1) return QNG_ERR_UNSUPPORTED;
    LaunchArgs a = {};
    a.theta = theta;
    a.parts_L = const_cast<double *>(L);
    a.parts_sigma = const_cast<double *>(sigma);
    a.parts_grad = grad;
    a.dt = dt;
    a.lambda = lambda;
    a.dtheta_out = dtheta;
    a.g_out = g_opt;
    return run(c, kJobSolve | kJobFromParts, a);
}

qng_status qng_graph_capture(qng_ctx *c, const double *theta, double dt, double lambda, double *dtheta, double *g_opt,
                             double *grad_opt, double *energy_opt) {
    if (!c || !dtheta) return QNG_ERR_ARG;
    if (!c->ws || !c->prepared) return QNG_ERR_WORKSPACE;
    if (!c->stream) return QNG_ERR_ARG;  // the legacy default stream cannot be captured
    if (c->graph_exec) { cudaGraphExecDestroy(c->graph_exec); c->graph_exec = nullptr; }
    if (c->graph) { cudaGraphDestroy(c->graph); c->graph = nullptr; }
    const bool prof = c->profiling;
    c->profiling = false;
    cudaError_t e = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) { c->profiling = prof; return cuda_status(e); }
    qng_status s = qng_step(c, theta, dt, lambda, dtheta, g_opt, grad_opt, energy_opt);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(c->stream, &graph);
    c->profiling = prof;
    if (s != QNG_OK) { if (graph) cudaGraphDestroy(graph); return s; }
    if (e != cudaSuccess) return cuda_status(e);
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    if (e != cudaSuccess) { cudaGraphDestroy(graph); return cuda_status(e); }
    c->graph = graph;
    c->graph_exec = exec;
    return QNG_OK;
}

qng_status qng_graph_launch(qng_ctx *c) {
    if (!c) return QNG_ERR_ARG;
    if (!c->graph_exec) return QNG_ERR_ARG;
    return cuda_status(cudaGraphLaunch(c->graph_exec, c->stream));
}

qng_status qng_autotune(qng_ctx *c, const double *theta, int reps, int64_t *report) {
    if (!c || reps < 1) return QNG_ERR_ARG;
    if (!c->ws || !c->prepared) return QNG_ERR_WORKSPACE;
    if (c->streaming) return QNG_OK;  // the streaming path has a single shape here
    if (c->graph_exec) { cudaGraphExecDestroy(c->graph_exec); c->graph_exec = nullptr; }
    if (c->graph) { cudaGraphDestroy(c->graph); c->graph = nullptr; }
    const size_t bytes = c->ws_cap;  // shapes must fit the workspace the caller set
    double *scratch_out = reinterpret_cast<double *>(c->ws + c->o_io_dtheta);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return QNG_ERR_CUDA;
    auto time_step = [&](float &ms) -> qng_status {
        qng_status s = qng_step(c, theta, 0.1, 1e-3, scratch_out, nullptr, nullptr, nullptr);  // warm-up
        if (s != QNG_OK) return s;
        cudaEventRecord(e0, c->stream);
        for (int r = 0; r < reps; ++r)
            if ((s = qng_step(c, theta, 0.1, 1e-3, scratch_out, nullptr, nullptr, nullptr)) != QNG_OK) return s;
        cudaEventRecord(e1, c->stream);
        if (cudaEventSynchronize(e1) != cudaSuccess) return QNG_ERR_CUDA;
        cudaEventElapsedTime(&ms, e0, e1);
        return QNG_OK;
    };
    std::vector<int> ns;
    for (const HostInst &h : c->inst) ns.push_back(h.n);
    std::sort(ns.begin(), ns.end());
    ns.erase(std::unique(ns.begin(), ns.end()), ns.end());
    int64_t tried = 0;
    qng_status st = QNG_OK;
    for (int n : ns) {
        float best = 3.4e38f;
        int best_cl = c->tuned_cl[n], best_th = c->tuned_threads[n];
        for (int cl = 0; cl <= std::min(kMaxClusterLog2, n - 1); ++cl) {
            for (int th : {64, 128, 256}) {
                if ((1 << (n - cl)) < th) continue;
                c->tuned_cl[n] = cl;
                c->tuned_threads[n] = th;
                if (plan(c) != QNG_OK || c->ws_bytes > bytes) continue;
                if ((st = upload(c)) != QNG_OK) break;
                float ms = 0.f;
                if ((st = time_step(ms)) != QNG_OK) break;
                ++tried;
                if (ms < best) { best = ms; best_cl = cl; best_th = th; }
            }
            if (st != QNG_OK) break;
        }
        c->tuned_cl[n] = best_cl;
        c->tuned_threads[n] = best_th;
        if (st != QNG_OK) break;
        // the checkpoint sweep's cluster and CTA size, at the chosen column shape
        if (best_cl < 0) continue;
        int best_fth = c->tuned_fwd[n], best_fcl = c->tuned_fcl[n];
        for (int fcl = best_cl; fcl <= std::min(kMaxFwdClusterLog2, std::min(best_cl + 1, n - 1)); ++fcl) {
            for (int fth : {64, 128, 256, 512}) {
                if ((1 << (n - fcl)) < fth) continue;
                c->tuned_fcl[n] = fcl;
                c->tuned_fwd[n] = fth;
                if (plan(c) != QNG_OK || c->ws_bytes > bytes) continue;
                if ((st = upload(c)) != QNG_OK) break;
                float ms = 0.f;
                if ((st = time_step(ms)) != QNG_OK) break;
                ++tried;
                if (ms < best) { best = ms; best_fth = fth; best_fcl = fcl; }
            }
            if (st != QNG_OK) break;
        }
        c->tuned_fcl[n] = best_fcl;
        c->tuned_fwd[n] = best_fth;
        if (st != QNG_OK) break;
    }
    // a single instance: the pipelined sweep's chunk count, at the chosen shapes
    if (st == QNG_OK && c->count == 1 && (st = plan(c)) == QNG_OK && (st = upload(c)) == QNG_OK) {
        float best = 3.4e38f;
        int best_req = c->pipe_req;
        for (int req : {1, 2, 3, 4}) {
            c->pipe_req = req;
            float ms = 0.f;
            if ((st = time_step(ms)) != QNG_OK) break;
            ++tried;
            if (ms < best) { best = ms; best_req = req; }
        }
        c->pipe_req = best_req;
    }
    // a batch of several launch groups: the groups in turn (1) or side by side on their own streams (2)
    if (st == QNG_OK && c->count > 1 && (st = plan(c)) == QNG_OK && (st = upload(c)) == QNG_OK && c->groups.size() > 1) {
        float best = 3.4e38f;
        int best_req = c->pipe_req;
        for (int req : {1, 2}) {
            c->pipe_req = req;
            float ms = 0.f;
            if ((st = time_step(ms)) != QNG_OK) break;
            ++tried;
            if (ms < best) { best = ms; best_req = req; }
        }
        c->pipe_req = best_req;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    qng_status s2 = plan(c);
    if (s2 == QNG_OK) s2 = upload(c);
    if (report) *report = tried;
    return st != QNG_OK ? st : s2;
}

qng_status qng_get_tuning(const qng_ctx *c, int n_qubits, int *cluster_log2, int *threads, int *forward_threads) {
    if (!c || n_qubits < 1 || n_qubits > kMaxQubits) return QNG_ERR_ARG;
    int cl = default_cl(n_qubits, c->precision);
    if (c->tuned_cl[n_qubits] >= 0) cl = c->tuned_cl[n_qubits];
    cl = std::max(0, std::min(cl, std::min(kMaxClusterLog2, n_qubits - 1)));
    int th = default_threads(n_qubits - cl);
    if (c->tuned_threads[n_qubits] > 0) th = c->tuned_threads[n_qubits];
    const int fth = fwd_threads_for(c, n_qubits, cl, fwd_cluster(c, n_qubits, cl));
    if (cluster_log2) *cluster_log2 = cl;
    if (threads) *threads = th;
    if (forward_threads) *forward_threads = fth;
    return QNG_OK;
}

qng_status qng_set_shape(qng_ctx *c, int n_qubits, int cluster_log2, int threads, int forward_threads) {
    if (!c || n_qubits < 1 || n_qubits > kMaxQubits) return QNG_ERR_ARG;
    if (cluster_log2 < -1 || cluster_log2 > kMaxClusterLog2) return QNG_ERR_ARG;
    if (threads != 0 && (threads < 64 || threads > 256 || threads % 32)) return QNG_ERR_ARG;
    if (forward_threads != 0 && (forward_threads < 64 || forward_threads > 512 || forward_threads % 32))
        return QNG_ERR_ARG;
    const int ocl = c->tuned_cl[n_qubits], oth = c->tuned_threads[n_qubits], ofth = c->tuned_fwd[n_qubits];
    c->tuned_cl[n_qubits] = cluster_log2;
    c->tuned_threads[n_qubits] = threads;
    c->tuned_fwd[n_qubits] = forward_threads;
    qng_status s = plan(c);
    if (s != QNG_OK || (c->ws && c->ws_bytes > c->ws_cap)) {
        c->tuned_cl[n_qubits] = ocl;
        c->tuned_threads[n_qubits] = oth;
        c->tuned_fwd[n_qubits] = ofth;
        plan(c);
        if (c->ws) upload(c);
        return s != QNG_OK ? s : QNG_ERR_WORKSPACE;
    }
    if (c->ws) return upload(c);
    return QNG_OK;
}

qng_status qng_set_forward_cluster(qng_ctx *c, int n_qubits, int cluster_log2) {
    if (!c || n_qubits < 1 || n_qubits > kMaxQubits) return QNG_ERR_ARG;
    if (cluster_log2 < -1 || cluster_log2 > kMaxFwdClusterLog2) return QNG_ERR_ARG;
    const int old = c->tuned_fcl[n_qubits];
    c->tuned_fcl[n_qubits] = cluster_log2;
    qng_status s = plan(c);
    if (s != QNG_OK || (c->ws && c->ws_bytes > c->ws_cap)) {
        c->tuned_fcl[n_qubits] = old;
        plan(c);
        if (c->ws) upload(c);
        return s != QNG_OK ? s : QNG_ERR_WORKSPACE;
    }
    if (c->ws) return upload(c);
    return QNG_OK;
}

qng_status qng_get_forward_cluster(const qng_ctx *c, int n_qubits, int *cluster_log2) {
    if (!c || !cluster_log2 || n_qubits < 1 || n_qubits > kMaxQubits) return QNG_ERR_ARG;
    int cl = default_cl(n_qubits, c->precision);
    if (c->tuned_cl[n_qubits] >= 0) cl = c->tuned_cl[n_qubits];
    cl = std::max(0, std::min(cl, std::min(kMaxClusterLog2, n_qubits - 1)));
    *cluster_log2 = fwd_cluster(c, n_qubits, cl);
    return QNG_OK;
}

qng_status qng_stream_traffic(const qng_ctx *c, int64_t *metric_bytes, int64_t *other_bytes, int64_t *metric_passes) {
    if (!c) return QNG_ERR_ARG;
    int64_t mb = 0, ob = 0, mp = 0;
    if (c->streaming) {
        const int64_t reg = (int64_t)amp_bytes(c->precision) << c->inst[0].n;
        for (const large::Launch &L : c->sched.launches) {
            if (L.kind != large::Launch::Pass) continue;
            const large::PassDesc &pd = c->sched.passes[L.pass];
            const int64_t b = reg * (__builtin_popcount(pd.loadmask) + __builtin_popcount(pd.storemask));
            if (L.segment == large::kSegMetric) { mb += b; ++mp; }
            else if (L.segment != large::kSegMetricIm) ob += b;  // not part of a step
        }
    }
    if (metric_bytes) *metric_bytes = mb;
    if (other_bytes) *other_bytes = ob;
    if (metric_passes) *metric_passes = mp;
    return QNG_OK;
}

qng_status qng_stream_segments(const qng_ctx *c, int64_t *bytes, int64_t *launches) {
    if (!c) return QNG_ERR_ARG;
    int64_t b[QNG_KERNEL_CLASSES] = {}, n[QNG_KERNEL_CLASSES] = {};
    if (c->streaming) {
        const int64_t reg = (int64_t)amp_bytes(c->precision) << c->inst[0].n;
        for (const large::Launch &L : c->sched.launches) {
            if (L.segment == large::kSegMetricIm) continue;  // a complex-metric call's, not a step's
            const int k = stream_class(L);
            if (L.kind == large::Launch::Pass) {
                const large::PassDesc &pd = c->sched.passes[L.pass];
                b[k] += reg * (__builtin_popcount(pd.loadmask & pd.regmask) + __builtin_popcount(pd.storemask & pd.regmask));
            } else if (L.kind == large::Launch::Hpsi) {
                b[k] += 2 * reg;
            } else {
                b[k] += (int64_t)sizeof(double) * (int64_t)L.nitems * c->l_grid;
            }
            ++n[k];
        }
    }
    for (int k = 0; k < QNG_KERNEL_CLASSES; ++k) {
        if (bytes) bytes[k] = b[k];
        if (launches) launches[k] = n[k];
    }
    return QNG_OK;
}

qng_status qng_profile(qng_ctx *c, int enable) {
    if (!c) return QNG_ERR_ARG;
    c->profiling = enable != 0;
    return QNG_OK;
}

qng_status qng_profile_read(qng_ctx *c, double *ms, int64_t *launches) {
    if (!c) return QNG_ERR_ARG;
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_status(e);
    for (auto &m : c->marks) {
        float t = 0.f;
        if ((e = cudaEventElapsedTime(&t, m.a, m.b)) != cudaSuccess) return cuda_status(e);
        c->prof_ms[m.cls] += t;
        c->prof_n[m.cls] += 1;
        c->spare.push_back(m.a);
        c->spare.push_back(m.b);
    }
    c->marks.clear();
    for (int k = 0; k < QNG_KERNEL_CLASSES; ++k) {
        if (ms) ms[k] = c->prof_ms[k];
        if (launches) launches[k] = c->prof_n[k];
        c->prof_ms[k] = 0.0;
        c->prof_n[k] = 0;
    }
    return QNG_OK;
}

qng_status qng_last_launch_count(const qng_ctx *c, int64_t *launches) {
    if (!c || !launches) return QNG_ERR_ARG;
    *launches = c->last_launches;
    return QNG_OK;
}

qng_status qng_set_pipeline(qng_ctx *c, int chunks) {
    if (!c || chunks < 0 || chunks > kPipeMax) return QNG_ERR_ARG;
    c->pipe_req = chunks;
    return QNG_OK;
}

qng_status qng_get_pipeline(const qng_ctx *c, int *chunks) {
    if (!c || !chunks) return QNG_ERR_ARG;
    *chunks = pipe_chunks(c);
    return QNG_OK;
}

qng_status qng_solve_report(qng_ctx *c, int *path, int32_t *handed_over) {
    if (!c || !path || !handed_over) return QNG_ERR_ARG;
    *path = c->last_solve;
    *handed_over = 0;
    if (c->last_solve != QNG_SOLVE_MIXED) return QNG_OK;
    std::vector<int32_t> flag((size_t)c->count);
    cudaError_t e = cudaMemcpyAsync(flag.data(), c->ws + c->o_irflag, sizeof(int32_t) * flag.size(),
                                    cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_status(e);
    for (int32_t f : flag) *handed_over += f != 0;
    return QNG_OK;
}

void qng_destroy(qng_ctx *c) { delete c; }

const char *qng_status_string(qng_status s) {
    switch (s) {
    case QNG_OK: return "ok";
    case QNG_ERR_ARG: return "invalid argument";
    case QNG_ERR_OOM: return "host allocation failed";
    case QNG_ERR_CUDA: return "CUDA error";
    case QNG_ERR_TIMEOUT: return "device wait timed out";
    case QNG_ERR_NOT_SPD: return "g + lambda I is not positive definite";
    case QNG_ERR_WORKSPACE: return "workspace missing, too small or misaligned";
    case QNG_ERR_UNSUPPORTED: return "unsupported request";
    }
    return "unknown status";
}

}  // extern "C"

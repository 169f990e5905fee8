// qng_metric_noalloc: the metric entry point for callers that cannot allocate device memory.
//
// Who needs it: code that runs inside a host application which owns all of the GPU's memory
// through its own pool or arena and forbids direct cudaMalloc/cudaFree (plugins, embedded
// solvers, real-time loops where the implicit synchronisation of cudaMalloc is not allowed), and
// code that cannot keep a workspace buffer alive between calls. Such callers pass only their
// inputs and outputs; everything else the kernels need lives in one file-scope device array.
//
// The array holds QNG_NOALLOC_SCRATCH_BYTES bytes on every GPU that loads the library, until the
// process exits. All calls on one device share it and it keeps what the last call left there:
// two calls whose work overlaps on the GPU (different streams, or different host threads) race on
// it and give wrong results, so callers must order them. The device status word at its start is
// cleared by every call. Every call looks up the array's device address on the current device
// (cudaGetSymbolAddress, which allocates nothing), so the address stays right if the device's
// context is ever re-created; the first call on a device may load the library's kernels, so make
// it before capturing any stream. No cudaMalloc, cudaFree or other allocating routine is called,
// on the device or on the host: the circuit tables are built in fixed-size arrays on the caller's
// stack and copied into the array with cudaMemcpyAsync from that (pageable) memory, which the
// CUDA runtime stages before the call returns; the host may wait for that staging. A stream that
// is being captured would record copies from stack memory that is gone by the time the graph
// runs, so the call refuses such a stream before it touches the device.
#include <cmath>
#include <cstring>

#include "qng_internal.h"

namespace {

using namespace qng;

constexpr int kNaMaxGates = 1024;
constexpr int kNaMaxParams = 320;
constexpr int kNaMaxDiag = 1024;

__device__ __align__(256) unsigned char g_noalloc_scratch[QNG_NOALLOC_SCRATCH_BYTES];

size_t up256(size_t x) { return (x + 255) & ~size_t(255); }

// Device address of the scratch array in the current device's context. The name
// g_noalloc_scratch in host code is only a host-side handle of the symbol, never an address a
// kernel may be given.
qng_status scratch_address(unsigned char **out) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return QNG_ERR_CUDA;
    *out = static_cast<unsigned char *>(p);
    return QNG_OK;
}

bool rot_kind(int k) { return k == QNG_GATE_RX || k == QNG_GATE_RY || k == QNG_GATE_RZ; }

}  // namespace

extern "C" qng_status qng_metric_noalloc(int n_qubits, const qng_gate *gates, int n_gates, int precision,
                                         const double *theta, double *g, void *stream) {
    if (n_qubits < 1 || n_qubits > kMaxQubitsSmall || n_gates < 0 || (n_gates > 0 && !gates)) return QNG_ERR_ARG;
    if (precision != QNG_C64 && precision != QNG_C128) return QNG_ERR_ARG;
    if (n_gates > kNaMaxGates) return QNG_ERR_WORKSPACE;
    const int n = n_qubits;

    // tables, built on the stack
    DevParam params[kNaMaxParams];
    DevFixed fixed[kNaMaxGates];
    DevDiag diag[kNaMaxDiag];
    DevWork work[kNaMaxParams];
    int P = 0, nfix = 0, ndiag = 0, pend_begin = 0;
    for (int k = 0; k < n_gates; ++k) {
        const qng_gate &x = gates[k];
        if (x.kind >= QNG_GATE_CRX && x.kind <= QNG_GATE_CRP) return QNG_ERR_UNSUPPORTED;  // qng_metric takes them
        if (x.q0 < 0 || x.q0 >= n) return QNG_ERR_ARG;
        if (rot_kind(x.kind)) {
            if (x.param != P) return QNG_ERR_ARG;
            if (P >= kNaMaxParams) return QNG_ERR_WORKSPACE;
            DevParam p = {};
            p.axis = x.kind == QNG_GATE_RX ? kAxisX : (x.kind == QNG_GATE_RY ? kAxisY : kAxisZ);
            p.q = x.q0;
            p.fix_begin = pend_begin;
            p.fix_count = nfix - pend_begin;
            bool all_diag = true;
            for (int f = pend_begin; f < nfix; ++f)
                if (fixed[f].kind != QNG_GATE_CZ && fixed[f].kind != QNG_GATE_Z) all_diag = false;
            p.zmask = 0;
            if (all_diag) {
                uint64_t sm[64] = {0};
                for (int f = pend_begin; f < nfix; ++f) {
                    if (fixed[f].kind == QNG_GATE_Z) {
                        p.zmask ^= 1ull << fixed[f].q0;
                    } else {
                        const int u = fixed[f].q0 < fixed[f].q1 ? fixed[f].q0 : fixed[f].q1;
                        const int v = fixed[f].q0 < fixed[f].q1 ? fixed[f].q1 : fixed[f].q0;
                        sm[v - u] ^= 1ull << u;
                    }
                }
                p.diag_begin = ndiag;
                for (int s = 1; s < 64; ++s) {
                    if (!sm[s]) continue;
                    if (ndiag >= kNaMaxDiag) return QNG_ERR_WORKSPACE;
                    diag[ndiag++] = DevDiag{s, 0, sm[s]};
                }
                p.diag_count = ndiag - p.diag_begin;
            } else {
                p.diag_begin = 0;
                p.diag_count = -1;
            }
            params[P++] = p;
            pend_begin = nfix;
        } else if (x.kind >= QNG_GATE_CZ && x.kind <= QNG_GATE_H) {
            if (x.param != -1) return QNG_ERR_ARG;
            if ((x.kind == QNG_GATE_CZ || x.kind == QNG_GATE_CNOT) && (x.q1 < 0 || x.q1 >= n || x.q1 == x.q0))
                return QNG_ERR_ARG;
            fixed[nfix++] = DevFixed{x.kind, x.q0, x.q1, 0};
        } else {
            return QNG_ERR_ARG;
        }
    }
    set_zruns(params, P);
    if (P == 0) return QNG_OK;  // an empty metric
    if (!theta || !g) return QNG_ERR_ARG;

    // launch shape: the defaults of the workspace path
    Group grp;
    grp.cl = n - 9;
    if (grp.cl < 0) grp.cl = 0;
    if (grp.cl > kMaxClusterLog2) grp.cl = kMaxClusterLog2;
    if (grp.cl > n - 1) grp.cl = n - 1;
    const uint32_t Nl = 1u << (n - grp.cl);
    grp.threads = Nl <= 256 ? 64 : (Nl <= 1024 ? 128 : 256);
    grp.fwd_threads = Nl / 2 < 64 ? 64 : (Nl / 2 > 512 ? 512 : (int)(Nl / 2));
    grp.fwd_cl = grp.cl;
    grp.max_n = n;
    grp.max_P = P;
    grp.first_inst = 0;
    grp.num_inst = 1;
    // metric columns 1..P-1 longest first, then column 0 (its <sigma_0> only)
    for (int j = 0; j < P; ++j) work[j] = DevWork{0, P - 1 - j};
    grp.first_met = 0;
    grp.num_met = P;
    grp.first_work = 0;
    grp.num_work = P;
    grp.first_grad = 0;
    grp.num_grad = 0;
    const size_t ab = precision == QNG_C128 ? 16 : 8;
    const size_t state = (size_t)Nl * ab * (grp.cl ? 3 : 1);
    const int nw = grp.threads / 32;
    grp.smem_fwd = state + 64 * sizeof(double);
    grp.smem_col = state + (size_t)(P + 1) * nw * sizeof(double) + (size_t)(P + 1) * sizeof(double);
    grp.smem_col_im = grp.smem_col;  // this entry point takes Re G only
    if (grp.smem_col > kMaxSmem) return QNG_ERR_UNSUPPORTED;

    DevInst in = {};
    in.n = n;
    in.P = P;
    in.cl = grp.cl;
    in.nterms = 0;
    in.param_tab = 0;
    in.w_begin = pend_begin;
    in.w_count = nfix - pend_begin;
    in.term_off = 0;
    const int32_t ginst = 0;

    // scratch layout
    size_t off = 0;
    auto take = [&](size_t bytes) { const size_t o = up256(off); off = o + (bytes ? bytes : 1); return o; };
    const size_t o_status = take(256), o_inst = take(sizeof(DevInst)), o_param = take(sizeof(DevParam) * P),
                 o_fixed = take(sizeof(DevFixed) * (nfix ? nfix : 1)), o_diag = take(sizeof(DevDiag) * (ndiag ? ndiag : 1)),
                 o_work = take(sizeof(DevWork) * P), o_ginst = take(sizeof(int32_t)), o_coef = take(sizeof(DevCoef) * P),
                 o_sigma = take(sizeof(double) * P), o_pctrl = take(sizeof(double) * P),
                 o_scale = take(sizeof(double) * (P + 2)),
                 o_L = take(sizeof(double) * (size_t)P * P), o_grad = take(sizeof(double) * P),
                 o_energy = take(sizeof(double)), o_ckpt = take(ab * ((size_t)(P + 1) << n)), o_eta = take(ab << n);
    if (up256(off) > (size_t)QNG_NOALLOC_SCRATCH_BYTES) return QNG_ERR_WORKSPACE;
    in.param_off = 0;
    in.metric_off = 0;
    in.ckpt_off = 0;
    in.eta_off = 0;
    in.scale_off = 0;

    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) return QNG_ERR_CUDA;
    if (cap != cudaStreamCaptureStatusNone) return QNG_ERR_UNSUPPORTED;
    unsigned char *base = nullptr;
    qng_status s = scratch_address(&base);
    if (s != QNG_OK) return s;
    cudaError_t e = cudaMemsetAsync(base + o_status, 0, 256, st);
    auto put = [&](size_t o, const void *src, size_t bytes) {
        if (e == cudaSuccess && bytes) e = cudaMemcpyAsync(base + o, src, bytes, cudaMemcpyHostToDevice, st);
    };
    put(o_inst, &in, sizeof(in));
    put(o_param, params, sizeof(DevParam) * P);
    put(o_fixed, fixed, sizeof(DevFixed) * nfix);
    put(o_diag, diag, sizeof(DevDiag) * ndiag);
    put(o_work, work, sizeof(DevWork) * P);
    put(o_ginst, &ginst, sizeof(ginst));
    if (e != cudaSuccess) return QNG_ERR_CUDA;
    if (prepare_kernels(precision, grp.smem_fwd, grp.smem_col, grp.smem_col) != cudaSuccess) return QNG_ERR_CUDA;

    Work w;
    w.status = reinterpret_cast<int32_t *>(base + o_status);
    w.inst = reinterpret_cast<const DevInst *>(base + o_inst);
    w.param = reinterpret_cast<const DevParam *>(base + o_param);
    w.gen = nullptr;  // no generalised rotations here
    w.fixed = reinterpret_cast<const DevFixed *>(base + o_fixed);
    w.diag = reinterpret_cast<const DevDiag *>(base + o_diag);
    w.term = nullptr;
    w.work = reinterpret_cast<const DevWork *>(base + o_work);
    w.group_inst = reinterpret_cast<const int32_t *>(base + o_ginst);
    w.coef = reinterpret_cast<DevCoef *>(base + o_coef);
    w.sigma = reinterpret_cast<double *>(base + o_sigma);
    w.pctrl = reinterpret_cast<double *>(base + o_pctrl);
    w.scale = reinterpret_cast<double *>(base + o_scale);
    w.L = reinterpret_cast<double *>(base + o_L);
    w.gradraw = reinterpret_cast<double *>(base + o_grad);
    w.energy = reinterpret_cast<double *>(base + o_energy);
    w.chol = w.L;  // the metric-only finish never factorises
    w.Lim = nullptr;
    w.srhs = w.sy = w.sdinv = nullptr;
    w.irflag = nullptr;
    w.ckpt = base + o_ckpt;
    w.eta = base + o_eta;

    LaunchArgs a = {};
    a.theta = theta;
    a.g_out = g;
    a.jobs = kJobMetric;
    if (launch_coef(w, theta, P, st) != cudaSuccess) return QNG_ERR_CUDA;
    if (launch_forward(w, grp, precision, 0, st) != cudaSuccess) return QNG_ERR_CUDA;
    if (launch_columns(w, grp, precision, 1, 0, 0, st) != cudaSuccess) return QNG_ERR_CUDA;
    if (launch_finish(w, 1, P, a, st) != cudaSuccess) return QNG_ERR_CUDA;
    return QNG_OK;
}

// Internal declarations shared by the host API (qng_api.cu) and the kernels (qng_kernels.cu).
// Device-visible tables live in the caller's workspace; every offset below is in elements.
#pragma once

#include <cstddef>
#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/qng.h"

namespace qng {

constexpr int kMaxQubits = 30;         // any single instance
constexpr int kMaxQubitsSmall = 16;    // instances run by the on-chip (cluster-resident) path
constexpr int kMaxClusterLog2 = 3;     // 8 CTAs per cluster (the portable maximum)
constexpr int kMaxFwdClusterLog2 = 4;  // the checkpoint sweep: up to 16 CTAs (non-portable size)
constexpr int kAxisX = 0, kAxisY = 1, kAxisZ = 2;
constexpr int kAxisGen = 3;  // generalised rotation: generator K = C (x) S, see DevParam::gx

// One parametric gate k of an instance: U_k = R_k F_k with R_k = exp(-i theta_k sigma / 2).
struct DevParam {
    int32_t axis;       // kAxisX / kAxisY / kAxisZ
    int32_t q;          // target qubit
    int32_t fix_begin;  // F_k: fixed gates [fix_begin, fix_begin + fix_count) of the fixed table, circuit order
    int32_t fix_count;
    int32_t diag_begin; // if F_k is all CZ / Z: its sign as (shift, mask) pairs [diag_begin, +diag_count)
    int32_t diag_count; //   of the diag table, plus zmask; diag_count = -1 when F_k is not all diagonal
    uint64_t zmask;     //   single-qubit Z factors of F_k
    int32_t zrun;       // Z rotations with diagonal F from k on (this one included, at most kZRunMax); 0 if k is not one
    int32_t zdown;      // Z rotations without fixed gates from k down (this one included); 0 if k is not one
};

// Generator of a kAxisGen parameter (same index as its DevParam): K = C (x) S with C the projector
// onto gctrl's qubits all 1 (gctrl = 0: C = 1) and S = i^gny X^gx Z^gz, so that
// (S x)[k] = i^gny (-1)^popcount((k ^ gx) & gz) x[k ^ gx].
struct DevGen {
    uint64_t gx, gz, gctrl;
    int32_t gny;
    int32_t pad;
};

constexpr int kZRunMax = 16;
constexpr size_t kMaxSmem = 227 * 1024;  // dynamic shared memory per CTA (opt-in maximum)

// Fill DevParam::zrun over the parameters [p, p + P) of one instance.
// zdown: the runs the complex64 column walk of a single instance composes (its own kernel
// instantiation; batches launch the column kernel without that code).
inline void set_zruns(DevParam *p, int P) {
    int run = 0;
    for (int k = P - 1; k >= 0; --k) {
        run = (p[k].axis == kAxisZ && p[k].diag_count >= 0) ? run + 1 : 0;
        p[k].zrun = run < kZRunMax ? run : kZRunMax;
    }
    int down = 0;
    for (int k = 0; k < P; ++k) {
        down = (p[k].axis == kAxisZ && p[k].fix_count == 0) ? down + 1 : 0;
        p[k].zdown = down;
    }
}

struct DevFixed {
    int32_t kind;  // QNG_GATE_CZ, CNOT, X, Y, Z, H
    int32_t q0;
    int32_t q1;
    int32_t pad;
};

// sign(k) of a set of CZ gates = (-1)^(sum over pairs of popcount(k & (k >> shift) & mask))
struct DevDiag {
    int32_t shift;
    int32_t pad;
    uint64_t mask;
};

struct DevTerm {
    double coeff;
    uint64_t x;
    uint64_t z;
    int32_t ny;   // number of Y factors mod 4
    int32_t pad;
};

// Per-instance descriptor.
struct DevInst {
    int32_t n, P;
    int32_t cl;             // log2 of CTAs per cluster used for this instance's chains
    int32_t nterms;
    int64_t param_off;      // theta, coef, sigma, grad, dtheta (P entries)
    int64_t metric_off;     // g, L, cholesky scratch (P*P entries)
    int64_t ckpt_off;       // checkpoints Psi[0..P] (amplitude units; (P+1) * 2^n)
    int64_t eta_off;        // adjoint seed eta (2^n amplitudes)
    int64_t scale_off;      // P + 2 scale factors: Psi[0..P], eta
    int32_t param_tab;      // first DevParam of the instance
    int32_t w_begin;        // trailing fixed gates W in the fixed table
    int32_t w_count;
    int32_t term_off;       // first DevTerm
};

struct DevWork {
    int32_t inst;
    int32_t col;  // 0..P-1: metric column; P: gradient (adjoint) column
};
constexpr int kSolveBlock = 16;      // block width of the block solve
constexpr int kBlockSolveMinP = 48;  // smaller instances use k_finish

// Coefficients of parameter k (float64): c = cos(theta/2), s = sin(theta/2), and the scaled
// form of the adjoint rotation R^dag = c I + i s sigma = f (I + i t sigma) (|c| >= |s|) or
// f (t I + i sigma) (|c| < |s|).
struct DevCoef {
    double c, s, t, f;
    int32_t caseB;
    int32_t pad;
    float cf, sf, tf;  // c, s, t rounded to float32 once here, for the complex64 kernels
    int32_t pad2;
};

// Pointers into the workspace.
struct Work {
    int32_t *status;          // device status word
    const DevInst *inst;
    const DevParam *param;
    const DevGen *gen;        // generators of kAxisGen parameters, indexed like param
    const DevFixed *fixed;
    const DevDiag *diag;
    const DevTerm *term;
    const DevWork *work;      // work items, all groups, each group contiguous
    const int32_t *group_inst;// instances of each group, contiguous per group
    DevCoef *coef;
    double *sigma;            // <psi_k|sigma_k|psi_k>
    double *scale;            // checkpoint and eta scale factors
    double *L;                // (1/4) Re L_ij, i < j, per instance P*P
    double *gradraw;          // d<E>/d theta
    double *energy;           // <E>
    double *chol;             // P*P per instance
    double *Lim;              // (1/4) Im L_ij, i < j (complex metric calls only; shares chol's region)
    double *pctrl;            // <C_k>: 1 for ordinary rotations, Prob(control = 1) for controlled ones
    double *srhs;             // block solve: running right-hand side (P)
    double *sy;               // block solve: y (P)
    double *sdinv;            // block solve: inverses of the diagonal blocks (nblk x 16 x 16)
    int32_t *irflag;          // per instance: 1 = the mixed-precision solve left the step to k_solve
    void *ckpt;               // checkpoint amplitudes
    void *eta;                // adjoint seeds
};

// A launch group: instances sharing one cluster size and CTA shape.
struct Group {
    int cl = 0;
    int threads = 128;      // CTA size of the column kernel
    int fwd_cl = 0;         // cluster size (log2) of the checkpoint sweep
    int fwd_threads = 256;  // CTA size of the checkpoint sweep (k_forward)
    bool general = false;   // some instance has generalised rotations (GEN kernel instantiations)
    int max_n = 0;
    int max_P = 0;
    int first_inst = 0;   // into group_inst
    int num_inst = 0;
    int first_work = 0;   // into work: metric + gradient columns, sorted by decreasing length
    int num_work = 0;
    int first_grad = 0;   // gradient columns only
    int num_grad = 0;
    int first_met = 0;    // metric columns only, sorted by decreasing length
    int num_met = 0;
    size_t smem_fwd = 0;
    size_t smem_col = 0;
    size_t smem_col_im = 0;  // column kernel with Im L partial sums (metric_im)
    int *queue = nullptr;        // device work counter of the persistent column launch (batched contexts)
    int resident_clusters = 0;   // clusters of the column kernel resident at once
};

enum Job : int {
    kJobMetric = 1,
    kJobGradient = 2,
    kJobEnergy = 4,
    kJobSolve = 8,
    kJobMetricIm = 16,  // with kJobMetric: Im G as well (no solve in the same call)
    kJobParts = 32,     // column partition: the raw L, sigma, grad and <E> go out, no assembly
    kJobFromParts = 64, // column partition: assemble and solve from gathered L, sigma and grad
};

struct LaunchArgs {
    const double *theta;
    double *g_out;        // may be null
    double *gim_out;      // Im G (kJobMetricIm), may be null
    double *sigma_out;    // may be null
    double *grad_out;     // may be null
    double *energy_out;   // may be null
    double *dtheta_out;   // may be null
    const double *grad_scale;  // device, one per instance (energy backward), may be null
    double *parts_L;           // column partition: L (P x P) out (kJobParts) or in (kJobFromParts)
    double *parts_sigma;       //   sigma (P), likewise
    const double *parts_grad;  //   grad (P) in (kJobFromParts)
    int ir_gate;               // k_solve: only the instances the mixed-precision solve handed over
    double dt, lambda;
    int jobs;
};

// Kernel-side launchers (qng_kernels.cu). Return cudaSuccess or the launch error.
cudaError_t launch_coef(const Work &w, const double *theta, int64_t total_params, cudaStream_t st);
cudaError_t launch_theta_update(const Work &w, double *theta, const double *dtheta, int64_t total, cudaStream_t st);
// The checkpoint sweep over parameters [k_begin, k_end) (clipped to P); last = 1 adds the
// trailing gates, <E> and eta. k_begin > 0 restarts from checkpoint k_begin.
cudaError_t launch_forward(const Work &w, const Group &g, int precision, int want_eta, cudaStream_t st, int k_begin = 0,
                           int k_end = 1 << 30, int last = 1);
cudaError_t launch_columns(const Work &w, const Group &g, int precision, int with_metric, int with_grad,
                           int metric_im, cudaStream_t st);
// Work items [first, first + num) of the group's list; persistent = false gives one cluster per
// item (no work queue), so finished clusters leave their SMs to other kernels.
cudaError_t launch_columns_range(const Work &w, const Group &g, int precision, int metric_im, int first, int num,
                                 bool persistent, cudaStream_t st);
cudaError_t launch_finish(const Work &w, int count, int max_P, const LaunchArgs &a, cudaStream_t st);
// block solve (qng_solve.cu). Largest own-row count of a CTA over all block columns: CTA 0
// holds the 16 diagonal-block rows (all P rows when it is alone); a CTA of rank >= 1 holds at most
// ceil((P - 16) / (C - 1)) rows below the block (block 0 is the worst case).
__host__ __device__ inline int sblock_rows_max(int P, int C) {
    if (C == 1) return P;
    const int per = (P - kSolveBlock + C - 2) / (C - 1);
    return per > kSolveBlock ? per : kSolveBlock;
}
size_t sblock_smem_bytes(int P, int C);
cudaError_t prepare_sblock(int P, int C);
cudaError_t launch_sblock(const Work &w, const LaunchArgs &a, int P, int C, int K, cudaStream_t st);
cudaError_t launch_sback(const Work &w, const LaunchArgs &a, int P, cudaStream_t st);
// mixed-precision solve (qng_solve_ir.cu): one cluster of C CTAs per instance
size_t solve_ir_smem_bytes(int P, int C);
cudaError_t prepare_solve_ir(int P, int C);
cudaError_t launch_solve_ir(const Work &w, int count, int max_P, int C, const LaunchArgs &a, cudaStream_t st);
cudaError_t launch_solve(const Work &w, int count, int max_P, int cl, const LaunchArgs &a, cudaStream_t st);
size_t solve_smem_bytes(int P, int cl);
cudaError_t prepare_solve(size_t smem);
int resident_clusters(const Group &g, int precision);
cudaError_t prepare_kernels(int precision, size_t smem_fwd, size_t smem_col, size_t smem_col_im);

// Raise fn's dynamic shared memory limit (cudaFuncAttributeMaxDynamicSharedMemorySize) on the
// current device to at least bytes; never lowers it. The attribute belongs to the kernel, not to a
// context, so every context and the allocation-free entry point share it: lowering it for a small
// problem would make the next launch of a larger live context fail.
cudaError_t raise_smem_limit(const void *fn, size_t bytes);

}  // namespace qng

// Streaming (HBM) path: pass program format shared by the host planner and the kernels.
#pragma once

#include <cstdint>
#include <vector>

#include "qng_internal.h"

namespace qng {
namespace large {

constexpr int kRegs = 4;      // register slots: 0 psi, 1 a (lambda / eta), 2 b (phi), 3 b2 (a second phi)
constexpr int kMaxWin = 7;    // tile qubits beyond the contiguous low block
constexpr int kMaxSlots = 32; // inner products per pass
constexpr int kRegPsi = 0, kRegA = 1, kRegB = 2, kRegB2 = 3;

enum OpKind : int32_t {
    kOpCopy = 0,       // r1 <- r0
    kOpZero = 1,       // r0 <- |0...0>
    kOpRot = 2,        // rotation param on every register of regs (adjoint: R^dag, else R)
    kOpFixed = 3,      // fixed gate fixed_kind(q0, q1) on every register of regs
    kOpSigma = 4,      // r0 <- sigma_{axis}(q0) r0
    kOpIp = 5,         // slot += Re (adjoint = 0) or Im (adjoint = 1) of <r0| sigma_{axis}(q0) |r1>; axis -1: no sigma
    kOpRecordFac = 6,  // slotfac[slot] <- scale(r0) * scale(r1)
    kOpSetScale = 7,   // scale(r1) <- scale(r0) (no data)
    kOpStep = 8,       // one recurrence step in one sweep: slot += Re/Im <r0|sigma_{axis}(q0)|r1> (adjoint
                       // 0/1; 2: Re into slot and Im into slot + 1), then, if param >= 0, the adjoint
                       // rotation of param (same axis and qubit) on r0 and r1
    kOpStep2 = 9,      // the step of two columns that share a (registers a, b and b2): Re <a|sigma|b> into
                       // slot and Re <a|sigma|b2> into slot + 1 (adjoint 0), or Re, Im of the first into
                       // slot, slot + 1 and of the second into slot + 2, slot + 3 (adjoint 2); then the
                       // adjoint rotation on a, b and b2
};

struct PassOp {
    int32_t kind;
    int32_t r0, r1;
    int32_t regs;
    int32_t q0, q1;
    int32_t axis;
    int32_t adjoint;
    int32_t param;
    int32_t fixed_kind;
    int32_t slot;
    // register-phase kernel (complex64 tiles of 2^12): position 0..3 among the phase's register
    // bits of the op's non-diagonal target qubit (kt), and of q0 / q1 where a diagonal part reads
    // their bit (dk0 / dk1); -1 where the qubit is not a register bit of the phase.
    // zrun: the op starts a run of diagonal operations on a and b that the kernel composes (its
    // length, plus kZrunIm when the run's steps take Im as well), -1 inside such a run, 0 otherwise
    int8_t kt, dk0, dk1, zrun;
};

struct PassDesc {
    int32_t n, t, low, win;
    int32_t wq[kMaxWin];
    int32_t regmask, loadmask, storemask;
    int32_t op_begin, nops;
    int32_t nslots, slot_base;
    int32_t parity;
    int32_t phase_begin, nphases;  // register phases (complex64 tiles of 2^12 only)
};

// Register-phase kernel of complex64 passes (tiles of 2^12 amplitudes, 256 threads). Within a phase
// thread i holds, of every register the phase touches, the 16 amplitudes at the tile's local indices
// l = tl(i) | dep(m), m = 0..15, where dep puts bit k of m at local bit rbit[k] and tl puts bit b of
// i at local bit tbit[b]. Every non-diagonal target of the phase's operations is one of the rbit, so
// the phase runs in registers; phases exchange amplitudes through the shared-memory tile.
constexpr int kPhaseAmps = 16;
constexpr int kPhaseTile = 12;      // local qubits of a register-phase tile
constexpr int kPhaseThreads = 256;
constexpr int kMaxPhaseOps = 96;    // operations per pass of the register-phase kernel
constexpr int kMaxPhases = 16;      // phases per pass
struct PassPhase {
    int32_t op_begin, op_end;  // the pass's operations [op_begin, op_end), relative to the pass
    int8_t rbit[4];            // local bits held in registers; rbit[0] == 0 selects 16-byte accesses
    int8_t tbit[8];            // local bits of the thread index bits 0..7
    int32_t rmask;             // registers the phase reads or writes (gathered from the tile)
    int32_t wmask;             // registers the phase writes (scattered back)
    int32_t macro;             // 0, or a straight-line form of the phase's last `count` operations
                               // (kMacro* | axis << 4 | count, kMacroRev for descending targets); the
                               // operations before them run one by one
};
// Straight-line phases: kMacroSteps, m recurrence steps (a, b, Re) on one axis with pair targets
// at register bits 0..m-1 in order; kMacroCnot, m CNOTs on a and b with targets at register bits
// 0..m-1 in order, the controls of the first m - 1 at register bits 1..m-1 and the last control a
// thread-uniform bit.
constexpr int32_t kMacroSteps = 1 << 8, kMacroCnot = 2 << 8;
// kMacroSteps2: the same with steps of two columns (kOpStep2, Re). kMacroRev (steps only): the
// targets are register bits m-1, ..., 0 in order instead.
constexpr int32_t kMacroSteps2 = 3 << 8, kMacroRev = 1 << 7;
// Runs of diagonal operations (PassOp::zrun): Z-axis recurrence steps and CZ / Z gates, either all on
// (a, b) or all on (a, b, b2) (kZrunDual), at least two steps, at most kMaxZrun operations, all steps
// Re (adjoint 0) or all Re and Im (2, kZrunIm).
constexpr int kMaxZrun = 31, kZrunIm = 32, kZrunDual = 64;

struct ReduceItem {
    int32_t slot;
    int32_t pad;
    double mul;
    double *dst;
};

struct PassArgs {
    const PassDesc *desc;
    const PassOp *ops;
    const DevCoef *coef;
    void *reg[kRegs];
    double *regscale;  // [2][kRegs]
    double *partial;   // [slots][grid]
    double *slotfac;   // [slots]
    const PassPhase *phases;  // register-phase kernel only
    int32_t *status;          // device status word (register-phase kernel: a malformed pass)
};

cudaError_t prepare_pass(int precision, size_t smem);
cudaError_t launch_pass(const PassArgs &pa, int precision, int grid, int threads, size_t smem, int metric_im,
                        cudaStream_t st);
// Register-phase kernel (complex64, tiles of 2^12): the pass's register mask picks the instantiation
// (stages of the shared-memory tile ring, psi held or not); grid CTAs of kPhaseThreads threads, each
// taking tiles b, b + grid, ...
size_t phased_smem_bytes(int nreg);
int phased_stages(int nreg);
cudaError_t prepare_pass_phased();
cudaError_t launch_pass_phased(const PassArgs &pa, int regmask, int grid, int metric_im, cudaStream_t st);
cudaError_t launch_hpsi(const void *in, void *out, const DevTerm *terms, int nterms, int n, int precision,
                        double *partial, int grid, cudaStream_t st);
cudaError_t launch_reduce(const double *partial, const double *slotfac, int nctas, const ReduceItem *items, int nitems,
                          int use_fac, cudaStream_t st);

// A planned launch of the streaming schedule.
struct Launch {
    enum Kind { Pass, Hpsi, Reduce } kind;
    int pass = -1;             // index into the pass table
    int item_begin = 0, nitems = 0;
    int use_fac = 1;
    int segment = 0;           // kSegForward, kSegEnergy, kSegAdjoint, kSegMetric, kSegMetricIm
};
// kSegMetricIm repeats kSegMetric with both parts of every inner product; a call runs one of the two.
enum Segment { kSegForward = 0, kSegEnergy = 1, kSegAdjoint = 2, kSegMetric = 3, kSegMetricIm = 4 };
enum Region { kRegionSigma = 0, kRegionL = 1, kRegionGrad = 2, kRegionEnergy = 3, kRegionLim = 4 };

// A reduce destination before the workspace address is known.
struct RedSpec {
    int32_t slot;
    double mul;
    int region;
    int64_t index;
};

struct Schedule {
    int n = 0, t = 0, low = 0;
    bool phased = false;  // complex64 with tiles of 2^12: the register-phase kernel runs every pass
    bool pairs = false;   // metric columns walk in pairs sharing a (register b2 in use)
    std::vector<PassDesc> passes;
    std::vector<PassOp> ops;
    std::vector<PassPhase> phases;
    std::vector<Launch> launches;
    std::vector<RedSpec> reds;
    int max_slots = 1;
};

// Build the streaming schedule of one instance: gates (circuit order), P parameters. want (P
// entries, may be null: all) selects the metric columns whose recurrence runs; for the others the
// metric segment only advances psi through U_j.
void build_schedule(const std::vector<qng_gate> &gates, int n, int P, int precision, Schedule &out,
                    const std::vector<uint8_t> *want = nullptr);

}  // namespace large
}  // namespace qng

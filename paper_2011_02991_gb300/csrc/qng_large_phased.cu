// sm_103a register-phase kernel of the streaming path, for complex64 registers in tiles of 2^12
// amplitudes (instances of 12 or more qubits). It runs the same passes as k_pass (qng_large.cu):
// one launch is one pass of Algorithm 1's O(1)-register recurrence (Sec. 3) over the registers it
// touches, a tile program of rotations, fixed gates, sigma, inner products and recurrence steps
// (Eq. L_recurrent_def: L_ij from <a|sigma_i|b>, then a, b <- U_i^dag). What differs is how a CTA
// moves the data, so that a pass runs at HBM rate:
//   - persistent: one CTA per SM takes tiles b, b + grid, ... through a ring of S shared-memory
//     stages; the 16-byte cp.async loads of the next S - 1 tiles are in flight while a tile is
//     computed, and a finished tile is stored with 16-byte vector stores straight from the ring;
//   - register phases: the pass's operations are cut (on the host) into phases whose pair targets
//     are four local qubits; in a phase each thread holds 16 amplitudes of every register it
//     touches, at the local indices spanned by those four bits, and applies the phase's operations
//     in registers. Phases exchange amplitudes through the shared-memory tile, whose 16-byte chunks
//     are XOR-swizzled so that the threads of a half-warp (or quarter-warp) hit distinct banks;
//   - rotations as in-place plane rotations: (cos alpha + i sin alpha sigma) turns 2 x 2 blocks of
//     real components by alpha, each by three shears (three FMAs, no temporaries); alpha = theta/2 is
//     taken in (-pi/2, pi/2], and the rotation by theta/2 - pi, which is minus the rotation by
//     theta/2, leaves a factor -1 that the register's float64 factor keeps (complex64 registers carry
//     only these signs, so nothing is ever renormalised).
// Inner products accumulate in float32 over a thread's 16 amplitudes and a warp (a shuffle tree),
// then in float64: lane s of every warp keeps slot s's running sum over the tiles in a register,
// and the CTA's partial sums are formed in a fixed order at the end (partial[slot][cta]), like k_pass.
#include <cuda_runtime.h>

#include <cstdint>

#include "qng_large.h"

namespace qng {
namespace large {

namespace {

constexpr int kT = 1 << kPhaseTile;        // amplitudes per register tile
constexpr int kRegTile = kT * 8;           // bytes of a register tile (complex64)
constexpr int kNT = kPhaseThreads;         // threads per CTA
constexpr int kA = kPhaseAmps;             // amplitudes per thread per register in a phase
constexpr int kNW = kNT / 32;

static_assert(kNT * kA == kT, "a phase covers the tile");

// Swizzled position of 16-byte chunk c (11 bits) of a register tile, and the 8-byte word of local
// index l. Both are linear over GF(2): wpos(l ^ l') = wpos(l) ^ wpos(l').
__device__ __forceinline__ uint32_t swz(uint32_t c) { return c ^ (((c >> 3) ^ (c >> 6) ^ (c >> 9)) & 7u); }
__device__ __forceinline__ uint32_t wpos(uint32_t l) { return (swz(l >> 1) << 1) | (l & 1u); }

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gmem_src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// An amplitude held in registers, the (re, im) half of one float4 of its register row: a row keeps
// its amplitudes in pairs (m, m + 1) that are the operands of 16-byte shared-memory accesses, so the
// compiler can keep each pair in the aligned register quad those accesses use.
struct Amp {
    float &x, &y;
    __device__ __forceinline__ operator float2() const { return make_float2(x, y); }
    __device__ __forceinline__ Amp &operator=(float2 v) { x = v.x; y = v.y; return *this; }
    __device__ __forceinline__ Amp &operator=(const Amp &o) {
        const float ox = o.x, oy = o.y;
        x = ox;
        y = oy;
        return *this;
    }
};
struct Row {
    float4 q[kA / 2];
    __device__ __forceinline__ Amp operator[](int m) {
        return Amp{(m & 1) ? q[m >> 1].z : q[m >> 1].x, (m & 1) ? q[m >> 1].w : q[m >> 1].y};
    }
};
// the registers a phase holds: slot 0 psi (passes that touch psi) or b2 (passes that do not), 1 a, 2 b
typedef Row Regs[3];

// ---- data movement between the shared-memory tile and the registers of a phase ----------------
// Word of amplitude m: P0 ^ (e0 if bit 0 of m) ^ (e1 if bit 1) ^ ..., the swizzled positions of the
// thread's base index and of the four register bits.
struct PhaseAddr {
    uint32_t P0, e0, e1, e2, e3;
    __device__ __forceinline__ uint32_t at(int m) const {
        return P0 ^ ((m & 1) ? e0 : 0u) ^ ((m & 2) ? e1 : 0u) ^ ((m & 4) ? e2 : 0u) ^ ((m & 8) ? e3 : 0u);
    }
};
template <int R> __device__ __forceinline__ void gather(Regs &X, const float2 *tile, const PhaseAddr &A, bool vmode) {
    if (vmode) {
#pragma unroll
        for (int m = 0; m < kA; m += 2) X[R].q[m >> 1] = reinterpret_cast<const float4 *>(tile)[A.at(m) >> 1];
    } else {
#pragma unroll
        for (int m = 0; m < kA; ++m) X[R][m] = tile[A.at(m)];
    }
}
template <int R> __device__ __forceinline__ void scatter(Regs &X, float2 *tile, const PhaseAddr &A, bool vmode) {
    if (vmode) {
#pragma unroll
        for (int m = 0; m < kA; m += 2) reinterpret_cast<float4 *>(tile)[A.at(m) >> 1] = X[R].q[m >> 1];
    } else {
#pragma unroll
        for (int m = 0; m < kA; ++m) tile[A.at(m)] = X[R][m];
    }
}

// ---- the operations, on registers held in a phase -------------------------------------------
// Every operation is compiled for its register(s), axis, register bit of the pair target and
// rotation case; a diagonal part reads its qubit's bit either as a compile-time pattern over the
// 16 amplitudes (the qubit is register bit DK) or as one bit per thread (a thread or tile bit).
template <int DK> __device__ __forceinline__ constexpr uint32_t pat() {
    return DK == 0 ? 0xAAAAu : (DK == 1 ? 0xCCCCu : (DK == 2 ? 0xF0F0u : (DK == 3 ? 0xFF00u : 0u)));
}

// A rotation exp(+- i alpha sigma) acts on the amplitude pairs of its target (X, Y) or on each
// amplitude (Z) as plane rotations by +-alpha of 2 x 2 blocks of real components. A block (u, v)
// turns by phi through three in-place shears, u -= a v, v += b u, u -= a v (a = tan(phi/2),
// b = sin(phi)): every FMA overwrites one component from the other's current value, so no
// temporaries are needed, and |phi| <= pi/2 keeps |a|, |b| <= 1.
template <bool NEG> __device__ __forceinline__ void shear3(float &u, float &v, float a, float b) {
    if (NEG) { u = fmaf(a, v, u); v = fmaf(-b, u, v); u = fmaf(a, v, u); }
    else     { u = fmaf(-a, v, u); v = fmaf(b, u, v); u = fmaf(-a, v, u); }
}
// (cos alpha + i sin alpha sigma) on the pair (x0, x1): X blocks (x0.x, x1.y), (x1.x, x0.y);
// Y blocks (x1.x, x0.x), (x1.y, x0.y); each turned by alpha
template <int AX> __device__ __forceinline__ void rot_pair(Amp x0, Amp x1, float a, float b) {
    if (AX == kAxisX) { shear3<false>(x0.x, x1.y, a, b); shear3<false>(x1.x, x0.y, a, b); }
    else              { shear3<false>(x1.x, x0.x, a, b); shear3<false>(x1.y, x0.y, a, b); }
}
// (cos alpha + i sin alpha (-1)^S) on one amplitude: the block (x.x, x.y) turned by +-alpha
template <bool S> __device__ __forceinline__ void rot_amp(Amp x, float a, float b) { shear3<S>(x.x, x.y, a, b); }

// inner product <A| sigma |B> (IM 0: Re, 1: Im, 2: both) over the register-bit-K pairs, then, when
// ROT, the rotation of the same axis on A and B
// The inner product reads every amplitude before the first shear overwrites one: the rotation
// coefficients are made to depend on the finished sums (an empty asm with operands, no instruction),
// so the compiler cannot interleave the two and keep old and new values alive together, which would
// cost a register copy per component. Four independent partial sums keep the FMA chains short.
__device__ __forceinline__ void after(float &a, float &b, float re, float im) {
    asm volatile("" : "+f"(a), "+f"(b) : "f"(re), "f"(im));
}
template <int RA, int RB, int IM, bool ROT, int K, int AX>
__device__ __forceinline__ void step_pairs(Regs &X, float a, float b, float &re, float &im) {
    // four accumulators per part, one per product of a pair: chains of 8 dependent FMAs, not 16
    float pr[4] = {0.0f, 0.0f, 0.0f, 0.0f}, pi[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int m0 = 0; m0 < kA; ++m0) {
        if (m0 & (1 << K)) continue;
        const int m1 = m0 | (1 << K);
        const float2 a0 = X[RA][m0], a1 = X[RA][m1], b0 = X[RB][m0], b1 = X[RB][m1];
        float2 s0, s1;  // (sigma b)_0, (sigma b)_1
        if (AX == kAxisX) { s0 = b1; s1 = b0; }
        else              { s0 = make_float2(b1.y, -b1.x); s1 = make_float2(-b0.y, b0.x); }
        if (IM != 1) {
            pr[0] = fmaf(a0.x, s0.x, pr[0]); pr[1] = fmaf(a0.y, s0.y, pr[1]);
            pr[2] = fmaf(a1.x, s1.x, pr[2]); pr[3] = fmaf(a1.y, s1.y, pr[3]);
        }
        if (IM != 0) {
            pi[0] = fmaf(a0.x, s0.y, pi[0]); pi[1] = fmaf(-a0.y, s0.x, pi[1]);
            pi[2] = fmaf(a1.x, s1.y, pi[2]); pi[3] = fmaf(-a1.y, s1.x, pi[3]);
        }
    }
    const float r = (pr[0] + pr[1]) + (pr[2] + pr[3]), i = (pi[0] + pi[1]) + (pi[2] + pi[3]);
    if (IM != 1) re += r;
    if (IM != 0) im += i;
    if (ROT) {
        after(a, b, r, i);
#pragma unroll
        for (int m0 = 0; m0 < kA; ++m0) {
            if (m0 & (1 << K)) continue;
            const int m1 = m0 | (1 << K);
            rot_pair<AX>(X[RA][m0], X[RA][m1], a, b);
            rot_pair<AX>(X[RB][m0], X[RB][m1], a, b);
        }
    }
}
// Z-axis step: the qubit's bit of amplitude m is bit m of pattern PT
template <int RA, int RB, int IM, bool ROT, uint32_t PT>
__device__ __forceinline__ void step_diag(Regs &X, float a, float b, float &re, float &im) {
    float pr[4] = {0.0f, 0.0f, 0.0f, 0.0f}, pi[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int m = 0; m < kA; ++m) {
        const bool sb = ((PT >> m) & 1u) != 0;
        const float2 av = X[RA][m], bv = X[RB][m];
        const float2 af = sb ? make_float2(-av.x, -av.y) : av;  // (Z b)_m = (-1)^bit b_m, folded into a
        if (IM != 1) pr[m & 3] = fmaf(af.x, bv.x, fmaf(af.y, bv.y, pr[m & 3]));
        if (IM != 0) pi[m & 3] = fmaf(af.x, bv.y, fmaf(-af.y, bv.x, pi[m & 3]));
    }
    const float r = (pr[0] + pr[1]) + (pr[2] + pr[3]), i = (pi[0] + pi[1]) + (pi[2] + pi[3]);
    if (IM != 1) re += r;
    if (IM != 0) im += i;
    if (ROT) {
        after(a, b, r, i);
#pragma unroll
        for (int m = 0; m < kA; ++m) {
            if ((PT >> m) & 1u) { rot_amp<true>(X[RA][m], a, b); rot_amp<true>(X[RB][m], a, b); }
            else                { rot_amp<false>(X[RA][m], a, b); rot_amp<false>(X[RB][m], a, b); }
        }
    }
}
// The step of two columns sharing a: inner products <a|sigma|b> and <a|sigma|b2> (b2 in slot 0), then,
// when ROT, the rotation on a, b and b2. acc: Re ab, Im ab, Re ab2, Im ab2 (Im only for IM 2).
template <int IM, bool ROT, int K, int AX>
__device__ __forceinline__ void step2_pairs(Regs &X, float a, float b, float (&acc)[4]) {
    // the products of a pair go to separate accumulators: chains of 8 dependent FMAs, not 16
    float pr[2][2] = {}, pi[2][2] = {}, qr[2][2] = {}, qi[2][2] = {};
#pragma unroll
    for (int m0 = 0; m0 < kA; ++m0) {
        if (m0 & (1 << K)) continue;
        const int m1 = m0 | (1 << K);
        const float2 a0 = X[1][m0], a1 = X[1][m1], b0 = X[2][m0], b1 = X[2][m1], c0 = X[0][m0], c1 = X[0][m1];
        float2 s0, s1, t0, t1;  // sigma b, sigma b2 at m0, m1
        if (AX == kAxisX) { s0 = b1; s1 = b0; t0 = c1; t1 = c0; }
        else {
            s0 = make_float2(b1.y, -b1.x); s1 = make_float2(-b0.y, b0.x);
            t0 = make_float2(c1.y, -c1.x); t1 = make_float2(-c0.y, c0.x);
        }
        pr[0][0] = fmaf(a0.x, s0.x, pr[0][0]); pr[0][1] = fmaf(a0.y, s0.y, pr[0][1]);
        pr[1][0] = fmaf(a1.x, s1.x, pr[1][0]); pr[1][1] = fmaf(a1.y, s1.y, pr[1][1]);
        qr[0][0] = fmaf(a0.x, t0.x, qr[0][0]); qr[0][1] = fmaf(a0.y, t0.y, qr[0][1]);
        qr[1][0] = fmaf(a1.x, t1.x, qr[1][0]); qr[1][1] = fmaf(a1.y, t1.y, qr[1][1]);
        if (IM == 2) {
            pi[0][0] = fmaf(a0.x, s0.y, pi[0][0]); pi[0][1] = fmaf(-a0.y, s0.x, pi[0][1]);
            pi[1][0] = fmaf(a1.x, s1.y, pi[1][0]); pi[1][1] = fmaf(-a1.y, s1.x, pi[1][1]);
            qi[0][0] = fmaf(a0.x, t0.y, qi[0][0]); qi[0][1] = fmaf(-a0.y, t0.x, qi[0][1]);
            qi[1][0] = fmaf(a1.x, t1.y, qi[1][0]); qi[1][1] = fmaf(-a1.y, t1.x, qi[1][1]);
        }
    }
    const float r1 = (pr[0][0] + pr[0][1]) + (pr[1][0] + pr[1][1]);
    const float r2 = (qr[0][0] + qr[0][1]) + (qr[1][0] + qr[1][1]);
    acc[0] += r1;
    acc[2] += r2;
    if (IM == 2) {
        acc[1] += (pi[0][0] + pi[0][1]) + (pi[1][0] + pi[1][1]);
        acc[3] += (qi[0][0] + qi[0][1]) + (qi[1][0] + qi[1][1]);
    }
    if (ROT) {
        after(a, b, r1, r2);
#pragma unroll
        for (int m0 = 0; m0 < kA; ++m0) {
            if (m0 & (1 << K)) continue;
            const int m1 = m0 | (1 << K);
            rot_pair<AX>(X[1][m0], X[1][m1], a, b);
            rot_pair<AX>(X[2][m0], X[2][m1], a, b);
            rot_pair<AX>(X[0][m0], X[0][m1], a, b);
        }
    }
}
template <int IM, bool ROT, uint32_t PT>
__device__ __forceinline__ void step2_diag(Regs &X, float a, float b, float (&acc)[4]) {
    float pr[4] = {}, pi[4] = {}, qr[4] = {}, qi[4] = {};
#pragma unroll
    for (int m = 0; m < kA; ++m) {
        const bool sb = ((PT >> m) & 1u) != 0;
        const float2 av = X[1][m], bv = X[2][m], cv = X[0][m];
        const float2 af = sb ? make_float2(-av.x, -av.y) : av;
        pr[m & 3] = fmaf(af.x, bv.x, fmaf(af.y, bv.y, pr[m & 3]));
        qr[m & 3] = fmaf(af.x, cv.x, fmaf(af.y, cv.y, qr[m & 3]));
        if (IM == 2) {
            pi[m & 3] = fmaf(af.x, bv.y, fmaf(-af.y, bv.x, pi[m & 3]));
            qi[m & 3] = fmaf(af.x, cv.y, fmaf(-af.y, cv.x, qi[m & 3]));
        }
    }
    const float r1 = (pr[0] + pr[1]) + (pr[2] + pr[3]), r2 = (qr[0] + qr[1]) + (qr[2] + qr[3]);
    acc[0] += r1;
    acc[2] += r2;
    if (IM == 2) {
        acc[1] += (pi[0] + pi[1]) + (pi[2] + pi[3]);
        acc[3] += (qi[0] + qi[1]) + (qi[2] + qi[3]);
    }
    if (ROT) {
        after(a, b, r1, r2);
#pragma unroll
        for (int m = 0; m < kA; ++m) {
            if ((PT >> m) & 1u) { rot_amp<true>(X[1][m], a, b); rot_amp<true>(X[2][m], a, b); rot_amp<true>(X[0][m], a, b); }
            else                { rot_amp<false>(X[1][m], a, b); rot_amp<false>(X[2][m], a, b); rot_amp<false>(X[0][m], a, b); }
        }
    }
}

// rotation of register R about axis AX (X or Y) on register bit K
template <int R, int K, int AX> __device__ __forceinline__ void rot_pairs(Regs &X, float a, float b) {
#pragma unroll
    for (int m0 = 0; m0 < kA; ++m0) {
        if (m0 & (1 << K)) continue;
        rot_pair<AX>(X[R][m0], X[R][m0 | (1 << K)], a, b);
    }
}
template <int R, uint32_t PT> __device__ __forceinline__ void rot_diag(Regs &X, float a, float b) {
#pragma unroll
    for (int m = 0; m < kA; ++m) {
        if ((PT >> m) & 1u) rot_amp<true>(X[R][m], a, b);
        else                rot_amp<false>(X[R][m], a, b);
    }
}
// sigma of register R on register bit K
template <int R, int K, int AX> __device__ __forceinline__ void sigma_pairs(Regs &X) {
#pragma unroll
    for (int m0 = 0; m0 < kA; ++m0) {
        if (m0 & (1 << K)) continue;
        const int m1 = m0 | (1 << K);
        const float2 x0 = X[R][m0], x1 = X[R][m1];
        if (AX == kAxisX) { X[R][m0] = x1; X[R][m1] = x0; }
        else              { X[R][m0] = make_float2(x1.y, -x1.x); X[R][m1] = make_float2(-x0.y, x0.x); }  // -i x1, i x0
    }
}
// sign flip of the amplitudes set in PT
template <int R, uint32_t PT> __device__ __forceinline__ void flip_pat(Regs &X) {
#pragma unroll
    for (int m = 0; m < kA; ++m)
        if ((PT >> m) & 1u) X[R][m] = make_float2(-X[R][m].x, -X[R][m].y);
}
// fixed gates on the pairs of register bit K: CNOT with its control register bit C (C < 0: all
// pairs, the caller has tested a thread-uniform control bit), X, Y, H (without 1/sqrt 2)
template <int R, int K, int C> __device__ __forceinline__ void cnot_pairs(Regs &X) {
#pragma unroll
    for (int m0 = 0; m0 < kA; ++m0) {
        if (m0 & (1 << K)) continue;
        if (C >= 0 && !((m0 >> C) & 1)) continue;
        const int m1 = m0 | (1 << K);
        const float2 x0 = X[R][m0];
        X[R][m0] = X[R][m1];
        X[R][m1] = x0;
    }
}
template <int R, int K, int KIND> __device__ __forceinline__ void fixed_pairs(Regs &X) {
#pragma unroll
    for (int m0 = 0; m0 < kA; ++m0) {
        if (m0 & (1 << K)) continue;
        const int m1 = m0 | (1 << K);
        const float2 x0 = X[R][m0], x1 = X[R][m1];
        if (KIND == QNG_GATE_X) {
            X[R][m0] = x1;
            X[R][m1] = x0;
        } else if (KIND == QNG_GATE_Y) {
            X[R][m0] = make_float2(x1.y, -x1.x);
            X[R][m1] = make_float2(-x0.y, x0.x);
        } else {  // H
            const float h = 0.70710678118654752440f;
            X[R][m0] = make_float2((x0.x + x1.x) * h, (x0.y + x1.y) * h);
            X[R][m1] = make_float2((x0.x - x1.x) * h, (x0.y - x1.y) * h);
        }
    }
}

// ---- variant numbering -------------------------------------------------------------------------
// Axis variant av of a step, inner product, rotation or sigma: 0..3 X on register bit av, 4..7 Y on
// register bit av - 4, 8 Z on a thread-uniform bit, 9..12 Z on register bit av - 9. Steps and
// rotations use av as well.
// Fixed-gate variant fv: 0..10 CZ (pattern cz_pattern(fv)); 11 Z uniform, 12..15 Z on register bit
// fv - 12; 16..35 CNOT (target register bit (fv - 16) / 5, control (fv - 16) % 5: 0 uniform, 1..4
// register bit - 1); 36..39 X, 40..43 Y, 44..47 H on register bit fv % 4.
// CZ patterns: both bits uniform; one register bit k; two register bits (k0 < k1)
__host__ __device__ constexpr uint32_t cz_pattern(int fv) {
    return fv == 0 ? 0xFFFFu
         : fv <= 4 ? (fv == 1 ? 0xAAAAu : fv == 2 ? 0xCCCCu : fv == 3 ? 0xF0F0u : 0xFF00u)
         : fv == 5 ? (0xAAAAu & 0xCCCCu) : fv == 6 ? (0xAAAAu & 0xF0F0u) : fv == 7 ? (0xAAAAu & 0xFF00u)
         : fv == 8 ? (0xCCCCu & 0xF0F0u) : fv == 9 ? (0xCCCCu & 0xFF00u) : (0xF0F0u & 0xFF00u);
}
__device__ __forceinline__ int cz_index(int k0, int k1) {  // register positions (-1: uniform)
    if (k0 > k1) { const int x = k0; k0 = k1; k1 = x; }
    if (k1 < 0) return 0;
    if (k0 < 0) return 1 + k1;
    const int base[3] = {5, 8, 10};
    return base[k0] + (k1 - k0 - 1);
}

// Runs variant v. u0 / u1: the thread-uniform bits of the op's qubits q0 / q1 (1 where the qubit
// is a register bit, whose bits the variant's pattern carries). Steps and inner products add their
// partial sums to re / im.
template <int RA, int RB, int IM, bool ROT>
__device__ __forceinline__ void step_av(Regs &X, int av, float a, float b, uint32_t u0, float &re, float &im) {
    switch (av) {
#define QNG_SP(K, AX) step_pairs<RA, RB, IM, ROT, K, AX>(X, a, b, re, im); break;
    case 0: QNG_SP(0, kAxisX) case 1: QNG_SP(1, kAxisX) case 2: QNG_SP(2, kAxisX) case 3: QNG_SP(3, kAxisX)
    case 4: QNG_SP(0, kAxisY) case 5: QNG_SP(1, kAxisY) case 6: QNG_SP(2, kAxisY) case 7: QNG_SP(3, kAxisY)
#undef QNG_SP
    case 8: {  // Z on a thread-uniform bit: its sign goes into the angle and the inner product
        float r2 = 0.0f, i2 = 0.0f;
        step_diag<RA, RB, IM, ROT, 0u>(X, u0 ? -a : a, u0 ? -b : b, r2, i2);
        re += u0 ? -r2 : r2;
        im += u0 ? -i2 : i2;
        break;
    }
    case 9: step_diag<RA, RB, IM, ROT, pat<0>()>(X, a, b, re, im); break;
    case 10: step_diag<RA, RB, IM, ROT, pat<1>()>(X, a, b, re, im); break;
    case 11: step_diag<RA, RB, IM, ROT, pat<2>()>(X, a, b, re, im); break;
    case 12: step_diag<RA, RB, IM, ROT, pat<3>()>(X, a, b, re, im); break;
    default: break;
    }
}

template <int IM>
__device__ __forceinline__ void step2_av(Regs &X, int av, float a, float b, uint32_t u0, float (&acc)[4]) {
    switch (av) {
#define QNG_SP2(K, AX) step2_pairs<IM, true, K, AX>(X, a, b, acc); break;
    case 0: QNG_SP2(0, kAxisX) case 1: QNG_SP2(1, kAxisX) case 2: QNG_SP2(2, kAxisX) case 3: QNG_SP2(3, kAxisX)
    case 4: QNG_SP2(0, kAxisY) case 5: QNG_SP2(1, kAxisY) case 6: QNG_SP2(2, kAxisY) case 7: QNG_SP2(3, kAxisY)
#undef QNG_SP2
    case 8: {  // Z on a thread-uniform bit: its sign goes into the angle and the inner products
        float t[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        step2_diag<IM, true, 0u>(X, u0 ? -a : a, u0 ? -b : b, t);
#pragma unroll
        for (int k = 0; k < 4; ++k) acc[k] += u0 ? -t[k] : t[k];
        break;
    }
    case 9: step2_diag<IM, true, pat<0>()>(X, a, b, acc); break;
    case 10: step2_diag<IM, true, pat<1>()>(X, a, b, acc); break;
    case 11: step2_diag<IM, true, pat<2>()>(X, a, b, acc); break;
    case 12: step2_diag<IM, true, pat<3>()>(X, a, b, acc); break;
    default: break;
    }
}

template <int R> __device__ __forceinline__ void rot_av(Regs &X, int av, float a, float b, uint32_t u0) {
    switch (av) {
    case 0: rot_pairs<R, 0, kAxisX>(X, a, b); break;
    case 1: rot_pairs<R, 1, kAxisX>(X, a, b); break;
    case 2: rot_pairs<R, 2, kAxisX>(X, a, b); break;
    case 3: rot_pairs<R, 3, kAxisX>(X, a, b); break;
    case 4: rot_pairs<R, 0, kAxisY>(X, a, b); break;
    case 5: rot_pairs<R, 1, kAxisY>(X, a, b); break;
    case 6: rot_pairs<R, 2, kAxisY>(X, a, b); break;
    case 7: rot_pairs<R, 3, kAxisY>(X, a, b); break;
    case 8: rot_diag<R, 0u>(X, u0 ? -a : a, u0 ? -b : b); break;
    case 9: rot_diag<R, pat<0>()>(X, a, b); break;
    case 10: rot_diag<R, pat<1>()>(X, a, b); break;
    case 11: rot_diag<R, pat<2>()>(X, a, b); break;
    case 12: rot_diag<R, pat<3>()>(X, a, b); break;
    default: break;
    }
}

template <int R> __device__ __forceinline__ void sigma_av(Regs &X, int av, uint32_t u0) {
    switch (av) {
    case 0: sigma_pairs<R, 0, kAxisX>(X); break;
    case 1: sigma_pairs<R, 1, kAxisX>(X); break;
    case 2: sigma_pairs<R, 2, kAxisX>(X); break;
    case 3: sigma_pairs<R, 3, kAxisX>(X); break;
    case 4: sigma_pairs<R, 0, kAxisY>(X); break;
    case 5: sigma_pairs<R, 1, kAxisY>(X); break;
    case 6: sigma_pairs<R, 2, kAxisY>(X); break;
    case 7: sigma_pairs<R, 3, kAxisY>(X); break;
    case 8: if (u0) flip_pat<R, 0xFFFFu>(X); break;
    case 9: flip_pat<R, pat<0>()>(X); break;
    case 10: flip_pat<R, pat<1>()>(X); break;
    case 11: flip_pat<R, pat<2>()>(X); break;
    case 12: flip_pat<R, pat<3>()>(X); break;
    default: break;
    }
}

template <int R> __device__ __forceinline__ void fixed_fv(Regs &X, int fv, uint32_t u0, uint32_t u1) {
    switch (fv) {
#define QNG_CZ(F) case F: if (u0 & u1) flip_pat<R, cz_pattern(F)>(X); break;
    QNG_CZ(0) QNG_CZ(1) QNG_CZ(2) QNG_CZ(3) QNG_CZ(4) QNG_CZ(5) QNG_CZ(6) QNG_CZ(7) QNG_CZ(8) QNG_CZ(9) QNG_CZ(10)
#undef QNG_CZ
    case 11: if (u0) flip_pat<R, 0xFFFFu>(X); break;
    case 12: flip_pat<R, pat<0>()>(X); break;
    case 13: flip_pat<R, pat<1>()>(X); break;
    case 14: flip_pat<R, pat<2>()>(X); break;
    case 15: flip_pat<R, pat<3>()>(X); break;
#define QNG_CN(K)                                                  \
    case 16 + 5 * K: if (u0) cnot_pairs<R, K, -1>(X); break;       \
    case 17 + 5 * K: cnot_pairs<R, K, 0>(X); break;                \
    case 18 + 5 * K: cnot_pairs<R, K, 1>(X); break;                \
    case 19 + 5 * K: cnot_pairs<R, K, 2>(X); break;                \
    case 20 + 5 * K: cnot_pairs<R, K, 3>(X); break;
    QNG_CN(0) QNG_CN(1) QNG_CN(2) QNG_CN(3)
#undef QNG_CN
    case 36: fixed_pairs<R, 0, QNG_GATE_X>(X); break;
    case 37: fixed_pairs<R, 1, QNG_GATE_X>(X); break;
    case 38: fixed_pairs<R, 2, QNG_GATE_X>(X); break;
    case 39: fixed_pairs<R, 3, QNG_GATE_X>(X); break;
    case 40: fixed_pairs<R, 0, QNG_GATE_Y>(X); break;
    case 41: fixed_pairs<R, 1, QNG_GATE_Y>(X); break;
    case 42: fixed_pairs<R, 2, QNG_GATE_Y>(X); break;
    case 43: fixed_pairs<R, 3, QNG_GATE_Y>(X); break;
    case 44: fixed_pairs<R, 0, QNG_GATE_H>(X); break;
    case 45: fixed_pairs<R, 1, QNG_GATE_H>(X); break;
    case 46: fixed_pairs<R, 2, QNG_GATE_H>(X); break;
    case 47: fixed_pairs<R, 3, QNG_GATE_H>(X); break;
    default: break;
    }
}

__device__ __forceinline__ void set_status(int32_t *status, int code) {
    if (status) atomicCAS(status, 0, code);
}

}  // namespace

// An operation of the pass, decoded once per CTA: one 16-byte shared-memory load.
struct __align__(16) OpD {
    uint8_t cat;    // kCat*
    uint8_t sub;    // step: register combo (0 (a, b, Re), 1 (a, b, Re and Im), 2 (psi, a, Im)); step of two
                    // columns: 0 Re, 1 Re and Im; inner product, sigma: 0 on b, 1 on b2; fixed: fv
    uint8_t var;    // step, rotation, inner product, sigma: av
    uint8_t regs;   // fixed gate: register mask
    int8_t q0u, q1u;  // qubit whose thread-uniform bit the variant reads, or -1 (a register bit: 1)
    uint8_t slot;
    uint8_t pad;      // first operation of a diagonal run: PassOp::zrun, else 0
    float a, b;     // rotation: tan(phi / 2), sin(phi) of its plane rotations (see shear3)
};
static_assert(sizeof(OpD) == 16, "one 16-byte shared-memory load per operation");
enum : uint8_t {
    kCatNop = 0, kCatCopyA, kCatCopyB, kCatZero, kCatStep, kCatIp, kCatRot, kCatSigma, kCatFixed, kCatStep2, kCatCopyAB2,
    kCatBad
};

// axis variant (see the numbering above) of an operation on axis ax with pair target kt and the
// diagonal qubit at register position dk
__device__ __forceinline__ int axis_variant(int ax, int kt, int dk) {
    if (ax == kAxisX) return kt >= 0 ? kt : -1;
    if (ax == kAxisY) return kt >= 0 ? 4 + kt : -1;
    if (ax == kAxisZ) return dk >= 0 ? 9 + dk : 8;
    return -1;
}

// Straight-line phases (PassPhase::macro): the whole phase is one basic block, so the compiler keeps
// the amplitudes in place from step to step and nothing is decoded per operation.
// Operation K of the run targets register bit K, or M - 1 - K when REV (targets in descending order).
template <int AX, int K, int M, bool REV>
__device__ __forceinline__ void steps_run(Regs &X, const OpD *d, float *part, int lane, int tid) {
    if constexpr (K < M) {
        const OpD o = d[K];
        float re = 0.0f, im = 0.0f;
        step_pairs<1, 2, 0, true, REV ? M - 1 - K : K, AX>(X, o.a, o.b, re, im);
        re += __shfl_xor_sync(0xffffffffu, re, 1);
        if (!(lane & 1)) part[o.slot * (kNT / 2) + (tid >> 1)] = re;
        steps_run<AX, K + 1, M, REV>(X, d, part, lane, tid);
    }
}
template <int AX, bool REV>
__device__ __forceinline__ void macro_steps(Regs &X, int m, const OpD *d, float *part, int lane, int tid) {
    switch (m) {
    case 1: steps_run<AX, 0, 1, REV>(X, d, part, lane, tid); break;
    case 2: steps_run<AX, 0, 2, REV>(X, d, part, lane, tid); break;
    case 3: steps_run<AX, 0, 3, REV>(X, d, part, lane, tid); break;
    default: steps_run<AX, 0, 4, REV>(X, d, part, lane, tid); break;
    }
}
template <int K, int M> __device__ __forceinline__ void cnots_run(Regs &X, uint32_t ulast) {
    if constexpr (K < M) {
        if constexpr (K < M - 1) {
            cnot_pairs<1, K, K + 1>(X);
            cnot_pairs<2, K, K + 1>(X);
        } else if (ulast) {
            cnot_pairs<1, K, -1>(X);
            cnot_pairs<2, K, -1>(X);
        }
        cnots_run<K + 1, M>(X, ulast);
    }
}
__device__ __forceinline__ void macro_cnots(Regs &X, int m, uint32_t ulast) {
    switch (m) {
    case 1: cnots_run<0, 1>(X, ulast); break;
    case 2: cnots_run<0, 2>(X, ulast); break;
    case 3: cnots_run<0, 3>(X, ulast); break;
    default: cnots_run<0, 4>(X, ulast); break;
    }
}
// the same two forms for the steps of two columns and for CNOTs on b2 as well (slot 0)
template <int AX, int K, int M, bool REV>
__device__ __forceinline__ void steps2_run(Regs &X, const OpD *d, float *part, int lane, int tid) {
    if constexpr (K < M) {
        const OpD o = d[K];
        float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        step2_pairs<0, true, REV ? M - 1 - K : K, AX>(X, o.a, o.b, acc);
        acc[0] += __shfl_xor_sync(0xffffffffu, acc[0], 1);
        acc[2] += __shfl_xor_sync(0xffffffffu, acc[2], 1);
        if (!(lane & 1)) {
            part[o.slot * (kNT / 2) + (tid >> 1)] = acc[0];
            part[(o.slot + 1) * (kNT / 2) + (tid >> 1)] = acc[2];
        }
        steps2_run<AX, K + 1, M, REV>(X, d, part, lane, tid);
    }
}
template <int AX, bool REV>
__device__ __forceinline__ void macro_steps2(Regs &X, int m, const OpD *d, float *part, int lane, int tid) {
    switch (m) {
    case 1: steps2_run<AX, 0, 1, REV>(X, d, part, lane, tid); break;
    case 2: steps2_run<AX, 0, 2, REV>(X, d, part, lane, tid); break;
    case 3: steps2_run<AX, 0, 3, REV>(X, d, part, lane, tid); break;
    default: steps2_run<AX, 0, 4, REV>(X, d, part, lane, tid); break;
    }
}
template <int K, int M> __device__ __forceinline__ void cnots3_run(Regs &X, uint32_t ulast) {
    if constexpr (K < M) {
        if constexpr (K < M - 1) {
            cnot_pairs<1, K, K + 1>(X);
            cnot_pairs<2, K, K + 1>(X);
            cnot_pairs<0, K, K + 1>(X);
        } else if (ulast) {
            cnot_pairs<1, K, -1>(X);
            cnot_pairs<2, K, -1>(X);
            cnot_pairs<0, K, -1>(X);
        }
        cnots3_run<K + 1, M>(X, ulast);
    }
}
__device__ __forceinline__ void macro_cnots3(Regs &X, int m, uint32_t ulast) {
    switch (m) {
    case 1: cnots3_run<0, 1>(X, ulast); break;
    case 2: cnots3_run<0, 2>(X, ulast); break;
    case 3: cnots3_run<0, 3>(X, ulast); break;
    default: cnots3_run<0, 4>(X, ulast); break;
    }
}

// ---- runs of diagonal operations (PassOp::zrun) ------------------------------------------------
// Z-axis recurrence steps on (a, b) and CZ / Z gates on a and b commute with one another, so every
// step's inner product <a|Z_q|b> equals the one on the run's starting registers, and the run's
// adjoint rotations (cos + i sin Z) and signs compose into one factor per amplitude. For the
// thread's amplitude m that factor is U times, for each register bit k, R_k (bit k of m clear) or its
// conjugate (set), times the sign of the run's gates at m: U collects the rotations on qubits whose
// bit is the same for all 16 amplitudes, R_k those on register bit k. The composed factors are exact
// (cos, sin) products, so a run leaves the registers' float64 signs as they were.
__device__ __forceinline__ float2 cmul(float2 x, float2 y) {
    return make_float2(fmaf(x.x, y.x, -(x.y * y.y)), fmaf(x.x, y.y, x.y * y.x));
}
__device__ __forceinline__ float2 cmulc(float2 x, float2 y) {  // x conj(y)
    return make_float2(fmaf(x.x, y.x, x.y * y.y), fmaf(x.y, y.x, -(x.x * y.y)));
}
// T = sum of v, W[k] = sum over m of (-1)^(bit k of m) v[m]: a butterfly over the four register bits
__device__ __forceinline__ void walsh4(const float (&v)[kA], float &T, float (&W)[4]) {
    float e1[8], e2[4], w0a = 0.0f, w0b = 0.0f;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        e1[i] = v[2 * i] + v[2 * i + 1];
        if (i & 1) w0b += v[2 * i] - v[2 * i + 1];
        else       w0a += v[2 * i] - v[2 * i + 1];
    }
    float w1 = 0.0f;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        e2[i] = e1[2 * i] + e1[2 * i + 1];
        w1 += e1[2 * i] - e1[2 * i + 1];
    }
    const float e30 = e2[0] + e2[1], e31 = e2[2] + e2[3];
    W[0] = w0a + w0b;
    W[1] = w1;
    W[2] = (e2[0] - e2[1]) + (e2[2] - e2[3]);
    W[3] = e30 - e31;
    T = e30 + e31;
}
// sign pattern (bit m: amplitude m changes sign) of a CZ (fv 0..10) or Z (fv 11..15) gate
__device__ __forceinline__ uint32_t diag_mask(int fv, uint32_t u0, uint32_t u1) {
    if (fv <= 10) {
        uint32_t p = 0xFFFFu;
        switch (fv) {
#define QNG_CZP(F) case F: p = cz_pattern(F); break;
        QNG_CZP(1) QNG_CZP(2) QNG_CZP(3) QNG_CZP(4) QNG_CZP(5) QNG_CZP(6) QNG_CZP(7) QNG_CZP(8) QNG_CZP(9) QNG_CZP(10)
#undef QNG_CZP
        default: break;
        }
        return (u0 & u1) ? p : 0u;
    }
    if (fv == 11) return u0 ? 0xFFFFu : 0u;
    return fv == 12 ? pat<0>() : (fv == 13 ? pat<1>() : (fv == 14 ? pat<2>() : pat<3>()));
}
// Inner products of a run with register R (b in slot 2, b2 in slot 0): T, W of Re conj(a) b and, for
// IM 2, of Im conj(a) b.
template <int R, int IM>
__device__ __forceinline__ void zsums(Regs &X, float &T, float (&W)[4], float &Ti, float (&Wi)[4]) {
    float v[kA];
#pragma unroll
    for (int m = 0; m < kA; ++m) v[m] = fmaf(X[1][m].x, X[R][m].x, X[1][m].y * X[R][m].y);
    walsh4(v, T, W);
    if (IM == 2) {
#pragma unroll
        for (int m = 0; m < kA; ++m) v[m] = fmaf(X[1][m].x, X[R][m].y, -(X[1][m].y * X[R][m].x));
        walsh4(v, Ti, Wi);
    }
}
__device__ __forceinline__ float zpick(int k, uint32_t u0, float T, const float (&W)[4]) {
    return k == 0 ? W[0] : (k == 1 ? W[1] : (k == 2 ? W[2] : (k == 3 ? W[3] : (u0 ? -T : T))));
}
// IM 0: each step's Re into its slot; IM 2: Re into its slot and Im into the next. DUAL: steps of two
// columns (b and b2), their values in the order of kOpStep2's slots.
template <int IM, bool DUAL>
__device__ __forceinline__ void zrun(Regs &X, const OpD *d, int len, uint64_t gl, float *part, int lane, int tid) {
    float T, W[4], Ti = 0.0f, Wi[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    float T2 = 0.0f, W2[4] = {0.0f, 0.0f, 0.0f, 0.0f}, T2i = 0.0f, W2i[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    zsums<2, IM>(X, T, W, Ti, Wi);
    if (DUAL) zsums<0, IM>(X, T2, W2, T2i, W2i);
    float2 U = make_float2(1.0f, 0.0f), R0 = U, R1 = U, R2 = U, R3 = U;
    uint32_t sg = 0;
    for (int r = 0; r < len; ++r) {
        const OpD o = d[r];
        const uint32_t u0 = o.q0u < 0 ? 1u : (uint32_t)(gl >> o.q0u) & 1u;
        if (o.cat == kCatStep || o.cat == kCatStep2) {
            const int k = (int)o.var - 9;  // register bit of the qubit, or -1: thread-uniform (variant 8)
            float v[4];
            int nv = 0;
            v[nv++] = zpick(k, u0, T, W);
            if (IM == 2) v[nv++] = zpick(k, u0, Ti, Wi);
            if (DUAL) {
                v[nv++] = zpick(k, u0, T2, W2);
                if (IM == 2) v[nv++] = zpick(k, u0, T2i, W2i);
            }
#pragma unroll
            for (int x = 0; x < nv; ++x) v[x] += __shfl_xor_sync(0xffffffffu, v[x], 1);
            if (!(lane & 1)) {
#pragma unroll
                for (int x = 0; x < nv; ++x) part[(o.slot + x) * (kNT / 2) + (tid >> 1)] = v[x];
            }
            const float2 f = make_float2(o.a, o.b);  // cos, sin of the step's half angle (1, 0 without rotation)
            if (k < 0) U = cmul(U, make_float2(f.x, u0 ? -f.y : f.y));
            else if (k == 0) R0 = cmul(R0, f);
            else if (k == 1) R1 = cmul(R1, f);
            else if (k == 2) R2 = cmul(R2, f);
            else R3 = cmul(R3, f);
        } else {
            const uint32_t u1 = o.q1u < 0 ? 1u : (uint32_t)(gl >> o.q1u) & 1u;
            sg ^= diag_mask(o.sub, u0, u1);
        }
    }
    float2 ph[kA];
    ph[0] = U;
    ph[1] = cmulc(ph[0], R0);
    ph[0] = cmul(ph[0], R0);
#pragma unroll
    for (int e = 0; e < 2; ++e) { ph[e | 2] = cmulc(ph[e], R1); ph[e] = cmul(ph[e], R1); }
#pragma unroll
    for (int e = 0; e < 4; ++e) { ph[e | 4] = cmulc(ph[e], R2); ph[e] = cmul(ph[e], R2); }
#pragma unroll
    for (int e = 0; e < 8; ++e) { ph[e | 8] = cmulc(ph[e], R3); ph[e] = cmul(ph[e], R3); }
    if (sg) {
#pragma unroll
        for (int m = 0; m < kA; ++m)
            if ((sg >> m) & 1u) ph[m] = make_float2(-ph[m].x, -ph[m].y);
    }
#pragma unroll
    for (int m = 0; m < kA; ++m) {
        X[1][m] = cmul(X[1][m], ph[m]);
        X[2][m] = cmul(X[2][m], ph[m]);
        if (DUAL) X[0][m] = cmul(X[0][m], ph[m]);
    }
}

// S: stages of the shared-memory tile ring; PSI: the pass touches register psi (passes of the
// metric columns do not, and their instantiation keeps only a and b in registers)
template <int S, bool PSI>
__global__ void __launch_bounds__(kNT, 1) k_pass_phased(PassArgs pa) {
    // dynamic: the ring [S][nreg][kRegTile], then the inner-product partials [slot][kNT / 2] (float)
    extern __shared__ __align__(128) unsigned char ring[];
    __shared__ uint64_t rowoff[1 << kMaxWin];
    __shared__ __align__(16) OpD opd[kMaxPhaseOps];
    __shared__ PassPhase ph_sh[kMaxPhases];
    __shared__ int8_t lbit[64];
    __shared__ int8_t freeq[64];
    __shared__ uint32_t btab[2][512];  // tile index -> global index of its first amplitude, 9 bits at a time
    __shared__ int s_bad;
    const PassDesc pd = *pa.desc;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const bool well_formed = pd.t == kPhaseTile && pd.low == 5 && pd.win == kMaxWin && pd.nops >= 1 &&
                             pd.nops <= kMaxPhaseOps && pd.nphases >= 1 && pd.nphases <= kMaxPhases &&
                             pd.nslots <= kMaxSlots && (pd.regmask & 9) != 9;
    if (!well_formed) {
        if (tid == 0 && blockIdx.x == 0) set_status(pa.status, QNG_ERR_UNSUPPORTED);
        return;
    }
    int slot_of[kRegs];
    int nreg = 0;
#pragma unroll
    for (int r = 0; r < kRegs; ++r) slot_of[r] = ((pd.regmask >> r) & 1) ? nreg++ : 0;
    {
        // the launch must have sized the ring for this pass's registers, and psi only with PSI
        uint32_t dyn = 0;
        asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn));
        const size_t need = (size_t)S * nreg * kRegTile + (size_t)kMaxSlots * (kNT / 2) * sizeof(float);
        if (dyn < need || (!PSI && (pd.regmask & 1)) || (PSI && (pd.regmask & 8))) {
            if (tid == 0 && blockIdx.x == 0) set_status(pa.status, QNG_ERR_UNSUPPORTED);
            return;
        }
    }
    float *part = reinterpret_cast<float *>(ring + (size_t)S * nreg * kRegTile);  // [slot][kNT / 2]
    if (tid == 0) {
        s_bad = 0;
        for (int q = 0; q < 64; ++q) lbit[q] = -1;
        for (int q = 0; q < pd.low; ++q) lbit[q] = (int8_t)q;
        for (int k = 0; k < pd.win; ++k) lbit[pd.wq[k]] = (int8_t)(pd.low + k);
        int nf = 0;
        for (int q = pd.low; q < pd.n; ++q)
            if (lbit[q] < 0) freeq[nf++] = (int8_t)q;
        for (int k = nf; k < 64; ++k) freeq[k] = -1;
    }
    for (int r = tid; r < (1 << pd.win); r += kNT) {
        uint64_t o = 0;
        for (int k = 0; k < pd.win; ++k) o |= (uint64_t)((r >> k) & 1) << pd.wq[k];
        rowoff[r] = o;
    }
    for (int p = tid; p < pd.nphases; p += kNT) ph_sh[p] = pa.phases[pd.phase_begin + p];
    __syncthreads();
    for (int i = tid; i < 1024; i += kNT) {
        const int half = i >> 9, v = i & 511;
        uint32_t b = 0;
        for (int k = 0; k < 9; ++k) {
            const int q = freeq[9 * half + k];
            if (q >= 0) b |= (uint32_t)((v >> k) & 1) << q;
        }
        btab[half][v] = b;
    }
    // offsets (from the tile's first amplitude) of the thread's 16-byte chunks: the same in every tile
    uint32_t goff[kT / 2 / kNT];
#pragma unroll
    for (int i = 0; i < kT / 2 / kNT; ++i) {
        const uint32_t l = (uint32_t)(tid + i * kNT) << 1;
        goff[i] = (uint32_t)rowoff[l >> 5] | (l & 31u);
    }
    __syncthreads();

    const uint32_t G = gridDim.x;
    const uint64_t ntiles = 1ull << (pd.n - kPhaseTile);
    auto tile_base = [&](uint64_t tile) -> uint64_t { return btab[0][tile & 511u] | btab[1][(tile >> 9) & 511u]; };
    auto stage_reg = [&](int stage, int r) { return ring + ((size_t)stage * nreg + slot_of[r]) * kRegTile; };
    // 16-byte cp.async of every loaded register of a tile into a ring stage
    auto issue = [&](uint64_t tile, int stage) {
        const uint64_t b = tile_base(tile);
#pragma unroll
        for (int r = 0; r < kRegs; ++r) {
            if (!((pd.loadmask & pd.regmask) >> r & 1)) continue;
            const float2 *src = reinterpret_cast<const float2 *>(pa.reg[r]);
            unsigned char *dst = stage_reg(stage, r);
#pragma unroll
            for (int i = 0; i < kT / 2 / kNT; ++i) {
                const uint32_t c = (uint32_t)(tid + i * kNT);
                cp_async16(dst + (size_t)swz(c) * 16, src + b + goff[i]);
            }
        }
    };
    // the first S - 1 tiles' loads go out before the per-pass set-up below
#pragma unroll
    for (int s = 0; s < S - 1; ++s) {
        const uint64_t tile = blockIdx.x + (uint64_t)s * G;
        if (tile < ntiles) issue(tile, s);
        cp_async_commit();
    }

    // decode the operations
    for (int o = tid; o < pd.nops; o += kNT) {
        const PassOp op = pa.ops[pd.op_begin + o];
        OpD d = {};
        d.q0u = (int8_t)((op.dk0 >= 0 || op.q0 < 0) ? -1 : op.q0);
        d.q1u = (int8_t)((op.dk1 >= 0 || op.q1 < 0) ? -1 : op.q1);
        d.slot = (uint8_t)(op.slot >= 0 ? op.slot : 0);
        d.pad = op.zrun > 0 ? (uint8_t)op.zrun : 0;
        if (op.zrun != 0 && (op.kind == kOpStep || op.kind == kOpStep2)) {
            // a step of a diagonal run: the exact cos, sin of its adjoint rotation (1, 0 without one)
            d.a = op.param >= 0 ? (float)pa.coef[op.param].c : 1.0f;
            d.b = op.param >= 0 ? (float)pa.coef[op.param].s : 0.0f;
        } else if ((op.kind == kOpRot || op.kind == kOpStep || op.kind == kOpStep2) && op.param >= 0) {
            // steps take the adjoint rotation cos + i sin sigma; kOpRot R (adjoint 0, cos - i sin
            // sigma) or R^dag (adjoint 1). alpha = theta / 2 in (-pi/2, pi/2]: when cos < 0 the
            // rotation by alpha - pi is used and the register's sign flips (decided below).
            const DevCoef co = pa.coef[op.param];
            const double sg = (op.kind == kOpStep || op.kind == kOpStep2 || op.adjoint) ? 1.0 : -1.0;
            const double flip = co.c < 0.0 ? -1.0 : 1.0;
            const double c = flip * co.c, sn = flip * sg * co.s;  // cos, sin of the plane angle phi
            d.a = (float)(sn / (1.0 + c));
            d.b = (float)sn;
        }
        const int av = axis_variant(op.axis, op.kt, op.dk0);
        switch (op.kind) {
        case kOpCopy:
            d.cat = op.r0 == kRegPsi && op.r1 == kRegA ? kCatCopyA : (op.r0 == kRegPsi && op.r1 == kRegB ? kCatCopyB : kCatBad);
            if (op.r0 == kRegA && op.r1 == kRegB2) d.cat = kCatCopyAB2;
            break;
        case kOpZero: d.cat = op.r0 == kRegPsi ? kCatZero : kCatBad; break;
        case kOpRot:
            d.cat = (op.regs == (1 << kRegPsi) && av >= 0) ? kCatRot : kCatBad;
            d.var = (uint8_t)av;
            break;
        case kOpSigma:
            d.cat = ((op.r0 == kRegB || op.r0 == kRegB2) && av >= 0) ? kCatSigma : kCatBad;
            d.sub = op.r0 == kRegB2 ? 1 : 0;
            d.var = (uint8_t)av;
            break;
        case kOpIp:
            d.cat = ((op.r0 == kRegB || op.r0 == kRegB2) && op.r1 == op.r0 && op.adjoint == 0 && av >= 0) ? kCatIp : kCatBad;
            d.sub = op.r0 == kRegB2 ? 1 : 0;
            d.var = (uint8_t)av;
            break;
        case kOpStep2:
            d.cat = (av >= 0 && (op.adjoint == 0 || op.adjoint == 2)) ? kCatStep2 : kCatBad;
            d.sub = op.adjoint == 2 ? 1 : 0;
            d.var = (uint8_t)av;
            break;
        case kOpStep:
            d.cat = kCatStep;
            if (op.r0 == kRegA && op.r1 == kRegB && op.adjoint == 0) d.sub = 0;
            else if (op.r0 == kRegA && op.r1 == kRegB && op.adjoint == 2) d.sub = 1;
            else if (op.r0 == kRegPsi && op.r1 == kRegA && op.adjoint == 1) d.sub = 2;
            else d.cat = kCatBad;
            if (av < 0) d.cat = kCatBad;
            d.var = (uint8_t)av;
            break;
        case kOpFixed: {
            d.cat = kCatFixed;
            d.regs = (uint8_t)op.regs;
            const int k = op.fixed_kind;
            if (k == QNG_GATE_CZ) d.sub = (uint8_t)cz_index(op.dk0, op.dk1);
            else if (k == QNG_GATE_Z) d.sub = (uint8_t)(op.dk0 >= 0 ? 12 + op.dk0 : 11);
            else if (op.kt < 0) d.cat = kCatBad;
            else if (k == QNG_GATE_CNOT) d.sub = (uint8_t)(16 + 5 * op.kt + (op.dk0 >= 0 ? 1 + op.dk0 : 0));
            else if (k == QNG_GATE_X) d.sub = (uint8_t)(36 + op.kt);
            else if (k == QNG_GATE_Y) d.sub = (uint8_t)(40 + op.kt);
            else if (k == QNG_GATE_H) d.sub = (uint8_t)(44 + op.kt);
            else d.cat = kCatBad;
            if (k == QNG_GATE_CNOT && op.dk0 >= 0 && op.dk0 == op.kt) d.cat = kCatBad;
            break;
        }
        case kOpRecordFac:
        case kOpSetScale: d.cat = kCatNop; break;
        default: d.cat = kCatBad;
        }
        opd[o] = d;
    }
    __syncthreads();
    // The registers' float64 factors evolve the same way in every tile; for complex64 they are
    // +-1 (a rotation taken as alpha - pi flips its registers' signs). Thread 0 of block 0 records
    // the factor of every inner product and the factors at the pass's end.
    if (tid == 0) {
        double sc[kRegs];
        for (int r = 0; r < kRegs; ++r) sc[r] = pa.regscale[(pd.parity & 1) * kRegs + r];
        const bool rec = blockIdx.x == 0;
        int bad = 0;
        for (int o = 0; o < pd.nops; ++o) {
            const PassOp op = pa.ops[pd.op_begin + o];
            bad |= opd[o].cat == kCatBad;
            double f = 1.0;
            if ((op.kind == kOpRot || op.kind == kOpStep || op.kind == kOpStep2) && op.param >= 0 && op.zrun == 0 &&
                pa.coef[op.param].c < 0.0)
                f = -1.0;
            switch (op.kind) {
            case kOpCopy: sc[op.r1] = sc[op.r0]; break;
            case kOpZero: sc[op.r0] = 1.0; break;
            case kOpRot: sc[kRegPsi] *= f; break;
            case kOpIp:
            case kOpRecordFac:
                if (rec) pa.slotfac[pd.slot_base + op.slot] = sc[op.r0] * sc[op.r1];
                break;
            case kOpStep:
                if (rec) {
                    pa.slotfac[pd.slot_base + op.slot] = sc[op.r0] * sc[op.r1];
                    if (op.adjoint == 2) pa.slotfac[pd.slot_base + op.slot + 1] = sc[op.r0] * sc[op.r1];
                }
                if (op.param >= 0) {
                    sc[op.r0] *= f;
                    sc[op.r1] *= f;
                }
                break;
            case kOpStep2: {
                const int nv = op.adjoint == 2 ? 2 : 1;  // values per column
                if (rec)
                    for (int k = 0; k < nv; ++k) {
                        pa.slotfac[pd.slot_base + op.slot + k] = sc[kRegA] * sc[kRegB];
                        pa.slotfac[pd.slot_base + op.slot + nv + k] = sc[kRegA] * sc[kRegB2];
                    }
                if (op.param >= 0) {
                    sc[kRegA] *= f;
                    sc[kRegB] *= f;
                    sc[kRegB2] *= f;
                }
                break;
            }
            case kOpSetScale: sc[op.r1] = sc[op.r0]; break;
            default: break;
            }
        }
        if (rec)
            for (int r = 0; r < kRegs; ++r) pa.regscale[((pd.parity + 1) & 1) * kRegs + r] = sc[r];
        if (bad && rec) set_status(pa.status, QNG_ERR_UNSUPPORTED);
        s_bad = bad;
    }
    __syncthreads();
    if (s_bad) {  // a pass this kernel does not run: nothing is written
        cp_async_wait<0>();
        return;
    }

    double dacc[kMaxSlots / kNW];  // lane 0 of warp w: running float64 sums of slots w, w + 8, ...
#pragma unroll
    for (int k = 0; k < kMaxSlots / kNW; ++k) dacc[k] = 0.0;

    int it = 0;
    for (uint64_t tile = blockIdx.x; tile < ntiles; tile += G, ++it) {
        const uint64_t tn = tile + (uint64_t)(S - 1) * G;
        if (tn < ntiles) issue(tn, (it + S - 1) % S);
        cp_async_commit();
        cp_async_wait<S - 1>();
        __syncthreads();
        const int stage = it % S;
        const uint64_t base = tile_base(tile);
        for (int p = 0; p < pd.nphases; ++p) {
            const PassPhase P = ph_sh[p];
            uint32_t tl = 0;  // the thread's local index with all register bits 0
#pragma unroll
            for (int b = 0; b < 8; ++b) tl |= (uint32_t)((tid >> b) & 1) << P.tbit[b];
            const PhaseAddr ad = {wpos(tl), wpos(1u << P.rbit[0]), wpos(1u << P.rbit[1]), wpos(1u << P.rbit[2]),
                                  wpos(1u << P.rbit[3])};
            const bool vm = P.rbit[0] == 0;
            const int rm = P.rmask & pd.regmask, wm = P.wmask & pd.regmask;
            // the phase's registers: every phase gathers the ones it touches and scatters the ones it
            // writes, so nothing is carried from one phase (or tile) to the next in registers
            Regs X;
            if (PSI && (rm & 1)) gather<0>(X, reinterpret_cast<const float2 *>(stage_reg(stage, 0)), ad, vm);
            if (!PSI && (rm & 8)) gather<0>(X, reinterpret_cast<const float2 *>(stage_reg(stage, 3)), ad, vm);
            if (rm & 2) gather<1>(X, reinterpret_cast<const float2 *>(stage_reg(stage, 1)), ad, vm);
            if (rm & 4) gather<2>(X, reinterpret_cast<const float2 *>(stage_reg(stage, 2)), ad, vm);
            // global index of the thread's amplitude m = 0: the bit of every qubit that is not a
            // register bit is the same for the thread's 16 amplitudes
            const uint64_t gl = base | rowoff[tl >> 5] | (tl & 31u);
            // the phase's last m operations may form a straight-line block (PassPhase::macro); the
            // operations before them run one by one
            const int mb = P.op_end - (P.macro ? (P.macro & 15) : 0);
            for (int o = P.op_begin; o < mb; ++o) {
                const OpD d = opd[o];
                if (d.pad) {  // a run of diagonal operations, composed
                    const int len = d.pad & kMaxZrun;
                    if (d.pad & kZrunDual) {
                        if constexpr (!PSI) {
                            if (d.pad & kZrunIm) zrun<2, true>(X, opd + o, len, gl, part, lane, tid);
                            else zrun<0, true>(X, opd + o, len, gl, part, lane, tid);
                        }
                    } else if (d.pad & kZrunIm) {
                        zrun<2, false>(X, opd + o, len, gl, part, lane, tid);
                    } else {
                        zrun<0, false>(X, opd + o, len, gl, part, lane, tid);
                    }
                    o += len - 1;
                    continue;
                }
                // the thread-uniform bits of q0 / q1, for the variants that read them
                auto ubit = [&](int q) -> uint32_t { return q < 0 ? 1u : (uint32_t)(gl >> q) & 1u; };
                const uint32_t u0 = ubit(d.q0u), u1 = ubit(d.q1u);
                const int cat = (!PSI && (d.cat == kCatCopyA || d.cat == kCatCopyB || d.cat == kCatZero ||
                                          d.cat == kCatRot || (d.cat == kCatStep && d.sub == 2)))
                                    ? (int)kCatNop : (int)d.cat;  // cannot occur: the pass has no psi
                switch (cat) {
                case kCatCopyA:
                    if (PSI) {
#pragma unroll
                        for (int m = 0; m < kA; ++m) X[1][m] = X[0][m];
                    }
                    break;
                case kCatCopyB:
                    if (PSI) {
#pragma unroll
                        for (int m = 0; m < kA; ++m) X[2][m] = X[0][m];
                    }
                    break;
                case kCatZero: {
                    const bool one = gl == 0;
                    if (PSI) {
#pragma unroll
                        for (int m = 0; m < kA; ++m) X[0][m] = make_float2((one && m == 0) ? 1.0f : 0.0f, 0.0f);
                    }
                    break;
                }
                case kCatRot: if (PSI) rot_av<0>(X, d.var, d.a, d.b, u0); break;
                case kCatSigma:
                    if (d.sub == 0) sigma_av<2>(X, d.var, u0);
                    else if constexpr (!PSI) sigma_av<0>(X, d.var, u0);
                    break;
                case kCatFixed:
                    if (PSI && (d.regs & 1)) fixed_fv<0>(X, d.sub, u0, u1);
                    if (!PSI && (d.regs & 8)) fixed_fv<0>(X, d.sub, u0, u1);
                    if (d.regs & 2) fixed_fv<1>(X, d.sub, u0, u1);
                    if (d.regs & 4) fixed_fv<2>(X, d.sub, u0, u1);
                    break;
                case kCatCopyAB2:
                    if constexpr (!PSI) {
#pragma unroll
                        for (int m = 0; m < kA; ++m) X[0][m] = X[1][m];
                    }
                    break;
                case kCatStep2:
                    if constexpr (!PSI) {
                        float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
                        if (d.sub) step2_av<2>(X, d.var, d.a, d.b, u0, acc);
                        else step2_av<0>(X, d.var, d.a, d.b, u0, acc);
                        // slots: Re ab, Re ab2; or Re ab, Im ab, Re ab2, Im ab2
                        float v[4] = {acc[0], d.sub ? acc[1] : acc[2], acc[2], acc[3]};
                        const int nv = d.sub ? 4 : 2;
#pragma unroll
                        for (int x = 0; x < 4; ++x)
                            if (x < nv) v[x] += __shfl_xor_sync(0xffffffffu, v[x], 1);
                        if (!(lane & 1)) {
#pragma unroll
                            for (int x = 0; x < 4; ++x)
                                if (x < nv) part[(d.slot + x) * (kNT / 2) + (tid >> 1)] = v[x];
                        }
                    }
                    break;
                case kCatIp:
                case kCatStep: {
                    float re = 0.0f, im = 0.0f;
                    if (d.cat == kCatIp) {
                        if (d.sub == 0) step_av<2, 2, 0, false>(X, d.var, 0.0f, 0.0f, u0, re, im);
                        else if constexpr (!PSI) step_av<0, 0, 0, false>(X, d.var, 0.0f, 0.0f, u0, re, im);
                    }
                    else if (d.sub == 0) step_av<1, 2, 0, true>(X, d.var, d.a, d.b, u0, re, im);
                    else if (d.sub == 1) step_av<1, 2, 2, true>(X, d.var, d.a, d.b, u0, re, im);
                    else if (PSI) { step_av<0, 1, 1, true>(X, d.var, d.a, d.b, u0, re, im); re = im; }
                    // thread pairs combine, then one float per pair goes to the tile's partials
                    re += __shfl_xor_sync(0xffffffffu, re, 1);
                    const bool two = d.cat == kCatStep && d.sub == 1;
                    if (two) im += __shfl_xor_sync(0xffffffffu, im, 1);
                    if (!(lane & 1)) {
                        part[d.slot * (kNT / 2) + (tid >> 1)] = re;
                        if (two) part[(d.slot + 1) * (kNT / 2) + (tid >> 1)] = im;
                    }
                    break;
                }
                default:
                    break;
                }
            }
            if (P.macro) {
                const int m = P.macro & 15;
                const bool rev = (P.macro & kMacroRev) != 0;
                const OpD *dm = opd + mb;
                if ((P.macro & ~0xFF) == kMacroSteps) {
                    if (((P.macro >> 4) & 7) == kAxisX) {
                        if (rev) macro_steps<kAxisX, true>(X, m, dm, part, lane, tid);
                        else macro_steps<kAxisX, false>(X, m, dm, part, lane, tid);
                    } else {
                        if (rev) macro_steps<kAxisY, true>(X, m, dm, part, lane, tid);
                        else macro_steps<kAxisY, false>(X, m, dm, part, lane, tid);
                    }
                } else if ((P.macro & ~0xFF) == kMacroSteps2) {
                    if constexpr (!PSI) {
                        if (((P.macro >> 4) & 7) == kAxisX) {
                            if (rev) macro_steps2<kAxisX, true>(X, m, dm, part, lane, tid);
                            else macro_steps2<kAxisX, false>(X, m, dm, part, lane, tid);
                        } else {
                            if (rev) macro_steps2<kAxisY, true>(X, m, dm, part, lane, tid);
                            else macro_steps2<kAxisY, false>(X, m, dm, part, lane, tid);
                        }
                    }
                } else {
                    const int q = dm[m - 1].q0u;
                    const uint32_t ul = q < 0 ? 1u : (uint32_t)(gl >> q) & 1u;
                    if ((P.macro >> 4) & 1) {
                        if constexpr (!PSI) macro_cnots3(X, m, ul);
                    } else {
                        macro_cnots(X, m, ul);
                    }
                }
            }
            if (PSI && (wm & 1)) scatter<0>(X, reinterpret_cast<float2 *>(stage_reg(stage, 0)), ad, vm);
            if (!PSI && (wm & 8)) scatter<0>(X, reinterpret_cast<float2 *>(stage_reg(stage, 3)), ad, vm);
            if (wm & 2) scatter<1>(X, reinterpret_cast<float2 *>(stage_reg(stage, 1)), ad, vm);
            if (wm & 4) scatter<2>(X, reinterpret_cast<float2 *>(stage_reg(stage, 2)), ad, vm);
            __syncthreads();
        }
        // the tile's inner products: warp w sums slots w, w + 8, ... over the 128 thread pairs in a
        // fixed order (float32), lane 0 adds each to its float64 running sum
#pragma unroll
        for (int k = 0; k < kMaxSlots / kNW; ++k) {
            const int sl = wid + kNW * k;
            if (sl < pd.nslots) {
                const float *ps = part + sl * (kNT / 2);
                float v = (ps[lane] + ps[lane + 32]) + (ps[lane + 64] + ps[lane + 96]);
                v = warp_sum(v);
                if (lane == 0) dacc[k] += (double)v;
            }
        }
        // store: 16-byte vector stores of the written registers, straight from the ring stage
#pragma unroll
        for (int r = 0; r < kRegs; ++r) {
            if (!((pd.storemask & pd.regmask) >> r & 1)) continue;
            float2 *dst = reinterpret_cast<float2 *>(pa.reg[r]);
            const unsigned char *srcs = stage_reg(stage, r);
#pragma unroll
            for (int i = 0; i < kT / 2 / kNT; ++i) {
                const uint32_t c = (uint32_t)(tid + i * kNT);
                const float4 v = *reinterpret_cast<const float4 *>(srcs + (size_t)swz(c) * 16);
                *reinterpret_cast<float4 *>(dst + base + goff[i]) = v;
            }
        }
        __syncthreads();  // the stage and the partials are free for the next tile
    }
    cp_async_wait<0>();
    // per-CTA partial sums (slot, cta)
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < kMaxSlots / kNW; ++k) {
            const int sl = wid + kNW * k;
            if (sl < pd.nslots) pa.partial[(size_t)(pd.slot_base + sl) * G + blockIdx.x] = dacc[k];
        }
    }
}

int phased_stages(int nreg) { return nreg >= 3 ? 2 : 3; }
size_t phased_smem_bytes(int nreg) {
    return (size_t)phased_stages(nreg) * nreg * kRegTile + (size_t)kMaxSlots * (kNT / 2) * sizeof(float);
}

cudaError_t prepare_pass_phased() {
    cudaError_t e = raise_smem_limit(reinterpret_cast<const void *>(k_pass_phased<2, true>), phased_smem_bytes(3));
    if (e != cudaSuccess) return e;
    if ((e = raise_smem_limit(reinterpret_cast<const void *>(k_pass_phased<2, false>), phased_smem_bytes(3))) != cudaSuccess)
        return e;
    if ((e = raise_smem_limit(reinterpret_cast<const void *>(k_pass_phased<3, true>), phased_smem_bytes(2))) != cudaSuccess)
        return e;
    return raise_smem_limit(reinterpret_cast<const void *>(k_pass_phased<3, false>), phased_smem_bytes(2));
}

cudaError_t launch_pass_phased(const PassArgs &pa, int regmask, int grid, int metric_im, cudaStream_t st) {
    (void)metric_im;  // the complex-metric steps are compiled into the same kernel
    const int nreg = __builtin_popcount(regmask & 15);
    if (nreg < 1 || nreg > 3 || (regmask & 9) == 9) return cudaErrorInvalidValue;
    const size_t smem = phased_smem_bytes(nreg);
    if (phased_stages(nreg) == 2 && (regmask & 1)) k_pass_phased<2, true><<<grid, kNT, smem, st>>>(pa);
    else if (phased_stages(nreg) == 2) k_pass_phased<2, false><<<grid, kNT, smem, st>>>(pa);
    else if (regmask & 1) k_pass_phased<3, true><<<grid, kNT, smem, st>>>(pa);
    else k_pass_phased<3, false><<<grid, kNT, smem, st>>>(pa);
    return cudaGetLastError();
}

}  // namespace large
}  // namespace qng

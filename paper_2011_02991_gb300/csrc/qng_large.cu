// sm_103a kernels of the streaming path, for one instance whose state vectors live in HBM
// (n > 16 qubits, 2^n amplitudes per register). Algorithm 1 keeps O(1) registers (Sec. 3): the
// rolling state psi, the prefix lambda (here "a") and phi (here "b"). Every kernel launch is one
// pass over the registers it touches: the state is cut into tiles of 2^t amplitudes (the low
// kLow qubits, contiguous in memory, plus a window of up to kMaxWin other qubits); a CTA loads a
// tile of each register into shared memory, runs a short program of operations on it (rotations,
// fixed gates, sigma, inner products) and writes it back. Operations on qubits outside the tile
// must be diagonal (Z rotations, CZ, Z, Z-axis inner products); the host forms passes so that all
// other operations act on tile qubits. Several steps of the recurrence share one pass, so HBM
// traffic per step is 4 S / (steps per pass) for the two column registers (S = bytes per register).
//
// Inner products accumulate per CTA into partial[slot][cta]; the column's reduce kernel sums them
// in a fixed order. float64 registers use the scaled form of the on-chip path: each register is a
// float64 factor times a vector, the factors live in a two-entry parity buffer per register
// (launch p reads entry p&1 and writes entry (p+1)&1), and every inner product records the product
// of its registers' factors in slotfac[slot].
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "qng_large.h"

namespace qng {
namespace large {

template <typename R> struct CX2;
template <> struct CX2<double> { using T = double2; };
template <> struct CX2<float> { using T = float2; };

__device__ __forceinline__ double lflip(double v, int p) {
    return __longlong_as_double(__double_as_longlong(v) ^ ((long long)(p & 1) << 63));
}
__device__ __forceinline__ float lflip(float v, int p) { return __int_as_float(__float_as_int(v) ^ ((p & 1) << 31)); }
template <typename T2> __device__ __forceinline__ T2 lflip2(T2 v, int p) {
    v.x = lflip(v.x, p);
    v.y = lflip(v.y, p);
    return v;
}
__device__ __forceinline__ uint32_t lins0(uint32_t p, int q) { return ((p >> q) << (q + 1)) | (p & ((1u << q) - 1u)); }

template <typename RA> __device__ __forceinline__ RA lwarp_sum(RA v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

struct TileCtx {
    int t;                 // tile qubits
    uint32_t T;            // 2^t
    int low;               // contiguous low qubits
    int win;               // window qubits
    int lbit[64];          // local bit of global qubit q, or -1 when q is outside the tile
    uint64_t base;         // global index of the tile's local index 0
};

constexpr int kOpsCached = 96;  // pass ops kept in shared memory (the rest are read from global memory)

// 16-byte asynchronous copy global -> shared (cp.async, cached in L2 only). Both addresses must be
// 16-byte aligned: tiles start on 16-byte boundaries and rows of the state are at least 128 bytes.
__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gmem_src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gmem_src) : "memory");
}

// global index of local index l in the current tile
__device__ __forceinline__ uint64_t gidx(const TileCtx &tc, const uint64_t *rowoff, uint32_t l) {
    return tc.base | rowoff[l >> tc.low] | (l & ((1u << tc.low) - 1u));
}

// bit q of global index of local l
__device__ __forceinline__ int gbit(const TileCtx &tc, uint32_t l, int q) {
    const int lb = tc.lbit[q];
    return lb >= 0 ? (int)((l >> lb) & 1u) : (int)((tc.base >> q) & 1ull);
}


// Partial inner product of one step: re and/or im as IM asks (0: Re, 1: Im, 2: both).
template <typename R> struct Acc2 {
    R re, im;
};

// One recurrence step on the registers A (left) and B (right) in one sweep of the tile: the inner
// product with sigma on the pairs of qubit lb (compile-time axis AX and part IM), then, when ROT,
// the adjoint rotation of the same axis on both registers. Every sign folds into an FMA operand.
template <typename R, int AX, int IM, bool ROT, int CB>
__device__ __forceinline__ Acc2<R> step_pairs(typename CX2<R>::T *A, typename CX2<R>::T *B, uint32_t T, int lb, R c,
                                              R s, R t) {
    using cx = typename CX2<R>::T;
    constexpr bool kScaled = std::is_same<R, double>::value;
    Acc2<R> acc = {0, 0};
    const uint32_t bit = 1u << lb;
    auto rot = [&](cx x, cx v) -> cx {
        cx y;
        if constexpr (kScaled) {
            if constexpr (CB) { y.x = fma(t, x.x, v.x); y.y = fma(t, x.y, v.y); }
            else              { y.x = fma(t, v.x, x.x); y.y = fma(t, v.y, x.y); }
        } else {
            y.x = fma(s, v.x, c * x.x); y.y = fma(s, v.y, c * x.y);
        }
        return y;
    };
    for (uint32_t p = threadIdx.x; p < (T >> 1); p += blockDim.x) {
        const uint32_t l0 = lins0(p, lb), l1 = l0 | bit;
        const cx a0 = A[l0], a1 = A[l1], b0 = B[l0], b1 = B[l1];
        cx s0, s1;  // (sigma b)_0, (sigma b)_1
        if constexpr (AX == kAxisX) { s0 = b1; s1 = b0; }
        else { s0 = cx{b1.y, -b1.x}; s1 = cx{-b0.y, b0.x}; }
        if constexpr (IM != 0) acc.im = fma(a0.x, s0.y, fma(-a0.y, s0.x, fma(a1.x, s1.y, fma(-a1.y, s1.x, acc.im))));
        if constexpr (IM != 1) acc.re = fma(a0.x, s0.x, fma(a0.y, s0.y, fma(a1.x, s1.x, fma(a1.y, s1.y, acc.re))));
        if constexpr (ROT) {
            // (i sigma x)_0, (i sigma x)_1
            if constexpr (AX == kAxisX) {
                A[l0] = rot(a0, cx{-a1.y, a1.x}); A[l1] = rot(a1, cx{-a0.y, a0.x});
                B[l0] = rot(b0, cx{-b1.y, b1.x}); B[l1] = rot(b1, cx{-b0.y, b0.x});
            } else {
                A[l0] = rot(a0, a1); A[l1] = rot(a1, cx{-a0.x, -a0.y});
                B[l0] = rot(b0, b1); B[l1] = rot(b1, cx{-b0.x, -b0.y});
            }
        }
    }
    return acc;
}

template <typename R, int IM, bool ROT, int CB>
__device__ __forceinline__ Acc2<R> step_diag(const TileCtx &tc, typename CX2<R>::T *A, typename CX2<R>::T *B, int q, R c,
                                             R s, R t) {
    using cx = typename CX2<R>::T;
    constexpr bool kScaled = std::is_same<R, double>::value;
    Acc2<R> acc = {0, 0};
    // the tile's fields in registers (the loop's shared-memory stores would force re-reads)
    const uint32_t T = tc.T;
    const int lb = tc.lbit[q];
    const int bfix = lb < 0 ? (int)((tc.base >> q) & 1ull) : 0;
    for (uint32_t l = threadIdx.x; l < T; l += blockDim.x) {
        const int beta = lb >= 0 ? (int)((l >> lb) & 1u) : bfix;
        const cx a = A[l], b = B[l];
        const cx af = lflip2(a, beta);  // (Z b)_beta = (-1)^beta b, folded into a
        if constexpr (IM != 0) acc.im = fma(af.x, b.y, fma(-af.y, b.x, acc.im));
        if constexpr (IM != 1) acc.re = fma(af.x, b.x, fma(af.y, b.y, acc.re));
        if constexpr (ROT) {
            const cx va = {lflip(a.y, beta ^ 1), lflip(a.x, beta)}, vb = {lflip(b.y, beta ^ 1), lflip(b.x, beta)};
            cx ya, yb;
            if constexpr (kScaled) {
                if constexpr (CB) {
                    ya.x = fma(t, a.x, va.x); ya.y = fma(t, a.y, va.y);
                    yb.x = fma(t, b.x, vb.x); yb.y = fma(t, b.y, vb.y);
                } else {
                    ya.x = fma(t, va.x, a.x); ya.y = fma(t, va.y, a.y);
                    yb.x = fma(t, vb.x, b.x); yb.y = fma(t, vb.y, b.y);
                }
            } else {
                ya.x = fma(s, va.x, c * a.x); ya.y = fma(s, va.y, c * a.y);
                yb.x = fma(s, vb.x, c * b.x); yb.y = fma(s, vb.y, c * b.y);
            }
            A[l] = ya;
            B[l] = yb;
        }
    }
    return acc;
}

template <typename R, int IM, int CB>
__device__ __forceinline__ Acc2<R> step_dispatch_cb(const TileCtx &tc, typename CX2<R>::T *A, typename CX2<R>::T *B,
                                                    int ax, int q, bool rot, R c, R s, R t) {
    if (ax == kAxisZ)
        return rot ? step_diag<R, IM, true, CB>(tc, A, B, q, c, s, t) : step_diag<R, IM, false, CB>(tc, A, B, q, c, s, t);
    const int lb = tc.lbit[q];
    if (ax == kAxisX)
        return rot ? step_pairs<R, kAxisX, IM, true, CB>(A, B, tc.T, lb, c, s, t)
                   : step_pairs<R, kAxisX, IM, false, CB>(A, B, tc.T, lb, c, s, t);
    return rot ? step_pairs<R, kAxisY, IM, true, CB>(A, B, tc.T, lb, c, s, t)
               : step_pairs<R, kAxisY, IM, false, CB>(A, B, tc.T, lb, c, s, t);
}

template <typename R, int IM>
__device__ __forceinline__ Acc2<R> step_dispatch(const TileCtx &tc, typename CX2<R>::T *A, typename CX2<R>::T *B, int ax,
                                                 int q, bool rot, R c, R s, R t, int caseB) {
    if (std::is_same<R, double>::value && caseB) return step_dispatch_cb<R, IM, 1>(tc, A, B, ax, q, rot, c, s, t);
    return step_dispatch_cb<R, IM, 0>(tc, A, B, ax, q, rot, c, s, t);
}

// The step of two columns that share a (kOpStep2): the inner products <A|sigma|B> into ab and
// <A|sigma|C> into ac, then, when ROT, the adjoint rotation on A, B and C, in one sweep of the tile.
template <typename R, int AX, int IM, bool ROT, int CB>
__device__ __forceinline__ void step2_pairs(typename CX2<R>::T *A, typename CX2<R>::T *B, typename CX2<R>::T *C,
                                           uint32_t T, int lb, R c, R s, R t, Acc2<R> &ab, Acc2<R> &ac) {
    using cx = typename CX2<R>::T;
    constexpr bool kScaled = std::is_same<R, double>::value;
    const uint32_t bit = 1u << lb;
    auto rot = [&](cx x, cx v) -> cx {
        cx y;
        if constexpr (kScaled) {
            if constexpr (CB) { y.x = fma(t, x.x, v.x); y.y = fma(t, x.y, v.y); }
            else              { y.x = fma(t, v.x, x.x); y.y = fma(t, v.y, x.y); }
        } else {
            y.x = fma(s, v.x, c * x.x); y.y = fma(s, v.y, c * x.y);
        }
        return y;
    };
    auto ip = [&](Acc2<R> &acc, cx a0, cx a1, cx s0, cx s1) {
        if constexpr (IM != 0) acc.im = fma(a0.x, s0.y, fma(-a0.y, s0.x, fma(a1.x, s1.y, fma(-a1.y, s1.x, acc.im))));
        if constexpr (IM != 1) acc.re = fma(a0.x, s0.x, fma(a0.y, s0.y, fma(a1.x, s1.x, fma(a1.y, s1.y, acc.re))));
    };
    for (uint32_t p = threadIdx.x; p < (T >> 1); p += blockDim.x) {
        const uint32_t l0 = lins0(p, lb), l1 = l0 | bit;
        const cx a0 = A[l0], a1 = A[l1], b0 = B[l0], b1 = B[l1], c0 = C[l0], c1 = C[l1];
        if constexpr (AX == kAxisX) {
            ip(ab, a0, a1, b1, b0);
            ip(ac, a0, a1, c1, c0);
        } else {
            ip(ab, a0, a1, cx{b1.y, -b1.x}, cx{-b0.y, b0.x});
            ip(ac, a0, a1, cx{c1.y, -c1.x}, cx{-c0.y, c0.x});
        }
        if constexpr (ROT) {
            if constexpr (AX == kAxisX) {
                A[l0] = rot(a0, cx{-a1.y, a1.x}); A[l1] = rot(a1, cx{-a0.y, a0.x});
                B[l0] = rot(b0, cx{-b1.y, b1.x}); B[l1] = rot(b1, cx{-b0.y, b0.x});
                C[l0] = rot(c0, cx{-c1.y, c1.x}); C[l1] = rot(c1, cx{-c0.y, c0.x});
            } else {
                A[l0] = rot(a0, a1); A[l1] = rot(a1, cx{-a0.x, -a0.y});
                B[l0] = rot(b0, b1); B[l1] = rot(b1, cx{-b0.x, -b0.y});
                C[l0] = rot(c0, c1); C[l1] = rot(c1, cx{-c0.x, -c0.y});
            }
        }
    }
}

template <typename R, int IM, bool ROT, int CB>
__device__ __forceinline__ void step2_diag(const TileCtx &tc, typename CX2<R>::T *A, typename CX2<R>::T *B,
                                           typename CX2<R>::T *C, int q, R c, R s, R t, Acc2<R> &ab, Acc2<R> &ac) {
    using cx = typename CX2<R>::T;
    constexpr bool kScaled = std::is_same<R, double>::value;
    const uint32_t T = tc.T;
    const int lb = tc.lbit[q];
    const int bfix = lb < 0 ? (int)((tc.base >> q) & 1ull) : 0;
    auto rotz = [&](cx x, int beta) -> cx {
        const cx v = {lflip(x.y, beta ^ 1), lflip(x.x, beta)};  // (i Z x)
        cx y;
        if constexpr (kScaled) {
            if constexpr (CB) { y.x = fma(t, x.x, v.x); y.y = fma(t, x.y, v.y); }
            else              { y.x = fma(t, v.x, x.x); y.y = fma(t, v.y, x.y); }
        } else {
            y.x = fma(s, v.x, c * x.x); y.y = fma(s, v.y, c * x.y);
        }
        return y;
    };
    for (uint32_t l = threadIdx.x; l < T; l += blockDim.x) {
        const int beta = lb >= 0 ? (int)((l >> lb) & 1u) : bfix;
        const cx a = A[l], b = B[l], cc = C[l];
        const cx af = lflip2(a, beta);  // (Z b)_beta = (-1)^beta b, folded into a
        if constexpr (IM != 0) {
            ab.im = fma(af.x, b.y, fma(-af.y, b.x, ab.im));
            ac.im = fma(af.x, cc.y, fma(-af.y, cc.x, ac.im));
        }
        if constexpr (IM != 1) {
            ab.re = fma(af.x, b.x, fma(af.y, b.y, ab.re));
            ac.re = fma(af.x, cc.x, fma(af.y, cc.y, ac.re));
        }
        if constexpr (ROT) {
            A[l] = rotz(a, beta);
            B[l] = rotz(b, beta);
            C[l] = rotz(cc, beta);
        }
    }
}

template <typename R, int IM, int CB>
__device__ __forceinline__ void step2_dispatch_cb(const TileCtx &tc, typename CX2<R>::T *A, typename CX2<R>::T *B,
                                                  typename CX2<R>::T *C, int ax, int q, bool rot, R c, R s, R t,
                                                  Acc2<R> &ab, Acc2<R> &ac) {
    if (ax == kAxisZ) {
        if (rot) step2_diag<R, IM, true, CB>(tc, A, B, C, q, c, s, t, ab, ac);
        else step2_diag<R, IM, false, CB>(tc, A, B, C, q, c, s, t, ab, ac);
        return;
    }
    const int lb = tc.lbit[q];
    if (ax == kAxisX) {
        if (rot) step2_pairs<R, kAxisX, IM, true, CB>(A, B, C, tc.T, lb, c, s, t, ab, ac);
        else step2_pairs<R, kAxisX, IM, false, CB>(A, B, C, tc.T, lb, c, s, t, ab, ac);
    } else {
        if (rot) step2_pairs<R, kAxisY, IM, true, CB>(A, B, C, tc.T, lb, c, s, t, ab, ac);
        else step2_pairs<R, kAxisY, IM, false, CB>(A, B, C, tc.T, lb, c, s, t, ab, ac);
    }
}

template <typename R, int IM>
__device__ __forceinline__ void step2_dispatch(const TileCtx &tc, typename CX2<R>::T *A, typename CX2<R>::T *B,
                                               typename CX2<R>::T *C, int ax, int q, bool rot, R c, R s, R t, int caseB,
                                               Acc2<R> &ab, Acc2<R> &ac) {
    if (std::is_same<R, double>::value && caseB) step2_dispatch_cb<R, IM, 1>(tc, A, B, C, ax, q, rot, c, s, t, ab, ac);
    else step2_dispatch_cb<R, IM, 0>(tc, A, B, C, ax, q, rot, c, s, t, ab, ac);
}

// MIM = 1: the pass may hold steps that take both parts of the inner product (adjoint = 2, slots
// slot and slot + 1); a separate instantiation keeps the registers of the other passes unchanged.
template <typename R, int MIM>
__global__ void __launch_bounds__(256) k_pass(PassArgs pa) {
    using cx = typename CX2<R>::T;
    constexpr bool kScaled = std::is_same<R, double>::value;
    constexpr uint32_t kAmpsPer16 = 16 / sizeof(cx);
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ uint64_t rowoff[1 << kMaxWin];
    __shared__ TileCtx tc;
    __shared__ PassOp ops_sh[kOpsCached];  // the pass's program, the same for every tile
    __shared__ double red[32];
    const PassDesc pd = *pa.desc;
    const int nt = blockDim.x, nw = nt >> 5, lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    cx *tile[kRegs];
    {
        cx *p = reinterpret_cast<cx *>(smem);
        for (int r = 0; r < kRegs; ++r) {
            tile[r] = p;
            if (pd.regmask & (1 << r)) p += (size_t)1 << pd.t;
        }
    }
    if (threadIdx.x == 0) {
        tc.t = pd.t;
        tc.T = 1u << pd.t;
        tc.low = pd.low;
        tc.win = pd.win;
        for (int q = 0; q < 64; ++q) tc.lbit[q] = -1;
        for (int q = 0; q < pd.low; ++q) tc.lbit[q] = q;
        for (int k = 0; k < pd.win; ++k) tc.lbit[pd.wq[k]] = pd.low + k;
    }
    for (int o = threadIdx.x; o < pd.nops && o < kOpsCached; o += nt) ops_sh[o] = pa.ops[pd.op_begin + o];
    for (uint32_t r = threadIdx.x; r < (1u << pd.win); r += nt) {
        uint64_t o = 0;
        for (int k = 0; k < pd.win; ++k) o |= (uint64_t)((r >> k) & 1u) << pd.wq[k];
        rowoff[r] = o;
    }
    // register scale factors at the start of this pass (float64 form)
    double scale[kRegs];
    for (int r = 0; r < kRegs; ++r) scale[r] = kScaled ? pa.regscale[(pd.parity & 1) * kRegs + r] : 1.0;
    double part[kMaxSlots];
    for (int k = 0; k < kMaxSlots; ++k) part[k] = 0.0;
    __syncthreads();
    const uint64_t ntiles = 1ull << (pd.n - pd.t);
    // free (non-tile) qubit positions above the low block, ascending
    for (uint64_t tile_id = blockIdx.x; tile_id < ntiles; tile_id += gridDim.x) {
        if (threadIdx.x == 0) {
            uint64_t b = 0, rem = tile_id;
            for (int q = pd.low; q < pd.n && rem; ++q) {
                if (tc.lbit[q] >= 0) continue;
                b |= (rem & 1ull) << q;
                rem >>= 1;
            }
            tc.base = b;
        }
        __syncthreads();
        // load: asynchronous 16-byte copies global -> shared (one complex128 amplitude, or two
        // adjacent complex64 ones of the same row), every copy of every register in flight before
        // one wait, so the pass has the memory parallelism to stream at HBM rate
        for (int r = 0; r < kRegs; ++r) {
            if (!(pd.regmask & (1 << r)) || !(pd.loadmask & (1 << r))) continue;
            const cx *src = reinterpret_cast<const cx *>(pa.reg[r]);
            for (uint32_t c = threadIdx.x; c < tc.T / kAmpsPer16; c += nt) {
                const uint32_t l = c * kAmpsPer16;
                cp_async16(tile[r] + l, src + gidx(tc, rowoff, l));
            }
        }
        asm volatile("cp.async.wait_all;\n" ::: "memory");
        __syncthreads();
        double sc[kRegs];
        for (int r = 0; r < kRegs; ++r) sc[r] = scale[r];
        for (int o = 0; o < pd.nops; ++o) {
            const PassOp op = o < kOpsCached ? ops_sh[o] : pa.ops[pd.op_begin + o];
            switch (op.kind) {
            case kOpCopy: {
                for (uint32_t l = threadIdx.x; l < tc.T; l += nt) tile[op.r1][l] = tile[op.r0][l];
                sc[op.r1] = sc[op.r0];
                break;
            }
            case kOpZero: {  // |0...0> into register r0 (scale 1)
                for (uint32_t l = threadIdx.x; l < tc.T; l += nt) {
                    cx z = {0, 0};
                    if (gidx(tc, rowoff, l) == 0) z.x = 1;
                    tile[op.r0][l] = z;
                }
                sc[op.r0] = 1.0;
                break;
            }
            case kOpRot: {  // y = c x + i s' sigma x on every register of op.regs (s' = +-s)
                const DevCoef co = pa.coef[op.param];
                const double sg = op.adjoint ? 1.0 : -1.0;
                const R c = (R)co.c, s = (R)(sg * co.s), t = (R)(sg * co.t);
                const int caseB = co.caseB;
                const double f = co.caseB ? sg * co.f : co.f;
                const int q = op.q0, ax = op.axis;
                for (int r = 0; r < kRegs; ++r) {
                    if (!(op.regs & (1 << r))) continue;
                    cx *X = tile[r];
                    if (ax == kAxisZ) {
                        const uint32_t T = tc.T;
                        const int lbz = tc.lbit[q];
                        const int bfix = lbz < 0 ? (int)((tc.base >> q) & 1ull) : 0;
                        for (uint32_t l = threadIdx.x; l < T; l += nt) {
                            const int beta = lbz >= 0 ? (int)((l >> lbz) & 1u) : bfix;
                            const cx x = X[l];
                            const cx v = {lflip(x.y, beta ^ 1), lflip(x.x, beta)};  // (i Z x)
                            cx y;
                            if (kScaled) {
                                if (caseB) { y.x = fma(t, x.x, v.x); y.y = fma(t, x.y, v.y); }
                                else       { y.x = fma(t, v.x, x.x); y.y = fma(t, v.y, x.y); }
                            } else {
                                y.x = fma(s, v.x, c * x.x); y.y = fma(s, v.y, c * x.y);
                            }
                            X[l] = y;
                        }
                    } else {
                        const int lb = tc.lbit[q];
                        const uint32_t bit = 1u << lb;
                        for (uint32_t p = threadIdx.x; p < (tc.T >> 1); p += nt) {
                            const uint32_t l0 = lins0(p, lb), l1 = l0 | bit;
                            const cx x0 = X[l0], x1 = X[l1];
                            cx v0, v1;
                            if (ax == kAxisX) { v0 = cx{-x1.y, x1.x}; v1 = cx{-x0.y, x0.x}; }
                            else              { v0 = x1; v1 = cx{-x0.x, -x0.y}; }
                            cx y0, y1;
                            if (kScaled) {
                                if (caseB) {
                                    y0.x = fma(t, x0.x, v0.x); y0.y = fma(t, x0.y, v0.y);
                                    y1.x = fma(t, x1.x, v1.x); y1.y = fma(t, x1.y, v1.y);
                                } else {
                                    y0.x = fma(t, v0.x, x0.x); y0.y = fma(t, v0.y, x0.y);
                                    y1.x = fma(t, v1.x, x1.x); y1.y = fma(t, v1.y, x1.y);
                                }
                            } else {
                                y0.x = fma(s, v0.x, c * x0.x); y0.y = fma(s, v0.y, c * x0.y);
                                y1.x = fma(s, v1.x, c * x1.x); y1.y = fma(s, v1.y, c * x1.y);
                            }
                            X[l0] = y0;
                            X[l1] = y1;
                        }
                    }
                    if (kScaled) sc[r] *= f;
                }
                break;
            }
            case kOpFixed: {  // a fixed gate on every register of op.regs (all fixed gates are self-adjoint)
                const int kind = op.fixed_kind;
                const R hs = kScaled ? (R)1 : (R)0.70710678118654752440;
                for (int r = 0; r < kRegs; ++r) {
                    if (!(op.regs & (1 << r))) continue;
                    cx *X = tile[r];
                    if (kind == QNG_GATE_CZ || kind == QNG_GATE_Z) {
                        for (uint32_t l = threadIdx.x; l < tc.T; l += nt) {
                            const int p = (kind == QNG_GATE_CZ) ? (gbit(tc, l, op.q0) & gbit(tc, l, op.q1)) : gbit(tc, l, op.q0);
                            if (p) X[l] = lflip2(X[l], 1);
                        }
                    } else {
                        const int qt = (kind == QNG_GATE_CNOT) ? op.q1 : op.q0;
                        const int lb = tc.lbit[qt];
                        const uint32_t bit = 1u << lb;
                        for (uint32_t p = threadIdx.x; p < (tc.T >> 1); p += nt) {
                            const uint32_t l0 = lins0(p, lb), l1 = l0 | bit;
                            const cx x0 = X[l0], x1 = X[l1];
                            cx y0, y1;
                            if (kind == QNG_GATE_CNOT) {
                                if (gbit(tc, l0, op.q0)) { y0 = x1; y1 = x0; } else { y0 = x0; y1 = x1; }
                            } else if (kind == QNG_GATE_X) {
                                y0 = x1; y1 = x0;
                            } else if (kind == QNG_GATE_Y) {
                                y0 = cx{x1.y, -x1.x}; y1 = cx{-x0.y, x0.x};
                            } else {  // H
                                y0 = cx{(x0.x + x1.x) * hs, (x0.y + x1.y) * hs};
                                y1 = cx{(x0.x - x1.x) * hs, (x0.y - x1.y) * hs};
                            }
                            X[l0] = y0;
                            X[l1] = y1;
                        }
                    }
                    if (kScaled && kind == QNG_GATE_H) sc[r] *= 0.70710678118654752440;
                }
                break;
            }
            case kOpSigma: {  // register r0 <- sigma_q register r0
                cx *X = tile[op.r0];
                const int q = op.q0, ax = op.axis;
                if (ax == kAxisZ) {
                    for (uint32_t l = threadIdx.x; l < tc.T; l += nt)
                        if (gbit(tc, l, q)) X[l] = lflip2(X[l], 1);
                } else {
                    const int lb = tc.lbit[q];
                    const uint32_t bit = 1u << lb;
                    for (uint32_t p = threadIdx.x; p < (tc.T >> 1); p += nt) {
                        const uint32_t l0 = lins0(p, lb), l1 = l0 | bit;
                        const cx x0 = X[l0], x1 = X[l1];
                        if (ax == kAxisX) { X[l0] = x1; X[l1] = x0; }
                        else { X[l0] = cx{x1.y, -x1.x}; X[l1] = cx{-x0.y, x0.x}; }  // -i x1, i x0
                    }
                }
                break;
            }
            case kOpIp: {  // part[slot] += Re/Im <r0| sigma_q |r1>  (axis -1: no sigma)
                const cx *A = tile[op.r0], *B = tile[op.r1];
                const int q = op.q0, ax = op.axis, im = op.adjoint;
                R acc = 0;
                if (ax < 0 || ax == kAxisZ) {
                    const uint32_t T = tc.T;
                    const int lbz = ax == kAxisZ ? tc.lbit[q] : -1;
                    const int bfix = (ax == kAxisZ && lbz < 0) ? (int)((tc.base >> q) & 1ull) : 0;
                    for (uint32_t l = threadIdx.x; l < T; l += nt) {
                        const int beta = lbz >= 0 ? (int)((l >> lbz) & 1u) : bfix;
                        const cx a = (ax == kAxisZ) ? lflip2(A[l], beta) : A[l];
                        const cx b = B[l];
                        acc = im ? fma(a.x, b.y, fma(-a.y, b.x, acc)) : fma(a.x, b.x, fma(a.y, b.y, acc));
                    }
                } else {
                    const int lb = tc.lbit[q];
                    const uint32_t bit = 1u << lb;
                    for (uint32_t p = threadIdx.x; p < (tc.T >> 1); p += nt) {
                        const uint32_t l0 = lins0(p, lb), l1 = l0 | bit;
                        const cx a0 = A[l0], a1 = A[l1], b0 = B[l0], b1 = B[l1];
                        cx s0, s1;  // (sigma b)_0, (sigma b)_1
                        if (ax == kAxisX) { s0 = b1; s1 = b0; }
                        else { s0 = cx{b1.y, -b1.x}; s1 = cx{-b0.y, b0.x}; }
                        if (im) acc = fma(a0.x, s0.y, fma(-a0.y, s0.x, fma(a1.x, s1.y, fma(-a1.y, s1.x, acc))));
                        else acc = fma(a0.x, s0.x, fma(a0.y, s0.y, fma(a1.x, s1.x, fma(a1.y, s1.y, acc))));
                    }
                }
                part[op.slot] += (double)acc;  // float64 from here on; reduced once per launch
                if (blockIdx.x == 0 && threadIdx.x == 0 && tile_id == 0) pa.slotfac[pd.slot_base + op.slot] = sc[op.r0] * sc[op.r1];
                break;
            }
            case kOpStep: {
                const bool rot = op.param >= 0;
                R c = 0, sv = 0, tv = 0;
                int caseB = 0;
                double f = 1.0;
                if (rot) {
                    const DevCoef co = pa.coef[op.param];  // adjoint rotation: s' = +s
                    c = (R)co.c; sv = (R)co.s; tv = (R)co.t; caseB = co.caseB; f = co.f;
                }
                if (MIM && op.adjoint == 2) {
                    const Acc2<R> acc = step_dispatch<R, 2>(tc, tile[op.r0], tile[op.r1], op.axis, op.q0, rot, c, sv, tv, caseB);
                    part[op.slot] += (double)acc.re;
                    part[op.slot + 1] += (double)acc.im;
                    if (blockIdx.x == 0 && threadIdx.x == 0 && tile_id == 0)
                        pa.slotfac[pd.slot_base + op.slot] = pa.slotfac[pd.slot_base + op.slot + 1] = sc[op.r0] * sc[op.r1];
                } else {
                    const Acc2<R> acc = op.adjoint
                        ? step_dispatch<R, 1>(tc, tile[op.r0], tile[op.r1], op.axis, op.q0, rot, c, sv, tv, caseB)
                        : step_dispatch<R, 0>(tc, tile[op.r0], tile[op.r1], op.axis, op.q0, rot, c, sv, tv, caseB);
                    part[op.slot] += (double)(op.adjoint ? acc.im : acc.re);
                    if (blockIdx.x == 0 && threadIdx.x == 0 && tile_id == 0)
                        pa.slotfac[pd.slot_base + op.slot] = sc[op.r0] * sc[op.r1];
                }
                if (kScaled && rot) { sc[op.r0] *= f; sc[op.r1] *= f; }
                break;
            }
            case kOpStep2: {
                const bool rot = op.param >= 0;
                R c = 0, sv = 0, tv = 0;
                int caseB = 0;
                double f = 1.0;
                if (rot) {
                    const DevCoef co = pa.coef[op.param];  // adjoint rotation: s' = +s
                    c = (R)co.c; sv = (R)co.s; tv = (R)co.t; caseB = co.caseB; f = co.f;
                }
                Acc2<R> ab = {0, 0}, ac = {0, 0};
                const bool both = MIM && op.adjoint == 2;
                if (both) step2_dispatch<R, 2>(tc, tile[kRegA], tile[kRegB], tile[kRegB2], op.axis, op.q0, rot, c, sv, tv, caseB, ab, ac);
                else step2_dispatch<R, 0>(tc, tile[kRegA], tile[kRegB], tile[kRegB2], op.axis, op.q0, rot, c, sv, tv, caseB, ab, ac);
                const double fb = sc[kRegA] * sc[kRegB], fc = sc[kRegA] * sc[kRegB2];
                const bool rec = blockIdx.x == 0 && threadIdx.x == 0 && tile_id == 0;
                if (both) {
                    part[op.slot] += (double)ab.re;
                    part[op.slot + 1] += (double)ab.im;
                    part[op.slot + 2] += (double)ac.re;
                    part[op.slot + 3] += (double)ac.im;
                    if (rec) {
                        pa.slotfac[pd.slot_base + op.slot] = pa.slotfac[pd.slot_base + op.slot + 1] = fb;
                        pa.slotfac[pd.slot_base + op.slot + 2] = pa.slotfac[pd.slot_base + op.slot + 3] = fc;
                    }
                } else {
                    part[op.slot] += (double)ab.re;
                    part[op.slot + 1] += (double)ac.re;
                    if (rec) {
                        pa.slotfac[pd.slot_base + op.slot] = fb;
                        pa.slotfac[pd.slot_base + op.slot + 1] = fc;
                    }
                }
                if (kScaled && rot) { sc[kRegA] *= f; sc[kRegB] *= f; sc[kRegB2] *= f; }
                break;
            }
            case kOpRecordFac: {
                if (blockIdx.x == 0 && threadIdx.x == 0 && tile_id == 0) pa.slotfac[pd.slot_base + op.slot] = sc[op.r0] * sc[op.r1];
                break;
            }
            case kOpSetScale: {
                sc[op.r1] = sc[op.r0];
                break;
            }
            default:
                break;
            }
            __syncthreads();
            // keep float64 scale factors far from underflow (exact power-of-two rescaling)
            if (kScaled) {
                for (int r = 0; r < kRegs; ++r) {
                    if (!(pd.regmask & (1 << r))) continue;
                    const int ex = (int)((__double_as_longlong(sc[r]) >> 52) & 0x7ff);
                    if (ex < 1023 - 200) {
                        for (uint32_t l = threadIdx.x; l < tc.T; l += nt) {
                            cx x = tile[r][l];
                            if constexpr (kScaled) { x.x *= 0x1p-200; x.y *= 0x1p-200; }
                            tile[r][l] = x;
                        }
                        sc[r] *= 0x1p200;
                        __syncthreads();
                    }
                }
            }
        }
        // store: 16-byte vector stores (a row of 2^low amplitudes is contiguous)
        for (int r = 0; r < kRegs; ++r) {
            if (!(pd.regmask & (1 << r)) || !(pd.storemask & (1 << r))) continue;
            cx *dst = reinterpret_cast<cx *>(pa.reg[r]);
            for (uint32_t c = threadIdx.x; c < tc.T / kAmpsPer16; c += nt) {
                const uint32_t l = c * kAmpsPer16;
                *reinterpret_cast<float4 *>(dst + gidx(tc, rowoff, l)) = *reinterpret_cast<const float4 *>(tile[r] + l);
            }
        }
        if (tile_id + gridDim.x >= ntiles && blockIdx.x == 0 && threadIdx.x == 0 && kScaled)
            for (int r = 0; r < kRegs; ++r) pa.regscale[((pd.parity + 1) & 1) * kRegs + r] = sc[r];
        __syncthreads();
    }
    // per-CTA partial sums: warp, then CTA, in a fixed order
    for (int k = 0; k < pd.nslots; ++k) {
        const double v = lwarp_sum(part[k]);
        if (lane == 0) red[wid] = v;
        __syncthreads();
        if (threadIdx.x == 0) {
            double tot = 0.0;
            for (int w = 0; w < nw; ++w) tot += red[w];
            pa.partial[(size_t)(pd.slot_base + k) * gridDim.x + blockIdx.x] = tot;
        }
        __syncthreads();
    }
}

// out[m] = sum_t c_t i^{ny} (-1)^{popcount((m ^ x) & z)} in[m ^ x]; partial <in|out> per CTA.
template <typename R>
__global__ void __launch_bounds__(256) k_hpsi(const void *in_, void *out_, const DevTerm *terms, int nterms, int n,
                                              double *partial) {
    using cx = typename CX2<R>::T;
    const cx *in = reinterpret_cast<const cx *>(in_);
    cx *out = reinterpret_cast<cx *>(out_);
    __shared__ double red[32];
    const uint64_t N = 1ull << n;
    double e = 0.0;
    for (uint64_t m = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; m < N; m += (uint64_t)gridDim.x * blockDim.x) {
        // each element in the amplitudes' own precision (complex64: float32, the precision it is
        // stored in); the inner product <in|out> below in float64. Terms come grouped by X mask,
        // so psi[m ^ x] is gathered once per distinct mask.
        R hr = 0, hi = 0;
        uint64_t xl = ~0ull;
        R vr = 0, vi = 0;
        for (int t = 0; t < nterms; ++t) {
            const DevTerm tm = terms[t];
            const uint64_t src = m ^ tm.x;
            if (tm.x != xl) {
                const cx v = in[src];
                vr = v.x;
                vi = v.y;
                xl = tm.x;
            }
            const int ph = (tm.ny + 2 * (__popcll(src & tm.z) & 1)) & 3;
            const R cf = (R)tm.coeff;
            if (ph == 0)      { hr = fma(cf, vr, hr);  hi = fma(cf, vi, hi); }
            else if (ph == 1) { hr = fma(-cf, vi, hr); hi = fma(cf, vr, hi); }
            else if (ph == 2) { hr = fma(-cf, vr, hr); hi = fma(-cf, vi, hi); }
            else              { hr = fma(cf, vi, hr);  hi = fma(-cf, vr, hi); }
        }
        const cx x = in[m];
        e += (double)x.x * (double)hr + (double)x.y * (double)hi;
        out[m] = cx{hr, hi};
    }
    e = lwarp_sum(e);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = e;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += red[w];
        partial[blockIdx.x] = tot;
    }
}

// Sum partial[slot][0..nctas) in a fixed order and scatter: dst[k] = mul * slotfac[slot] * sum.
__global__ void k_reduce(const double *partial, const double *slotfac, int nctas, const ReduceItem *items, int nitems,
                         int use_fac) {
    const int k = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (k >= nitems) return;
    const ReduceItem it = items[k];
    double v = 0.0;
    for (int c = lane; c < nctas; c += 32) v += partial[(size_t)it.slot * nctas + c];
    v = lwarp_sum(v);
    if (lane == 0) *it.dst = it.mul * (use_fac ? slotfac[it.slot] : 1.0) * v;
}

// ------------------------------------------------------------------------------------------
cudaError_t prepare_pass(int precision, size_t smem) {
    cudaError_t e;
    if (precision == QNG_C128) {
        if ((e = raise_smem_limit(reinterpret_cast<const void *>(k_pass<double, 0>), smem)) != cudaSuccess) return e;
        return raise_smem_limit(reinterpret_cast<const void *>(k_pass<double, 1>), smem);
    }
    if ((e = raise_smem_limit(reinterpret_cast<const void *>(k_pass<float, 0>), smem)) != cudaSuccess) return e;
    return raise_smem_limit(reinterpret_cast<const void *>(k_pass<float, 1>), smem);
}

cudaError_t launch_pass(const PassArgs &pa, int precision, int grid, int threads, size_t smem, int metric_im,
                        cudaStream_t st) {
    if (precision == QNG_C128) {
        if (metric_im) k_pass<double, 1><<<grid, threads, smem, st>>>(pa);
        else k_pass<double, 0><<<grid, threads, smem, st>>>(pa);
    } else {
        if (metric_im) k_pass<float, 1><<<grid, threads, smem, st>>>(pa);
        else k_pass<float, 0><<<grid, threads, smem, st>>>(pa);
    }
    return cudaGetLastError();
}

cudaError_t launch_hpsi(const void *in, void *out, const DevTerm *terms, int nterms, int n, int precision,
                        double *partial, int grid, cudaStream_t st) {
    if (precision == QNG_C128) k_hpsi<double><<<grid, 256, 0, st>>>(in, out, terms, nterms, n, partial);
    else k_hpsi<float><<<grid, 256, 0, st>>>(in, out, terms, nterms, n, partial);
    return cudaGetLastError();
}

cudaError_t launch_reduce(const double *partial, const double *slotfac, int nctas, const ReduceItem *items, int nitems,
                          int use_fac, cudaStream_t st) {
    if (nitems <= 0) return cudaSuccess;
    const int per = 8;  // warps per block
    k_reduce<<<(nitems + per - 1) / per, per * 32, 0, st>>>(partial, slotfac, nctas, items, nitems, use_fac);
    return cudaGetLastError();
}

}  // namespace large
}  // namespace qng

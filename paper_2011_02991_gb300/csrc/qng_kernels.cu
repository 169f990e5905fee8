// sm_103a kernels of the on-chip path: every state vector of an instance lives in the shared
// memory of one thread-block cluster (2^cl CTAs, each holding 2^(n-cl) amplitudes), so the
// O(P^2) recurrence of Algorithm 1 runs without touching HBM except to read checkpoints.
//
//   k_coef     per-parameter cos/sin of theta/2 and the scaled rotation form
//   k_forward  psi_k = U_k ... U_1 |0> for every k (checkpoints), W psi, H W psi, <E>, and the
//              adjoint seed eta = W^dag H W psi (Sec. 2: psi_i and T_i; Eq. 2 for <E>)
//   k_columns  one cluster per column j of L: phi walks down from dU_j psi_{j-1} by one adjoint
//              gate per element, L_ij = prod[dU_i psi_{i-1}, phi_{i+1,j}] (Eq. L_recurrent_def,
//              the inner loop of Algorithm 1); the extra column P walks eta down the same way
//              and yields d<E>/d theta_i (reverse sweep)
//   k_finish   G_ij = L_ij - T_i^* T_j (Eq. g_t_L_def), g = Re G, and the float64 Cholesky solve
//              of (g + lambda I) dtheta = -dt grad<E> (Eq. 3)
//
// Notation used throughout (0-based parameters k = 0..P-1):
//   Psi[k]    the state after U_{k-1} (Psi[0] = |0>), stored as a checkpoint;
//   R_k^dag = c + i s sigma_k, R_k = c - i s sigma_k, with c = cos(theta_k/2), s = sin(theta_k/2);
//   dU_k Psi[k] = (-i/2) sigma_k Psi[k+1], hence L_ij = (1/4) <Psi[i+1]| sigma_i |b_ij> with
//   b_ij = U_{i+1}^dag ... U_j^dag sigma_j Psi[j+1], and T_k = -(i/2) <Psi[k+1]|sigma_k|Psi[k+1]>.
// Complex128 amplitudes are kept as (scalar factor) x (vector): a rotation becomes one FMA per
// real component (see DevCoef), halving the float64 work on a part whose float64 rate is 1/64 of
// its float32 rate; the factors are applied to each inner product.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "qng_internal.h"

namespace cg = cooperative_groups;

namespace qng {

template <typename R> struct CX;
template <> struct CX<double> { using T = double2; };
template <> struct CX<float> { using T = float2; };

__device__ __forceinline__ uint32_t ins0(uint32_t p, int q) {
    return ((p >> q) << (q + 1)) | (p & ((1u << q) - 1u));
}

// (-1)^parity of an all-diagonal fixed block F (CZ and Z gates) at basis index k
__device__ __forceinline__ int diag_parity(uint64_t k, const DevParam &pd, const DevDiag *dt) {
    int par = __popcll(k & pd.zmask);
    for (int e = 0; e < pd.diag_count; ++e) {
        const DevDiag d = dt[pd.diag_begin + e];
        par += __popcll(k & (k >> d.shift) & d.mask);
    }
    return par & 1;
}

template <typename T2> __device__ __forceinline__ T2 neg_if(T2 v, int p) {
    if (p) { v.x = -v.x; v.y = -v.y; }
    return v;
}

// (i sigma x)_beta for the pair component with bit value beta, own value xm, partner value xo
template <typename T2> __device__ __forceinline__ T2 i_sigma(int axis, int beta, T2 xm, T2 xo) {
    T2 v;
    if (axis == kAxisX) {          // i x_other
        v.x = -xo.y; v.y = xo.x;
    } else if (axis == kAxisY) {   // beta=0: i(-i x1) = x1 ; beta=1: i(i x0) = -x0
        if (beta) { v.x = -xo.x; v.y = -xo.y; } else { v = xo; }
    } else {                       // beta=0: i x0 ; beta=1: -i x1
        if (beta) { v.x = xm.y; v.y = -xm.x; } else { v.x = -xm.y; v.y = xm.x; }
    }
    return v;
}

// (sigma x)_beta
template <typename T2> __device__ __forceinline__ T2 sigma_of(int axis, int beta, T2 xm, T2 xo) {
    T2 v;
    if (axis == kAxisX) {
        v = xo;
    } else if (axis == kAxisY) {   // beta=0: -i x1 ; beta=1: i x0
        if (beta) { v.x = -xo.y; v.y = xo.x; } else { v.x = xo.y; v.y = -xo.x; }
    } else {
        v = beta ? T2{-xm.x, -xm.y} : xm;
    }
    return v;
}

// Rotation y = c x + i s' sigma x in one of three forms (see DevCoef).
template <typename R> struct Rot {
    R c, s, t;
    int caseB;
    __device__ __forceinline__ typename CX<R>::T apply(typename CX<R>::T x, typename CX<R>::T v) const {
        typename CX<R>::T y;
        if (std::is_same<R, double>::value) {
            if (caseB) { y.x = fma(t, x.x, v.x); y.y = fma(t, x.y, v.y); }
            else       { y.x = fma(t, v.x, x.x); y.y = fma(t, v.y, x.y); }
        } else {
            y.x = fma(s, v.x, c * x.x); y.y = fma(s, v.y, c * x.y);
        }
        return y;
    }
};

// The same rotation with its scaled form fixed at compile time (no per-amplitude branch).
template <typename R, int CB> struct RotC {
    R c, s, t;
    __device__ __forceinline__ typename CX<R>::T apply(typename CX<R>::T x, typename CX<R>::T v) const {
        typename CX<R>::T y;
        if constexpr (std::is_same<R, double>::value) {
            if constexpr (CB) { y.x = fma(t, x.x, v.x); y.y = fma(t, x.y, v.y); }
            else              { y.x = fma(t, v.x, x.x); y.y = fma(t, v.y, x.y); }
        } else {
            y.x = fma(s, v.x, c * x.x); y.y = fma(s, v.y, c * x.y);
        }
        return y;
    }
};

// adjoint (R^dag) or forward (R) coefficients of parameter k; f receives the scale factor
template <typename R> __device__ __forceinline__ Rot<R> make_rot(const DevCoef &co, bool adjoint, double &f) {
    Rot<R> r;
    if constexpr (std::is_same<R, float>::value) {  // the float32 copies: no float64 work per step
        const float sg = adjoint ? 1.0f : -1.0f;
        r.c = co.cf;
        r.s = sg * co.sf;
        r.t = sg * co.tf;
        r.caseB = co.caseB;
        f = 1.0;  // complex64 registers carry no float64 factor
    } else {
        const double sg = adjoint ? 1.0 : -1.0;
        r.c = (R)co.c;
        r.s = (R)(sg * co.s);
        r.t = (R)(sg * co.t);
        r.caseB = co.caseB;
        f = co.caseB ? sg * co.f : co.f;
    }
    return r;
}

template <typename RA> __device__ __forceinline__ RA warp_sum(RA v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Warp sums of 8 values at once: a[k] of every lane is summed over the warp; the lane returns the
// sum of a[(lane >> 2) & 7]. 9 additions and 18 shuffles for 8 sums instead of 40 and 80.
template <typename RA> __device__ __forceinline__ RA warp_sum8(const RA (&a)[8], int lane) {
    const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4;
    RA t[4], u[2];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const RA mine = b4 ? a[4 + k] : a[k], other = b4 ? a[k] : a[4 + k];
        t[k] = mine + __shfl_xor_sync(0xffffffffu, other, 16);
    }
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const RA mine = b3 ? t[2 + k] : t[k], other = b3 ? t[k] : t[2 + k];
        u[k] = mine + __shfl_xor_sync(0xffffffffu, other, 8);
    }
    RA v = (b2 ? u[1] : u[0]) + __shfl_xor_sync(0xffffffffu, b2 ? u[0] : u[1], 4);
    v += __shfl_xor_sync(0xffffffffu, v, 2);
    v += __shfl_xor_sync(0xffffffffu, v, 1);
    return v;
}

// ------------------------------------------------------------------------------------------
// Cluster-resident state: CTA `rank` holds amplitudes [rank * Nl, (rank + 1) * Nl) in buf.
// Qubits >= nl are distributed; a pair on such a qubit has its halves in two CTAs at the same
// local index. A distributed op pushes the CTA's half into the partner's receive buffer (two
// buffers used alternately), then one cluster barrier, then each CTA writes its own half.
// Every CTA of a cluster runs the same op sequence, so the barriers match.
template <typename R> struct Eng {
    using cx = typename CX<R>::T;
    cx *buf, *rv0, *rv1;
    int n, nl, cl, rank, phase;
    uint32_t Nl;
    uint64_t base;  // global index of buf[0]

    __device__ void csync() const {
        if (cl) cg::this_cluster().sync(); else __syncthreads();
    }

    // push my slice to the partner across distributed qubit q; returns my receive buffer
    __device__ cx *exchange(int q) { return exchange_rank(rank ^ (1 << (q - nl))); }

    // push my slice to CTA `partner` of the cluster (which pushes its own to me); returns my
    // receive buffer holding the partner's slice
    __device__ cx *exchange_rank(int partner) {
        cx *mine = phase ? rv1 : rv0;
        cx *remote = cg::this_cluster().map_shared_rank(mine, partner);
        for (uint32_t l = threadIdx.x; l < Nl; l += blockDim.x) remote[l] = buf[l];
        cg::this_cluster().sync();
        phase ^= 1;
        return mine;
    }

    // one fixed gate (all are self-adjoint); scale absorbs the 1/sqrt2 of H in float64
    __device__ void fixed_gate(const DevFixed g, double &scale) {
        const int kind = g.kind;
        if (kind == QNG_GATE_CZ || kind == QNG_GATE_Z) {
            const uint64_t m = (kind == QNG_GATE_CZ) ? ((1ull << g.q0) | (1ull << g.q1)) : (1ull << g.q0);
            for (uint32_t l = threadIdx.x; l < Nl; l += blockDim.x) {
                const uint64_t k = base | l;
                if ((k & m) == m) { cx x = buf[l]; x.x = -x.x; x.y = -x.y; buf[l] = x; }
            }
            __syncthreads();
            return;
        }
        const int q = (kind == QNG_GATE_CNOT) ? g.q1 : g.q0;
        const uint64_t cm = (kind == QNG_GATE_CNOT) ? (1ull << g.q0) : 0ull;
        const bool kScaled = std::is_same<R, double>::value;
        const R hs = kScaled ? (R)1 : (R)0.70710678118654752440;
        if (q < nl) {
            const uint32_t bit = 1u << q, half = Nl >> 1;
            for (uint32_t p = threadIdx.x; p < half; p += blockDim.x) {
                const uint32_t l0 = ins0(p, q), l1 = l0 | bit;
                cx x0 = buf[l0], x1 = buf[l1], y0, y1;
                if (kind == QNG_GATE_CNOT) {
                    if ((base | l0) & cm) { y0 = x1; y1 = x0; } else { y0 = x0; y1 = x1; }
                } else if (kind == QNG_GATE_X) {
                    y0 = x1; y1 = x0;
                } else if (kind == QNG_GATE_Y) {
                    y0.x = x1.y; y0.y = -x1.x; y1.x = -x0.y; y1.y = x0.x;
                } else {  // H
                    y0.x = (x0.x + x1.x) * hs; y0.y = (x0.y + x1.y) * hs;
                    y1.x = (x0.x - x1.x) * hs; y1.y = (x0.y - x1.y) * hs;
                }
                buf[l0] = y0; buf[l1] = y1;
            }
            __syncthreads();
        } else {
            const cx *rv = exchange(q);
            const int beta = (rank >> (q - nl)) & 1;
            for (uint32_t l = threadIdx.x; l < Nl; l += blockDim.x) {
                const cx xm = buf[l], xo = rv[l];
                cx y;
                if (kind == QNG_GATE_CNOT) {
                    y = ((base | l) & cm) ? xo : xm;
                } else if (kind == QNG_GATE_X) {
                    y = xo;
                } else if (kind == QNG_GATE_Y) {
                    y = beta ? cx{-xo.y, xo.x} : cx{xo.y, -xo.x};
                } else {  // H: y0 = x0 + x1, y1 = x0 - x1
                    y = beta ? cx{(xo.x - xm.x) * hs, (xo.y - xm.y) * hs} : cx{(xm.x + xo.x) * hs, (xm.y + xo.y) * hs};
                }
                buf[l] = y;
            }
            __syncthreads();
        }
        if (kind == QNG_GATE_H && kScaled) scale *= 0.70710678118654752440;
    }

    // fixed gates gs[0..count) in circuit order (reverse = true: their adjoint, last gate first);
    // consecutive diagonal ones (CZ, Z) commute and go through one sign pass with one barrier
    __device__ void fixed_gates(const DevFixed *gs, int count, double &scale, bool reverse) {
        for (int f = 0; f < count;) {
            const DevFixed g = gs[reverse ? count - 1 - f : f];
            if (g.kind != QNG_GATE_CZ && g.kind != QNG_GATE_Z) {
                fixed_gate(g, scale);
                ++f;
                continue;
            }
            int r = f + 1;
            while (r < count) {
                const int kd = gs[reverse ? count - 1 - r : r].kind;
                if (kd != QNG_GATE_CZ && kd != QNG_GATE_Z) break;
                ++r;
            }
            if (r - f == 1) {
                fixed_gate(g, scale);
                ++f;
                continue;
            }
            for (uint32_t l = threadIdx.x; l < Nl; l += blockDim.x) {
                const uint64_t k = base | l;
                int par = 0;
                for (int u = f; u < r; ++u) {
                    const DevFixed d = gs[reverse ? count - 1 - u : u];
                    const uint64_t m = (d.kind == QNG_GATE_CZ) ? ((1ull << d.q0) | (1ull << d.q1)) : (1ull << d.q0);
                    par += (k & m) == m;
                }
                if (par & 1) { cx x = buf[l]; x.x = -x.x; x.y = -x.y; buf[l] = x; }
            }
            __syncthreads();
            f = r;
        }
    }

    // keep the float64 scale factor far from underflow: fold 2^-200 into the vector (exact)
    __device__ void maybe_renorm(double &scale) {
        if constexpr (std::is_same<R, double>::value) {
            const double lim = 0x1p-200;
            const int ex = (int)((__double_as_longlong(scale) >> 52) & 0x7ff);  // integer test, no float64 op
            if (ex < 1023 - 200) {
                for (uint32_t l = threadIdx.x; l < Nl; l += blockDim.x) {
                    cx x = buf[l];
                    x.x *= lim; x.y *= lim;
                    buf[l] = x;
                }
                scale *= 0x1p200;
                __syncthreads();
            }
        }
    }
};

template <typename R> __device__ __forceinline__ Eng<R> make_eng(unsigned char *smem, int n, int cl) {
    Eng<R> e;
    using cx = typename CX<R>::T;
    e.n = n;
    e.cl = cl;
    e.nl = n - cl;
    e.Nl = 1u << e.nl;
    e.rank = cl ? (int)cg::this_cluster().block_rank() : 0;
    e.base = (uint64_t)e.rank << e.nl;
    e.buf = reinterpret_cast<cx *>(smem);
    e.rv0 = e.buf + e.Nl;
    e.rv1 = e.rv0 + e.Nl;
    e.phase = 0;
    // distributed shared memory may only be touched once every CTA of the cluster is running
    if (cl) cg::this_cluster().sync();
    return e;
}

// Sum a per-thread double over the CTA, then over the cluster; the result lands in rank 0's
// thread 0. red must hold blockDim/32 doubles of shared memory.
__device__ double cluster_sum(double v, double *red, int cl) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    v = warp_sum(v);
    if (lane == 0) red[wid] = v;
    __syncthreads();
    if (cl) cg::this_cluster().sync();
    double tot = 0.0;
    if (threadIdx.x == 0 && (!cl || cg::this_cluster().block_rank() == 0)) {
        const int C = 1 << cl;
        for (int r = 0; r < C; ++r) {
            const double *rr = cl ? cg::this_cluster().map_shared_rank(red, r) : red;
            for (int w = 0; w < nw; ++w) tot += rr[w];
        }
    }
    if (cl) cg::this_cluster().sync();
    return tot;
}


// ------------------------------------------------------------------------------------------
// Compile-time Pauli axis and bit value: every sign below folds into an FMA operand or is a
// sign-bit flip on the integer pipe, so a pair costs only its essential float64 FMAs.
__device__ __forceinline__ double flip(double v, int p) {
    return __longlong_as_double(__double_as_longlong(v) ^ ((long long)(p & 1) << 63));
}
__device__ __forceinline__ float flip(float v, int p) { return __int_as_float(__float_as_int(v) ^ ((p & 1) << 31)); }
template <typename T2> __device__ __forceinline__ T2 flip2(T2 v, int p) {
    v.x = flip(v.x, p);
    v.y = flip(v.y, p);
    return v;
}

// (i sigma x)_BETA and (sigma x)_BETA from own value xm and partner value xo
template <int AX, int BETA, typename T2> __device__ __forceinline__ T2 isig(T2 xm, T2 xo) {
    if constexpr (AX == kAxisX) return T2{-xo.y, xo.x};
    else if constexpr (AX == kAxisY) return BETA ? T2{-xo.x, -xo.y} : xo;
    else return BETA ? T2{xm.y, -xm.x} : T2{-xm.y, xm.x};
}
template <int AX, int BETA, typename T2> __device__ __forceinline__ T2 sig(T2 xm, T2 xo) {
    if constexpr (AX == kAxisX) return xo;
    else if constexpr (AX == kAxisY) return BETA ? T2{-xo.y, xo.x} : T2{xo.y, -xo.x};
    else return BETA ? T2{-xm.x, -xm.y} : xm;
}
// Partial inner products of one step: re = Re<a|s>, im = Im<a|s> (only the parts IM asks for).
template <typename RA> struct RI {
    RA re, im;
};
// IM = 0: Re(conj(a) s); IM = 1: Im(conj(a) s); IM = 2: both
template <int IM, typename RA, typename T2> __device__ __forceinline__ void ipacc(RI<RA> &part, T2 a, T2 s) {
    if constexpr (IM != 1) part.re = fma(a.x, s.x, fma(a.y, s.y, part.re));
    if constexpr (IM != 0) part.im = fma(a.x, s.y, fma(-a.y, s.x, part.im));
}

// One fused step of a column on a local X/Y qubit: inner product with sigma on the pairs,
// then the adjoint rotation R^dag on the same pairs, then the diagonal fixed block F^dag.
template <typename R, int AX, int IM, int CB>
__device__ __forceinline__ RI<R> col_pairs(Eng<R> &e, const typename CX<R>::T *a, int q, bool rot_on,
                                           const RotC<R, CB> &rot, bool post, const DevParam &pi, const DevDiag *dt) {
    using cx = typename CX<R>::T;
    RI<R> part = {0, 0};
    const uint32_t bit = 1u << q, half = e.Nl >> 1;
    for (uint32_t p = threadIdx.x; p < half; p += blockDim.x) {
        const uint32_t l0 = ins0(p, q), l1 = l0 | bit;
        const cx x0 = e.buf[l0], x1 = e.buf[l1];
        const cx a0 = a[e.base | l0], a1 = a[e.base | l1];
        ipacc<IM>(part, a0, sig<AX, 0>(x0, x1));
        ipacc<IM>(part, a1, sig<AX, 1>(x1, x0));
        if (rot_on) {
            cx y0 = rot.apply(x0, isig<AX, 0>(x0, x1));
            cx y1 = rot.apply(x1, isig<AX, 1>(x1, x0));
            if (post) {
                y0 = flip2(y0, diag_parity(e.base | l0, pi, dt));
                y1 = flip2(y1, diag_parity(e.base | l1, pi, dt));
            }
            e.buf[l0] = y0;
            e.buf[l1] = y1;
        }
    }
    return part;
}

// The same step on a distributed X/Y qubit, this CTA holding the BETA half of every pair.
template <typename R, int AX, int IM, int BETA, int CB>
__device__ __forceinline__ RI<R> col_dist(Eng<R> &e, const typename CX<R>::T *rv, const typename CX<R>::T *a,
                                          bool rot_on, const RotC<R, CB> &rot, bool post, const DevParam &pi,
                                          const DevDiag *dt) {
    using cx = typename CX<R>::T;
    RI<R> part = {0, 0};
    for (uint32_t l = threadIdx.x; l < e.Nl; l += blockDim.x) {
        const uint64_t kk = e.base | l;
        const cx xm = e.buf[l], xo = rv[l];
        ipacc<IM>(part, a[kk], sig<AX, BETA>(xm, xo));
        if (rot_on) {
            cx y = rot.apply(xm, isig<AX, BETA>(xm, xo));
            if (post) y = flip2(y, diag_parity(kk, pi, dt));
            e.buf[l] = y;
        }
    }
    return part;
}

// The same step for a Z rotation (diagonal: any qubit, no pairing).
template <typename R, int IM, int CB>
__device__ __forceinline__ RI<R> col_diag(Eng<R> &e, const typename CX<R>::T *a, int q, bool rot_on,
                                          const RotC<R, CB> &rot, bool post, const DevParam &pi, const DevDiag *dt) {
    using cx = typename CX<R>::T;
    RI<R> part = {0, 0};
    for (uint32_t l = threadIdx.x; l < e.Nl; l += blockDim.x) {
        const uint64_t kk = e.base | l;
        const int beta = (int)((kk >> q) & 1);
        const cx x = e.buf[l];
        ipacc<IM>(part, flip2(a[kk], beta), x);  // (Z x)_beta = (-1)^beta x
        if (rot_on) {
            const cx v = {flip(x.y, beta ^ 1), flip(x.x, beta)};  // (i Z x)_beta
            cx y = rot.apply(x, v);
            if (post) y = flip2(y, diag_parity(kk, pi, dt));
            e.buf[l] = y;
        }
    }
    return part;
}

template <typename R, int IM, int CB>
__device__ __forceinline__ RI<R> col_step_cb(Eng<R> &e, const typename CX<R>::T *a, const DevParam &pi, bool rot_on,
                                             const RotC<R, CB> &rot, bool post, const DevDiag *dt) {
    RI<R> part;
    if (pi.axis == kAxisZ) {
        part = col_diag<R, IM, CB>(e, a, pi.q, rot_on, rot, post, pi, dt);
    } else if (pi.q < e.nl) {
        part = (pi.axis == kAxisX) ? col_pairs<R, kAxisX, IM, CB>(e, a, pi.q, rot_on, rot, post, pi, dt)
                                   : col_pairs<R, kAxisY, IM, CB>(e, a, pi.q, rot_on, rot, post, pi, dt);
    } else {
        const typename CX<R>::T *rv = e.exchange(pi.q);
        const int beta = (e.rank >> (pi.q - e.nl)) & 1;
        if (pi.axis == kAxisX)
            part = beta ? col_dist<R, kAxisX, IM, 1, CB>(e, rv, a, rot_on, rot, post, pi, dt)
                        : col_dist<R, kAxisX, IM, 0, CB>(e, rv, a, rot_on, rot, post, pi, dt);
        else
            part = beta ? col_dist<R, kAxisY, IM, 1, CB>(e, rv, a, rot_on, rot, post, pi, dt)
                        : col_dist<R, kAxisY, IM, 0, CB>(e, rv, a, rot_on, rot, post, pi, dt);
    }
    __syncthreads();
    return part;
}

template <typename R, int IM>
__device__ __forceinline__ RI<R> col_step(Eng<R> &e, const typename CX<R>::T *a, const DevParam &pi, bool rot_on,
                                          const Rot<R> &rot, bool post, const DevDiag *dt) {
    if (std::is_same<R, double>::value && rot.caseB)
        return col_step_cb<R, IM, 1>(e, a, pi, rot_on, RotC<R, 1>{rot.c, rot.s, rot.t}, post, dt);
    return col_step_cb<R, IM, 0>(e, a, pi, rot_on, RotC<R, 0>{rot.c, rot.s, rot.t}, post, dt);
}

// ------------------------------------------------------------------------------------------
// Generalised rotations (Sec. 2: one Pauli string, optionally controlled): generator K = C (x) S,
// R(theta) = exp(-i theta K / 2) = 1 - C + C (cos(theta/2) - i sin(theta/2) S), dR = (-i/2) K R.
// Runtime masks and the plain (cos, sin) form: with a control there is no single float64 factor.

// (S x)[k] = i^q x[k ^ gx]: q from S's Y count and the Z signs of the source index
__device__ __forceinline__ int gen_q(uint64_t k, const DevGen &p) {
    return (p.gny + 2 * (__popcll((k ^ p.gx) & p.gz) & 1)) & 3;
}
// v * i^q by a swap and sign-bit flips (no float64 operation)
template <typename T2> __device__ __forceinline__ T2 mul_iq(T2 v, int q) {
    const T2 t = (q & 1) ? T2{v.y, v.x} : v;
    return T2{flip(t.x, ((q + 1) >> 1) & 1), flip(t.y, (q >> 1) & 1)};
}
// c x + ss w, with w = i (S x)[k]: the rotation (ss = -s) or its adjoint (ss = +s)
template <typename R, typename T2> __device__ __forceinline__ T2 gen_rot(T2 x, T2 w, R c, R ss) {
    return T2{fma(ss, w.x, c * x.x), fma(ss, w.y, c * x.y)};
}

// Visit every amplitude of the CTA with its partner under S: f(l, k, x[k], x[k ^ gx]). Partners
// inside the CTA are visited as pairs by one thread after reading both, so f may write buf[l];
// a partner in another CTA of the cluster comes from the exchanged copy of that CTA's slice.
template <typename R, typename F>
__device__ __forceinline__ void gen_visit(Eng<R> &e, const DevGen &p, F &&f) {
    using cx = typename CX<R>::T;
    const uint32_t lx = (uint32_t)(p.gx & (uint64_t)(e.Nl - 1));
    const int dx = (int)(p.gx >> e.nl);
    if (dx) {
        const cx *rv = e.exchange_rank(e.rank ^ dx);
        for (uint32_t l = threadIdx.x; l < e.Nl; l += blockDim.x) f(l, e.base | l, e.buf[l], rv[l ^ lx]);
    } else if (lx) {
        const int b = __ffs(lx) - 1;
        for (uint32_t pr = threadIdx.x; pr < (e.Nl >> 1); pr += blockDim.x) {
            const uint32_t l0 = ins0(pr, b), l1 = l0 ^ lx;
            const cx x0 = e.buf[l0], x1 = e.buf[l1];
            f(l0, e.base | l0, x0, x1);
            f(l1, e.base | l1, x1, x0);
        }
    } else {
        for (uint32_t l = threadIdx.x; l < e.Nl; l += blockDim.x) {
            const cx x = e.buf[l];
            f(l, e.base | l, x, x);
        }
    }
}

// Forward generalised rotation (the fixed block F_k has been applied), writing the checkpoint.
template <typename R>
__device__ __forceinline__ void fwd_step_gen(Eng<R> &e, typename CX<R>::T *out, const DevGen &p, R c, R s) {
    using cx = typename CX<R>::T;
    gen_visit(e, p, [&](uint32_t l, uint64_t kk, cx xm, cx xo) {
        cx y = xm;
        if ((kk & p.gctrl) == p.gctrl) y = gen_rot(xm, mul_iq(xo, gen_q(kk, p) + 1), c, -s);
        e.buf[l] = y;
        out[kk] = y;
    });
    __syncthreads();
}

// One column step with a generalised rotation: part += <a|K b> (Re / Im / both per IM), then
// b <- R^dag b when rot_on (F^dag is applied by the caller).
template <typename R, int IM>
__device__ __forceinline__ RI<R> col_step_gen(Eng<R> &e, const typename CX<R>::T *a, const DevGen &p, bool rot_on,
                                              R c, R s) {
    using cx = typename CX<R>::T;
    RI<R> part = {0, 0};
    gen_visit(e, p, [&](uint32_t l, uint64_t kk, cx xm, cx xo) {
        if ((kk & p.gctrl) != p.gctrl) return;  // K = 0 and R^dag = 1 there
        const int q = gen_q(kk, p);
        ipacc<IM>(part, a[kk], mul_iq(xo, q));
        if (rot_on) e.buf[l] = gen_rot(xm, mul_iq(xo, q + 1), c, s);
    });
    __syncthreads();
    return part;
}

// Column start of a generalised rotation j (Sec. 2): x = F_j Psi[j]; returns this thread's part of
// e_j = <x|K x>, leaves b = F_j^dag K x in the state buffer, multiplies scale_b by the float64
// factors of F_j and F_j^dag and sets escale to that of F_j alone; the warp sums of <x|C x> (the
// control probability, L_jj = <C_j>/4) go to pcred[warp].
template <typename R>
__device__ __forceinline__ R gen_column_start(Eng<R> &e, const Work &w, const DevInst &in, int j,
                                              const typename CX<R>::T *psi, double *pcred, double &escale,
                                              double &scale_b) {
    using cx = typename CX<R>::T;
    const DevParam pj = w.param[in.param_tab + j];
    const DevGen gj = w.gen[in.param_tab + j];
    double sF = 1.0;
    for (uint32_t l = threadIdx.x; l < e.Nl; l += blockDim.x) e.buf[l] = psi[e.base | l];
    __syncthreads();
    for (int f = 0; f < pj.fix_count; ++f) e.fixed_gate(w.fixed[pj.fix_begin + f], sF);
    escale = sF;
    R ep = 0, pc = 0;
    gen_visit(e, gj, [&](uint32_t l, uint64_t kk, cx xm, cx xo) {
        cx v = {0, 0};
        if ((kk & gj.gctrl) == gj.gctrl) {
            v = mul_iq(xo, gen_q(kk, gj));
            pc += xm.x * xm.x + xm.y * xm.y;
        }
        ep += xm.x * v.x + xm.y * v.y;
        e.buf[l] = v;
    });
    __syncthreads();
    for (int f = pj.fix_count - 1; f >= 0; --f) e.fixed_gate(w.fixed[pj.fix_begin + f], sF);
    scale_b *= sF;
    const double pcw = warp_sum((double)pc);
    if ((threadIdx.x & 31) == 0) pcred[threadIdx.x >> 5] = pcw;
    return ep;
}

// Forward rotation R_k with the diagonal fixed block F_k applied to the inputs (pre), writing
// both the shared-memory state and the checkpoint out.
template <typename R, int AX, int CB>
__device__ __forceinline__ void fwd_pairs(Eng<R> &e, typename CX<R>::T *out, int q, const RotC<R, CB> &rot, bool pre,
                                          const DevParam &pk, const DevDiag *dt) {
    using cx = typename CX<R>::T;
    const uint32_t bit = 1u << q, half = e.Nl >> 1;
    for (uint32_t p = threadIdx.x; p < half; p += blockDim.x) {
        const uint32_t l0 = ins0(p, q), l1 = l0 | bit;
        cx x0 = e.buf[l0], x1 = e.buf[l1];
        if (pre) {
            x0 = flip2(x0, diag_parity(e.base | l0, pk, dt));
            x1 = flip2(x1, diag_parity(e.base | l1, pk, dt));
        }
        const cx y0 = rot.apply(x0, isig<AX, 0>(x0, x1));
        const cx y1 = rot.apply(x1, isig<AX, 1>(x1, x0));
        e.buf[l0] = y0;
        e.buf[l1] = y1;
        out[e.base | l0] = y0;
        out[e.base | l1] = y1;
    }
}

template <typename R, int AX, int BETA, int CB>
__device__ __forceinline__ void fwd_dist(Eng<R> &e, const typename CX<R>::T *rv, typename CX<R>::T *out, int q,
                                         const RotC<R, CB> &rot, bool pre, const DevParam &pk, const DevDiag *dt) {
    using cx = typename CX<R>::T;
    const uint64_t m = 1ull << q;
    for (uint32_t l = threadIdx.x; l < e.Nl; l += blockDim.x) {
        const uint64_t kk = e.base | l;
        cx xm = e.buf[l], xo = rv[l];
        if (pre) {
            xm = flip2(xm, diag_parity(kk, pk, dt));
            xo = flip2(xo, diag_parity(kk ^ m, pk, dt));
        }
        const cx y = rot.apply(xm, isig<AX, BETA>(xm, xo));
        e.buf[l] = y;
        out[kk] = y;
    }
}

template <typename R, int CB>
__device__ __forceinline__ void fwd_diag(Eng<R> &e, typename CX<R>::T *out, int q, const RotC<R, CB> &rot, bool pre,
                                         const DevParam &pk, const DevDiag *dt) {
    using cx = typename CX<R>::T;
    for (uint32_t l = threadIdx.x; l < e.Nl; l += blockDim.x) {
        const uint64_t kk = e.base | l;
        cx x = e.buf[l];
        if (pre) x = flip2(x, diag_parity(kk, pk, dt));
        const int beta = (int)((kk >> q) & 1);
        const cx v = {flip(x.y, beta ^ 1), flip(x.x, beta)};
        const cx y = rot.apply(x, v);
        e.buf[l] = y;
        out[kk] = y;
    }
}

template <typename R, int CB>
__device__ __forceinline__ void fwd_step_cb(Eng<R> &e, typename CX<R>::T *out, const DevParam &pk, const RotC<R, CB> &rot,
                                            bool pre, const DevDiag *dt) {
    if (pk.axis == kAxisZ) {
        fwd_diag<R, CB>(e, out, pk.q, rot, pre, pk, dt);
    } else if (pk.q < e.nl) {
        if (pk.axis == kAxisX) fwd_pairs<R, kAxisX, CB>(e, out, pk.q, rot, pre, pk, dt);
        else fwd_pairs<R, kAxisY, CB>(e, out, pk.q, rot, pre, pk, dt);
    } else {
        const typename CX<R>::T *rv = e.exchange(pk.q);
        const int beta = (e.rank >> (pk.q - e.nl)) & 1;
        if (pk.axis == kAxisX) {
            if (beta) fwd_dist<R, kAxisX, 1, CB>(e, rv, out, pk.q, rot, pre, pk, dt);
            else fwd_dist<R, kAxisX, 0, CB>(e, rv, out, pk.q, rot, pre, pk, dt);
        } else {
            if (beta) fwd_dist<R, kAxisY, 1, CB>(e, rv, out, pk.q, rot, pre, pk, dt);
            else fwd_dist<R, kAxisY, 0, CB>(e, rv, out, pk.q, rot, pre, pk, dt);
        }
    }
    __syncthreads();
}

template <typename R>
__device__ __forceinline__ void fwd_step(Eng<R> &e, typename CX<R>::T *out, const DevParam &pk, const Rot<R> &rot,
                                         bool pre, const DevDiag *dt) {
    if (std::is_same<R, double>::value && rot.caseB) fwd_step_cb<R, 1>(e, out, pk, RotC<R, 1>{rot.c, rot.s, rot.t}, pre, dt);
    else fwd_step_cb<R, 0>(e, out, pk, RotC<R, 0>{rot.c, rot.s, rot.t}, pre, dt);
}

// ------------------------------------------------------------------------------------------
__global__ void k_coef(const double *theta, DevCoef *coef, double *pctrl, int64_t total, int32_t *status) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= total) return;
    pctrl[k] = 1.0;  // <C_k> of an uncontrolled rotation; controlled ones are overwritten by their column
    const double th = theta[k];
    if (!isfinite(th)) atomicCAS(status, 0, (int)QNG_ERR_ARG);
    double s, c;
    sincos(0.5 * th, &s, &c);
    DevCoef co;
    co.c = c;
    co.s = s;
    if (fabs(c) >= fabs(s)) { co.caseB = 0; co.f = c; co.t = s / c; }
    else                    { co.caseB = 1; co.f = s; co.t = c / s; }
    co.pad = 0;
    co.cf = (float)co.c;
    co.sf = (float)co.s;
    co.tf = (float)co.t;
    co.pad2 = 0;
    coef[k] = co;
}

// ------------------------------------------------------------------------------------------
// A run of m consecutive Z rotations (each with an all-diagonal fixed block, or none) in one
// elementwise pass: every amplitude goes through the m rotations in registers and each
// intermediate state is written to its checkpoint; no barrier between the rotations. The float64
// scale of each checkpoint is the running product of the rotations' factors (uniform, so every
// thread computes the same sequence and renormalises at the same steps).
template <typename R, int AMPS>
__device__ __forceinline__ void fwd_zrun_t(Eng<R> &e, typename CX<R>::T *__restrict__ ckpt, uint64_t N,
                                           const DevParam *__restrict__ params, const DevCoef *__restrict__ coefs,
                                           int k0, int m, const DevDiag *__restrict__ dt, double sc, double *sbcast,
                                           double *scales, bool write_scales) {
    using cx = typename CX<R>::T;
    constexpr bool kScaled = std::is_same<R, double>::value;
    cx x[AMPS];
    uint64_t kk[AMPS];
#pragma unroll
    for (int a = 0; a < AMPS; ++a) {
        const uint32_t l = threadIdx.x + a * blockDim.x;
        kk[a] = e.base | l;
        x[a] = e.buf[l];
    }
    DevParam pk = params[k0];
    DevCoef co = coefs[k0];
    for (int u = 0; u < m; ++u) {  // the thread's amplitudes advance together: AMPS independent chains
        const int un = u + 1 < m ? u + 1 : u;
        const DevParam pn = params[k0 + un];  // next step's tables, loaded while this step computes
        const DevCoef cn = coefs[k0 + un];
        // sign of the diagonal block F_k on each amplitude: one table read per (shift, mask) pair
        int par[AMPS];
#pragma unroll
        for (int a = 0; a < AMPS; ++a) par[a] = __popcll(kk[a] & pk.zmask);
        for (int d = 0; d < pk.diag_count; ++d) {
            const DevDiag dd = dt[pk.diag_begin + d];
#pragma unroll
            for (int a = 0; a < AMPS; ++a) par[a] += __popcll(kk[a] & (kk[a] >> dd.shift) & dd.mask);
        }
        cx *out = ckpt + (uint64_t)(k0 + u + 1) * N;
#pragma unroll
        for (int a = 0; a < AMPS; ++a) {
            x[a] = flip2(x[a], par[a] & 1);
            const int beta = (int)((kk[a] >> pk.q) & 1);
            const cx v = {flip(x[a].y, beta ^ 1), flip(x[a].x, beta)};  // (i Z x)_beta
            if constexpr (kScaled) {  // forward rotation: t' = -t
                if (co.caseB) { x[a].x = fma(-co.t, x[a].x, v.x); x[a].y = fma(-co.t, x[a].y, v.y); }
                else          { x[a].x = fma(-co.t, v.x, x[a].x); x[a].y = fma(-co.t, v.y, x[a].y); }
            } else {
                const R c = (R)co.c, sv = (R)(-co.s);
                x[a].x = fma(sv, v.x, c * x[a].x); x[a].y = fma(sv, v.y, c * x[a].y);
            }
            out[kk[a]] = x[a];
        }
        if (threadIdx.x == 0) {  // thread 0 carries the run's scale sequence (one float64 multiply a step)
            if constexpr (kScaled) sc *= co.caseB ? -co.f : co.f;
            if (write_scales) scales[k0 + u + 1] = sc;
        }
        pk = pn;
        co = cn;
    }
#pragma unroll
    for (int a = 0; a < AMPS; ++a) e.buf[threadIdx.x + a * blockDim.x] = x[a];
    if (threadIdx.x == 0) *sbcast = sc;
}

// returns false (and does nothing) when the CTA shape has no compiled amplitude count
template <typename R>
__device__ __forceinline__ bool fwd_zrun(Eng<R> &e, typename CX<R>::T *ckpt, uint64_t N, const DevParam *params,
                                         const DevCoef *coefs, int k0, int m, const DevDiag *dt, double &scale,
                                         double *scales, bool write_scales) {
    if (e.Nl % blockDim.x) return false;
    const uint32_t amps = e.Nl / blockDim.x;
    __shared__ double sbcast;  // the scale after the run, from thread 0 to the CTA
    switch (amps) {
    case 1: fwd_zrun_t<R, 1>(e, ckpt, N, params, coefs, k0, m, dt, scale, &sbcast, scales, write_scales); break;
    case 2: fwd_zrun_t<R, 2>(e, ckpt, N, params, coefs, k0, m, dt, scale, &sbcast, scales, write_scales); break;
    case 4: fwd_zrun_t<R, 4>(e, ckpt, N, params, coefs, k0, m, dt, scale, &sbcast, scales, write_scales); break;
    case 8: fwd_zrun_t<R, 8>(e, ckpt, N, params, coefs, k0, m, dt, scale, &sbcast, scales, write_scales); break;
    default: return false;
    }
    __syncthreads();
    scale = sbcast;
    return true;
}

// ------------------------------------------------------------------------------------------
// k_forward: one cluster per instance of the group.
// GEN = 1: the group has generalised rotations (a separate instantiation keeps the registers of
// the ordinary one unchanged).
template <typename R, int GEN>
__global__ void __launch_bounds__(512) k_forward(Work w, int group_first, int cl, int want_eta, int k_begin, int k_end,
                                                 int last) {
    using cx = typename CX<R>::T;
    extern __shared__ __align__(16) unsigned char smem[];
    const DevInst in = w.inst[w.group_inst[group_first + (blockIdx.x >> cl)]];
    Eng<R> e = make_eng<R>(smem, in.n, cl);
    double *red = reinterpret_cast<double *>(e.buf + (cl ? 3 : 1) * e.Nl);
    const uint64_t N = 1ull << in.n;
    cx *ckpt = reinterpret_cast<cx *>(w.ckpt) + in.ckpt_off;
    double *scales = w.scale + in.scale_off;

    // parameters [k_begin, k_end) of the sweep: from |0> at k_begin = 0, else from checkpoint
    // k_begin as an earlier launch wrote it (the carried state is that checkpoint, renormalised
    // exactly as the uninterrupted sweep would have renormalised it)
    const int kb = min(k_begin, in.P), ke = min(k_end, in.P);
    double scale = 1.0;
    if (kb == 0) {
        for (uint32_t l = threadIdx.x; l < e.Nl; l += blockDim.x) {
            cx z = {0, 0};
            if ((e.base | l) == 0) z.x = 1;
            e.buf[l] = z;
            ckpt[e.base | l] = z;
        }
        if (e.rank == 0 && threadIdx.x == 0) scales[0] = 1.0;
    } else {
        const cx *src = ckpt + (uint64_t)kb * N;
        for (uint32_t l = threadIdx.x; l < e.Nl; l += blockDim.x) e.buf[l] = src[e.base | l];
        scale = scales[kb];
    }
    __syncthreads();
    if (kb > 0) e.maybe_renorm(scale);

    DevParam pk_n;
    DevCoef co_n;
    if (kb < ke) { pk_n = w.param[in.param_tab + kb]; co_n = w.coef[in.param_off + kb]; }
    for (int k = kb; k < ke; ++k) {
        // a run of Z rotations with diagonal fixed blocks: one pass, no barriers in between
        // (clipped at the end of the range)
        if (pk_n.zrun > 1 && ke - k > 1) {
            const int m = min((int)pk_n.zrun, ke - k);
            // the whole run stays above the renormalisation threshold: each factor is >= 1/sqrt2
            const int ex = (int)((__double_as_longlong(scale) >> 52) & 0x7ff);
            if ((!std::is_same<R, double>::value || ex - (m + 1) / 2 - 1 >= 1023 - 200) &&
                fwd_zrun<R>(e, ckpt, N, w.param + in.param_tab, w.coef + in.param_off, k, m, w.diag, scale, scales,
                            e.rank == 0 && threadIdx.x == 0)) {
                k += m - 1;
                if (k + 1 < ke) { pk_n = w.param[in.param_tab + k + 1]; co_n = w.coef[in.param_off + k + 1]; }
                continue;
            }
        }
        const DevParam pk = pk_n;
        const DevCoef co = co_n;
        if (k + 1 < ke) { pk_n = w.param[in.param_tab + k + 1]; co_n = w.coef[in.param_off + k + 1]; }
        if constexpr (GEN) {
            if (pk.axis == kAxisGen) {  // generalised rotation: F_k gate by gate, then the plain (cos, sin) form
                for (int f = 0; f < pk.fix_count; ++f) e.fixed_gate(w.fixed[pk.fix_begin + f], scale);
                fwd_step_gen<R>(e, ckpt + (uint64_t)(k + 1) * N, w.gen[in.param_tab + k], (R)co.c, (R)co.s);
                if (e.rank == 0 && threadIdx.x == 0) scales[k + 1] = scale;
                e.maybe_renorm(scale);
                continue;
            }
        }
        if (pk.diag_count < 0) e.fixed_gates(w.fixed + pk.fix_begin, pk.fix_count, scale, false);
        const bool pre = pk.diag_count > 0 || pk.zmask != 0;
        double fs;
        const Rot<R> rot = make_rot<R>(co, false, fs);
        cx *out = ckpt + (uint64_t)(k + 1) * N;
        fwd_step<R>(e, out, pk, rot, pre, w.diag);
        if (std::is_same<R, double>::value) scale *= fs;
        if (e.rank == 0 && threadIdx.x == 0) scales[k + 1] = scale;  // the scale of checkpoint k+1 as written
        e.maybe_renorm(scale);                                         // then the state carried on to k+2
    }

    if (!last) return;
    // trailing fixed gates W, then H W psi, <E> and eta = W^dag H W psi
    e.fixed_gates(w.fixed + in.w_begin, in.w_count, scale, false);
    cx *eta = reinterpret_cast<cx *>(w.eta) + in.eta_off;
    for (uint32_t l = threadIdx.x; l < e.Nl; l += blockDim.x) eta[e.base | l] = e.buf[l];
    __syncthreads();
    e.csync();  // W psi visible to the whole cluster through global memory
    double epart = 0.0;
    for (uint32_t l = threadIdx.x; l < e.Nl; l += blockDim.x) {
        const uint64_t kk = e.base | l;
        double hr = 0.0, hi = 0.0;
#pragma unroll 4  // independent gathers of W psi in flight together (each is an L2 round trip)
        for (int t = 0; t < in.nterms; ++t) {
            const DevTerm tm = w.term[in.term_off + t];
            const uint64_t src = kk ^ tm.x;
            const cx v = __ldcg(eta + src);
            const int ph = (tm.ny + 2 * (__popcll(src & tm.z) & 1)) & 3;
            const double vr = (double)v.x, vi = (double)v.y;
            // i^ph * coeff * v
            if (ph == 0)      { hr = fma(tm.coeff, vr, hr);  hi = fma(tm.coeff, vi, hi); }
            else if (ph == 1) { hr = fma(-tm.coeff, vi, hr); hi = fma(tm.coeff, vr, hi); }
            else if (ph == 2) { hr = fma(-tm.coeff, vr, hr); hi = fma(-tm.coeff, vi, hi); }
            else              { hr = fma(tm.coeff, vi, hr);  hi = fma(-tm.coeff, vr, hi); }
        }
        const cx x = e.buf[l];
        epart += (double)x.x * hr + (double)x.y * hi;
        e.buf[l] = cx{(R)hr, (R)hi};
    }
    __syncthreads();
    const double esum = cluster_sum(epart, red, cl);  // also orders the reads of eta before the writes below
    if (e.rank == 0 && threadIdx.x == 0) w.energy[w.group_inst[group_first + (blockIdx.x >> cl)]] = esum * scale * scale;
    if (want_eta) {
        e.fixed_gates(w.fixed + in.w_begin, in.w_count, scale, true);
        for (uint32_t l = threadIdx.x; l < e.Nl; l += blockDim.x) eta[e.base | l] = e.buf[l];
        if (e.rank == 0 && threadIdx.x == 0) scales[in.P + 1] = scale;
    }
}

// ------------------------------------------------------------------------------------------
// complex64 column walk through a run of L Z rotations without fixed gates, from parameter i down.
// Diagonal operators commute: Psi[i'+1] and b at step i' of the run are Psi[i+1] and the run's
// starting b times the same diagonal unitary D, so <Psi[i'+1]|Z_q|b> = <Psi[i+1]|Z_q|b_start>. Every
// inner product of the run therefore comes from the one checkpoint Psi[i+1], and the run's adjoint
// rotations (cos + i sin Z) compose into one factor per amplitude: one checkpoint read and one
// barrier for the run instead of one per step.
constexpr int kColRun = 4;  // steps per run at most (a longer run is taken in pieces)
template <typename R, int AMPS, int MODE>
__device__ __forceinline__ void col_zrun_t(Eng<R> &e, const typename CX<R>::T *__restrict__ a,
                                           const DevParam *__restrict__ params, const DevCoef *__restrict__ coefs,
                                           int i, int L, RI<R> (&parts)[kColRun]) {
    using cx = typename CX<R>::T;
    // per amplitude only the products and the composed factor stay in registers; b is read again
    // from shared memory at the end (the run does not write it before then)
    cx ph[AMPS];
    R pr[AMPS], pm[AMPS];
#pragma unroll
    for (int u = 0; u < AMPS; ++u) {
        const uint32_t l = threadIdx.x + u * blockDim.x;
        const cx xv = e.buf[l];
        const cx av = a[e.base | l];
        pr[u] = av.x * xv.x + av.y * xv.y;  // Re conj(a) b
        pm[u] = av.x * xv.y - av.y * xv.x;  // Im conj(a) b
        ph[u] = cx{(R)1, (R)0};
    }
#pragma unroll
    for (int r = 0; r < kColRun; ++r) {
        if (r >= L) break;
        const int ii = i - r;
        const DevParam pk = params[ii];
        RI<R> pt = {0, 0};
#pragma unroll
        for (int u = 0; u < AMPS; ++u) {
            const bool beta = ((e.base | (threadIdx.x + u * blockDim.x)) >> pk.q) & 1;  // (Z b)_beta = (-1)^beta b
            if (MODE != 1) pt.re += beta ? -pr[u] : pr[u];
            if (MODE != 0) pt.im += beta ? -pm[u] : pm[u];
        }
        parts[r] = pt;
        if (ii > 0) {  // the last step of a column (i = 0) takes no rotation
            const DevCoef co = coefs[ii];
            const R c = co.cf, sn = co.sf;
#pragma unroll
            for (int u = 0; u < AMPS; ++u) {
                const R sv = (((e.base | (threadIdx.x + u * blockDim.x)) >> pk.q) & 1) ? -sn : sn;
                ph[u] = cx{fma(c, ph[u].x, -sv * ph[u].y), fma(c, ph[u].y, sv * ph[u].x)};
            }
        }
    }
#pragma unroll
    for (int u = 0; u < AMPS; ++u) {
        const uint32_t l = threadIdx.x + u * blockDim.x;
        const cx x = e.buf[l];
        const cx y = {fma(x.x, ph[u].x, -x.y * ph[u].y), fma(x.x, ph[u].y, x.y * ph[u].x)};
        e.buf[l] = y;
    }
}
// false (nothing done) when the CTA shape has no compiled amplitude count
template <typename R, int MODE>
__device__ __forceinline__ bool col_zrun(Eng<R> &e, const typename CX<R>::T *a, const DevParam *params,
                                         const DevCoef *coefs, int i, int L, RI<R> (&parts)[kColRun]) {
    if (e.Nl % blockDim.x) return false;
    switch (e.Nl / blockDim.x) {
    case 1: col_zrun_t<R, 1, MODE>(e, a, params, coefs, i, L, parts); return true;
    case 2: col_zrun_t<R, 2, MODE>(e, a, params, coefs, i, L, parts); return true;
    case 4: col_zrun_t<R, 4, MODE>(e, a, params, coefs, i, L, parts); return true;
    default: return false;
    }
}
// The partial sums of step sx into the warp's shift register acc, flushed to red every 8 steps (4
// with both parts, mode 2) and at the last step.
template <typename RA, int MIM>
__device__ __forceinline__ void push_part(RA (&acc)[8], int &cnt, int mode, int sx, int nsteps, RI<RA> part,
                                          double *red, double *red_im, int lane, int nw, int wid) {
    if (!MIM || mode != 2) {
#pragma unroll
        for (int k = 7; k > 0; --k) acc[k] = acc[k - 1];
        acc[0] = mode ? part.im : part.re;
        if (++cnt == 8 || sx == nsteps - 1) {
            const int idx = (lane >> 2) & 7;
            const double pw = (double)warp_sum8(acc, lane);
            if ((lane & 3) == 0 && idx < cnt) red[(size_t)(sx - idx) * nw + wid] = pw;
#pragma unroll
            for (int k = 0; k < 8; ++k) acc[k] = 0;
            cnt = 0;
        }
    } else {
#pragma unroll
        for (int k = 7; k > 1; --k) acc[k] = acc[k - 2];
        acc[0] = part.re;
        acc[1] = part.im;
        if (++cnt == 4 || sx == nsteps - 1) {
            const int idx = (lane >> 2) & 7, off = idx >> 1;
            const double pw = (double)warp_sum8(acc, lane);
            if ((lane & 3) == 0 && off < cnt) ((idx & 1) ? red_im : red)[(size_t)(sx - off) * nw + wid] = pw;
#pragma unroll
            for (int k = 0; k < 8; ++k) acc[k] = 0;
            cnt = 0;
        }
    }
}

// ------------------------------------------------------------------------------------------
// k_columns: one cluster per work item (instance, column).
template <typename R, int MIM, int GEN, int ZR>
__device__ __forceinline__ void column_item(const Work &w, const DevWork wk, int cl, int max_P, unsigned char *smem);

// One cluster per work item, or (queue != nullptr) a persistent grid of clusters that take work
// items, longest first, from a device counter until all num_work are done. MIM = 1: metric
// columns take Im L_ij as well (into w.Lim); their partial sums need Group::smem_col_im bytes.
// GEN = 1: the group has generalised rotations. ZR = 1 (complex64, a group of one instance): runs
// of Z rotations are composed (col_zrun_t); a separate instantiation, so that the batches' column
// kernel stays as it was (with the run code compiled in, a 256-instance batch measured slower).
template <typename R, int MIM, int GEN, int ZR = 0>
__global__ void __launch_bounds__(256, (MIM || GEN) ? 2 : 3) k_columns(Work w, int work_first, int cl, int max_P, int *queue,
                                                                       int num_work) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int item_sh;
    if (!queue) {
        column_item<R, MIM, GEN, ZR>(w, w.work[work_first + (blockIdx.x >> cl)], cl, max_P, smem);
        return;
    }
    for (;;) {
        if (threadIdx.x == 0 && (!cl || cg::this_cluster().block_rank() == 0)) item_sh = atomicAdd(queue, 1);
        if (cl) {
            cg::this_cluster().sync();
            const int item = *cg::this_cluster().map_shared_rank(&item_sh, 0);
            cg::this_cluster().sync();  // rank 0 keeps item_sh until every CTA has read it
            if (item >= num_work) return;
            column_item<R, MIM, GEN, ZR>(w, w.work[work_first + item], cl, max_P, smem);
        } else {
            __syncthreads();
            const int item = item_sh;
            __syncthreads();
            if (item >= num_work) return;
            column_item<R, MIM, GEN, ZR>(w, w.work[work_first + item], cl, max_P, smem);
        }
    }
}

template <typename R, int MIM, int GEN, int ZR>
__device__ __forceinline__ void column_item(const Work &w, const DevWork wk, int cl, int max_P, unsigned char *smem) {
    using cx = typename CX<R>::T;
    using RA = R;  // per-thread partial sums; float64 from the warp level on
    const DevInst in = w.inst[wk.inst];
    Eng<R> e = make_eng<R>(smem, in.n, cl);
    const int nw = blockDim.x >> 5, lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    double *red = reinterpret_cast<double *>(e.buf + (cl ? 3 : 1) * e.Nl);  // [(max_P + 1) * nw]
    double *fac = red + (size_t)(max_P + 1) * nw;                              // [max_P + 1]
    double *red_im = fac + (max_P + 1);  // [(max_P + 1) * nw], metric_im only
    const uint64_t N = 1ull << in.n;
    const cx *ckpt = reinterpret_cast<const cx *>(w.ckpt) + in.ckpt_off;
    const double *scales = w.scale + in.scale_off;
    const int P = in.P;
    const int col = wk.col;
    const bool grad_col = col == P;

    double scale_b;
    int nsteps, i0;
    bool gen_start = false;     // generalised rotation: <C_j> is reduced too
    __shared__ double pcred[8]; // per-warp partial sums of <C_j> (at most 8 warps)
    if (!grad_col) {
        // b = F_j^dag sigma_j F_j Psi[j] = U_j^dag sigma_j Psi[j+1]; e_j = <Psi[j]|b>
        const int j = col;
        const DevParam pj = w.param[in.param_tab + j];
        const cx *psi = ckpt + (uint64_t)j * N;
        scale_b = scales[j];
        double escale = 1.0;  // scale of F_j Psi[j] relative to Psi[j] (float64 form with H gates)
        RA ep = 0;
        if (GEN && pj.axis == kAxisGen) {
            gen_start = true;
            if constexpr (GEN) ep = gen_column_start<R>(e, w, in, j, psi, pcred, escale, scale_b);
        } else if (pj.diag_count >= 0) {
            const uint64_t m = (pj.axis == kAxisZ) ? 0ull : (1ull << pj.q);
            const bool diag = pj.diag_count > 0 || pj.zmask != 0;
            for (uint32_t l = threadIdx.x; l < e.Nl; l += blockDim.x) {
                const uint64_t kk = e.base | l, kp = kk ^ m;
                const int beta = (int)((kk >> pj.q) & 1);
                const cx xo = psi[kp];
                const cx xm = m ? psi[kk] : xo;
                cx v = sigma_of(pj.axis, beta, xo, xo);  // (sigma y)[kk] from y[kp]
                if (diag) v = neg_if(v, diag_parity(kk, pj, w.diag) ^ diag_parity(kp, pj, w.diag));
                e.buf[l] = v;
                ep += xm.x * v.x + xm.y * v.y;
            }
            __syncthreads();
        } else {
            // general F_j: load Psi[j], apply F_j, take e_j and apply sigma_j, then undo F_j
            double sF = 1.0;
            for (uint32_t l = threadIdx.x; l < e.Nl; l += blockDim.x) e.buf[l] = psi[e.base | l];
            __syncthreads();
            for (int f = 0; f < pj.fix_count; ++f) e.fixed_gate(w.fixed[pj.fix_begin + f], sF);
            escale = sF;
            const int q = pj.q, axis = pj.axis;
            if (axis == kAxisZ) {
                for (uint32_t l = threadIdx.x; l < e.Nl; l += blockDim.x) {
                    const uint64_t kk = e.base | l;
                    const cx x = e.buf[l];
                    const cx v = sigma_of(axis, (int)((kk >> q) & 1), x, x);
                    ep += x.x * v.x + x.y * v.y;
                    e.buf[l] = v;
                }
                __syncthreads();
            } else if (q < e.nl) {
                const uint32_t bit = 1u << q, half = e.Nl >> 1;
                for (uint32_t p = threadIdx.x; p < half; p += blockDim.x) {
                    const uint32_t l0 = ins0(p, q), l1 = l0 | bit;
                    const cx x0 = e.buf[l0], x1 = e.buf[l1];
                    const cx v0 = sigma_of(axis, 0, x0, x1), v1 = sigma_of(axis, 1, x1, x0);
                    ep += x0.x * v0.x + x0.y * v0.y + x1.x * v1.x + x1.y * v1.y;
                    e.buf[l0] = v0; e.buf[l1] = v1;
                }
                __syncthreads();
            } else {
                const cx *rv = e.exchange(q);
                const int beta = (e.rank >> (q - e.nl)) & 1;
                for (uint32_t l = threadIdx.x; l < e.Nl; l += blockDim.x) {
                    const cx xm = e.buf[l];
                    const cx v = sigma_of(axis, beta, xm, rv[l]);
                    ep += xm.x * v.x + xm.y * v.y;
                    e.buf[l] = v;
                }
                __syncthreads();
            }
            for (int f = pj.fix_count - 1; f >= 0; --f) e.fixed_gate(w.fixed[pj.fix_begin + f], sF);
            scale_b *= sF;
        }
        const double epw = warp_sum((double)ep);
        if (lane == 0) red[(size_t)max_P * nw + wid] = epw;
        if (threadIdx.x == 0) fac[max_P] = scales[j] * escale * scales[j] * escale;
        nsteps = j;
        i0 = j - 1;
    } else {
        const cx *eta = reinterpret_cast<const cx *>(w.eta) + in.eta_off;
        for (uint32_t l = threadIdx.x; l < e.Nl; l += blockDim.x) e.buf[l] = eta[e.base | l];
        scale_b = scales[P + 1];
        nsteps = P;
        i0 = P - 1;
        __syncthreads();
    }

    // 0: Re <a|sigma b> (metric), 1: Im (gradient column), 2: both (metric with Im L)
    const int mode = grad_col ? 1 : (MIM ? 2 : 0);
    RA acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};  // acc[k]: partial sum of step s - k (mode 2: re/im of step s - k/2)
    int cnt = 0;
    constexpr bool kScaled = std::is_same<R, double>::value;
    __shared__ int rn_flag[2];  // renormalise b after step s (written by thread 0, parity of s)
    const uint32_t slice_bytes = e.Nl * (uint32_t)sizeof(cx);
    for (int s = 0; s < nsteps; ++s) {
        const int i = i0 - s;
        const DevParam pi = w.param[in.param_tab + i];
        const double sci = scales[i + 1];
        const cx *a = ckpt + (uint64_t)(i + 1) * N;
        if constexpr (!kScaled && !GEN && ZR) {
            // complex64: a run of Z rotations without fixed gates in one pass (col_zrun_t)
            const int L = min(min(pi.zdown, nsteps - s), kColRun);
            if (L >= 2) {
                RI<RA> zp[kColRun];
                const DevParam *pt = w.param + in.param_tab;
                const DevCoef *ct = w.coef + in.param_off;
                bool done = false;
                if (mode == 0) done = col_zrun<R, 0>(e, a, pt, ct, i, L, zp);
                else if (mode == 1) done = col_zrun<R, 1>(e, a, pt, ct, i, L, zp);
                else if constexpr (MIM) done = col_zrun<R, 2>(e, a, pt, ct, i, L, zp);
                if (done) {
                    if (s + L < nsteps) {  // the step after the run reads checkpoint i - L + 1
                        const char *nxt = reinterpret_cast<const char *>(ckpt + (uint64_t)(i - L + 1) * N + e.base);
                        for (uint32_t off = threadIdx.x * 128u; off < slice_bytes; off += blockDim.x * 128u)
                            asm volatile("prefetch.global.L1 [%0];" ::"l"(nxt + off));
                    }
                    if (threadIdx.x == 0)  // every inner product of the run is taken on checkpoint i + 1
                        for (int r = 0; r < L; ++r) fac[s + r] = sci * scale_b;
#pragma unroll
                    for (int r = 0; r < kColRun; ++r)
                        if (r < L) push_part<RA, MIM>(acc, cnt, mode, s + r, nsteps, zp[r], red, red_im, lane, nw, wid);
                    __syncthreads();
                    s += L - 1;
                    continue;
                }
            }
        }

        // the next step reads this CTA's slice of checkpoint i: start it towards L1 now, so the
        // step after this one does not wait on L2
        if (s + 1 < nsteps) {
            const char *nxt = reinterpret_cast<const char *>(ckpt + (uint64_t)i * N + e.base);
            for (uint32_t off = threadIdx.x * 128u; off < slice_bytes; off += blockDim.x * 128u)
                asm volatile("prefetch.global.L1 [%0];" ::"l"(nxt + off));
        }
        const bool rot_on = (i > 0);
        const bool gen = GEN && pi.axis == kAxisGen;  // generalised rotation: plain (cos, sin) form, factor 1
        double fs = 1.0;
        const DevCoef co = w.coef[in.param_off + i];
        const Rot<R> rot = make_rot<R>(co, true, fs);
        if (gen) fs = 1.0;
        if (threadIdx.x == 0) {  // thread 0 owns the scale of b
            fac[s] = sci * scale_b;
            rn_flag[s & 1] = 0;
            if (kScaled && rot_on) {
                scale_b *= fs;
                rn_flag[s & 1] = ((int)((__double_as_longlong(scale_b) >> 52) & 0x7ff) < 1023 - 200);
            }
        }
        const bool post = !gen && rot_on && (pi.diag_count > 0 || pi.zmask != 0);
        RI<RA> part;
        if (GEN && gen) {
            if constexpr (GEN) {
                const DevGen gi = w.gen[in.param_tab + i];
                part = (mode == 1) ? col_step_gen<R, 1>(e, a, gi, rot_on, (R)co.c, (R)co.s)
                                   : col_step_gen<R, MIM ? 2 : 0>(e, a, gi, rot_on, (R)co.c, (R)co.s);
            }
        } else if (mode == 1) {
            part = col_step<R, 1>(e, a, pi, rot_on, rot, post, w.diag);
        } else {
            part = col_step<R, MIM ? 2 : 0>(e, a, pi, rot_on, rot, post, w.diag);
        }
        if (rot_on) {
            if (pi.diag_count < 0 || gen) {  // F_i^dag gate by gate
                for (int f = pi.fix_count - 1; f >= 0; --f) e.fixed_gate(w.fixed[pi.fix_begin + f], scale_b);
                if (threadIdx.x == 0 && kScaled)
                    rn_flag[s & 1] = ((int)((__double_as_longlong(scale_b) >> 52) & 0x7ff) < 1023 - 200);
                __syncthreads();
            }
            if constexpr (kScaled) {
                if (rn_flag[s & 1]) {  // rare: fold 2^-200 into the vector (exact)
                    for (uint32_t l = threadIdx.x; l < e.Nl; l += blockDim.x) {
                        cx x = e.buf[l];
                        x.x *= 0x1p-200; x.y *= 0x1p-200;
                        e.buf[l] = x;
                    }
                    if (threadIdx.x == 0) scale_b *= 0x1p200;
                    __syncthreads();
                }
            }
        }
        if (!MIM || mode != 2) {
#pragma unroll
            for (int k = 7; k > 0; --k) acc[k] = acc[k - 1];
            acc[0] = mode ? part.im : part.re;
            if (++cnt == 8 || s == nsteps - 1) {
                const int idx = (lane >> 2) & 7;
                const double pw = (double)warp_sum8(acc, lane);
                if ((lane & 3) == 0 && idx < cnt) red[(size_t)(s - idx) * nw + wid] = pw;
#pragma unroll
                for (int k = 0; k < 8; ++k) acc[k] = 0;
                cnt = 0;
            }
        } else {
#pragma unroll
            for (int k = 7; k > 1; --k) acc[k] = acc[k - 2];
            acc[0] = part.re;
            acc[1] = part.im;
            if (++cnt == 4 || s == nsteps - 1) {
                const int idx = (lane >> 2) & 7, off = idx >> 1;
                const double pw = (double)warp_sum8(acc, lane);
                if ((lane & 3) == 0 && off < cnt) ((idx & 1) ? red_im : red)[(size_t)(s - off) * nw + wid] = pw;
#pragma unroll
                for (int k = 0; k < 8; ++k) acc[k] = 0;
                cnt = 0;
            }
        }
    }

    // reduce the per-warp partial sums over the cluster (rank 0) and write the results
    __syncthreads();
    if (cl) cg::this_cluster().sync();
    if (e.rank == 0) {
        const int C = 1 << cl;
        const int rows = grad_col ? nsteps : nsteps + 1;
        for (int s = threadIdx.x; s < rows; s += blockDim.x) {
            const int row = (s < nsteps) ? s : max_P;
            double tot = 0.0;
            for (int r = 0; r < C; ++r) {
                const double *rr = cl ? cg::this_cluster().map_shared_rank(red, r) : red;
                for (int ww = 0; ww < nw; ++ww) tot += rr[(size_t)row * nw + ww];
            }
            tot *= fac[row];
            if (grad_col) {
                w.gradraw[in.param_off + (i0 - s)] = -tot;
            } else if (s < nsteps) {
                w.L[in.metric_off + (int64_t)(i0 - s) * P + col] = 0.25 * tot;
                if (MIM) {
                    double ti = 0.0;
                    for (int r = 0; r < C; ++r) {
                        const double *rr = cl ? cg::this_cluster().map_shared_rank(red_im, r) : red_im;
                        for (int ww = 0; ww < nw; ++ww) ti += rr[(size_t)row * nw + ww];
                    }
                    w.Lim[in.metric_off + (int64_t)(i0 - s) * P + col] = 0.25 * ti * fac[row];
                }
            } else {
                w.sigma[in.param_off + col] = tot;
            }
        }
        if (GEN && gen_start && threadIdx.x == 0) {  // <C_j> = <x|C x> with the same float64 factor as e_j
            double t = 0.0;
            for (int r = 0; r < C; ++r) {
                const double *pr = cl ? cg::this_cluster().map_shared_rank(pcred, r) : pcred;
                for (int ww = 0; ww < nw; ++ww) t += pr[ww];
            }
            w.pctrl[in.param_off + col] = t * fac[max_P];
        }
    }
    if (cl) cg::this_cluster().sync();
}

// ------------------------------------------------------------------------------------------
// k_finish: one CTA per instance. Assembly of g (Eq. g_t_L_def with L_ii = 1/4 and
// T_k = -(i/2) sigma_k), outputs, and the Cholesky solve of (g + lambda I) dtheta = -dt grad.
__global__ void __launch_bounds__(512) k_finish(Work w, LaunchArgs a) {
    __shared__ double sh[2];
    __shared__ int bad;
    const int b = blockIdx.x;
    const DevInst in = w.inst[b];
    const int P = in.P;
    const double *sg = w.sigma + in.param_off;
    const double *pc = w.pctrl + in.param_off;  // <C_i>: the diagonal L_ii = <C_i>/4 (Sec. 2)
    const double *L = w.L + in.metric_off;
    const bool metric = a.jobs & (kJobMetric | kJobSolve);
    double *A = w.chol + in.metric_off;
    if (metric) {
        for (int64_t idx = threadIdx.x; idx < (int64_t)P * P; idx += blockDim.x) {
            const int i = (int)(idx / P), j = (int)(idx % P);
            double v;
            if (i == j) v = 0.25 * (pc[i] - sg[i] * sg[i]);
            else if (i < j) v = L[(int64_t)i * P + j] - 0.25 * sg[i] * sg[j];
            else v = L[(int64_t)j * P + i] - 0.25 * sg[i] * sg[j];
            if (a.g_out) a.g_out[in.metric_off + idx] = v;
            if (a.jobs & kJobSolve) A[idx] = v + (i == j ? a.lambda : 0.0);
        }
        if ((a.jobs & kJobMetricIm) && a.gim_out) {  // Im G = Im L: T_i^* T_j is real; Hermitian
            const double *Li = w.Lim + in.metric_off;
            for (int64_t idx = threadIdx.x; idx < (int64_t)P * P; idx += blockDim.x) {
                const int i = (int)(idx / P), j = (int)(idx % P);
                a.gim_out[in.metric_off + idx] = i < j ? Li[(int64_t)i * P + j] : (i > j ? -Li[(int64_t)j * P + i] : 0.0);
            }
        }
        if (a.sigma_out)
            for (int k = threadIdx.x; k < P; k += blockDim.x) a.sigma_out[in.param_off + k] = sg[k];
    }
    if (a.jobs & kJobGradient) {
        const double gs = a.grad_scale ? a.grad_scale[b] : 1.0;
        if (a.grad_out)
            for (int k = threadIdx.x; k < P; k += blockDim.x) a.grad_out[in.param_off + k] = gs * w.gradraw[in.param_off + k];
    }
    if ((a.jobs & (kJobGradient | kJobEnergy)) && a.energy_out && threadIdx.x == 0) a.energy_out[b] = w.energy[b];
    if (!(a.jobs & kJobSolve) || P == 0) return;
    __syncthreads();
    // right-looking Cholesky, lower triangle, in place
    if (threadIdx.x == 0) bad = 0;
    for (int k = 0; k < P; ++k) {
        if (threadIdx.x == 0) {
            const double d = A[(int64_t)k * P + k];
            if (!(d > 0.0)) { bad = 1; atomicCAS(w.status, 0, (int)QNG_ERR_NOT_SPD); }
            const double r = sqrt(d);
            A[(int64_t)k * P + k] = r;
            sh[0] = 1.0 / r;
        }
        __syncthreads();
        if (bad) return;
        const double inv = sh[0];
        for (int i = k + 1 + threadIdx.x; i < P; i += blockDim.x) A[(int64_t)i * P + k] *= inv;
        __syncthreads();
        const int m = P - k - 1;
        for (int64_t t = threadIdx.x; t < (int64_t)m * m; t += blockDim.x) {
            const int i = k + 1 + (int)(t / m), j = k + 1 + (int)(t % m);
            if (j <= i) A[(int64_t)i * P + j] -= A[(int64_t)i * P + k] * A[(int64_t)j * P + k];
        }
        __syncthreads();
    }
    // forward substitution L y = -dt grad, then L^T x = y (x in dtheta)
    double *x = a.dtheta_out + in.param_off;
    const double *gr = w.gradraw + in.param_off;
    for (int k = threadIdx.x; k < P; k += blockDim.x) x[k] = -a.dt * gr[k];
    __syncthreads();
    for (int k = 0; k < P; ++k) {
        if (threadIdx.x == 0) { x[k] /= A[(int64_t)k * P + k]; sh[1] = x[k]; }
        __syncthreads();
        const double xk = sh[1];
        for (int i = k + 1 + threadIdx.x; i < P; i += blockDim.x) x[i] -= A[(int64_t)i * P + k] * xk;
        __syncthreads();
    }
    for (int k = P - 1; k >= 0; --k) {
        if (threadIdx.x == 0) { x[k] /= A[(int64_t)k * P + k]; sh[1] = x[k]; }
        __syncthreads();
        const double xk = sh[1];
        for (int i = threadIdx.x; i < k; i += blockDim.x) x[i] -= A[(int64_t)k * P + i] * xk;
        __syncthreads();
    }
}

// ------------------------------------------------------------------------------------------
// k_solve: one cluster of 2^cl CTAs per instance. Assembly of g (Eq. g_t_L_def), then the float64
// Cholesky factorisation of A = g + lambda I and the solve of A dtheta = -dt grad (Eq. 3). Row i of
// A lives in the shared memory of CTA i mod C. Blocked right-looking factorisation, block width kNb:
//   (B) barrier: the diagonal block and its right-hand side have been pushed to every CTA;
//   (C) every CTA factors the diagonal block itself and solves that block of L y = b;
//   (D) each CTA turns its own rows below the block into panel rows of L, updates its entries of
//       b, and pushes its panel rows to every CTA (remote stores only, no remote loads);
//   (E) barrier: the whole panel is in every CTA;
//   (F) each CTA updates its own trailing rows, then pushes its rows of the next diagonal block.
// Single buffers are safe: a buffer is rewritten only after a barrier that every reader reached
// after its last read. The back substitution L^T x = y runs block by block from the end: partial
// sums of the own rows are pushed to every CTA (two parity buffers), one barrier per block, and
// every CTA solves the block with the diagonal blocks of L it kept from (C).
constexpr int kNb = 16;

struct SolveSmem {
    double *A;      // [R][P] own rows
    double *PLt;    // [kNb][P] panel of the current block, column-major (column c, row j - t0)
    double *Ld;     // [nblk][kNb][kNb] factored diagonal blocks (the current one is factored in place)
    double *ys;     // [P] y, then x
    double *part;   // [2][C][kNb] pushed partial sums of the back substitution
    double *b;      // [R] own entries of the right-hand side
    double *inv;    // [kNb] reciprocal pivots of the current block
    int *flag;
};

__device__ __forceinline__ SolveSmem solve_smem(unsigned char *smem, int R, int P, int C) {
    const int nblk = (P + kNb - 1) / kNb;
    SolveSmem s;
    s.A = reinterpret_cast<double *>(smem);
    s.PLt = s.A + (size_t)R * P;
    s.Ld = s.PLt + (size_t)kNb * P;
    s.ys = s.Ld + (size_t)nblk * kNb * kNb;
    s.part = s.ys + P;
    s.b = s.part + 2 * C * kNb;
    s.inv = s.b + R;
    s.flag = reinterpret_cast<int *>(s.inv + kNb);
    return s;
}

// named barrier of warps 0..3 (threads 0..127)
__device__ __forceinline__ void sync128() { asm volatile("bar.sync 1, 128;" ::: "memory"); }

__global__ void __launch_bounds__(256) k_solve(Work w, LaunchArgs a, int cl) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ unsigned char tri_r[kNb * (kNb - 1) / 2], tri_c[kNb * (kNb - 1) / 2];
    const int C = 1 << cl;
    const int b = blockIdx.x >> cl;
    const int rank = cl ? (int)cg::this_cluster().block_rank() : 0;
    // after the mixed-precision solve: only the instances it handed over (same word in every CTA)
    if (a.ir_gate && w.irflag[b] == 0) return;
    const DevInst in = w.inst[b];
    const int P = in.P;
    const int R = (P + C - 1) / C;
    SolveSmem sm = solve_smem(smem, R, P, C);
    const double *sg = w.sigma + in.param_off;
    const double *pc = w.pctrl + in.param_off;  // <C_i>: the diagonal L_ii = <C_i>/4 (Sec. 2)
    const double *L = w.L + in.metric_off;
    const double *gr = w.gradraw + in.param_off;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5, tid = threadIdx.x;
    auto csync = [&]() { if (cl) cg::this_cluster().sync(); else __syncthreads(); };
    auto rptr = [&](double *p, int r) -> double * { return cl ? cg::this_cluster().map_shared_rank(p, r) : p; };
    const int nblk = (P + kNb - 1) / kNb;
    const int nown = (rank < P) ? (P - 1 - rank) / C + 1 : 0;

    // lower-triangle enumeration of a (kNb-1) x (kNb-1) block by rows: entry t <-> (r, c), c <= r
    if (tid == 0) {
        int t = 0;
        for (int r = 0; r < kNb - 1; ++r)
            for (int c = 0; c <= r; ++c) { tri_r[t] = (unsigned char)r; tri_c[t] = (unsigned char)c; ++t; }
    }
    // assembly of own rows, outputs
    for (int t = tid; t < nown * P; t += blockDim.x) {
        const int il = t / P, j = t % P, i = il * C + rank;
        double v;
        if (i == j) v = 0.25 * (pc[i] - sg[i] * sg[i]);
        else if (i < j) v = L[(int64_t)i * P + j] - 0.25 * sg[i] * sg[j];
        else v = L[(int64_t)j * P + i] - 0.25 * sg[i] * sg[j];
        if (a.g_out) a.g_out[in.metric_off + (int64_t)i * P + j] = v;
        sm.A[(size_t)il * P + j] = v + (i == j ? a.lambda : 0.0);
    }
    for (int il = tid; il < nown; il += blockDim.x) sm.b[il] = -a.dt * gr[il * C + rank];
    if (rank == 0) {
        if (a.grad_out)
            for (int k = tid; k < P; k += blockDim.x) a.grad_out[in.param_off + k] = gr[k];
        if (a.sigma_out)
            for (int k = tid; k < P; k += blockDim.x) a.sigma_out[in.param_off + k] = sg[k];
        if (a.energy_out && tid == 0) a.energy_out[b] = w.energy[b];
    }
    if (tid == 0) *sm.flag = 0;
    __syncthreads();
    csync();  // every CTA is running before any distributed shared memory access
    auto push_diag = [&](int kb) {  // rows of diagonal block kb (own ones) and their b entries, to every CTA
        const int c0 = kb * kNb, nb = min(kNb, P - c0);
        double *dst = sm.Ld + (size_t)kb * kNb * kNb;
        for (int t = tid; t < nb * (nb + 1) * C; t += blockDim.x) {
            const int q = t % C, e = t / C, r = e / (nb + 1), c = e % (nb + 1), i = c0 + r;
            if (i % C != rank) continue;
            if (c < nb) rptr(dst, q)[r * kNb + c] = (c <= r) ? sm.A[(size_t)(i / C) * P + c0 + c] : 0.0;
            else rptr(sm.ys, q)[i] = sm.b[i / C];
        }
    };
    push_diag(0);

    bool failed = false;
    for (int kb = 0; kb < nblk; ++kb) {
        const int c0 = kb * kNb, nb = min(kNb, P - c0), t0 = c0 + nb;
        double *D = sm.Ld + (size_t)kb * kNb * kNb;
        __syncthreads();
        csync();  // (B) the diagonal block and its b entries are here
        // (C) factor the diagonal block in place (warps 0..3), then its part of L y = b (warp 0)
        if (tid < 128) {
            for (int k = 0; k < nb; ++k) {
                if (tid == 0) {
                    const double d = D[k * kNb + k];
                    if (!(d > 0.0)) *sm.flag = 1;
                    else { const double iv = rsqrt(d); D[k * kNb + k] = d * iv; sm.inv[k] = iv; }
                }
                sync128();
                if (*sm.flag) break;
                const double iv = sm.inv[k];
                if (tid > k && tid < nb) D[tid * kNb + k] *= iv;
                sync128();
                const int s = nb - k - 1;
                if (tid < s * (s + 1) / 2) {
                    const int r = k + 1 + tri_r[tid], c = k + 1 + tri_c[tid];
                    D[r * kNb + c] = fma(-D[r * kNb + k], D[c * kNb + k], D[r * kNb + c]);
                }
                sync128();
            }
            if (wid == 0 && !*sm.flag) {
                for (int c = 0; c < nb; ++c) {
                    if (lane == 0) sm.ys[c0 + c] *= sm.inv[c];
                    __syncwarp();
                    const double yc = sm.ys[c0 + c];
                    if (lane > c && lane < nb) sm.ys[c0 + lane] = fma(-D[lane * kNb + c], yc, sm.ys[c0 + lane]);
                    __syncwarp();
                }
            }
        }
        __syncthreads();
        if (*sm.flag) { failed = true; break; }  // identical in every CTA: all stop together
        // (D) own rows of the diagonal block take L; own rows below become panel rows
        const int first_below = (t0 > rank) ? (t0 - rank + C - 1) / C : 0;  // first own il with i >= t0
        const int npr = max(0, nown - first_below);
        for (int t = tid; t < nown * nb; t += blockDim.x) {
            const int il = t / nb, c = t % nb, i = il * C + rank;
            if (i >= c0 && i < t0 && c <= i - c0) sm.A[(size_t)il * P + c0 + c] = D[(i - c0) * kNb + c];
        }
        for (int c = 0; c < nb; ++c) {  // right-looking triangular solve of the panel, spread over the CTA
            for (int t = tid; t < npr; t += blockDim.x) {
                const int il = first_below + t;
                double *row = sm.A + (size_t)il * P + c0;
                const double v = row[c] * sm.inv[c];
                row[c] = v;
                sm.b[il] = fma(-v, sm.ys[c0 + c], sm.b[il]);
            }
            __syncthreads();
            const int rest = nb - c - 1;
            for (int t = tid; t < npr * rest; t += blockDim.x) {
                const int il = first_below + t / rest, c2 = c + 1 + t % rest;
                double *row = sm.A + (size_t)il * P + c0;
                row[c2] = fma(-row[c], D[c2 * kNb + c], row[c2]);
            }
            __syncthreads();
        }
        for (int t = tid; t < npr * nb * C; t += blockDim.x) {  // push the panel rows to every CTA
            const int q = t % C, e = t / C, il = first_below + e / nb, c = e % nb;
            const int jj = il * C + rank - t0;
            rptr(sm.PLt, q)[(size_t)c * P + jj] = sm.A[(size_t)il * P + c0 + c];
        }
        __syncthreads();
        csync();  // (E) the whole panel is here
        // (F) trailing update of own rows: A_ij -= sum_c L_ic L_jc for t0 <= j <= i
        for (int il = first_below + wid; il < nown; il += nw) {
            const int i = il * C + rank, ii = i - t0;
            double *row = sm.A + (size_t)il * P;
            for (int j = t0 + lane; j <= i; j += 32) {
                const int jj = j - t0;
                double v = row[j];
#pragma unroll 4
                for (int c = 0; c < nb; ++c) v = fma(-sm.PLt[(size_t)c * P + ii], sm.PLt[(size_t)c * P + jj], v);
                row[j] = v;
            }
        }
        __syncthreads();
        if (kb + 1 < nblk) push_diag(kb + 1);
    }
    if (failed) {
        if (rank == 0 && tid == 0) atomicCAS(w.status, 0, (int)QNG_ERR_NOT_SPD);
        csync();
        return;
    }
    // back substitution L^T x = y, last block first; ys turns into x block by block
    for (int kb = nblk - 1; kb >= 0; --kb) {
        const int c0 = kb * kNb, nb = min(kNb, P - c0), t0 = c0 + nb;
        double *part = sm.part + (kb & 1) * C * kNb;
        const double *D = sm.Ld + (size_t)kb * kNb * kNb;
        for (int c = wid; c < nb; c += nw) {  // partial sums over own rows below the block, one warp per column
            double v = 0.0;
            for (int il = lane; il < nown; il += 32) {
                const int i = il * C + rank;
                if (i >= t0) v = fma(sm.A[(size_t)il * P + c0 + c], sm.ys[i], v);
            }
            v = warp_sum(v);
            if (lane < C) rptr(part, lane)[rank * kNb + c] = v;
        }
        __syncthreads();
        csync();
        if (wid == 0) {
            if (lane < nb) {
                double sacc = 0.0;
                for (int r = 0; r < C; ++r) sacc += part[r * kNb + lane];
                sm.ys[c0 + lane] -= sacc;
                sm.inv[lane] = 1.0 / D[lane * kNb + lane];
            }
            __syncwarp();
            for (int c = nb - 1; c >= 0; --c) {
                if (lane == 0) sm.ys[c0 + c] *= sm.inv[c];
                __syncwarp();
                const double xc = sm.ys[c0 + c];
                if (lane < c) sm.ys[c0 + lane] = fma(-D[c * kNb + lane], xc, sm.ys[c0 + lane]);
                __syncwarp();
            }
        }
        __syncthreads();
    }
    if (rank == 0)
        for (int k = tid; k < P; k += blockDim.x) a.dtheta_out[in.param_off + k] = sm.ys[k];
    csync();
}

size_t solve_smem_bytes(int P, int cl) {
    const int C = 1 << cl, R = (P + C - 1) / C, nblk = (P + kNb - 1) / kNb;
    return sizeof(double) * ((size_t)R * P + (size_t)kNb * P + (size_t)nblk * kNb * kNb + P + 2 * C * kNb + R + kNb) + 16;
}

// ------------------------------------------------------------------------------------------
// launchers
template <typename K, typename... Args>
static cudaError_t launch_cluster(K kern, int grid, int threads, size_t smem, int cl, cudaStream_t st, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    if (cl > 0) {
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = 1u << cl;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
    }
    return cudaLaunchKernelEx(&cfg, kern, args...);
}

template <typename K> static cudaError_t set_attrs(K kern, size_t smem) {
    cudaError_t e = raise_smem_limit(reinterpret_cast<const void *>(kern), smem);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
}

// smem_fwd / smem_col: the largest dynamic shared memory any group launches the kernels with
cudaError_t prepare_kernels(int precision, size_t smem_fwd, size_t smem_col, size_t smem_col_im) {
    cudaError_t e;
    if (precision == QNG_C128) {
        if ((e = set_attrs(k_forward<double, 0>, smem_fwd)) != cudaSuccess) return e;
        if ((e = set_attrs(k_forward<double, 1>, smem_fwd)) != cudaSuccess) return e;
        if ((e = set_attrs(k_columns<double, 0, 0>, smem_col)) != cudaSuccess) return e;
        if ((e = set_attrs(k_columns<double, 0, 1>, smem_col)) != cudaSuccess) return e;
        if ((e = set_attrs(k_columns<double, 1, 0>, smem_col_im)) != cudaSuccess) return e;
        return set_attrs(k_columns<double, 1, 1>, smem_col_im);
    }
    if ((e = set_attrs(k_forward<float, 0>, smem_fwd)) != cudaSuccess) return e;
    if ((e = set_attrs(k_forward<float, 1>, smem_fwd)) != cudaSuccess) return e;
    if ((e = set_attrs(k_columns<float, 0, 0>, smem_col)) != cudaSuccess) return e;
    if ((e = set_attrs(k_columns<float, 0, 0, 1>, smem_col)) != cudaSuccess) return e;
    if ((e = set_attrs(k_columns<float, 1, 0, 1>, smem_col_im)) != cudaSuccess) return e;
    if ((e = set_attrs(k_columns<float, 0, 1>, smem_col)) != cudaSuccess) return e;
    if ((e = set_attrs(k_columns<float, 1, 0>, smem_col_im)) != cudaSuccess) return e;
    return set_attrs(k_columns<float, 1, 1>, smem_col_im);
}

// theta <- theta + dtheta (the parameter update of Eq. 3), skipped once the device status word
// holds an error so that a failed solve leaves theta at its last good value.
__global__ void k_theta_update(double *theta, const double *dtheta, int64_t total, const int32_t *status) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= total || *status != 0) return;
    theta[k] += dtheta[k];
}

cudaError_t launch_theta_update(const Work &w, double *theta, const double *dtheta, int64_t total, cudaStream_t st) {
    if (total <= 0) return cudaSuccess;
    const int t = 256;
    k_theta_update<<<(unsigned)((total + t - 1) / t), t, 0, st>>>(theta, dtheta, total, w.status);
    return cudaGetLastError();
}

cudaError_t launch_coef(const Work &w, const double *theta, int64_t total, cudaStream_t st) {
    if (total <= 0) return cudaSuccess;
    const int t = 256;
    k_coef<<<(unsigned)((total + t - 1) / t), t, 0, st>>>(theta, w.coef, w.pctrl, total, w.status);
    return cudaGetLastError();
}

cudaError_t launch_forward(const Work &w, const Group &g, int precision, int want_eta, cudaStream_t st, int k_begin,
                           int k_end, int last) {
    if (g.num_inst == 0) return cudaSuccess;
    const int grid = g.num_inst << g.fwd_cl;
#define QNG_FWD(RT, G) launch_cluster(k_forward<RT, G>, grid, g.fwd_threads, g.smem_fwd, g.fwd_cl, st, w, g.first_inst, g.fwd_cl, \
                                      want_eta, k_begin, k_end, last)
    if (precision == QNG_C128) return g.general ? QNG_FWD(double, 1) : QNG_FWD(double, 0);
    return g.general ? QNG_FWD(float, 1) : QNG_FWD(float, 0);
#undef QNG_FWD
}

cudaError_t launch_columns(const Work &w, const Group &g, int precision, int with_metric, int with_grad,
                           int metric_im, cudaStream_t st) {
    int first, num;
    if (with_metric && with_grad) { first = g.first_work; num = g.num_work; }
    else if (with_metric)         { first = g.first_met; num = g.num_met; }
    else                          { first = g.first_grad; num = g.num_grad; }
    return launch_columns_range(w, g, precision, metric_im, first, num, true, st);
}

cudaError_t launch_columns_range(const Work &w, const Group &g, int precision, int metric_im, int first, int num,
                                 bool persistent, cudaStream_t st) {
    if (num == 0) return cudaSuccess;
    int *queue = nullptr;
    int clusters = num;
    if (persistent && g.queue && g.resident_clusters > 0 && g.resident_clusters < num) {
        queue = g.queue;
        clusters = g.resident_clusters;
        cudaError_t e = cudaMemsetAsync(queue, 0, sizeof(int), st);
        if (e != cudaSuccess) return e;
    }
    const int grid = clusters << g.cl;
    const size_t smem = metric_im ? g.smem_col_im : g.smem_col;
#define QNG_COLS(RT, M, G) launch_cluster(k_columns<RT, M, G>, grid, g.threads, smem, g.cl, st, w, first, g.cl, g.max_P, queue, num)
    if (precision == QNG_C128) {
        if (metric_im) return g.general ? QNG_COLS(double, 1, 1) : QNG_COLS(double, 1, 0);
        return g.general ? QNG_COLS(double, 0, 1) : QNG_COLS(double, 0, 0);
    }
    if (g.num_inst == 1 && !g.general) {  // a single instance: the instantiation with composed Z runs
        if (metric_im) return launch_cluster(k_columns<float, 1, 0, 1>, grid, g.threads, smem, g.cl, st, w, first, g.cl, g.max_P, queue, num);
        return launch_cluster(k_columns<float, 0, 0, 1>, grid, g.threads, smem, g.cl, st, w, first, g.cl, g.max_P, queue, num);
    }
    if (metric_im) return g.general ? QNG_COLS(float, 1, 1) : QNG_COLS(float, 1, 0);
    return g.general ? QNG_COLS(float, 0, 1) : QNG_COLS(float, 0, 0);
#undef QNG_COLS
}

// Clusters of this group's column kernel that fit on the GPU at once (0 if unknown).
int resident_clusters(const Group &g, int precision) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(1u << g.cl);
    cfg.blockDim = dim3(g.threads);
    cfg.dynamicSmemBytes = g.smem_col;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 1u << g.cl;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    cudaError_t e;
    if (precision == QNG_C128)
        e = g.general ? cudaOccupancyMaxActiveClusters(&n, k_columns<double, 0, 1>, &cfg)
                      : cudaOccupancyMaxActiveClusters(&n, k_columns<double, 0, 0>, &cfg);
    else
        e = g.general ? cudaOccupancyMaxActiveClusters(&n, k_columns<float, 0, 1>, &cfg)
                      : cudaOccupancyMaxActiveClusters(&n, k_columns<float, 0, 0>, &cfg);
    if (e != cudaSuccess) { cudaGetLastError(); return 0; }
    return n;
}

cudaError_t prepare_solve(size_t smem) {
    return raise_smem_limit(reinterpret_cast<const void *>(k_solve), smem);
}

cudaError_t launch_solve(const Work &w, int count, int max_P, int cl, const LaunchArgs &a, cudaStream_t st) {
    const size_t smem = solve_smem_bytes(max_P, cl);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)count << cl);
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    if (cl > 0) {
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = 1u << cl;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
    }
    return cudaLaunchKernelEx(&cfg, k_solve, w, a, cl);
}

cudaError_t launch_finish(const Work &w, int count, int max_P, const LaunchArgs &a, cudaStream_t st) {
    const int t = max_P >= 128 ? 512 : 128;
    k_finish<<<count, t, 0, st>>>(w, a);
    return cudaGetLastError();
}

}  // namespace qng

// Mixed-precision solve of (g + lambda I) dtheta = -dt grad (Eq. 3): float32 Cholesky
// factorisation, float64 iterative refinement.
//
// On GB300 a dependent float64 operation takes 64 cycles and a float64 rsqrt about 374, so the
// P sequential pivots of a float64 factorisation cost some 500-700 cycles each; float32 takes
// 4.5 and about 40. Here A = g + lambda I is assembled in float64 and factored in float32,
// A ~ L L^T; then, with x_0 = 0,
//   r_k = b - A x_k (float64),   d_k = L^-T L^-1 r_k (float32),   x_{k+1} = x_k + d_k,
// which converges to the float64 solution at a rate of about cond(A) times float32 rounding
// (a few iterations for the metrics of this method, whose condition numbers are in the 10^3 range
// with lambda = 1e-3). The step stops when the error the last correction leaves, estimated as
// the correction times its ratio to the previous one, is below 1e-13 of x, or when it stops
// shrinking. The result is accepted on two tests: the estimated error is at most 1e-12 of |x|, and
// a final residual r = b - A x computed in float64 gives a normwise backward error
// |r|_inf / (|A|_inf |x|_inf + |b|_inf) of at most 2 P eps (eps = 2^-53, the bound of a
// backward-stable float64 solve up to the rounding of r itself). A float32 pivot that is not
// positive, or a result that fails either test, marks the instance for the float64 cluster solve
// (k_solve), which is launched right after and stands down for the instances this kernel finished.
//
// One cluster of C CTAs (512 threads) per instance. CTA 0 holds the float32 matrix (full square,
// row stride P + 1) and does the factorisation and the triangular solves; CTAs 1..C-1 hold the
// float64 rows of A (contiguous slices) and take the residual.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "qng_internal.h"

namespace cg = cooperative_groups;

namespace qng {

namespace {

constexpr int kIb = 16;        // block width of the triangular solves
constexpr int kIrMaxIter = 12; // refinement steps at most

struct IrGeom {
    int P, C, R;     // rows of A per CTA of rank >= 1
    int ld;          // row stride of the float32 matrix
    int Pp;          // P rounded up to 16 (row length of the transposed panel)
    size_t o_xt, o_di, o_y, o_x;  // float offsets in CTA 0's shared memory
    size_t smem;
};

__host__ __device__ inline size_t up4(size_t x) { return (x + 3) & ~(size_t)3; }

__host__ __device__ inline IrGeom ir_geom(int P, int C) {
    IrGeom g;
    g.P = P;
    g.C = C;
    g.R = (P + C - 2) / (C - 1);
    g.ld = P + 1;
    g.Pp = (P + kIb - 1) / kIb * kIb;
    const int nblk = (P + kIb - 1) / kIb;
    g.o_xt = up4((size_t)P * g.ld);                  // Lm [P][ld]
    g.o_di = g.o_xt + (size_t)kIb * g.Pp;             // Xt [16][Pp], 16-byte aligned rows
    g.o_y = g.o_di + (size_t)nblk * kIb * kIb;        // Di [nblk][16][16]
    g.o_x = up4(g.o_y + (size_t)P);                   // yv [P]; then float64 x, r
    const size_t cta0 = sizeof(float) * g.o_x + sizeof(double) * 2 * (size_t)P;
    const size_t other = sizeof(double) * ((size_t)g.R * P + P);
    g.smem = cta0 > other ? cta0 : other;
    return g;
}

// One warp: the diagonal block at (k0, k0) of the float32 matrix (row stride ld), already updated
// by every earlier panel, with nb <= 16 real rows (the rest padded with the identity) -> its
// Cholesky factor L_K in place and L_K^-1 in D (16 x 16, zero past nb). Lane r holds row r; a
// column takes one rsqrt, and 1/L_cc = rsqrt(d) also serves the inverse. False if a pivot is not
// positive.
__device__ __noinline__ bool chol_diag16(float *Lm, int ld, int k0, int nb, float *D, int lane) {
    float row[kIb], rdiag[kIb];
#pragma unroll
    for (int c = 0; c < kIb; ++c)
        row[c] = (lane < nb) ? (c <= lane ? Lm[(size_t)(k0 + lane) * ld + k0 + c] : 0.0f) : (lane == c ? 1.0f : 0.0f);
    bool bad = false;
#pragma unroll
    for (int c = 0; c < kIb; ++c) {
        const float d = __shfl_sync(0xffffffffu, row[c], c);
        bad = bad || !(d > 0.0f);
        const float ri = rsqrtf(d);
        rdiag[c] = ri;
        const float lc = (lane == c) ? d * ri : row[c] * ri;
        if (lane >= c) row[c] = lc;
#pragma unroll
        for (int j = c + 1; j < kIb; ++j) {
            const float lj = __shfl_sync(0xffffffffu, lc, j);  // L[j][c]
            if (lane >= j) row[j] = fmaf(-lc, lj, row[j]);
        }
    }
    if (lane < nb) {
#pragma unroll
        for (int c = 0; c < kIb; ++c)
            if (c <= lane) Lm[(size_t)(k0 + lane) * ld + k0 + c] = row[c];
    }
    // lane c (mod 16) forms column c of L_K^-1 by forward substitution, rows taken from the warp
    const int c = lane & (kIb - 1);
    float xc[kIb];
#pragma unroll
    for (int r = 0; r < kIb; ++r) {
        float sum = (r == c) ? 1.0f : 0.0f;
#pragma unroll
        for (int m = 0; m < r; ++m) sum = fmaf(-__shfl_sync(0xffffffffu, row[m], r), xc[m], sum);
        xc[r] = (r >= c) ? sum * rdiag[r] : 0.0f;
    }
    if (lane < kIb) {
#pragma unroll
        for (int r = 0; r < kIb; ++r) D[r * kIb + c] = (r < nb && c < nb) ? xc[r] : 0.0f;
    }
    return !bad;
}

}  // namespace

size_t solve_ir_smem_bytes(int P, int C) { return ir_geom(P, C).smem + 64; }

__global__ void __launch_bounds__(512, 1) k_solve_ir(Work w, LaunchArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_fail, s_done;
    __shared__ double s_est;
    __shared__ float s_red[2][16];
    const int C = (int)cg::this_cluster().num_blocks();
    const int b = blockIdx.x / C;
    const int rank = (int)cg::this_cluster().block_rank();
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nwarp = blockDim.x >> 5, nt = blockDim.x;
    const DevInst in = w.inst[b];
    const int P = in.P;
    const IrGeom G = ir_geom(P, C);
    const int nblk = (P + kIb - 1) / kIb;
    const double *sg = w.sigma + in.param_off;
    const double *pc = w.pctrl + in.param_off;
    const double *L = w.L + in.metric_off;
    const double *gr = w.gradraw + in.param_off;
    auto cl = cg::this_cluster();

    // CTA 0: float32 matrix, inverse diagonal blocks, float64 x, r and the float32 work vector
    float *Lm = reinterpret_cast<float *>(smem);                       // [P][ld]
    float *Xt = Lm + G.o_xt;                                           // [16][Pp]: the panel, transposed
    float *Di = Lm + G.o_di;                                           // [nblk][16][16]
    float *yv = Lm + G.o_y;                                            // [P]
    double *xv = reinterpret_cast<double *>(Lm + G.o_x);               // [P]
    double *rv = xv + P;                                               // [P]
    // CTAs >= 1: float64 rows [r0, r1) of A and a copy of x
    double *Arow = reinterpret_cast<double *>(smem);                   // [R][P]
    double *xc = Arow + (size_t)G.R * P;                               // [P]
    const int r0 = rank > 0 ? min(P, (rank - 1) * G.R) : 0, r1 = rank > 0 ? min(P, rank * G.R) : 0;

    if (tid == 0) { s_fail = 0; s_done = 0; }
    cl.sync();  // every CTA runs before the first distributed shared memory store

    // (A) assembly (Eq. g_t_L_def): float64 rows in CTAs >= 1, g for those rows, and the float32
    // lower triangle pushed to CTA 0
    if (rank > 0) {
        float *L0 = cl.map_shared_rank(Lm, 0);
        for (int t = tid; t < (r1 - r0) * P; t += nt) {
            const int il = t / P, j = t % P, i = r0 + il;
            double v;
            if (i == j) v = 0.25 * (pc[i] - sg[i] * sg[i]);
            else if (i < j) v = L[(int64_t)i * P + j] - 0.25 * sg[i] * sg[j];
            else v = L[(int64_t)j * P + i] - 0.25 * sg[i] * sg[j];
            if (a.g_out) a.g_out[in.metric_off + (int64_t)i * P + j] = v;
            v += (i == j ? a.lambda : 0.0);
            Arow[t] = v;
            if (j <= i) L0[(size_t)i * G.ld + j] = (float)v;
        }
    }
    cl.sync();

    // (B) CTA 0: float32 Cholesky in place (lower triangle), blocked by 16 with look-ahead. Warp 0
    // factors diagonal block K + 1 in registers (and inverts it) while the other warps apply the
    // rank-16 update of panel K to the rest of the trailing triangle; the panel itself is
    // X = A_panel D_K^-T, one independent 16-term dot product per entry. Two barriers per block.
    if (rank == 0) {
        // kb = -1 only factors block 0; block kb is full whenever block kb + 1 exists
        for (int kb = -1; !s_fail; ++kb) {
            const int k0 = kb * kIb, nb = kIb, k1 = k0 + nb;
            if (k1 >= P) break;  // no block kb + 1
            // panel: X[i][c] = sum_{m <= c} A[i][m] Dinv[c][m], also into Xt (zero past P)
            const float *D = Di + (size_t)max(kb, 0) * kIb * kIb;
            for (int i = k1 + tid; kb >= 0 && i < G.Pp; i += nt) {
                float x[kIb];
                if (i < P) {
                    float av[kIb];
                    float *rowp = Lm + (size_t)i * G.ld + k0;
#pragma unroll
                    for (int mm = 0; mm < kIb; ++mm) av[mm] = (mm < nb) ? rowp[mm] : 0.0f;
#pragma unroll
                    for (int cc = 0; cc < kIb; ++cc) {
                        float v = 0.0f;
#pragma unroll
                        for (int mm = 0; mm <= cc; ++mm) v = fmaf(av[mm], D[cc * kIb + mm], v);
                        x[cc] = v;
                    }
#pragma unroll
                    for (int cc = 0; cc < kIb; ++cc)
                        if (cc < nb) rowp[cc] = x[cc];
                } else {
#pragma unroll
                    for (int cc = 0; cc < kIb; ++cc) x[cc] = 0.0f;
                }
#pragma unroll
                for (int cc = 0; cc < kIb; ++cc) Xt[(size_t)cc * G.Pp + i] = (cc < nb) ? x[cc] : 0.0f;
            }
            __syncthreads();
            // look-ahead: warp 0 updates and factors the next diagonal block; the other warps take
            // the rest of the trailing triangle in 4 x 4 tiles (those of the next block skipped)
            const int nb2 = min(kIb, P - k1);
            const int mrem = P - k1, mt = (mrem + 3) >> 2, ntile = mt * (mt + 1) / 2;
            const int t2 = (nb2 + 3) >> 2, skip = t2 * (t2 + 1) / 2;  // tiles inside the next block
            if (wid == 0) {
                // A[r][j] -= sum_c X[r][c] X[j][c] for r, j in block kb + 1, j <= r: lane (r, half)
                // takes j in [8 half, 8 half + 8), eight independent sums (Xt is zero past P)
                const int r = lane & (kIb - 1), jh = (lane >> 4) * 8;
                if (kb >= 0 && r < nb2 && jh <= r) {
                    float acc[8];
#pragma unroll
                    for (int q = 0; q < 8; ++q) acc[q] = 0.0f;
#pragma unroll
                    for (int cc = 0; cc < kIb; ++cc) {
                        const float *xrow = Xt + (size_t)cc * G.Pp + k1;
                        const float xr = xrow[r];
                        const float4 u = *reinterpret_cast<const float4 *>(xrow + jh);
                        const float4 v = *reinterpret_cast<const float4 *>(xrow + jh + 4);
                        acc[0] = fmaf(xr, u.x, acc[0]);
                        acc[1] = fmaf(xr, u.y, acc[1]);
                        acc[2] = fmaf(xr, u.z, acc[2]);
                        acc[3] = fmaf(xr, u.w, acc[3]);
                        acc[4] = fmaf(xr, v.x, acc[4]);
                        acc[5] = fmaf(xr, v.y, acc[5]);
                        acc[6] = fmaf(xr, v.z, acc[6]);
                        acc[7] = fmaf(xr, v.w, acc[7]);
                    }
                    float *arow = Lm + (size_t)(k1 + r) * G.ld + k1 + jh;
#pragma unroll
                    for (int q = 0; q < 8; ++q)
                        if (jh + q <= r) arow[q] -= acc[q];
                }
                __syncwarp();
                const bool ok = chol_diag16(Lm, G.ld, k1, min(kIb, P - k1), Di + (size_t)(kb + 1) * kIb * kIb, lane);
                if (!ok && lane == 0) s_fail = 1;
            } else if (kb >= 0) {
                for (int t = skip + tid - 32; t < ntile; t += nt - 32) {
                    int ti = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
                    while (ti * (ti + 1) / 2 > t) --ti;
                    while ((ti + 1) * (ti + 2) / 2 <= t) ++ti;
                    const int tj = t - ti * (ti + 1) / 2;
                    const int i0 = k1 + 4 * ti, j0 = k1 + 4 * tj;
                    float acc[4][4];
#pragma unroll
                    for (int u = 0; u < 4; ++u)
#pragma unroll
                        for (int v = 0; v < 4; ++v) acc[u][v] = 0.0f;
#pragma unroll 4
                    for (int cc = 0; cc < kIb; ++cc) {
                        const float4 xa = *reinterpret_cast<const float4 *>(Xt + (size_t)cc * G.Pp + i0);
                        const float4 xb = *reinterpret_cast<const float4 *>(Xt + (size_t)cc * G.Pp + j0);
                        const float av[4] = {xa.x, xa.y, xa.z, xa.w}, bv[4] = {xb.x, xb.y, xb.z, xb.w};
#pragma unroll
                        for (int u = 0; u < 4; ++u)
#pragma unroll
                            for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(av[u], bv[v], acc[u][v]);
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u)
#pragma unroll
                        for (int v = 0; v < 4; ++v) {
                            const int i = i0 + u, j = j0 + v;
                            if (i < P && j <= i) Lm[(size_t)i * G.ld + j] -= acc[u][v];
                        }
                }
            }
            __syncthreads();
        }
        for (int i = tid; i < P; i += nt) { xv[i] = 0.0; rv[i] = -a.dt * gr[i]; }
        __syncthreads();
    }
    // the failure flag to every CTA (all stop together)
    if (rank == 0 && tid == 0)
        for (int q = 1; q < C; ++q) *cl.map_shared_rank(&s_fail, q) = s_fail;
    cl.sync();
    bool fallback = s_fail != 0;

    // (C) refinement: CTA 0 solves L L^T d = r in float32 and updates x; CTAs >= 1 take r = b - A x
    double dn_prev = 0.0;
    double en = 0.0, xn = 0.0;
    for (int it = 0; !fallback && it < kIrMaxIter; ++it) {
        if (rank == 0) {
            for (int i = tid; i < P; i += nt) yv[i] = (float)rv[i];
            __syncthreads();
            __shared__ float s_blk[kIb];
            // forward L y = r by blocks: y_K = D_K^-1 y_K (16 threads), then every row below at once
            for (int kb = 0; kb < nblk; ++kb) {
                const int k0 = kb * kIb, nb = min(kIb, P - k0), k1 = k0 + nb;
                if (tid < nb) {  // row tid of D: zero past the diagonal, so a fixed 16 terms
                    const float *D = Di + (size_t)kb * kIb * kIb + tid * kIb;
                    float t0 = 0.0f, t1 = 0.0f;
#pragma unroll
                    for (int m = 0; m < kIb; m += 2) {
                        t0 = fmaf(D[m], (m < nb) ? yv[k0 + m] : 0.0f, t0);
                        t1 = fmaf(D[m + 1], (m + 1 < nb) ? yv[k0 + m + 1] : 0.0f, t1);
                    }
                    s_blk[tid] = t0 + t1;
                }
                __syncthreads();
                if (tid < nb) yv[k0 + tid] = s_blk[tid];
                for (int i = k1 + tid; i < P; i += nt) {  // rows below K exist only when K is full
                    const float *row = Lm + (size_t)i * G.ld + k0;
                    float s0 = yv[i], s1 = 0.0f;
#pragma unroll
                    for (int m = 0; m < kIb; m += 2) {
                        s0 = fmaf(-row[m], s_blk[m], s0);
                        s1 = fmaf(-row[m + 1], s_blk[m + 1], s1);
                    }
                    yv[i] = s0 + s1;
                }
                __syncthreads();
            }
            // back L^T d = y by blocks from the end: warp c forms t_c = y_c - sum_{i >= k1} L[i][c] d_i,
            // then 16 threads take d_K = D_K^-T t
            for (int kb = nblk - 1; kb >= 0; --kb) {
                const int k0 = kb * kIb, nb = min(kIb, P - k0), k1 = k0 + nb;
                if (wid < nb) {
                    float sacc = 0.0f;
                    for (int i = k1 + lane; i < P; i += 32) sacc = fmaf(Lm[(size_t)i * G.ld + k0 + wid], yv[i], sacc);
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) sacc += __shfl_xor_sync(0xffffffffu, sacc, o);
                    if (lane == 0) s_blk[wid] = yv[k0 + wid] - sacc;
                }
                __syncthreads();
                if (tid < nb) {  // column tid of D: zero above the diagonal and past nb
                    const float *D = Di + (size_t)kb * kIb * kIb;
                    float v0 = 0.0f, v1 = 0.0f;
#pragma unroll
                    for (int m = 0; m < kIb; m += 2) {
                        v0 = fmaf(D[m * kIb + tid], (m < nb) ? s_blk[m] : 0.0f, v0);
                        v1 = fmaf(D[(m + 1) * kIb + tid], (m + 1 < nb) ? s_blk[m + 1] : 0.0f, v1);
                    }
                    yv[k0 + tid] = v0 + v1;
                }
                __syncthreads();
            }
            // x += d; max |d| and max |x| (float32 magnitudes decide as well as float64 ones)
            float md = 0.0f, mx = 0.0f;
            for (int i = tid; i < P; i += nt) {
                const float d = yv[i];
                const double x = xv[i] + (double)d;
                xv[i] = x;
                md = fmaxf(md, fabsf(d));
                mx = fmaxf(mx, fabsf((float)x));
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                md = fmaxf(md, __shfl_xor_sync(0xffffffffu, md, o));
                mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            }
            if (lane == 0) { s_red[0][wid] = md; s_red[1][wid] = mx; }
            __syncthreads();
            if (tid == 0) {
                float a0 = 0.0f, a1 = 0.0f;
                for (int q = 0; q < nwarp; ++q) { a0 = fmaxf(a0, s_red[0][q]); a1 = fmaxf(a1, s_red[1][q]); }
                s_red[0][0] = a0;
                s_red[1][0] = a1;
                // error left after this correction: itself, or itself times its ratio to the last
                const double a0d = a0;
                s_est = it == 0 ? a0d : fmin(a0d, a0d * a0d / dn_prev);
                // done when the correction is negligible, or when the error it leaves (about the
                // correction times its ratio to the previous one) is, or when it stops shrinking
                const bool small = (double)a0 <= 1e-14 * a1 || (it >= 2 && (double)a0 * a0 <= 1e-13 * a1 * dn_prev);
                const bool stalled = it >= 2 && a0 > 0.5 * dn_prev;
                s_done = (small || stalled || it + 1 == kIrMaxIter) ? 1 : 0;
            }
            __syncthreads();
            dn_prev = s_red[0][0];
            en = s_est;
            xn = s_red[1][0];
            // x and the decision to every CTA
            for (int q = 1; q < C; ++q) {
                double *xr = cl.map_shared_rank(xc, q);
                for (int i = tid; i < P; i += nt) xr[i] = xv[i];
                if (tid == 0) *cl.map_shared_rank(&s_done, q) = s_done;
            }
        }
        cl.sync();
        if (s_done) break;
        // r = b - A x over the own rows (a warp per row), into CTA 0
        if (rank > 0) {
            double *r0p = cl.map_shared_rank(rv, 0);
            for (int il = wid; il < r1 - r0; il += nwarp) {
                const double *row = Arow + (size_t)il * P;
                double s = 0.0;
                for (int j = lane; j < P; j += 32) s = fma(row[j], xc[j], s);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
                if (lane == 0) r0p[r0 + il] = -a.dt * gr[r0 + il] - s;
            }
        }
        cl.sync();
    }
    // (D) computed backward error of the final x: CTAs >= 1 take r = b - A x over their own rows
    // with the row sums of |A| (x is the copy CTA 0 pushed before the last barrier) and hand their
    // maxima of |r_i|, sum_j |A_ij| and |b_i| to CTA 0
    __shared__ double s_wmax[3][32];
    __shared__ double s_rmax[3][8];
    if (!fallback && rank > 0) {
        double mr = 0.0, ma = 0.0, mb = 0.0;
        for (int il = wid; il < r1 - r0; il += nwarp) {
            const double *row = Arow + (size_t)il * P;
            double s = 0.0, sa = 0.0;
            for (int j = lane; j < P; j += 32) {
                s = fma(row[j], xc[j], s);
                sa += fabs(row[j]);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                s += __shfl_xor_sync(0xffffffffu, s, o);
                sa += __shfl_xor_sync(0xffffffffu, sa, o);
            }
            const double bi = -a.dt * gr[r0 + il];
            mr = fmax(mr, fabs(bi - s));
            ma = fmax(ma, sa);
            mb = fmax(mb, fabs(bi));
        }
        if (lane == 0) { s_wmax[0][wid] = mr; s_wmax[1][wid] = ma; s_wmax[2][wid] = mb; }
        __syncthreads();
        if (tid < 3) {
            double m = 0.0;
            for (int q = 0; q < nwarp; ++q) m = fmax(m, s_wmax[tid][q]);
            *cl.map_shared_rank(&s_rmax[tid][rank], 0) = m;
        }
    }
    cl.sync();
    // outputs, or the float64 solve's turn
    if (rank == 0) {
        if (!fallback) {
            double mr = 0.0, ma = 0.0, mb = 0.0;
            for (int q = 1; q < C; ++q) {
                mr = fmax(mr, s_rmax[0][q]);
                ma = fmax(ma, s_rmax[1][q]);
                mb = fmax(mb, s_rmax[2][q]);
            }
            const bool backward_ok = mr <= 2.0 * P * 0x1p-53 * (ma * xn + mb);
            if (!(en <= 1e-12 * xn) || !backward_ok) fallback = true;
        }
        if (tid == 0) w.irflag[b] = fallback ? 1 : 0;
        if (!fallback)
            for (int i = tid; i < P; i += nt) a.dtheta_out[in.param_off + i] = xv[i];
        if (a.grad_out)
            for (int k = tid; k < P; k += nt) a.grad_out[in.param_off + k] = gr[k];
        if (a.sigma_out)
            for (int k = tid; k < P; k += nt) a.sigma_out[in.param_off + k] = sg[k];
        if (a.energy_out && tid == 0) a.energy_out[b] = w.energy[b];
    }
    cl.sync();
}

cudaError_t prepare_solve_ir(int P, int C) {
    return raise_smem_limit(reinterpret_cast<const void *>(k_solve_ir), solve_ir_smem_bytes(P, C));
}

cudaError_t launch_solve_ir(const Work &w, int count, int max_P, int C, const LaunchArgs &a, cudaStream_t st) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(count * C));
    cfg.blockDim = dim3(512);
    cfg.dynamicSmemBytes = solve_ir_smem_bytes(max_P, C);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_solve_ir, w, a);
}

}  // namespace qng

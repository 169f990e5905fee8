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
// the correction times its ratio to the previous one, is below 1e-15 of x, or when it stops
// shrinking. A float32 pivot that is not positive, or a correction still above 1e-10 of x when it
// stops, marks the instance for the float64 cluster solve (k_solve), which is launched right after
// and stands down for the instances this kernel finished.
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
    size_t smem;
};

__host__ __device__ inline IrGeom ir_geom(int P, int C) {
    IrGeom g;
    g.P = P;
    g.C = C;
    g.R = (P + C - 2) / (C - 1);
    g.ld = P + 1;
    const size_t cta0 = sizeof(float) * ((size_t)P * g.ld + (size_t)((P + kIb - 1) / kIb) * kIb * kIb + P) +
                        sizeof(double) * 3 * (size_t)P;
    const size_t other = sizeof(double) * ((size_t)g.R * P + P);
    g.smem = cta0 > other ? cta0 : other;
    return g;
}

}  // namespace

size_t solve_ir_smem_bytes(int P, int C) { return ir_geom(P, C).smem + 64; }

__global__ void __launch_bounds__(512) k_solve_ir(Work w, LaunchArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_fail, s_done;
    __shared__ double s_red[2][16];
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
    float *Di = Lm + (size_t)P * G.ld;                                 // [nblk][16][16]
    float *yv = Di + (size_t)nblk * kIb * kIb;                         // [P]
    double *xv = reinterpret_cast<double *>(yv + P + (P & 1));         // [P] (8-byte aligned)
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

    // (B) CTA 0: float32 Cholesky in place (lower triangle), blocked by 16: a warp factors the
    // diagonal block in registers, one thread per row solves the panel, and the trailing lower
    // triangle takes a rank-16 update in 4 x 4 register tiles. Three barriers per block.
    if (rank == 0) {
        __shared__ float s_dinv[kIb];
        for (int kb = 0; kb < nblk; ++kb) {
            const int k0 = kb * kIb, nb = min(kIb, P - k0), k1 = k0 + nb;
            if (wid == 0) {
                // lane r < nb holds row r of the diagonal block
                float row[kIb];
#pragma unroll
                for (int c = 0; c < kIb; ++c)
                    row[c] = (lane < nb && c <= lane) ? Lm[(size_t)(k0 + lane) * G.ld + k0 + c] : 0.0f;
                bool bad = false;
#pragma unroll
                for (int c = 0; c < kIb; ++c) {
                    if (c < nb && !bad) {
                        const float d = __shfl_sync(0xffffffffu, row[c], c);
                        if (!(d > 0.0f)) {
                            bad = true;
                        } else {
                            const float ri = rsqrtf(d);
                            if (lane == c) row[c] = d * ri;
                            else if (lane > c) row[c] *= ri;
                            const float lc = row[c];
#pragma unroll
                            for (int j = c + 1; j < kIb; ++j) {
                                const float lj = __shfl_sync(0xffffffffu, lc, j);  // L[j][c]
                                if (lane >= j) row[j] = fmaf(-lc, lj, row[j]);
                            }
                        }
                    }
                }
                if (lane < nb)
#pragma unroll
                    for (int c = 0; c < kIb; ++c)
                        if (c <= lane) Lm[(size_t)(k0 + lane) * G.ld + k0 + c] = row[c];
                if (lane < nb) s_dinv[lane] = 1.0f / row[lane];
                if (bad && lane == 0) s_fail = 1;
            }
            __syncthreads();
            if (s_fail) break;
            // panel: rows i >= k1, X[i][c] = (A[i][c] - sum_{m<c} X[i][m] L[c][m]) / L[c][c]
            for (int i = k1 + tid; i < P; i += nt) {
                float *row = Lm + (size_t)i * G.ld + k0;
                float x[kIb];
#pragma unroll
                for (int c = 0; c < kIb; ++c) {
                    if (c < nb) {
                        float v = row[c];
#pragma unroll
                        for (int m = 0; m < c; ++m) v = fmaf(-x[m], Lm[(size_t)(k0 + c) * G.ld + k0 + m], v);
                        x[c] = v * s_dinv[c];
                        row[c] = x[c];
                    }
                }
            }
            __syncthreads();
            // trailing update: A[i][j] -= sum_c X[i][c] X[j][c] for k1 <= j <= i < P, 4 x 4 tiles of
            // the lower triangle (tile (ti, tj), tj <= ti), decoded from a linear index
            const int m = P - k1, mt = (m + 3) >> 2, ntile = mt * (mt + 1) / 2;
            for (int t = tid; t < ntile; t += nt) {
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
                for (int c = 0; c < nb; ++c) {
                    float xa[4], xb[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        xa[u] = (i0 + u < P) ? Lm[(size_t)(i0 + u) * G.ld + k0 + c] : 0.0f;
                        xb[u] = (j0 + u < P) ? Lm[(size_t)(j0 + u) * G.ld + k0 + c] : 0.0f;
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u)
#pragma unroll
                        for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(xa[u], xb[v], acc[u][v]);
                }
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int v = 0; v < 4; ++v) {
                        const int i = i0 + u, j = j0 + v;
                        if (i < P && j <= i) Lm[(size_t)i * G.ld + j] -= acc[u][v];
                    }
            }
            __syncthreads();
        }
        // inverses of the 16 x 16 diagonal blocks of L (a warp per block, lane c holds column c)
        if (!s_fail) {
            for (int kb = wid; kb < nblk; kb += nwarp) {
                const int k0 = kb * kIb, nb = min(kIb, P - k0);
                float *D = Di + (size_t)kb * kIb * kIb;  // D[r][c], lower
                const int c = lane & (kIb - 1);
                float xcol[kIb];
#pragma unroll
                for (int r = 0; r < kIb; ++r) xcol[r] = 0.0f;
                // column c of D^-1: forward substitution of e_c (lanes >= 16 duplicate 0..15)
#pragma unroll
                for (int r = 0; r < kIb; ++r) {
                    if (r < nb) {
                        float s = (r == c) ? 1.0f : 0.0f;
#pragma unroll
                        for (int m = 0; m < r; ++m) s = fmaf(-Lm[(size_t)(k0 + r) * G.ld + k0 + m], xcol[m], s);
                        xcol[r] = s / Lm[(size_t)(k0 + r) * G.ld + k0 + r];
                    }
                }
                if (lane < kIb)
#pragma unroll
                    for (int r = 0; r < kIb; ++r) D[r * kIb + c] = (r < nb && c < nb) ? xcol[r] : 0.0f;
            }
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
    double dn = 0.0, xn = 0.0;
    for (int it = 0; !fallback && it < kIrMaxIter; ++it) {
        if (rank == 0) {
            for (int i = tid; i < P; i += nt) yv[i] = (float)rv[i];
            __syncthreads();
            __shared__ float s_blk[kIb];
            // forward L y = r by blocks: y_K = D_K^-1 y_K (16 threads), then every row below at once
            for (int kb = 0; kb < nblk; ++kb) {
                const int k0 = kb * kIb, nb = min(kIb, P - k0), k1 = k0 + nb;
                if (tid < nb) {
                    const float *D = Di + (size_t)kb * kIb * kIb + tid * kIb;
                    float t = 0.0f;
                    for (int m = 0; m <= tid; ++m) t = fmaf(D[m], yv[k0 + m], t);
                    s_blk[tid] = t;
                }
                __syncthreads();
                if (tid < nb) yv[k0 + tid] = s_blk[tid];
                for (int i = k1 + tid; i < P; i += nt) {
                    const float *row = Lm + (size_t)i * G.ld + k0;
                    float s0 = yv[i], s1 = 0.0f;
                    for (int m = 0; m + 1 < nb; m += 2) {
                        s0 = fmaf(-row[m], s_blk[m], s0);
                        s1 = fmaf(-row[m + 1], s_blk[m + 1], s1);
                    }
                    if (nb & 1) s0 = fmaf(-row[nb - 1], s_blk[nb - 1], s0);
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
                if (tid < nb) {
                    const float *D = Di + (size_t)kb * kIb * kIb;
                    float v = 0.0f;
                    for (int m = tid; m < nb; ++m) v = fmaf(D[m * kIb + tid], s_blk[m], v);
                    yv[k0 + tid] = v;
                }
                __syncthreads();
            }
            // x += d; max |d| and max |x|
            double md = 0.0, mx = 0.0;
            for (int i = tid; i < P; i += nt) {
                const double d = (double)yv[i];
                const double x = xv[i] + d;
                xv[i] = x;
                md = fmax(md, fabs(d));
                mx = fmax(mx, fabs(x));
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                md = fmax(md, __shfl_xor_sync(0xffffffffu, md, o));
                mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            }
            if (lane == 0) { s_red[0][wid] = md; s_red[1][wid] = mx; }
            __syncthreads();
            if (tid == 0) {
                double a0 = 0.0, a1 = 0.0;
                for (int q = 0; q < nwarp; ++q) { a0 = fmax(a0, s_red[0][q]); a1 = fmax(a1, s_red[1][q]); }
                s_red[0][0] = a0;
                s_red[1][0] = a1;
                // done when the correction is negligible, or when the error it leaves (about the
                // correction times its ratio to the previous one) is, or when it stops shrinking
                const bool small = a0 <= 1e-14 * a1 || (it >= 2 && a0 * a0 <= 1e-15 * a1 * dn_prev);
                const bool stalled = it >= 2 && a0 > 0.5 * dn_prev;
                s_done = (small || stalled || it + 1 == kIrMaxIter) ? 1 : 0;
            }
            __syncthreads();
            dn = s_red[0][0];
            xn = s_red[1][0];
            dn_prev = dn;
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
    // outputs, or the float64 solve's turn
    if (rank == 0) {
        if (!fallback && !(dn <= 1e-10 * xn)) fallback = true;
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
    return cudaFuncSetAttribute(k_solve_ir, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)solve_ir_smem_bytes(P, C));
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

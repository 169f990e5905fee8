// Block solve of (g + lambda I) dtheta = -dt grad (Eq. 3) for one instance with many parameters.
//
// The cluster solve (k_solve) keeps every row of the matrix in the shared memory of one cluster,
// which stops fitting above P of about 330; k_finish, one CTA, takes O(P^3) float64 work on one SM.
// This solve keeps the Cholesky factor in global memory (L2-resident) and takes one 16-column block
// per launch, so it scales to P of about 1300 on one 8-CTA cluster.
//
// Let J be the reversal (J_kl = 1 when k + l = P - 1) and A = g + lambda I. B = J A J has, below
// its diagonal in column k, the entries of A's column j = P - 1 - k above the diagonal read
// upwards: the (1/4) Re L_ij, i < j, of recurrence column j (Eq. L_recurrent_def), with the
// T_i^* T_j terms of Eq. g_t_L_def from <sigma>. The left-looking blocked factorisation
// B = Lf Lf^T takes block column K (B columns [16K, 16K + 16)) per launch:
//   forward:  Lf y = J(-dt grad)   (block by block, inside the factorisation)
//   back:     Lf^T z = y           (k_sback)
//   result:   dtheta = J z
// Lf is column-major (Lf[k * P + l], l >= k) in the Cholesky scratch. Each 16 x 16 diagonal block
// D_K is also kept as its inverse (lower triangular), so that the panel rows and both
// substitutions are short dot products rather than 16-step chains.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "qng_internal.h"

namespace cg = cooperative_groups;

namespace qng {

namespace {

constexpr int kSb = kSolveBlock;  // block width

__device__ __forceinline__ void sbar128() { asm volatile("bar.sync 2, 128;" ::: "memory"); }

struct SbGeom {
    int k0, nb, k1;  // block columns [k0, k1), nb = k1 - k0
    int per;         // rows below the block per CTA of rank >= 1
    int rows_max;    // row capacity of the per-CTA buffers
    int mch;         // update terms m per CTA
};

__device__ __forceinline__ SbGeom sb_geom(int P, int C, int K) {
    SbGeom g;
    g.k0 = K * kSb;
    g.nb = min(kSb, P - g.k0);
    g.k1 = g.k0 + g.nb;
    g.per = C > 1 ? (P - g.k1 + C - 2) / (C - 1) : 0;
    g.rows_max = sblock_rows_max(P, C);
    g.mch = (g.k0 + C - 1) / C;
    return g;
}

// rows [rb, re) of B owned by CTA q: the diagonal block (and everything with one CTA) in CTA 0,
// the rows below it split evenly over the others
__device__ __forceinline__ void sb_rows(const SbGeom &g, int P, int C, int q, int &rb, int &re) {
    if (q == 0) {
        rb = g.k0;
        re = C == 1 ? P : g.k1;
    } else {
        rb = min(P, g.k1 + (q - 1) * g.per);
        re = min(P, g.k1 + q * g.per);
    }
}

}  // namespace

size_t sblock_smem_bytes(int P, int C) {
    const int rows = sblock_rows_max(P, C);
    const int mch = (P + C - 1) / C;
    // stage[mch][16] + pan[rows][16] + recv[C][rows][16] + Dinv[16][16] + y[16]
    return sizeof(double) * ((size_t)mch * kSb + (size_t)rows * kSb + (size_t)C * rows * kSb + kSb * kSb + kSb);
}

// One block column K of the factorisation; one cluster of C = gridDim.x CTAs (256
// threads). Reads the recurrence output L and <sigma> of columns [P-1-k1+1, P-1-k0] of A, the
// earlier block columns of Lf, and the running right-hand side r (r = J(-dt grad) minus the
// contributions of the earlier blocks, rows l >= k0). Writes Lf columns [k0, k1), the inverse
// of D_K, y_K, r for rows >= k1, and g (both triangles of the entries it assembles).
__global__ void __launch_bounds__(256) k_sblock(Work w, LaunchArgs a, int K) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ unsigned char tri_r[kSb * (kSb - 1) / 2], tri_c[kSb * (kSb - 1) / 2];
    __shared__ double sinv[kSb];
    __shared__ int fail;
    const int C = gridDim.x;
    const int rank = C > 1 ? (int)cg::this_cluster().block_rank() : 0;
    const int tid = threadIdx.x, lane = tid & 31;
    auto csync = [&]() { if (C > 1) cg::this_cluster().sync(); else __syncthreads(); };
    auto rptr = [&](double *p, int q) -> double * { return C > 1 ? cg::this_cluster().map_shared_rank(p, q) : p; };
    // An earlier block failed (or theta was invalid): every CTA sees the same word and stops
    // before any cluster barrier.
    if (*(volatile int32_t *)w.status != 0) return;
    const DevInst in = w.inst[0];
    const int P = in.P;
    const SbGeom g = sb_geom(P, C, K);
    double *stage = reinterpret_cast<double *>(smem);         // [mch][16]: Lf[m][k0 + c], own m
    double *pan = stage + (size_t)g.mch * kSb;                  // [rows_max][16]: own panel rows
    double *recv = pan + (size_t)g.rows_max * kSb;              // [C][rows_max][16]: partial sums
    double *Dv = recv + (size_t)C * g.rows_max * kSb;           // [16][16]: inverse of D_K
    double *yk = Dv + kSb * kSb;                                // [16]: y_K
    double *Lf = w.chol + in.metric_off;
    const double *sg = w.sigma + in.param_off;
    const double *pc = w.pctrl + in.param_off;  // <C_i>: the diagonal L_ii = <C_i>/4 (Sec. 2)
    const double *L = w.L + in.metric_off;
    const double *gr = w.gradraw + in.param_off;
    double *rv = w.srhs;
    int rb, re;
    sb_rows(g, P, C, rank, rb, re);
    const int nown = re - rb;

    if (tid == 0) {
        fail = 0;
        int t = 0;
        for (int r = 0; r < kSb - 1; ++r)
            for (int c = 0; c <= r; ++c) { tri_r[t] = (unsigned char)r; tri_c[t] = (unsigned char)c; ++t; }
    }
    // (A) own panel rows of B (lower part of the diagonal block), g for the same entries
    for (int t = tid; t < nown * kSb; t += blockDim.x) {
        const int r = t >> 4, c = t & (kSb - 1), l = rb + r, col = g.k0 + c;
        double v = 0.0;
        if (c < g.nb && col <= l) {
            const int i = P - 1 - l, j = P - 1 - col;  // i <= j
            const double gv = (i == j) ? 0.25 * (pc[i] - sg[i] * sg[i]) : L[(int64_t)i * P + j] - 0.25 * sg[i] * sg[j];
            if (a.g_out) {
                a.g_out[in.metric_off + (int64_t)i * P + j] = gv;
                if (i != j) a.g_out[in.metric_off + (int64_t)j * P + i] = gv;
            }
            v = gv + (i == j ? a.lambda : 0.0);
        }
        pan[t] = v;
    }
    // (B) left-looking update, split over the CTAs along m: partial sums of
    // sum_{m in own chunk} Lf[m][l] Lf[m][k0 + c] for every row l >= k0, pushed to l's owner
    const int mb = min(g.k0, rank * g.mch), me = min(g.k0, mb + g.mch);
    for (int t = tid; t < (me - mb) * kSb; t += blockDim.x) {
        const int m = mb + (t >> 4), c = t & (kSb - 1);
        stage[t] = c < g.nb ? Lf[(int64_t)m * P + g.k0 + c] : 0.0;
    }
    __syncthreads();
    csync();  // every CTA of the cluster runs before the first distributed shared memory store
    if (g.k0 > 0) {
        for (int t = tid; t < (P - g.k0) * kSb; t += blockDim.x) {
            const int l = g.k0 + (t >> 4), c = t & (kSb - 1);
            const double *lcol = Lf + l;
            double s = 0.0, s2 = 0.0;  // two chains, loads of four terms in flight
            int m = mb;
            for (; m + 4 <= me; m += 4) {
                const double v0 = lcol[(int64_t)m * P], v1 = lcol[(int64_t)(m + 1) * P];
                const double v2 = lcol[(int64_t)(m + 2) * P], v3 = lcol[(int64_t)(m + 3) * P];
                s = fma(v0, stage[(m - mb) * kSb + c], s);
                s2 = fma(v1, stage[(m + 1 - mb) * kSb + c], s2);
                s = fma(v2, stage[(m + 2 - mb) * kSb + c], s);
                s2 = fma(v3, stage[(m + 3 - mb) * kSb + c], s2);
            }
            for (; m < me; ++m) s = fma(lcol[(int64_t)m * P], stage[(m - mb) * kSb + c], s);
            s += s2;
            int q = 0;
            if (l >= g.k1 && C > 1) q = 1 + (l - g.k1) / g.per;
            int qb, qe;
            sb_rows(g, P, C, q, qb, qe);
            rptr(recv, q)[((size_t)rank * g.rows_max + (l - qb)) * kSb + c] = s;
        }
    }
    csync();  // partial sums delivered
    if (g.k0 > 0) {
        for (int t = tid; t < nown * kSb; t += blockDim.x) {
            double s = 0.0;
            for (int q = 0; q < C; ++q) s += recv[(size_t)q * g.rows_max * kSb + t];
            pan[t] -= s;
        }
    }
    __syncthreads();

    // (C) CTA 0: Cholesky of the diagonal block D_K (rows 0..nb-1 of pan), its inverse, y_K
    if (rank == 0) {
        if (tid < 128) {
            for (int k = 0; k < g.nb; ++k) {
                if (tid == 0) {
                    const double d = pan[k * kSb + k];
                    if (!(d > 0.0)) fail = 1;
                    else { const double iv = rsqrt(d); pan[k * kSb + k] = d * iv; sinv[k] = iv; }
                }
                sbar128();
                if (fail) break;
                const double iv = sinv[k];
                if (tid > k && tid < g.nb) pan[tid * kSb + k] *= iv;
                sbar128();
                const int s = g.nb - k - 1;
                if (tid < s * (s + 1) / 2) {
                    const int r = k + 1 + tri_r[tid], c = k + 1 + tri_c[tid];
                    pan[r * kSb + c] = fma(-pan[r * kSb + k], pan[c * kSb + k], pan[r * kSb + c]);
                }
                sbar128();
            }
        }
        __syncthreads();
        if (!fail) {
            // inverse of the lower-triangular factor, all 16 columns at once: X = D^-1, row by row
            // (x_r = (e_r - sum_{m<r} D_rm x_m) / D_rr); thread (r, c) holds X[r][c]
            double *X = Dv;
            for (int t = tid; t < kSb * kSb; t += blockDim.x) X[t] = 0.0;
            __syncthreads();
            const int r = tid >> 4, c = tid & (kSb - 1);
            for (int k = 0; k < g.nb; ++k) {
                // column k of D eliminates row k: X[k][c] is final, then rows below take it
                if (r == k && c <= k) X[k * kSb + c] = ((c == k ? 1.0 : 0.0) + X[k * kSb + c]) * sinv[k];
                __syncthreads();
                if (r > k && r < g.nb && c <= k) X[r * kSb + c] = fma(-pan[r * kSb + k], X[k * kSb + c], X[r * kSb + c]);
                __syncthreads();
            }
            // Lf's diagonal block, and y_K = D^-1 r_K
            if (r < g.nb && c <= r) Lf[(int64_t)(g.k0 + c) * P + g.k0 + r] = pan[r * kSb + c];
            if (tid < g.nb) {
                const int l = g.k0 + tid;
                sinv[tid] = K == 0 ? -a.dt * gr[P - 1 - l] : rv[l];  // r_K (sinv reused)
            }
            __syncthreads();
            if (tid < g.nb) {
                double y = 0.0;
                for (int k = 0; k <= tid; ++k) y = fma(X[tid * kSb + k], sinv[k], y);
                yk[tid] = y;
                w.sy[g.k0 + tid] = y;
            }
            for (int t = tid; t < kSb * kSb; t += blockDim.x) w.sdinv[(size_t)K * kSb * kSb + t] = X[t];
            __syncthreads();
        }
        if (fail && tid == 0) atomicCAS(w.status, 0, (int)QNG_ERR_NOT_SPD);
        // D^-1, y_K and the failure flag to every other CTA
        for (int q = 1; q < C; ++q) {
            for (int t = tid; t < kSb * kSb + kSb; t += blockDim.x) rptr(Dv, q)[t] = Dv[t];  // Dv and yk are adjacent
            if (tid == 0) *(cg::this_cluster().map_shared_rank(&fail, q)) = fail;
        }
    }
    csync();
    if (fail) return;  // identical in every CTA after the barrier; no barrier follows

    // (D) own rows below the block: Lf[k0 + c][l] = sum_{c' <= c} pan[l][c'] D^-1[c][c'], and
    // r_l -= sum_c Lf[k0 + c][l] y_c. Sixteen lanes per row (a half warp), whole warps per pass.
    const int first = (rank == 0) ? g.nb : 0;  // CTA 0's rows below the block exist with one CTA only
    const int nrows = nown - first;
    if (nrows > 0) {
        const int total = ((nrows * kSb + 31) >> 5) << 5;
        for (int t = tid; t < total; t += blockDim.x) {
            const int rr = t >> 4, c = t & (kSb - 1);
            const bool valid = rr < nrows;
            const int r = first + (valid ? rr : 0), l = rb + r;
            double x = 0.0;
            if (valid && c < g.nb)
                for (int k = 0; k <= c; ++k) x = fma(pan[r * kSb + k], Dv[c * kSb + k], x);
            if (valid && c < g.nb) Lf[(int64_t)(g.k0 + c) * P + l] = x;
            double ry = (valid && c < g.nb) ? x * yk[c] : 0.0;
            ry += __shfl_xor_sync(0xffffffffu, ry, 8);
            ry += __shfl_xor_sync(0xffffffffu, ry, 4);
            ry += __shfl_xor_sync(0xffffffffu, ry, 2);
            ry += __shfl_xor_sync(0xffffffffu, ry, 1);
            if (valid && c == 0) rv[l] = (K == 0 ? -a.dt * gr[P - 1 - l] : rv[l]) - ry;
        }
    }
    (void)lane;
}

// Back substitution Lf^T z = y, last block first, then dtheta = J z; also the step's other
// outputs (gradient, <sigma>, <E>). One CTA of 256 threads.
__global__ void __launch_bounds__(256) k_sback(Work w, LaunchArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double tb[kSb];
    __shared__ double di[kSb * kSb];
    const DevInst in = w.inst[0];
    const int P = in.P;
    const int tid = threadIdx.x;
    if (a.grad_out)
        for (int k = tid; k < P; k += blockDim.x) a.grad_out[in.param_off + k] = w.gradraw[in.param_off + k];
    if (a.sigma_out)
        for (int k = tid; k < P; k += blockDim.x) a.sigma_out[in.param_off + k] = w.sigma[in.param_off + k];
    if (a.energy_out && tid == 0) a.energy_out[0] = w.energy[0];
    if (*(volatile int32_t *)w.status != 0) return;
    double *z = reinterpret_cast<double *>(smem);  // [P]
    const double *Lf = w.chol + in.metric_off;
    const int nblk = (P + kSb - 1) / kSb;
    const int c = tid >> 4, part = tid & 15;  // column c of the block, 16 partial sums each
    for (int K = nblk - 1; K >= 0; --K) {
        const int k0 = K * kSb, nb = min(kSb, P - k0), k1 = k0 + nb;
        // t_c = y_c - sum_{l >= k1} Lf[k0 + c][l] z_l
        for (int t = tid; t < kSb * kSb; t += blockDim.x) di[t] = w.sdinv[(size_t)K * kSb * kSb + t];
        double s = 0.0, s2 = 0.0;
        if (c < nb) {
            const double *col = Lf + (int64_t)(k0 + c) * P;
            int l = k1 + part;
            for (; l + 16 < P; l += 32) {
                const double v0 = col[l], v1 = col[l + 16];
                s = fma(v0, z[l], s);
                s2 = fma(v1, z[l + 16], s2);
            }
            if (l < P) s = fma(col[l], z[l], s);
            s += s2;
        }
        s += __shfl_xor_sync(0xffffffffu, s, 8);
        s += __shfl_xor_sync(0xffffffffu, s, 4);
        s += __shfl_xor_sync(0xffffffffu, s, 2);
        s += __shfl_xor_sync(0xffffffffu, s, 1);
        if (part == 0 && c < nb) tb[c] = w.sy[k0 + c] - s;
        __syncthreads();
        // z_K = (D^-1)^T t: z_c = sum_{c' >= c} Dinv[c'][c] t_c'
        if (tid < nb) {
            double v = 0.0;
            for (int k = tid; k < nb; ++k) v = fma(di[k * kSb + tid], tb[k], v);
            z[k0 + tid] = v;
        }
        __syncthreads();
    }
    for (int i = tid; i < P; i += blockDim.x) a.dtheta_out[in.param_off + i] = z[P - 1 - i];
}

cudaError_t prepare_sblock(int P, int C) {
    cudaError_t e = raise_smem_limit(reinterpret_cast<const void *>(k_sblock), sblock_smem_bytes(P, C));
    if (e != cudaSuccess) return e;
    return raise_smem_limit(reinterpret_cast<const void *>(k_sback), sizeof(double) * P);
}

cudaError_t launch_sblock(const Work &w, const LaunchArgs &a, int P, int C, int K, cudaStream_t st) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)C);
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = sblock_smem_bytes(P, C);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    int na = 0;
    if (C > 1) {
        attr[na].id = cudaLaunchAttributeClusterDimension;
        attr[na].val.clusterDim.x = (unsigned)C;
        attr[na].val.clusterDim.y = 1;
        attr[na].val.clusterDim.z = 1;
        ++na;
    }
    cfg.attrs = attr;
    cfg.numAttrs = na;
    return cudaLaunchKernelEx(&cfg, k_sblock, w, a, K);
}

cudaError_t launch_sback(const Work &w, const LaunchArgs &a, int P, cudaStream_t st) {
    k_sback<<<1, 256, sizeof(double) * P, st>>>(w, a);
    return cudaGetLastError();
}

}  // namespace qng

// FINGER construction on the device: Algorithm 2 and the precomputed tables of
// Supplementary G (arXiv 2206.11408).
//
//   k_sample      neighbour-pair draw per node (counter-based, see finger.h)
//   k_pair_b      b = c^T d / c^T c for the D_res member of every pair
//   k_gram        G = sum d_res d_res^T (m x m): 64 x 64 output tiles, FP32 per
//                 chunk of pairs, FP64 across chunks
//   k_jacobi      cyclic parallel-order Jacobi on G in FP64 (cooperative grid);
//                 the eigenvectors of the r largest eigenvalues are the left
//                 singular vectors U_{1:r} of D_res (Proposition 1)
//   k_node_proj   P c for every node (tiled FFMA)
//   k_edge        per layer-0 edge (c, d): b, ||d_res|| = ||d - b c|| (explicit),
//                 u = (P d - b P c) / ||P d - b P c|| (= P d_res normalised)
//   k_pair_cos    X = cos(d_res, d'_res) (explicit residuals), Y = u_d . u_d'
//   k_sum*        deterministic block reductions for mu, sigma, mu_hat,
//                 sigma_hat (standard deviations, 1/N) and eps
//   k_lp_codes    FP8-e4m3 codes of u * code_scale in fragment order (reduced precision)
#include <cooperative_groups.h>
#include <math.h>

#include <algorithm>
#include <chrono>
#include <vector>

#include "internal.cuh"

namespace cg = cooperative_groups;

namespace fg {

namespace {

__device__ __forceinline__ float wsum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ uint64_t smix(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

__global__ void k_xnorm2(const float4* X, int64_t n, int m4, float* out) {
    const int lane = threadIdx.x & 31;
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (w >= n) return;
    float acc = 0.f;
    for (int k = lane; k < m4; k += 32) {
        const float4 x = X[w * m4 + k];
        acc = fmaf(x.x, x.x, acc);
        acc = fmaf(x.y, x.y, acc);
        acc = fmaf(x.z, x.z, acc);
        acc = fmaf(x.w, x.w, acc);
    }
    acc = wsum(acc);
    if (lane == 0) out[w] = acc;
}

__global__ void k_to_bf16(const float* X, int64_t n, int m_pad, int m8, __nv_bfloat16* out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int w = m8 * 8;
    if (i >= n * w) return;
    const int64_t r = i / w;
    const int k = (int)(i % w);
    out[i] = __float2bfloat16_rn(k < m_pad ? X[r * m_pad + k] : 0.f);
}

// pair rows (c, slot_i, slot_j); c = -1 when the node has < 2 neighbours
__global__ void k_sample(const uint32_t* adj0, int64_t n, int deg0, uint64_t seed, int spn,
                         int3* out) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * spn) return;
    const int64_t c = t / spn;
    const uint32_t* row = adj0 + c * deg0;
    int deg = 0;
    for (int j = 0; j < deg0; ++j) deg += row[j] != PAD;
    if (deg < 2) {
        out[t] = make_int3(-1, -1, -1);
        return;
    }
    const uint64_t h1 = smix(seed ^ (uint64_t)t);
    const uint64_t h2 = smix(h1);
    const int i = (int)(h1 % (uint64_t)deg);
    int j = (int)(h2 % (uint64_t)(deg - 1));
    j += j >= i;
    // slots of the i-th and j-th valid entries in row order
    int si = -1, sj = -1, v = 0;
    for (int s = 0; s < deg0; ++s) {
        if (row[s] == PAD) continue;
        if (v == i) si = s;
        if (v == j) sj = s;
        v++;
    }
    out[t] = make_int3((int)c, si, sj);
}

// b of the pair's first member (warp per pair)
__global__ void k_pair_b(const float4* X, int m4, const float* xn2, const uint32_t* adj0, int deg0,
                         const int3* pairs, int64_t np, float* b_out) {
    const int lane = threadIdx.x & 31;
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (w >= np) return;
    const int3 p = pairs[w];
    if (p.x < 0) {
        if (lane == 0) b_out[w] = 0.f;
        return;
    }
    const uint32_t d = adj0[(int64_t)p.x * deg0 + p.y];
    float acc = 0.f;
    for (int k = lane; k < m4; k += 32) {
        const float4 a = X[(int64_t)p.x * m4 + k], b = X[(int64_t)d * m4 + k];
        acc = fmaf(a.x, b.x, acc);
        acc = fmaf(a.y, b.y, acc);
        acc = fmaf(a.z, b.z, acc);
        acc = fmaf(a.w, b.w, acc);
    }
    acc = wsum(acc);
    const float cc = xn2[p.x];
    if (lane == 0) b_out[w] = cc > 0.f ? acc / cc : 0.f;
}

constexpr int GT = 64;      // Gram output tile
constexpr int GKP = 32;     // pairs per stage
constexpr int GCHUNK = 4096;

// G[I, J] += sum over a chunk of pairs of R[p, I] R[p, J], R = d - b c
__global__ void __launch_bounds__(256) k_gram(const float* X, int m_pad, int m, const uint32_t* adj0,
                                              int deg0, const int3* pairs, const float* bq,
                                              int64_t np, double* G) {
    __shared__ float Ri[GKP][GT + 1];
    __shared__ float Rj[GKP][GT + 1];
    const int ti = blockIdx.x * GT, tj = blockIdx.y * GT;
    const int64_t p0 = (int64_t)blockIdx.z * GCHUNK;
    const int64_t p1 = np < p0 + GCHUNK ? np : p0 + GCHUNK;
    const int t = threadIdx.x;
    const int oi = (t >> 4) * 4, oj = (t & 15) * 4;
    float acc[4][4] = {};
    for (int64_t pb = p0; pb < p1; pb += GKP) {
        __syncthreads();
        for (int e = t; e < GKP * GT; e += 256) {
            const int pp = e / GT, k = e % GT;
            const int64_t pi = pb + pp;
            float ri = 0.f, rj = 0.f;
            if (pi < p1) {
                const int3 p = pairs[pi];
                if (p.x >= 0) {
                    const uint32_t d = adj0[(int64_t)p.x * deg0 + p.y];
                    const float b = bq[pi];
                    const int ki = ti + k, kj = tj + k;
                    if (ki < m) ri = X[(int64_t)d * m_pad + ki] - b * X[(int64_t)p.x * m_pad + ki];
                    if (kj < m) rj = X[(int64_t)d * m_pad + kj] - b * X[(int64_t)p.x * m_pad + kj];
                }
            }
            Ri[pp][k] = ri;
            Rj[pp][k] = rj;
        }
        __syncthreads();
#pragma unroll 4
        for (int pp = 0; pp < GKP; ++pp) {
            float a[4], b[4];
#pragma unroll
            for (int x = 0; x < 4; ++x) {
                a[x] = Ri[pp][oi + x];
                b[x] = Rj[pp][oj + x];
            }
#pragma unroll
            for (int x = 0; x < 4; ++x)
#pragma unroll
                for (int y = 0; y < 4; ++y) acc[x][y] = fmaf(a[x], b[y], acc[x][y]);
        }
    }
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) {
            const int gi = ti + oi + x, gj = tj + oj + y;
            if (gi < m && gj < m) atomicAdd(&G[(int64_t)gi * m + gj], (double)acc[x][y]);
        }
}

// Parallel-order cyclic Jacobi on the symmetric m x m matrix A (row-major FP64),
// accumulating V (initialised to I).  Round r of a sweep rotates the m/2
// disjoint pairs of the round-robin schedule; each rotation zeroes A[p][q]:
//   tau = (A_qq - A_pp) / (2 A_pq), t = sign(tau) / (|tau| + sqrt(1 + tau^2)),
//   c = 1 / sqrt(1 + t^2), s = t c,  A <- J^T A J,  V <- V J,
// with J = I except J_pp = J_qq = c, J_pq = s, J_qp = -s.
__global__ void k_jacobi(double* A, double* V, int m, double2* rot, int2* pr, double* red,
                         int max_sweeps, double tol, int* sweeps_out) {
    cg::grid_group grid = cg::this_grid();
    const int mm = (m + 1) & ~1;   // even number of slots; slot m (if m odd) is a dummy
    const int half = mm / 2;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nth = (int64_t)gridDim.x * blockDim.x;
    __shared__ double sred[32];
    int sweep = 0;
    for (; sweep < max_sweeps; ++sweep) {
        // off-diagonal and total Frobenius mass
        double off = 0.0, tot = 0.0;
        for (int64_t i = tid; i < (int64_t)m * m; i += nth) {
            const double v = A[i] * A[i];
            tot += v;
            if (i / m != i % m) off += v;
        }
        for (int o = 16; o > 0; o >>= 1) {
            off += __shfl_xor_sync(0xffffffffu, off, o);
            tot += __shfl_xor_sync(0xffffffffu, tot, o);
        }
        if ((threadIdx.x & 31) == 0) {
            sred[threadIdx.x >> 5] = off;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double s = 0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sred[w];
            red[2 * blockIdx.x] = s;
        }
        __syncthreads();
        if ((threadIdx.x & 31) == 0) sred[threadIdx.x >> 5] = tot;
        __syncthreads();
        if (threadIdx.x == 0) {
            double s = 0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sred[w];
            red[2 * blockIdx.x + 1] = s;
        }
        grid.sync();
        double OFF = 0, TOT = 0;
        for (int b = 0; b < (int)gridDim.x; ++b) {
            OFF += red[2 * b];
            TOT += red[2 * b + 1];
        }
        grid.sync();
        if (OFF <= tol * tol * TOT || OFF == 0.0) break;
        for (int r = 0; r < mm - 1; ++r) {
            // pairs and rotations of this step of the sweep
            for (int64_t k = tid; k < half; k += nth) {
                int a, b;
                if (k == 0) a = 0;
                else a = (int)((k + r - 1) % (mm - 1)) + 1;
                b = (int)((mm - 1 - k + r - 1) % (mm - 1)) + 1;
                if (k == 0) b = (int)((mm - 1 + r - 1) % (mm - 1)) + 1;
                int p = min(a, b), q = max(a, b);
                double c = 1.0, s = 0.0;
                if (q < m) {
                    const double apq = A[(int64_t)p * m + q];
                    if (apq != 0.0) {
                        const double app = A[(int64_t)p * m + p], aqq = A[(int64_t)q * m + q];
                        const double tau = (aqq - app) / (2.0 * apq);
                        const double t = (tau >= 0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                        c = 1.0 / sqrt(1.0 + t * t);
                        s = t * c;
                    }
                }
                pr[k] = make_int2(p, q);
                rot[k] = make_double2(c, s);
            }
            grid.sync();
            // rows: A <- J^T A
            for (int64_t e = tid; e < (int64_t)half * m; e += nth) {
                const int k = (int)(e / m), j = (int)(e % m);
                const int2 pq = pr[k];
                if (pq.y >= m) continue;
                const double2 cs = rot[k];
                const double ap = A[(int64_t)pq.x * m + j], aq = A[(int64_t)pq.y * m + j];
                A[(int64_t)pq.x * m + j] = cs.x * ap - cs.y * aq;
                A[(int64_t)pq.y * m + j] = cs.y * ap + cs.x * aq;
            }
            grid.sync();
            // columns: A <- A J, V <- V J
            for (int64_t e = tid; e < (int64_t)half * m; e += nth) {
                const int k = (int)(e / m), i = (int)(e % m);
                const int2 pq = pr[k];
                if (pq.y >= m) continue;
                const double2 cs = rot[k];
                const double ap = A[(int64_t)i * m + pq.x], aq = A[(int64_t)i * m + pq.y];
                A[(int64_t)i * m + pq.x] = cs.x * ap - cs.y * aq;
                A[(int64_t)i * m + pq.y] = cs.y * ap + cs.x * aq;
                const double vp = V[(int64_t)i * m + pq.x], vq = V[(int64_t)i * m + pq.y];
                V[(int64_t)i * m + pq.x] = cs.x * vp - cs.y * vq;
                V[(int64_t)i * m + pq.y] = cs.y * vp + cs.x * vq;
            }
            grid.sync();
        }
    }
    if (tid == 0) *sweeps_out = sweep;
}

// P rows = eigenvectors of the r largest eigenvalues (ties by index), FP32,
// padded to r_pad x m_pad with zeros.  Single block.
__global__ void k_pick_basis(const double* A, const double* V, int m, int r, int r_pad, int m_pad,
                             float* P, double* evals) {
    extern __shared__ int order[];
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        const double di = A[(int64_t)i * m + i];
        int rank = 0;
        for (int j = 0; j < m; ++j) {
            const double dj = A[(int64_t)j * m + j];
            rank += (dj > di) || (dj == di && j < i);
        }
        order[rank] = i;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < r_pad * m_pad; e += blockDim.x) {
        const int k = e / m_pad, j = e % m_pad;
        float v = 0.f;
        if (k < r && j < m) v = (float)V[(int64_t)j * m + order[k]];
        P[e] = v;
    }
    for (int i = threadIdx.x; i < m; i += blockDim.x) evals[i] = A[(int64_t)order[i] * m + order[i]];
}

// Pc[n][r_pad] = X P^T: CTA of 64 nodes x 64 outputs, k-chunks of 32
__global__ void __launch_bounds__(256) k_node_proj(const float* X, int64_t n, int m_pad,
                                                   const float* P, int r_pad, float* Pc) {
    __shared__ float Xs[32][65];
    __shared__ float Ps[32][65];
    const int64_t n0 = (int64_t)blockIdx.x * 64;
    const int r0 = blockIdx.y * 64;
    const int t = threadIdx.x;
    const int on = (t >> 4) * 4, orr = (t & 15) * 4;
    float acc[4][4] = {};
    for (int k0 = 0; k0 < m_pad; k0 += 32) {
        __syncthreads();
        for (int e = t; e < 64 * 32; e += 256) {
            const int i = e / 32, k = e % 32;
            const int64_t gn = n0 + i;
            const int gk = k0 + k;
            Xs[k][i] = (gn < n && gk < m_pad) ? X[gn * m_pad + gk] : 0.f;
            const int gr = r0 + i;
            Ps[k][i] = (gr < r_pad && gk < m_pad) ? P[(int64_t)gr * m_pad + gk] : 0.f;
        }
        __syncthreads();
#pragma unroll 8
        for (int k = 0; k < 32; ++k) {
            float a[4], b[4];
#pragma unroll
            for (int x = 0; x < 4; ++x) {
                a[x] = Xs[k][on + x];
                b[x] = Ps[k][orr + x];
            }
#pragma unroll
            for (int x = 0; x < 4; ++x)
#pragma unroll
                for (int y = 0; y < 4; ++y) acc[x][y] = fmaf(a[x], b[y], acc[x][y]);
        }
    }
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) {
            const int64_t gn = n0 + on + x;
            const int gr = r0 + orr + y;
            if (gn < n && gr < r_pad) Pc[gn * r_pad + gr] = acc[x][y];
        }
}

// per layer-0 edge (c, d): warp per node c
__global__ void k_edge(const float4* X, int m4, const float* xn2, const uint32_t* adj0,
                       int64_t n, int deg0, const float* Pc, int r_pad, float* edge_u,
                       float2* edge_s) {
    const int lane = threadIdx.x & 31;
    const int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (c >= n) return;
    float4 xc[8];
#pragma unroll
    for (int v = 0; v < 8; ++v) {
        const int k = lane + 32 * v;
        xc[v] = k < m4 ? X[c * m4 + k] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    const float cc = xn2[c];
    const float pc0 = lane < r_pad ? Pc[c * r_pad + lane] : 0.f;
    const float pc1 = lane + 32 < r_pad ? Pc[c * r_pad + lane + 32] : 0.f;
    for (int j = 0; j < deg0; ++j) {
        const int64_t e = c * deg0 + j;
        const uint32_t d = adj0[e];
        if (d == PAD) {
            if (lane < r_pad) edge_u[e * r_pad + lane] = 0.f;
            if (lane + 32 < r_pad) edge_u[e * r_pad + lane + 32] = 0.f;
            if (lane == 0) edge_s[e] = make_float2(0.f, 0.f);
            continue;
        }
        float4 xd[8];
        float dot = 0.f;
#pragma unroll
        for (int v = 0; v < 8; ++v) {
            const int k = lane + 32 * v;
            xd[v] = k < m4 ? X[(int64_t)d * m4 + k] : make_float4(0.f, 0.f, 0.f, 0.f);
            dot = fmaf(xc[v].x, xd[v].x, dot);
            dot = fmaf(xc[v].y, xd[v].y, dot);
            dot = fmaf(xc[v].z, xd[v].z, dot);
            dot = fmaf(xc[v].w, xd[v].w, dot);
        }
        dot = wsum(dot);
        const float b = cc > 0.f ? dot / cc : 0.f;
        float rn = 0.f;
#pragma unroll
        for (int v = 0; v < 8; ++v) {
            float t;
            t = xd[v].x - b * xc[v].x; rn = fmaf(t, t, rn);
            t = xd[v].y - b * xc[v].y; rn = fmaf(t, t, rn);
            t = xd[v].z - b * xc[v].z; rn = fmaf(t, t, rn);
            t = xd[v].w - b * xc[v].w; rn = fmaf(t, t, rn);
        }
        rn = wsum(rn);
        const float u0 = lane < r_pad ? Pc[(int64_t)d * r_pad + lane] - b * pc0 : 0.f;
        const float u1 = lane + 32 < r_pad ? Pc[(int64_t)d * r_pad + lane + 32] - b * pc1 : 0.f;
        const float nu = wsum(u0 * u0 + u1 * u1);
        const float inv = nu > 0.f ? rsqrtf(nu) : 0.f;
        if (lane < r_pad) edge_u[e * r_pad + lane] = u0 * inv;
        if (lane + 32 < r_pad) edge_u[e * r_pad + lane + 32] = u1 * inv;
        if (lane == 0) edge_s[e] = make_float2(sqrtf(rn), b);
    }
}

// X_i, Y_i for every drawn pair (warp per pair); invalid pairs get NaN
__global__ void k_pair_cos(const float4* X, int m4, const uint32_t* adj0, int deg0,
                           const int3* pairs, int64_t np, const float* edge_u, const float2* edge_s,
                           int r_pad, double* Xc, double* Yc) {
    const int lane = threadIdx.x & 31;
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (w >= np) return;
    const int3 p = pairs[w];
    if (p.x < 0) {
        if (lane == 0) {
            Xc[w] = NAN;
            Yc[w] = NAN;
        }
        return;
    }
    const int64_t e1 = (int64_t)p.x * deg0 + p.y, e2 = (int64_t)p.x * deg0 + p.z;
    const uint32_t d1 = adj0[e1], d2 = adj0[e2];
    const float b1 = edge_s[e1].y, b2 = edge_s[e2].y;
    float s12 = 0.f, s11 = 0.f, s22 = 0.f;
    for (int k = lane; k < m4; k += 32) {
        const float4 c = X[(int64_t)p.x * m4 + k];
        const float4 x = X[(int64_t)d1 * m4 + k];
        const float4 y = X[(int64_t)d2 * m4 + k];
        const float r1[4] = {x.x - b1 * c.x, x.y - b1 * c.y, x.z - b1 * c.z, x.w - b1 * c.w};
        const float r2[4] = {y.x - b2 * c.x, y.y - b2 * c.y, y.z - b2 * c.z, y.w - b2 * c.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            s12 = fmaf(r1[i], r2[i], s12);
            s11 = fmaf(r1[i], r1[i], s11);
            s22 = fmaf(r2[i], r2[i], s22);
        }
    }
    s12 = wsum(s12);
    s11 = wsum(s11);
    s22 = wsum(s22);
    float uu = 0.f;
    for (int k = lane; k < r_pad; k += 32) uu = fmaf(edge_u[e1 * r_pad + k], edge_u[e2 * r_pad + k], uu);
    uu = wsum(uu);
    if (lane == 0) {
        const double den = sqrt((double)s11) * sqrt((double)s22);
        Xc[w] = den > 0 ? (double)s12 / den : 0.0;
        Yc[w] = (double)uu;
    }
}

// Rank rule (Supplementary E): X = cos(d_res, d'_res) and, for every
// candidate rank r_i = min((i+1) step, r_max), Y_i = cos of the projections on
// the first r_i basis rows, in one pass (warp per pair; both residuals staged
// in shared memory, one warp reduction per basis row).  Y is [nr][np].
constexpr int PREFIX_WARPS = 4;
__global__ void __launch_bounds__(32 * PREFIX_WARPS)
    k_pair_cos_prefix(const float4* X, int m4, const float* xn2, const uint32_t* adj0, int deg0,
                      const int3* pairs, int64_t np, const float* P, int m_pad, int r_max,
                      int step, double* Xc, double* Yk) {
    extern __shared__ float4 res_s[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int64_t w = (int64_t)blockIdx.x * PREFIX_WARPS + wib;
    if (w >= np) return;
    const int nr = (r_max + step - 1) / step;
    const int3 p = pairs[w];
    if (p.x < 0) {
        if (lane == 0) {
            Xc[w] = NAN;
            for (int i = 0; i < nr; ++i) Yk[(int64_t)i * np + w] = NAN;
        }
        return;
    }
    float4* r1 = res_s + (size_t)wib * 2 * m4;
    float4* r2 = r1 + m4;
    const uint32_t d1 = adj0[(int64_t)p.x * deg0 + p.y], d2 = adj0[(int64_t)p.x * deg0 + p.z];
    float cd1 = 0.f, cd2 = 0.f;
    for (int k = lane; k < m4; k += 32) {
        const float4 c = X[(int64_t)p.x * m4 + k];
        const float4 x = X[(int64_t)d1 * m4 + k];
        const float4 y = X[(int64_t)d2 * m4 + k];
        cd1 += c.x * x.x + c.y * x.y + c.z * x.z + c.w * x.w;
        cd2 += c.x * y.x + c.y * y.y + c.z * y.z + c.w * y.w;
    }
    cd1 = wsum(cd1);
    cd2 = wsum(cd2);
    const float cc = xn2[p.x];
    const float b1 = cc > 0.f ? cd1 / cc : 0.f, b2 = cc > 0.f ? cd2 / cc : 0.f;
    float s12 = 0.f, s11 = 0.f, s22 = 0.f;
    for (int k = lane; k < m4; k += 32) {
        const float4 c = X[(int64_t)p.x * m4 + k];
        const float4 x = X[(int64_t)d1 * m4 + k];
        const float4 y = X[(int64_t)d2 * m4 + k];
        const float4 a = make_float4(x.x - b1 * c.x, x.y - b1 * c.y, x.z - b1 * c.z, x.w - b1 * c.w);
        const float4 b = make_float4(y.x - b2 * c.x, y.y - b2 * c.y, y.z - b2 * c.z, y.w - b2 * c.w);
        r1[k] = a;
        r2[k] = b;
        s12 += a.x * b.x + a.y * b.y + a.z * b.z + a.w * b.w;
        s11 += a.x * a.x + a.y * a.y + a.z * a.z + a.w * a.w;
        s22 += b.x * b.x + b.y * b.y + b.z * b.z + b.w * b.w;
    }
    s12 = wsum(s12);
    s11 = wsum(s11);
    s22 = wsum(s22);
    if (lane == 0) {
        const double den = sqrt((double)s11) * sqrt((double)s22);
        Xc[w] = den > 0 ? (double)s12 / den : 0.0;
    }
    __syncwarp();
    const float4* P4 = reinterpret_cast<const float4*>(P);
    const int mp4 = m_pad / 4;
    double t12 = 0, t11 = 0, t22 = 0;
    for (int k = 0; k < r_max; ++k) {
        float u = 0.f, v = 0.f;
        for (int j = lane; j < m4; j += 32) {
            const float4 pk = P4[(int64_t)k * mp4 + j];
            const float4 a = r1[j], b = r2[j];
            u += pk.x * a.x + pk.y * a.y + pk.z * a.z + pk.w * a.w;
            v += pk.x * b.x + pk.y * b.y + pk.z * b.z + pk.w * b.w;
        }
        u = wsum(u);
        v = wsum(v);
        t12 += (double)u * v;
        t11 += (double)u * u;
        t22 += (double)v * v;
        if (lane == 0 && ((k + 1) % step == 0 || k + 1 == r_max)) {
            const double den = sqrt(t11) * sqrt(t22);
            Yk[(int64_t)(k / step) * np + w] = den > 0 ? t12 / den : 0.0;
        }
    }
}

// deterministic reductions: per-block partial sums, then one block sums them
// mode 0: sum X, sum Y, count;  mode 1: sum (X-mu)^2, sum (Y-muh)^2,
// sum (X-mu)(Y-muh);  mode 2: sum |(Y - muh) ratio + mu - X|
__global__ void k_sum_part(const double* Xc, const double* Yc, int64_t np, int mode, double mu,
                           double muh, double ratio, double* part) {
    __shared__ double s[3][256];
    double a = 0, b = 0, c = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < np;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double x = Xc[i], y = Yc[i];
        if (x != x) continue;
        if (mode == 0) {
            a += x;
            b += y;
            c += 1.0;
        } else if (mode == 1) {
            a += (x - mu) * (x - mu);
            b += (y - muh) * (y - muh);
            c += (x - mu) * (y - muh);
        } else {
            a += fabs((y - muh) * ratio + mu - x);
        }
    }
    s[0][threadIdx.x] = a;
    s[1][threadIdx.x] = b;
    s[2][threadIdx.x] = c;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o)
            for (int k = 0; k < 3; ++k) s[k][threadIdx.x] += s[k][threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int k = 0; k < 3; ++k) part[blockIdx.x * 3 + k] = s[k][0];
}

__global__ void k_sum_final(const double* part, int nb, double* out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double a = 0, b = 0, c = 0;
    for (int i = 0; i < nb; ++i) {
        a += part[3 * i];
        b += part[3 * i + 1];
        c += part[3 * i + 2];
    }
    out[0] = a;
    out[1] = b;
    out[2] = c;
}

// FP8-e4m3 codes of scale * u, 16 bytes per (node c, tile T, step kk of 32
// codes, lane l = 4g + t).  With k32 (a block of at most four such products,
// the shapes the search kernel multiplies in FP8) they are in the A-fragment
// order of mma.m16n8k32 with 8-bit operands: rows 16T + g (words 0, 2) and
// 16T + g + 8 (words 1, 3) at codes 32kk + 4t .. + 3 (words 0, 1) and
// 32kk + 16 + 4t .. + 3 (words 2, 3), the lower code in the lower byte.
// Otherwise they follow the FP16 A-fragment order of m16n8k16 for the k steps
// 2kk (bytes 0..7) and 2kk + 1 (bytes 8..15): rows 16T + g and 16T + g + 8 at
// codes 16ks + 2t, +1, +8, +9 (the kernel converts them to FP16 pairs).
__global__ void k_lp_codes(const float* edge_u, int64_t n, int deg0, int r_pad, int tiles,
                           int kp_n, float scale, int k32, uint4* out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n * tiles * kp_n * 32) return;
    const int l = (int)(i & 31);
    int64_t f = i >> 5;
    const int kk = (int)(f % kp_n);
    f /= kp_n;
    const int T = (int)(f % tiles);
    const int64_t c = f / tiles;
    const int g = l >> 2, t = l & 3;
    auto code = [&](int row, int k) -> uint32_t {
        const float v = row < deg0 && k < r_pad ? edge_u[((size_t)c * deg0 + row) * r_pad + k] * scale : 0.f;
        return (uint32_t)__nv_cvt_float_to_fp8(v, __NV_SATFINITE, __NV_E4M3);
    };
    uint32_t w[4];
    if (k32) {
        for (int q = 0; q < 4; ++q) {
            const int row = 16 * T + g + ((q & 1) ? 8 : 0);
            const int k0 = 32 * kk + 4 * t + ((q & 2) ? 16 : 0);
            w[q] = code(row, k0) | code(row, k0 + 1) << 8 | code(row, k0 + 2) << 16 | code(row, k0 + 3) << 24;
        }
    } else {
        for (int h = 0; h < 2; ++h) {
            const int ks = 2 * kk + h;
            const int r0 = 16 * T + g, r1 = r0 + 8, k0 = 16 * ks + 2 * t, k1 = k0 + 8;
            w[2 * h] = code(r0, k0) | code(r0, k0 + 1) << 8 | code(r1, k0) << 16 | code(r1, k0 + 1) << 24;
            w[2 * h + 1] = code(r0, k1) | code(r0, k1 + 1) << 8 | code(r1, k1) << 16 | code(r1, k1 + 1) << 24;
        }
    }
    out[i] = make_uint4(w[0], w[1], w[2], w[3]);
}

// FP16 codes in m16n8k16 A-fragment order: thread i writes the 16 bytes of
// lane l = i % 32 for (node c, tile T, k step ks) = i / 32, i.e. rows
// 16T + g and 16T + g + 8 (g = l / 4) at codes 16ks + 2t, +1, +8, +9
// (t = l % 4), each edge_u entry rounded to nearest even (0 beyond the node's
// deg0 rows and beyond r_pad codes; padding slots hold 0 in edge_u already).
__global__ void k_half_codes(const float* edge_u, int64_t n, int deg0, int r_pad, int tiles,
                             int ks_n, uint4* out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n * tiles * ks_n * 32) return;
    const int l = (int)(i & 31);
    int64_t f = i >> 5;
    const int ks = (int)(f % ks_n);
    f /= ks_n;
    const int T = (int)(f % tiles);
    const int64_t c = f / tiles;
    const int g = l >> 2, t = l & 3;
    auto code = [&](int row, int k) -> float {
        return row < deg0 && k < r_pad ? edge_u[((size_t)c * deg0 + row) * r_pad + k] : 0.f;
    };
    const int r0 = 16 * T + g, r1 = r0 + 8, k0 = 16 * ks + 2 * t, k1 = k0 + 8;
    __half2 w[4];
    w[0] = __floats2half2_rn(code(r0, k0), code(r0, k0 + 1));
    w[1] = __floats2half2_rn(code(r1, k0), code(r1, k0 + 1));
    w[2] = __floats2half2_rn(code(r0, k1), code(r0, k1 + 1));
    w[3] = __floats2half2_rn(code(r1, k1), code(r1, k1 + 1));
    out[i] = *reinterpret_cast<const uint4*>(w);
}

// layer-0 degree of every node
__global__ void k_degree(const uint32_t* adj0, int64_t n, int deg0, int32_t* deg) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    int d = 0;
    for (int j = 0; j < deg0; ++j) d += adj0[v * deg0 + j] != PAD;
    deg[v] = d;
}

// adjacency with each neighbour id tagged (bit 30) when its degree exceeds thr
__global__ void k_tag_adj(const uint32_t* adj0, int64_t ne, const int32_t* deg, int thr,
                          uint32_t* out) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ne) return;
    const uint32_t u = adj0[e];
    out[e] = u == PAD ? PAD : (deg[u] > thr ? u | 0x40000000u : u);
}

template <class T>
T* dalloc(size_t count) {
    void* p = nullptr;
    if (cudaMalloc(&p, count * sizeof(T) + 16) != cudaSuccess) return nullptr;
    return static_cast<T*>(p);
}

}  // namespace

cudaError_t launch_xnorm2(const float4* X, int64_t n, int m4, float* out, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    k_xnorm2<<<(unsigned)((n * 32 + 255) / 256), 256, 0, s>>>(X, n, m4, out);
    return cudaGetLastError();
}

cudaError_t launch_to_bf16(const float* X, int64_t n, int m_pad, int m8, __nv_bfloat16* out,
                           cudaStream_t s) {
    const int64_t tot = n * m8 * 8;
    if (tot == 0) return cudaSuccess;
    k_to_bf16<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(X, n, m_pad, m8, out);
    return cudaGetLastError();
}

}  // namespace fg

// The modes that read a centre's whole code block (FP16 and LP) take its layer-0
// adjacency from a tagged copy: a neighbour's id has bit 30 set when its
// degree exceeds 16 (32 when deg0 > 32), i.e. when the second half of its code
// block holds rows; ids must stay below 2^30.  Built once for both modes.
cudaError_t build_tagged_adj(finger_index* ix) {
    using namespace fg;
    if (ix->adj_t) return cudaSuccess;
    if (ix->n >= (int64_t(1) << 30)) return cudaErrorInvalidValue;
    const int tiles = ix->deg0 > 32 ? 4 : 2;
    const int64_t ne = ix->n * ix->deg0;
    int32_t* deg = nullptr;
    cudaError_t e = cudaMalloc(&ix->adj_t, sizeof(uint32_t) * (size_t)ne + 16);
    if (e == cudaSuccess) e = cudaMalloc(&deg, sizeof(int32_t) * (size_t)ix->n);
    if (e != cudaSuccess) {
        cudaFree(deg);
        cudaFree(ix->adj_t);
        ix->adj_t = nullptr;
        return e;
    }
    k_degree<<<(unsigned)((ix->n + 255) / 256), 256>>>(ix->adj0, ix->n, ix->deg0, deg);
    k_tag_adj<<<(unsigned)((ne + 255) / 256), 256>>>(ix->adj0, ne, deg, 8 * tiles, ix->adj_t);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    cudaFree(deg);
    if (e != cudaSuccess) {
        cudaFree(ix->adj_t);
        ix->adj_t = nullptr;
    }
    return e;
}

// FP8-e4m3 residual codes from the FP32 tables (modes LP and FINGER_F8): codes
// of code_scale * u in the tensor cores' fragment order, per node 2 tiles of 16
// slots (4 when deg0 > 32) x 1 (r <= 32) or 2 k pairs x 512 bytes, plus the
// tagged adjacency
cudaError_t fp8_rebuild(finger_index* ix) {
    using namespace fg;
    cudaFree(ix->edge_q);
    ix->edge_q = nullptr;
    const int64_t n = ix->n;
    if (n >= (int64_t(1) << 30)) return cudaErrorInvalidValue;
    const int hks = ix->r > 32 ? 4 : 2;
    const int tiles = ix->deg0 > 32 ? 4 : 2;
    const int64_t units = n * tiles * (hks / 2) * 32;
    cudaError_t e = cudaMalloc(&ix->edge_q, sizeof(uint4) * (size_t)units + 16);
    if (e != cudaSuccess) {
        ix->edge_q = nullptr;
        return e;
    }
    // FP8 products where a block needs at most four of them (the search
    // kernel's rule), else the FP16 layout its conversions expect
    const int k32 = tiles * (hks / 2) <= 4;
    k_lp_codes<<<(unsigned)((units + 255) / 256), 256>>>(ix->edge_u, n, ix->deg0, ix->r_pad, tiles,
                                                         hks / 2, ix->code_scale, k32,
                                                         reinterpret_cast<uint4*>(ix->edge_q));
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        cudaFree(ix->edge_q);
        ix->edge_q = nullptr;
        return e;
    }
    ix->hks = hks;
    return build_tagged_adj(ix);
}

// BF16 rows (mode LP) and the FP8 codes
cudaError_t lp_rebuild(finger_index* ix) {
    using namespace fg;
    cudaFree(ix->Xh);
    ix->Xh = nullptr;
    const int64_t n = ix->n;
    cudaError_t e = cudaMalloc(&ix->Xh, sizeof(__nv_bfloat16) * (size_t)n * ix->m8 * 8 + 16);
    if (e != cudaSuccess) {
        ix->Xh = nullptr;
        return e;
    }
    e = launch_to_bf16(ix->X, n, ix->m_pad, ix->m8, ix->Xh, 0);
    if (e == cudaSuccess) e = fp8_rebuild(ix);
    if (e != cudaSuccess) {
        cudaFree(ix->Xh);
        ix->Xh = nullptr;
    }
    return e;
}

// FP16 unit residual codes from the FP32 tables (mode FINGER_F16), in the
// tensor cores' A-fragment order: per node 2 tiles of 16 slots (4 when
// deg0 > 32; rows beyond deg0 are zero) x 2 k steps of 16 codes (4 when
// r > 32) x 512 bytes
cudaError_t half_rebuild(finger_index* ix) {
    using namespace fg;
    cudaFree(ix->edge_h);
    ix->edge_h = nullptr;
    if (ix->n >= (int64_t(1) << 30)) return cudaErrorInvalidValue;
    const int hks = ix->r > 32 ? 4 : 2;
    const int tiles = ix->deg0 > 32 ? 4 : 2;
    const int64_t units = ix->n * tiles * hks * 32;
    cudaError_t e = cudaMalloc(&ix->edge_h, sizeof(uint4) * (size_t)units + 16);
    if (e != cudaSuccess) return e;
    k_half_codes<<<(unsigned)((units + 255) / 256), 256>>>(ix->edge_u, ix->n, ix->deg0,
                                                          ix->r_pad, tiles, hks,
                                                          reinterpret_cast<uint4*>(ix->edge_h));
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return e;
    ix->hks = hks;
    return build_tagged_adj(ix);
}

namespace fg {

#define CKT(x)                        \
    do {                              \
        if ((x) != cudaSuccess) {     \
            status = FINGER_ERR_CUDA; \
            goto done;                \
        }                             \
    } while (0)

// Eigen-decomposition of G = sum over the drawn pairs of d_res d_res^T, kept
// in the index (diagonalised G and eigenvectors V) for the (seed, spn) draw it
// was computed from; a rebuild at another rank reuses it.
static finger_status ensure_eigen(finger_index* ix, const int3* pairs, int64_t np, uint64_t seed,
                                  int spn, cudaStream_t s) {
    if (ix->eig_G && ix->eig_seed == seed && ix->eig_spn == spn) return FINGER_OK;
    cudaFree(ix->eig_G);
    cudaFree(ix->eig_V);
    ix->eig_G = ix->eig_V = nullptr;
    const int m = ix->m, m4 = ix->m4, deg0 = ix->deg0;
    finger_status status = FINGER_OK;
    double* G = dalloc<double>((size_t)m * m);
    double* V = dalloc<double>((size_t)m * m);
    const int jb = std::max(1, std::min(ix->num_sms, (m + 63) / 64 * 4));
    double* red = dalloc<double>(2 * (size_t)jb);
    double2* rot = dalloc<double2>((size_t)m);
    int2* pr = dalloc<int2>((size_t)m);
    int* sweeps = dalloc<int>(1);
    float* bq = dalloc<float>((size_t)np);
    if (!G || !V || !red || !rot || !pr || !sweeps || !bq) {
        status = FINGER_ERR_OOM;
        goto done;
    }
    k_pair_b<<<(unsigned)((np * 32 + 255) / 256), 256, 0, s>>>(
        reinterpret_cast<const float4*>(ix->X), m4, ix->xnorm2, ix->adj0, deg0, pairs, np, bq);
    CKT(cudaGetLastError());
    CKT(cudaMemsetAsync(G, 0, sizeof(double) * m * m, s));
    {
        const dim3 grid((m + GT - 1) / GT, (m + GT - 1) / GT, (unsigned)((np + GCHUNK - 1) / GCHUNK));
        k_gram<<<grid, 256, 0, s>>>(ix->X, ix->m_pad, m, ix->adj0, deg0, pairs, bq, np, G);
        CKT(cudaGetLastError());
    }
    {
        std::vector<double> I((size_t)m * m, 0.0);
        for (int i = 0; i < m; ++i) I[(size_t)i * m + i] = 1.0;
        CKT(cudaMemcpyAsync(V, I.data(), sizeof(double) * I.size(), cudaMemcpyHostToDevice, s));
        int max_sweeps = 40;
        double tol = 1e-15;
        int mm = m;
        void* args[] = {&G, &V, (void*)&mm, &rot, &pr, &red, &max_sweeps, &tol, &sweeps};
        CKT(cudaLaunchCooperativeKernel((void*)k_jacobi, dim3(jb), dim3(256), args, 0, s));
        CKT(cudaStreamSynchronize(s));
    }
    ix->eig_G = G;
    ix->eig_V = V;
    ix->eig_seed = seed;
    ix->eig_spn = spn;
    G = V = nullptr;
done:
    cudaFree(G);
    cudaFree(V);
    cudaFree(red);
    cudaFree(rot);
    cudaFree(pr);
    cudaFree(sweeps);
    cudaFree(bq);
    return status;
}

static finger_status run_sums(const double* Xc, const double* Yc, int64_t np, int mode, double mu,
                              double muh, double ratio, double* part, double* sums, double h[3],
                              cudaStream_t s) {
    const int nbp = 512;
    k_sum_part<<<nbp, 256, 0, s>>>(Xc, Yc, np, mode, mu, muh, ratio, part);
    k_sum_final<<<1, 32, 0, s>>>(part, nbp, sums);
    if (cudaMemcpyAsync(h, sums, 3 * sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return FINGER_ERR_CUDA;
    return FINGER_OK;
}

// Algorithm 2's statistics over the pairs (X, Y): mu, sigma, mu_hat, sigma_hat
// (standard deviations, 1/N), eps, and the correlation of X and Y.  flags:
// FINGER_BUILD_NO_MATCHING keeps t_hat (mu = mu_hat = 0, sigma = sigma_hat =
// 1, eps = mean |Y - X|); FINGER_BUILD_NO_EPS sets eps = 0.
static finger_status pair_stats(const double* Xc, const double* Yc, int64_t np, int flags,
                                double* part, double* sums, double st[5], double* corr,
                                cudaStream_t s) {
    double h[3];
    finger_status status = run_sums(Xc, Yc, np, 0, 0, 0, 0, part, sums, h, s);
    if (status != FINGER_OK) return status;
    const double N = h[2] > 0 ? h[2] : 1.0;
    const double mu = h[0] / N, muh = h[1] / N;
    status = run_sums(Xc, Yc, np, 1, mu, muh, 0, part, sums, h, s);
    if (status != FINGER_OK) return status;
    const double sigma = sqrt(h[0] / N), sigmah = sqrt(h[1] / N);
    *corr = (h[0] > 0 && h[1] > 0) ? h[2] / sqrt(h[0] * h[1]) : 0.0;
    if (flags & FINGER_BUILD_NO_MATCHING) {
        st[0] = 0.0;
        st[1] = 1.0;
        st[2] = 0.0;
        st[3] = 1.0;
    } else {
        st[0] = mu;
        st[1] = sigma;
        st[2] = muh;
        st[3] = sigmah;
    }
    st[4] = 0.0;
    if (!(flags & FINGER_BUILD_NO_EPS)) {
        const double ratio = st[3] > 0 ? st[1] / st[3] : 0.0;
        status = run_sums(Xc, Yc, np, 2, st[0], st[2], ratio, part, sums, h, s);
        if (status != FINGER_OK) return status;
        st[4] = h[0] / N;
    }
    return FINGER_OK;
}

finger_status build_tables(finger_index* ix, const finger_build_params* p, cudaStream_t s) {
    const auto t0 = std::chrono::steady_clock::now();
    if (!ix->adj0) return FINGER_ERR_NOT_BUILT;
    const int r = p->r;
    if (r < 1 || r > MAX_R || r > ix->m) return FINGER_ERR_INVALID_ARG;
    if (p->flags & ~(FINGER_BUILD_NO_MATCHING | FINGER_BUILD_NO_EPS | FINGER_BUILD_HALF_CODES |
                     FINGER_BUILD_FP8_CODES))
        return FINGER_ERR_INVALID_ARG;
    if ((p->flags & (FINGER_BUILD_HALF_CODES | FINGER_BUILD_FP8_CODES) || p->build_lp) &&
        ix->n >= (int64_t(1) << 30))
        return FINGER_ERR_UNSUPPORTED;   // the code modes tag ids in bit 30
    const int spn = p->samples_per_node > 0 ? p->samples_per_node : 1;
    const int64_t n = ix->n;
    const int m = ix->m, m_pad = ix->m_pad, m4 = ix->m4, deg0 = ix->deg0;
    const int r_pad = (r + 3) & ~3;
    const int64_t np = n * spn;
    const int64_t ne = n * deg0;
    finger_status status = FINGER_OK;
    int3* pairs = nullptr;
    double* evals = nullptr;
    double *Xc = nullptr, *Yc = nullptr, *part = nullptr, *sums = nullptr;
    float* P = dalloc<float>((size_t)r_pad * m_pad);
    float* Pc = dalloc<float>((size_t)n * r_pad);
    float* edge_u = dalloc<float>((size_t)ne * r_pad);
    float2* edge_s = dalloc<float2>((size_t)ne);
    double st[5] = {0, 0, 0, 0, 0};
    double corr = 0.0;
    if (!P || !Pc || !edge_u || !edge_s) {
        status = FINGER_ERR_OOM;
        goto done;
    }
    pairs = dalloc<int3>((size_t)np);
    Xc = dalloc<double>((size_t)np);
    Yc = dalloc<double>((size_t)np);
    part = dalloc<double>(3 * 512);
    sums = dalloc<double>(3);
    evals = dalloc<double>((size_t)m);
    if (!pairs || !Xc || !Yc || !part || !sums || !evals) {
        status = FINGER_ERR_OOM;
        goto done;
    }
    k_sample<<<(unsigned)((np + 255) / 256), 256, 0, s>>>(ix->adj0, n, deg0, p->seed, spn, pairs);
    CKT(cudaGetLastError());
    if (p->basis_host) {
        std::vector<float> hp((size_t)r_pad * m_pad, 0.f);
        for (int k = 0; k < r; ++k)
            for (int j = 0; j < m; ++j) hp[(size_t)k * m_pad + j] = p->basis_host[(size_t)k * m + j];
        CKT(cudaMemcpyAsync(P, hp.data(), sizeof(float) * hp.size(), cudaMemcpyHostToDevice, s));
        CKT(cudaStreamSynchronize(s));
    } else {
        status = ensure_eigen(ix, pairs, np, p->seed, spn, s);
        if (status != FINGER_OK) goto done;
        k_pick_basis<<<1, 256, sizeof(int) * m, s>>>(ix->eig_G, ix->eig_V, m, r, r_pad, m_pad, P,
                                                     evals);
        CKT(cudaGetLastError());
    }
    {
        const dim3 grid((unsigned)((n + 63) / 64), (r_pad + 63) / 64);
        k_node_proj<<<grid, 256, 0, s>>>(ix->X, n, m_pad, P, r_pad, Pc);
        CKT(cudaGetLastError());
    }
    k_edge<<<(unsigned)((n * 32 + 127) / 128), 128, 0, s>>>(reinterpret_cast<const float4*>(ix->X),
                                                            m4, ix->xnorm2, ix->adj0, n, deg0, Pc,
                                                            r_pad, edge_u, edge_s);
    CKT(cudaGetLastError());
    k_pair_cos<<<(unsigned)((np * 32 + 255) / 256), 256, 0, s>>>(
        reinterpret_cast<const float4*>(ix->X), m4, ix->adj0, deg0, pairs, np, edge_u, edge_s,
        r_pad, Xc, Yc);
    CKT(cudaGetLastError());
    status = pair_stats(Xc, Yc, np, p->flags, part, sums, st, &corr, s);
    if (status != FINGER_OK) goto done;
    if (p->stats_host)
        for (int i = 0; i < 5; ++i) st[i] = p->stats_host[i];
    CKT(cudaStreamSynchronize(s));
    // reduced-precision tables
    cudaFree(ix->Xh);
    cudaFree(ix->edge_q);
    cudaFree(ix->edge_h);
    cudaFree(ix->adj_t);
    ix->Xh = nullptr;
    ix->edge_q = nullptr;
    ix->edge_h = nullptr;
    ix->adj_t = nullptr;
    ix->hks = 0;
done:
    cudaFree(pairs);
    cudaFree(evals);
    cudaFree(Xc);
    cudaFree(Yc);
    cudaFree(part);
    cudaFree(sums);
    if (status != FINGER_OK) {
        cudaFree(P);
        cudaFree(Pc);
        cudaFree(edge_u);
        cudaFree(edge_s);
        return status;
    }
    cudaFree(ix->P);
    cudaFree(ix->Pc);
    cudaFree(ix->edge_u);
    cudaFree(ix->edge_s);
    ix->P = P;
    ix->Pc = Pc;
    ix->edge_u = edge_u;
    ix->edge_s = edge_s;
    ix->r = r;
    ix->r_pad = r_pad;
    for (int i = 0; i < 5; ++i) ix->stats[i] = st[i];
    ix->corr = corr;
    if (p->build_lp && lp_rebuild(ix) != cudaSuccess) {
        cudaGetLastError();
        return FINGER_ERR_CUDA;
    }
    if ((p->flags & FINGER_BUILD_HALF_CODES) && half_rebuild(ix) != cudaSuccess) {
        cudaGetLastError();
        return FINGER_ERR_CUDA;
    }
    if ((p->flags & FINGER_BUILD_FP8_CODES) && !ix->edge_q && fp8_rebuild(ix) != cudaSuccess) {
        cudaGetLastError();
        return FINGER_ERR_CUDA;
    }
    ix->build_ms =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return FINGER_OK;
}

// Rank rule of Supplementary E (see finger_select_rank in finger.h).
finger_status select_rank(finger_index* ix, const finger_build_params* p, double threshold,
                          int r_step, int r_max, int* r_out, double* corr_trace, cudaStream_t s) {
    if (!ix->adj0) return FINGER_ERR_NOT_BUILT;
    if (p->basis_host || r_step < 1 || r_max < 1 || r_max > MAX_R || r_max > ix->m || !r_out ||
        !(threshold == threshold))
        return FINGER_ERR_INVALID_ARG;
    const int spn = p->samples_per_node > 0 ? p->samples_per_node : 1;
    const int64_t n = ix->n, np = n * spn;
    const int m = ix->m, m_pad = ix->m_pad, deg0 = ix->deg0;
    const int rp_max = (r_max + 3) & ~3;
    const int nr = (r_max + r_step - 1) / r_step;
    finger_status status = FINGER_OK;
    int3* pairs = dalloc<int3>((size_t)np);
    double* Xc = dalloc<double>((size_t)np);
    double* Yk = dalloc<double>((size_t)np * nr);
    double* part = dalloc<double>(3 * 512);
    double* sums = dalloc<double>(3);
    double* evals = dalloc<double>((size_t)m);
    float* P = dalloc<float>((size_t)rp_max * m_pad);
    int chosen = std::min(nr * r_step, r_max);
    const size_t smem = sizeof(float4) * 2 * (size_t)ix->m4 * PREFIX_WARPS;
    if (!pairs || !Xc || !Yk || !part || !sums || !evals || !P) {
        status = FINGER_ERR_OOM;
        goto done;
    }
    if (smem > 200 * 1024) {
        status = FINGER_ERR_UNSUPPORTED;
        goto done;
    }
    k_sample<<<(unsigned)((np + 255) / 256), 256, 0, s>>>(ix->adj0, n, deg0, p->seed, spn, pairs);
    CKT(cudaGetLastError());
    status = ensure_eigen(ix, pairs, np, p->seed, spn, s);
    if (status != FINGER_OK) goto done;
    k_pick_basis<<<1, 256, sizeof(int) * m, s>>>(ix->eig_G, ix->eig_V, m, r_max, rp_max, m_pad, P,
                                                 evals);
    CKT(cudaGetLastError());
    if (smem > 48 * 1024)
        CKT(cudaFuncSetAttribute(k_pair_cos_prefix, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem));
    k_pair_cos_prefix<<<(unsigned)((np + PREFIX_WARPS - 1) / PREFIX_WARPS), 32 * PREFIX_WARPS, smem,
                        s>>>(reinterpret_cast<const float4*>(ix->X), ix->m4, ix->xnorm2, ix->adj0,
                             deg0, pairs, np, P, m_pad, r_max, r_step, Xc, Yk);
    CKT(cudaGetLastError());
    for (int i = 0; i < nr; ++i) {
        double st[5], corr = 0.0;
        status = pair_stats(Xc, Yk + (size_t)i * np, np, FINGER_BUILD_NO_EPS, part, sums, st, &corr,
                            s);
        if (status != FINGER_OK) goto done;
        if (corr_trace) corr_trace[i] = corr;
        if (corr >= threshold || i == nr - 1) {
            chosen = std::min((i + 1) * r_step, r_max);
            break;
        }
    }
done:
    cudaFree(pairs);
    cudaFree(Xc);
    cudaFree(Yk);
    cudaFree(part);
    cudaFree(sums);
    cudaFree(evals);
    cudaFree(P);
    if (status != FINGER_OK) return status;
    finger_build_params q = *p;
    q.r = chosen;
    status = build_tables(ix, &q, s);
    if (status == FINGER_OK) *r_out = chosen;
    return status;
}

}  // namespace fg

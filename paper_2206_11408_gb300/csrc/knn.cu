// Exact K-nearest-neighbour search by brute force (ground truth for recall,
// Sec. 1, and the candidate lists of the graph builder).
//
// A CTA owns QB = 32 queries and streams every base row.  Tiles of
// 32 queries x 128 rows are computed with FP32 FFMA on (q - x)^2 in k-chunks of
// 32 dimensions staged transposed in shared memory (each thread a 4 x 4 block).
// After a tile, values below a query's current K-th key are appended to that
// query's candidate buffer and one warp per query inserts them into a sorted
// top-K list kept in shared memory.  Keys are (distance, id).  In causal mode
// (queries and base rows the same array) query row i considers base rows < i
// only, and tiles above the diagonal are not computed.
#include <float.h>

#include "internal.cuh"

namespace fg {

namespace {

constexpr int QB = 32, XB = 128, KC = 32, NT = 256;

__device__ __forceinline__ bool klt(float da, int ia, float db, int ib) {
    return da < db || (da == db && ia < ib);
}

__global__ void __launch_bounds__(NT) k_knn(const float4* __restrict__ X, int64_t nb, int m4,
                                            const float* __restrict__ Q, int64_t q_stride,
                                            int q_m, int64_t nq, int K, int exclude_self,
                                            int causal, const int32_t* __restrict__ remap,
                                            int64_t* out_ids, float* out_d) {
    extern __shared__ __align__(16) unsigned char sm[];
    float* Qs = reinterpret_cast<float*>(sm);          // KC x QB
    float* Xs = Qs + KC * QB;                          // KC x XB
    float* bd = Xs + KC * XB;                          // QB x XB candidate dists
    int* bi = reinterpret_cast<int*>(bd + QB * XB);    // QB x XB candidate ids
    int* bc = bi + QB * XB;                            // QB counts
    float* ld = reinterpret_cast<float*>(bc + QB);     // QB x K list dists
    int* li = reinterpret_cast<int*>(ld + QB * K);     // QB x K list ids
    float* thr_d = reinterpret_cast<float*>(li + QB * K);
    int* thr_i = reinterpret_cast<int*>(thr_d + QB);
    int* lsz = thr_i + QB;

    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int64_t q0 = (int64_t)blockIdx.x * QB;
    const int tq = t >> 5;     // 0..7 -> queries tq*4 .. +4
    const int tx = t & 31;     // 0..31 -> rows tx*4 .. +4
    for (int i = t; i < QB; i += NT) {
        bc[i] = 0;
        lsz[i] = 0;
        thr_d[i] = INFINITY;
        thr_i[i] = 0x7fffffff;
    }
    const int m = m4 * 4;
    const int64_t x_end = causal ? (q0 + QB < nb ? q0 + QB : nb) : nb;
    for (int64_t x0 = 0; x0 < x_end; x0 += XB) {
        float acc[4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
        for (int k0 = 0; k0 < m; k0 += KC) {
            __syncthreads();
            // stage Q chunk (transposed): QB x KC
            for (int i = t; i < QB * KC; i += NT) {
                const int qq = i / KC, kk = i % KC;
                const int64_t gq = q0 + qq;
                const int gk = k0 + kk;
                Qs[kk * QB + qq] = (gq < nq && gk < q_m) ? Q[gq * q_stride + gk] : 0.f;
            }
            // stage X chunk (transposed): XB rows x KC dims
            {
                const int row = t & (XB - 1), half = t >> 7;   // 2 threads per row
                const int64_t gx = x0 + row;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int kk = half * 16 + j * 4;
                    const int c4 = (k0 + kk) >> 2;
                    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (gx < nb && c4 < m4) v = __ldg(X + gx * m4 + c4);
                    Xs[(kk + 0) * XB + row] = v.x;
                    Xs[(kk + 1) * XB + row] = v.y;
                    Xs[(kk + 2) * XB + row] = v.z;
                    Xs[(kk + 3) * XB + row] = v.w;
                }
            }
            __syncthreads();
#pragma unroll 8
            for (int kk = 0; kk < KC; ++kk) {
                const float4 qv = *reinterpret_cast<const float4*>(Qs + kk * QB + tq * 4);
                const float4 xv = *reinterpret_cast<const float4*>(Xs + kk * XB + tx * 4);
                const float qa[4] = {qv.x, qv.y, qv.z, qv.w};
                const float xa[4] = {xv.x, xv.y, xv.z, xv.w};
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int b = 0; b < 4; ++b) {
                        const float d = qa[a] - xa[b];
                        acc[a][b] = fmaf(d, d, acc[a][b]);
                    }
            }
        }
        // candidates below the current threshold
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            const int qq = tq * 4 + a;
            const int64_t gq = q0 + qq;
            if (gq >= nq) continue;
            const int64_t self = exclude_self ? (remap ? (int64_t)remap[gq] : gq) : -1;
            const float td = thr_d[qq];
            const int ti = thr_i[qq];
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const int64_t gx = x0 + tx * 4 + b;
                if (gx >= nb || (causal && gx >= gq)) continue;
                const int gid = remap ? remap[gx] : (int)gx;
                if (gid == self) continue;
                if (klt(acc[a][b], gid, td, ti)) {
                    const int pos = atomicAdd(&bc[qq], 1);
                    bd[qq * XB + pos] = acc[a][b];
                    bi[qq * XB + pos] = gid;
                }
            }
        }
        __syncthreads();
        // merge: one warp per query (8 warps, 4 queries each)
        for (int qq = warp; qq < QB; qq += NT / 32) {
            const int nc = bc[qq];
            float* L = ld + qq * K;
            int* Li = li + qq * K;
            int sz = lsz[qq];
            for (int c = 0; c < nc; ++c) {
                const float d = bd[qq * XB + c];
                const int id = bi[qq * XB + c];
                if (sz == K && !klt(d, id, L[K - 1], Li[K - 1])) continue;
                int p = 0;
                for (int b0 = 0; b0 < sz; b0 += 32) {
                    const int i = b0 + lane;
                    p += __popc(__ballot_sync(0xffffffffu, i < sz && klt(L[i], Li[i], d, id)));
                }
                const int last = sz < K ? sz : K - 1;
                for (int top = last - 1; top >= p; top -= 32) {
                    const int i = top - lane;
                    float vd = 0.f;
                    int vi = 0;
                    if (i >= p) {
                        vd = L[i];
                        vi = Li[i];
                    }
                    __syncwarp();
                    if (i >= p) {
                        L[i + 1] = vd;
                        Li[i + 1] = vi;
                    }
                    __syncwarp();
                }
                if (lane == 0) {
                    L[p] = d;
                    Li[p] = id;
                }
                __syncwarp();
                if (sz < K) sz++;
            }
            if (lane == 0) {
                lsz[qq] = sz;
                bc[qq] = 0;
                if (sz == K) {
                    thr_d[qq] = L[K - 1];
                    thr_i[qq] = Li[K - 1];
                }
            }
        }
        __syncthreads();
    }
    for (int i = t; i < QB * K; i += NT) {
        const int qq = i / K, k = i % K;
        const int64_t gq = q0 + qq;
        if (gq >= nq) continue;
        const bool ok = k < lsz[qq];
        out_ids[gq * K + k] = ok ? (int64_t)li[qq * K + k] : (int64_t)-1;
        out_d[gq * K + k] = ok ? ld[qq * K + k] : INFINITY;
    }
}

}  // namespace

size_t knn_smem(int K) {
    return sizeof(float) * (KC * QB + KC * XB + QB * XB) + sizeof(int) * (QB * XB + QB) +
           (sizeof(float) + sizeof(int)) * QB * K + (sizeof(float) + 2 * sizeof(int)) * QB;
}

// Q: nq rows with stride q_stride floats of which the first q_m are read (the
// rest count as 0, matching the zero padding of the base rows).  remap (optional) maps base row -> id
// reported (and query row -> its own id for exclusion).
cudaError_t launch_knn(const float4* Xb, int64_t nb, int m4, const float* Q, int64_t q_stride,
                       int q_m, int64_t nq, int K, bool exclude_self,
                       const int32_t* remap, int64_t* out_ids, float* out_d, cudaStream_t s,
                       bool causal) {
    if (nq == 0) return cudaSuccess;
    const size_t smem = knn_smem(K);
    cudaError_t e = cudaFuncSetAttribute(k_knn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    const int64_t grid = (nq + QB - 1) / QB;
    k_knn<<<(unsigned)grid, NT, smem, s>>>(Xb, nb, m4, Q, q_stride, q_m, nq, K, exclude_self ? 1 : 0,
                                           causal ? 1 : 0, remap, out_ids, out_d);
    return cudaGetLastError();
}

}  // namespace fg

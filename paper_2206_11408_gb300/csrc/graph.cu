// HNSW-style graph construction on the device (the graph FINGER accelerates;
// FINGER is built on top of a given graph, Sec. 3.3).
//
// Levels are drawn as in HNSW: level(v) = floor(-ln U_v / ln M) with U_v from
// the counter-based generator splitmix64(seed ^ v).  Nodes are inserted in id
// order (the rows are i.i.d., so this is a random order).  For every level l
// the nodes with level >= l form a layer; its edges come from
//   1. the exact `candidates` nearest neighbours among the layer's nodes with a
//      smaller id (HNSW's efConstruction search over the nodes inserted
//      before, made exact; brute force with a causal mask, knn.cu; up to 256 on
//      the small upper layers).  The first nodes of a cluster thus link to
//      other clusters, as in HNSW.  `symmetric` takes all of the layer's nodes;
//   2. the HNSW neighbour-selection heuristic over those candidates, sorted by
//      (distance, id): keep a candidate only if it is strictly closer to the
//      node than to every neighbour kept so far, up to M forward links;
//   3. reverse links: every forward link v -> u offers v to u;
//   4. a second heuristic pass over forward links plus the closest offered
//      reverse links, up to the layer cap (2M on layer 0, M above).
// The entry point is the lowest id among the nodes of the top level.
#include <math.h>

#include <algorithm>
#include <vector>

#include "internal.cuh"

namespace fg {

namespace {

constexpr int IN_CAP = 64;   // reverse links considered per node (closest first)

__device__ __forceinline__ bool klt(float da, uint32_t ia, float db, uint32_t ib) {
    return da < db || (da == db && ia < ib);
}

__device__ __forceinline__ float wsum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Heuristic selection for one node per warp.  cand row w: ids (int64, -1 ends
// the list) and dists, ascending.  Writes up to Mmax kept ids (PAD filled) to
// out row w (width out_w) and their distances to out_d.
__global__ void k_select(const float4* __restrict__ X, int m4, const int64_t* __restrict__ cid,
                         const float* __restrict__ cd, int kc, int64_t rows, int Mmax,
                         uint32_t* out, float* out_d, int out_w, const int64_t* __restrict__ out_row) {
    __shared__ uint32_t kept_s[4][64];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int64_t w = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib;
    if (w >= rows) return;
    uint32_t* kept = kept_s[wib];
    float kd[2] = {0.f, 0.f};   // lane j holds dist of kept j (j < 32) and j+32
    int nk = 0;
    for (int i = 0; i < kc && nk < Mmax; ++i) {
        const int64_t e = cid[w * kc + i];
        if (e < 0) break;
        const float de = cd[w * kc + i];
        float4 xe[8];
#pragma unroll
        for (int v = 0; v < 8; ++v) {
            const int k = lane + 32 * v;
            xe[v] = k < m4 ? __ldg(X + e * m4 + k) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        bool good = true;
        for (int j = 0; j < nk && good; ++j) {
            const uint32_t kj = kept[j];
            float acc = 0.f;
#pragma unroll
            for (int v = 0; v < 8; ++v) {
                const int k = lane + 32 * v;
                if (k < m4) {
                    const float4 y = __ldg(X + (size_t)kj * m4 + k);
                    float d;
                    d = xe[v].x - y.x; acc = fmaf(d, d, acc);
                    d = xe[v].y - y.y; acc = fmaf(d, d, acc);
                    d = xe[v].z - y.z; acc = fmaf(d, d, acc);
                    d = xe[v].w - y.w; acc = fmaf(d, d, acc);
                }
            }
            const float dek = wsum(acc);
            if (!(de < dek)) good = false;
        }
        if (good) {
            if (lane == 0) kept[nk] = (uint32_t)e;
            if (lane == (nk & 31)) kd[nk >> 5] = de;
            __syncwarp();
            nk++;
        }
    }
    const int64_t orow = out_row ? out_row[w] : w;
    for (int j = lane; j < out_w; j += 32) {
        out[orow * out_w + j] = j < nk ? kept[j] : PAD;
        if (out_d) out_d[orow * out_w + j] = j < nk ? kd[j >> 5] : INFINITY;
    }
}

__global__ void k_count_in(const uint32_t* fwd, int64_t rows, int w, const int32_t* cmap,
                           int* in_cnt) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rows * w) return;
    const uint32_t u = fwd[i];
    if (u == PAD) return;
    atomicAdd(&in_cnt[cmap ? cmap[u] : (int)u], 1);
}

__global__ void k_fill_in(const uint32_t* fwd, const float* fwd_d, int64_t rows, int w,
                          const int32_t* cmap, const int32_t* nodes, const int64_t* in_off,
                          int* in_fill, uint32_t* in_src, float* in_d) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rows * w) return;
    const uint32_t u = fwd[i];
    if (u == PAD) return;
    const int cu = cmap ? cmap[u] : (int)u;
    const int64_t v_row = i / w;
    const uint32_t v = nodes ? (uint32_t)nodes[v_row] : (uint32_t)v_row;
    const int pos = atomicAdd(&in_fill[cu], 1);
    in_src[in_off[cu] + pos] = v;
    in_d[in_off[cu] + pos] = fwd_d[i];
}

// per node (warp): candidates = forward links (sorted) + the IN_CAP closest
// reverse links, merged by (distance, id) with duplicates removed.
__global__ void k_merge_cands(const uint32_t* fwd, const float* fwd_d, int fw, int64_t rows,
                              const int64_t* in_off, const uint32_t* in_src, const float* in_d,
                              int64_t* cid, float* cd, int kc) {
    __shared__ float sd[4][IN_CAP];
    __shared__ uint32_t si[4][IN_CAP];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int64_t w = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib;
    if (w >= rows) return;
    float* L = sd[wib];
    uint32_t* Li = si[wib];
    int sz = 0;
    const int64_t b = in_off[w], e = in_off[w + 1];
    for (int64_t t = b; t < e; ++t) {
        const float d = in_d[t];
        const uint32_t id = in_src[t];
        if (sz == IN_CAP && !klt(d, id, L[IN_CAP - 1], Li[IN_CAP - 1])) continue;
        int p = 0;
        for (int b0 = 0; b0 < sz; b0 += 32) {
            const int i = b0 + lane;
            p += __popc(__ballot_sync(0xffffffffu, i < sz && klt(L[i], Li[i], d, id)));
        }
        const int last = sz < IN_CAP ? sz : IN_CAP - 1;
        for (int top = last - 1; top >= p; top -= 32) {
            const int i = top - lane;
            float vd = 0.f;
            uint32_t vi = 0;
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
        if (sz < IN_CAP) sz++;
    }
    if (lane == 0) {
        int a = 0, c = 0, o = 0;
        const uint32_t* F = fwd + w * fw;
        const float* Fd = fwd_d + w * fw;
        int fn = 0;
        while (fn < fw && F[fn] != PAD) fn++;
        uint32_t lastid = PAD;
        while ((a < fn || c < sz) && o < kc) {
            bool takeF;
            if (a >= fn) takeF = false;
            else if (c >= sz) takeF = true;
            else takeF = !klt(L[c], Li[c], Fd[a], F[a]);
            const uint32_t id = takeF ? F[a] : Li[c];
            const float d = takeF ? Fd[a] : L[c];
            if (takeF) a++; else c++;
            if (id == lastid) continue;
            lastid = id;
            cid[w * kc + o] = id;
            cd[w * kc + o] = d;
            o++;
        }
        for (; o < kc; ++o) {
            cid[w * kc + o] = -1;
            cd[w * kc + o] = INFINITY;
        }
    }
}

__global__ void k_gather_rows(const float4* X, int m4, const int32_t* nodes, int64_t cnt,
                              float4* out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= cnt * m4) return;
    const int64_t r = i / m4, k = i % m4;
    out[i] = X[(int64_t)nodes[r] * m4 + k];
}

uint64_t splitmix64(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

#define CK(x)                                   \
    do {                                        \
        cudaError_t e_ = (x);                   \
        if (e_ != cudaSuccess) {                \
            status = FINGER_ERR_CUDA;           \
            goto done;                          \
        }                                       \
    } while (0)

template <class T>
T* dalloc(size_t count) {
    void* p = nullptr;
    if (cudaMalloc(&p, count * sizeof(T) + 16) != cudaSuccess) return nullptr;
    return static_cast<T*>(p);
}

// one layer: nodes (device, compact -> global id, or null for all n), returns rows
// of width out_w at out_row[...] (global rows for layer 0, up_adj rows above)
finger_status build_layer(finger_index* ix, const int32_t* d_nodes, int64_t cnt, int kc, int Mf,
                          int Mmax, uint32_t* out, int out_w, const int64_t* d_out_row,
                          const int32_t* d_cmap, bool causal, bool tensor, cudaStream_t s) {
    finger_status status = FINGER_OK;
    const int m4 = ix->m4;
    float4* Xl = nullptr;
    int64_t* cid = nullptr;
    float* cd = nullptr;
    uint32_t* fwd = nullptr;
    float* fwd_d = nullptr;
    int* in_cnt = nullptr;
    int64_t* in_off = nullptr;
    uint32_t* in_src = nullptr;
    float* in_d = nullptr;
    int64_t* cid2 = nullptr;
    float* cd2 = nullptr;
    std::vector<int> h_cnt;
    std::vector<int64_t> h_off;
    const int kc2 = Mf + IN_CAP;
    const int kk = (int)std::min<int64_t>(kc, cnt - 1);
    const int64_t wblocks = (cnt + 3) / 4;
    if (cnt <= 1 || kk <= 0) {
        // a single node has no neighbours
        std::vector<uint32_t> pad((size_t)cnt * out_w, PAD);
        if (cnt == 1) {
            int64_t row = 0;
            if (d_out_row) CK(cudaMemcpy(&row, d_out_row, sizeof(int64_t), cudaMemcpyDeviceToHost));
            CK(cudaMemcpy(out + row * out_w, pad.data(), sizeof(uint32_t) * out_w,
                          cudaMemcpyHostToDevice));
        }
        return FINGER_OK;
    }
    if (d_nodes) {
        Xl = dalloc<float4>((size_t)cnt * m4);
        if (!Xl) return FINGER_ERR_OOM;
        k_gather_rows<<<(unsigned)((cnt * m4 + 255) / 256), 256, 0, s>>>(
            reinterpret_cast<const float4*>(ix->X), m4, d_nodes, cnt, Xl);
        CK(cudaGetLastError());
    }
    cid = dalloc<int64_t>((size_t)cnt * kk);
    cd = dalloc<float>((size_t)cnt * kk);
    fwd = dalloc<uint32_t>((size_t)cnt * Mf);
    fwd_d = dalloc<float>((size_t)cnt * Mf);
    in_cnt = dalloc<int>((size_t)cnt);
    in_off = dalloc<int64_t>((size_t)cnt + 1);
    cid2 = dalloc<int64_t>((size_t)cnt * kc2);
    cd2 = dalloc<float>((size_t)cnt * kc2);
    if (!cid || !cd || !fwd || !fwd_d || !in_cnt || !in_off || !cid2 || !cd2) {
        status = FINGER_ERR_OOM;
        goto done;
    }
    if (tensor && causal && !d_nodes)   // layer 0: causal candidates on the tensor cores
        CK(launch_knn_tc_causal(ix, kk, cid, cd, s));
    else
        CK(launch_knn(d_nodes ? Xl : reinterpret_cast<const float4*>(ix->X), cnt, m4,
                      d_nodes ? reinterpret_cast<const float*>(Xl) : ix->X, (int64_t)m4 * 4,
                      m4 * 4, cnt, kk, true, d_nodes, cid, cd, s, causal));
    k_select<<<(unsigned)wblocks, 128, 0, s>>>(reinterpret_cast<const float4*>(ix->X), m4, cid, cd,
                                               kk, cnt, Mf, fwd, fwd_d, Mf, nullptr);
    CK(cudaGetLastError());
    CK(cudaMemsetAsync(in_cnt, 0, sizeof(int) * cnt, s));
    k_count_in<<<(unsigned)((cnt * Mf + 255) / 256), 256, 0, s>>>(fwd, cnt, Mf, d_cmap, in_cnt);
    CK(cudaGetLastError());
    h_cnt.resize(cnt);
    h_off.resize(cnt + 1);
    CK(cudaMemcpyAsync(h_cnt.data(), in_cnt, sizeof(int) * cnt, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    h_off[0] = 0;
    for (int64_t i = 0; i < cnt; ++i) h_off[i + 1] = h_off[i] + h_cnt[i];
    CK(cudaMemcpyAsync(in_off, h_off.data(), sizeof(int64_t) * (cnt + 1), cudaMemcpyHostToDevice, s));
    in_src = dalloc<uint32_t>((size_t)std::max<int64_t>(h_off[cnt], 1));
    in_d = dalloc<float>((size_t)std::max<int64_t>(h_off[cnt], 1));
    if (!in_src || !in_d) {
        status = FINGER_ERR_OOM;
        goto done;
    }
    CK(cudaMemsetAsync(in_cnt, 0, sizeof(int) * cnt, s));
    k_fill_in<<<(unsigned)((cnt * Mf + 255) / 256), 256, 0, s>>>(fwd, fwd_d, cnt, Mf, d_cmap,
                                                                 d_nodes, in_off, in_cnt, in_src,
                                                                 in_d);
    CK(cudaGetLastError());
    k_merge_cands<<<(unsigned)wblocks, 128, 0, s>>>(fwd, fwd_d, Mf, cnt, in_off, in_src, in_d,
                                                    cid2, cd2, kc2);
    CK(cudaGetLastError());
    k_select<<<(unsigned)wblocks, 128, 0, s>>>(reinterpret_cast<const float4*>(ix->X), m4, cid2,
                                               cd2, kc2, cnt, Mmax, out, nullptr, out_w, d_out_row);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(s));
done:
    cudaFree(Xl);
    cudaFree(cid);
    cudaFree(cd);
    cudaFree(fwd);
    cudaFree(fwd_d);
    cudaFree(in_cnt);
    cudaFree(in_off);
    cudaFree(in_src);
    cudaFree(in_d);
    cudaFree(cid2);
    cudaFree(cd2);
    return status;
}

}  // namespace

finger_status build_graph(finger_index* ix, const finger_graph_params* p, cudaStream_t s) {
    const int M = p->M;
    const int deg0 = 2 * M;
    if (M < 2 || deg0 > MAX_DEG0 || M > MAX_MUP) return FINGER_ERR_INVALID_ARG;
    int kc = p->candidates > 0 ? p->candidates : 2 * deg0;
    if (kc > 256 || kc < M) return FINGER_ERR_INVALID_ARG;
    const bool causal = p->symmetric == 0;
    const int64_t n = ix->n;
    finger_status status = FINGER_OK;
    // levels
    std::vector<int32_t> level(n);
    const double mL = 1.0 / log((double)M);
    int maxlevel = 0;
    for (int64_t i = 0; i < n; ++i) {
        const uint64_t h = splitmix64(p->level_seed ^ (uint64_t)i);
        const double u = (double)((h >> 11) + 1) * (1.0 / 9007199254740992.0);
        int l = p->flat ? 0 : (int)floor(-log(u) * mL);
        if (l > 30) l = 30;
        level[i] = l;
        maxlevel = std::max(maxlevel, l);
    }
    int entry = 0;
    for (int64_t i = 0; i < n; ++i)
        if (level[i] == maxlevel) {
            entry = (int)i;
            break;
        }
    std::vector<int64_t> up_off(n);
    int64_t rows = 0;
    for (int64_t i = 0; i < n; ++i) {
        up_off[i] = level[i] > 0 ? rows : -1;
        rows += level[i];
    }
    // release the previous graph and everything derived from it
    cudaFree(ix->adj0);
    cudaFree(ix->up_off);
    cudaFree(ix->up_adj);
    ix->adj0 = nullptr;
    ix->up_off = nullptr;
    ix->up_adj = nullptr;
    uint32_t* adj0 = dalloc<uint32_t>((size_t)n * deg0);
    int64_t* d_up_off = dalloc<int64_t>((size_t)n);
    uint32_t* up_adj = dalloc<uint32_t>((size_t)std::max<int64_t>(rows, 1) * M);
    int32_t* d_nodes = nullptr;
    int64_t* d_rows = nullptr;
    int32_t* d_cmap = nullptr;
    if (!adj0 || !d_up_off || !up_adj) {
        cudaFree(adj0);
        cudaFree(d_up_off);
        cudaFree(up_adj);
        return FINGER_ERR_OOM;
    }
    {
        CK(cudaMemcpy(d_up_off, up_off.data(), sizeof(int64_t) * n, cudaMemcpyHostToDevice));
        status = build_layer(ix, nullptr, n, kc, M, deg0, adj0, deg0, nullptr, nullptr, causal,
                             p->fp32_candidates == 0, s);
        if (status != FINGER_OK) goto done;
        if (maxlevel > 0) {
            d_nodes = dalloc<int32_t>((size_t)n);
            d_rows = dalloc<int64_t>((size_t)n);
            d_cmap = dalloc<int32_t>((size_t)n);
            if (!d_nodes || !d_rows || !d_cmap) {
                status = FINGER_ERR_OOM;
                goto done;
            }
        }
        for (int l = 1; l <= maxlevel; ++l) {
            std::vector<int32_t> nodes;
            std::vector<int64_t> orow;
            for (int64_t i = 0; i < n; ++i)
                if (level[i] >= l) {
                    nodes.push_back((int32_t)i);
                    orow.push_back(up_off[i] + l - 1);
                }
            const int64_t cnt = (int64_t)nodes.size();
            std::vector<int32_t> cmap(n, -1);
            for (int64_t j = 0; j < cnt; ++j) cmap[nodes[j]] = (int32_t)j;
            CK(cudaMemcpy(d_nodes, nodes.data(), sizeof(int32_t) * cnt, cudaMemcpyHostToDevice));
            CK(cudaMemcpy(d_rows, orow.data(), sizeof(int64_t) * cnt, cudaMemcpyHostToDevice));
            CK(cudaMemcpy(d_cmap, cmap.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice));
            // upper layers are small: offer up to 256 exact candidates so that the
            // selection sees beyond a node's own cluster and keeps long links
            status = build_layer(ix, d_nodes, cnt, (int)std::min<int64_t>(cnt - 1, 256), M, M,
                                 up_adj, M, d_rows, d_cmap, causal, false, s);
            if (status != FINGER_OK) goto done;
        }
    }
done:
    cudaFree(d_nodes);
    cudaFree(d_rows);
    cudaFree(d_cmap);
    if (status != FINGER_OK) {
        cudaFree(adj0);
        cudaFree(d_up_off);
        cudaFree(up_adj);
        return status;
    }
    ix->adj0 = adj0;
    ix->up_off = d_up_off;
    ix->up_adj = up_adj;
    ix->deg0 = deg0;
    ix->M = M;
    ix->maxlevel = maxlevel;
    ix->entry = entry;
    ix->up_rows = rows;
    ix->h_level = level;
    return FINGER_OK;
}

}  // namespace fg

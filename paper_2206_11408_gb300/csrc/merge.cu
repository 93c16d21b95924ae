// Top-K merge of per-shard search results (database-partitioned search).
//
// The K nearest neighbours of a query over a partitioned database are the K
// smallest (distance, id) keys of the union of the partitions' own K nearest
// (the kNN problem of Sec. 1 applied to the union; keys ordered as in the
// search, distance then id).  One warp per query ranks every candidate of the
// S lists against all others and writes those of rank < K to their slot.
#include "internal.cuh"

namespace fg {

namespace {

constexpr int MAX_SHARDS = 64;

struct ShardOffsets {
    int64_t off[MAX_SHARDS];
};

__global__ void k_merge_shards(const int64_t* __restrict__ ids, const float* __restrict__ d, int S,
                               int64_t nq, int K, ShardOffsets a, int64_t* out_ids, float* out_d) {
    const int lane = threadIdx.x & 31;
    const int64_t q = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (q >= nq) return;
    const int nc = S * K;
    int valid = 0;
    for (int i = lane; i < nc; i += 32) {
        const int s = i / K, k = i - s * K;
        const size_t x = ((size_t)s * nq + q) * K + k;
        const int64_t id = ids[x];
        if (id < 0) continue;
        valid++;
        const int64_t gi = id + a.off[s];
        const float di = d[x];
        int rank = 0;
        for (int j = 0; j < nc; ++j) {
            const int sj = j / K, kj = j - sj * K;
            const size_t y = ((size_t)sj * nq + q) * K + kj;
            const int64_t idj = ids[y];
            if (idj < 0) continue;
            const float dj = d[y];
            const int64_t gj = idj + a.off[sj];
            rank += dj < di || (dj == di && gj < gi);
        }
        if (rank < K) {
            out_ids[q * K + rank] = gi;
            out_d[q * K + rank] = di;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) valid += __shfl_xor_sync(0xffffffffu, valid, o);
    for (int k = valid + lane; k < K; k += 32) {
        out_ids[q * K + k] = -1;
        out_d[q * K + k] = INFINITY;
    }
}

}  // namespace

}  // namespace fg

using namespace fg;

extern "C" {

finger_status finger_merge_topk(const int64_t* ids, const float* dists, int shards, int64_t nq,
                                int K, const int64_t* id_offsets, int64_t* out_ids,
                                float* out_dists, void* stream) {
    if (shards < 1 || shards > MAX_SHARDS || nq < 0 || K < 1 || K > 1024 || !id_offsets)
        return FINGER_ERR_INVALID_ARG;
    if (nq == 0) return FINGER_OK;
    if (!ids || !dists || !out_ids || !out_dists) return FINGER_ERR_INVALID_ARG;
    ShardOffsets a{};
    for (int s = 0; s < shards; ++s) {
        if (id_offsets[s] < 0) return FINGER_ERR_INVALID_ARG;
        a.off[s] = id_offsets[s];
    }
    const int wpb = 4;
    k_merge_shards<<<(unsigned)((nq + wpb - 1) / wpb), 32 * wpb, 0, (cudaStream_t)stream>>>(
        ids, dists, shards, nq, K, a, out_ids, out_dists);
    if (cudaGetLastError() != cudaSuccess) return FINGER_ERR_CUDA;
    return FINGER_OK;
}

}  // extern "C"

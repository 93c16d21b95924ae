// Internal declarations of libfinger.so (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <stdint.h>

#include <map>
#include <string>
#include <vector>

#include "../../include/finger.h"

namespace fg {

constexpr uint32_t PAD = 0xFFFFFFFFu;     // empty adjacency slot / empty hash slot
constexpr uint32_t EXP = 0x80000000u;     // "expanded" flag kept in the result-list ids
constexpr int MAX_M = 1024;
constexpr int MAX_DEG0 = 64;
constexpr int MAX_MUP = 32;
constexpr int MAX_R = 64;
// BF16 padding of the predictor's shared-memory feature rows: a row stride of
// 8 mod 16 elements keeps the 16-byte feature stores and the MMA fragment loads
// free of bank conflicts
constexpr int MLP_PAD = 8;
constexpr int MAX_EF = 1024;
constexpr int MLP_H = 64;                 // hidden width of the learned predictor

// Device view of an index, passed by value to the kernels.
struct DevIndex {
    int64_t n;
    int m, m4, m8;          // dims; float4 chunks per FP32 row; uint4 chunks per BF16 row
    int deg0, Mup, maxlevel, entry;
    const float4* X;        // n x m4
    const float* xnorm2;    // n
    const uint32_t* adj0;   // n x deg0
    const int64_t* up_off;  // n
    const uint32_t* up_adj; // up_rows x Mup
    // FINGER tables
    int r, r4;              // rank; float4 chunks of r_pad
    const float4* P;        // r_pad x m4
    const float4* Pc;       // n x r4
    const float4* edge_u;   // (n*deg0) x r4
    const float2* edge_s;   // n*deg0: {||d_res||, b}
    float alpha, beta;      // t = t_hat * alpha + beta
    // reduced precision
    const uint4* Xh;        // n x m8 (BF16)
    // FP8-e4m3 codes of edge_u * code_scale (modes LP and FINGER_F8) in the 8-bit
    // A-fragment order of mma.m16n8k32: per node 2 NPL tiles x hks / 2 steps of
    // 32 codes x 32 lanes x 16 bytes
    const uint4* edge_q;
    float code_inv;         // 1 / code_scale
    // FP16 unit residual codes (mode FINGER_F16) in m16n8k16 A-fragment order:
    // per node 2 NPL tiles of 16 slots x hks k steps x 32 lanes x 16 bytes
    const uint4* edge_h;
    int hks;                // k steps of 16 codes: 2 (r <= 32) or 4 (r <= 64)
    // layer-0 adjacency for that mode: ids with bit 30 set when the neighbour
    // has more than 16 NPL neighbours (second half of its code block needed)
    const uint32_t* adj_t;
    // learned predictor: BF16 W1 (H x kp, zero padded beyond r+4) and W2 (H x H)
    // stored fragment-major for m16n8k16 B operands (uint2 per lane per
    // (n8 tile, k16 step)), w3 (H, BF16-valued FP32), FP32 biases
    const uint2* W1f;
    const uint2* W2f;
    const float* w3;
    const float* b1;
    const float* b2;
    float b3, mlp_eps;
    float mlp_delta;        // predictor only within mlp_delta * ub of ub; < 0: everywhere
    int mlp_kp;
};

struct SearchArgs {
    const float* Q;         // nq x m (row stride m)
    int64_t nq;
    int K, ef;              // uniform K / ef (batch arrays override when non-null)
    const int32_t* K_arr;
    const int32_t* ef_arr;
    const int64_t* out_off;
    int64_t* out_ids;
    float* out_d;
    int warmup;
    int ef_cap, H, rerank;
    int h16;                // 1: visited hash in 16-bit slots (n <= 4096 H)
    int max_expansions;
    uint32_t* work;         // [0] = next query
    int* err;
    unsigned long long* cnt;   // 8 summed counters
    int32_t* cnt_q;            // nq x 8 or null
    uint32_t* bitmap;          // slots x words
    int64_t words;
    uint32_t* spill;           // slots x spill_cap
    int spill_cap;
    int warp_smem;             // bytes per warp
    int blk_smem;              // bytes at the start of the block's smem (predictor weights)
    // harvest (learned predictor training data); used by the harvest mode only
    float* hv_feat;            // cap x (r+4)
    float* hv_target;          // cap
    int32_t* hv_trip;          // cap x 3: query, centre, neighbour
    unsigned long long* hv_count;
    int64_t hv_cap;
};

constexpr int MODE_HARVEST = 12;    // FINGER traversal that records predictor training data
// kernel instances of the public mode FINGER_F16 by k steps of the code table
constexpr int MODE_F16_K2 = 6;      // r <= 32
constexpr int MODE_F16_K4 = 7;      // r <= 64
// kernel instances of the public mode FINGER_LP (FP8 codes) by k steps
constexpr int MODE_LP_K2 = 8;
constexpr int MODE_LP_K4 = 9;
// kernel instances of the public mode FINGER_F8 (FP32 rows, FP8 codes) by k steps
constexpr int MODE_F8_K2 = 10;
constexpr int MODE_F8_K4 = 11;

// exact rows in flight per group of G lanes (VPL 16-byte chunks per lane)
__host__ __device__ constexpr int rows_per_group(int VPL) { return VPL >= 8 ? 1 : VPL >= 4 ? 2 : 4; }
// and per warp
__host__ __device__ constexpr int rows_in_flight(int G, int VPL) {
    return (32 / G) * rows_per_group(VPL);
}

struct SearchPlan {
    int mode;
    int G, VPL, NPL;
    int wpb;            // warps per block
    int blocks;
    int ef_cap, H;
    int h16;            // visited hash in 16-bit slots
    int occ;            // resident blocks of 4 warps per SM the kernel variant is compiled for
    int bps;            // resident blocks per SM of this plan (its register and shared-memory limit)
    int shape;          // row shape: 0 the default (G, VPL), 1 rows on all 32 lanes
    int smem_per_warp;
    int blk_smem;       // per-block shared memory before the warp regions
};

// kernels / launchers (search.cu)
cudaError_t launch_search(const DevIndex& ix, const SearchArgs& a, const SearchPlan& p,
                          cudaStream_t s);
int search_smem_per_warp(const DevIndex& ix, int mode, int ef_cap, int H, int NPL, int h16);
cudaError_t search_occupancy(const DevIndex& ix, const SearchPlan& p, int* blocks_per_sm);
void choose_groups(int nchunks, int* G, int* VPL);

// brute force (knn.cu); causal: query row i sees base rows < i only
cudaError_t launch_knn(const float4* Xb, int64_t nb, int m4, const float* Q, int64_t q_stride,
                       int q_m, int64_t nq, int K, bool exclude_self, const int32_t* remap,
                       int64_t* out_ids, float* out_d, cudaStream_t s, bool causal = false);
size_t knn_smem(int K);
// tensor-core exact kNN (knn_tc.cu): K <= knn_tc_max_k()
int knn_tc_max_k();
cudaError_t launch_knn_tc(finger_index* ix, const float* Q, int64_t nq, int K, int64_t* out_ids,
                          float* out_d, cudaStream_t s);
cudaError_t launch_knn_tc_causal(finger_index* ix, int K, int64_t* out_ids, float* out_d,
                                 cudaStream_t s);

// graph construction (graph.cu)
finger_status build_graph(finger_index* ix, const finger_graph_params* p, cudaStream_t s);
// FINGER tables (tables.cu)
finger_status build_tables(finger_index* ix, const finger_build_params* p, cudaStream_t s);
finger_status select_rank(finger_index* ix, const finger_build_params* p, double threshold,
                          int r_step, int r_max, int* r_out, double* corr_trace, cudaStream_t s);
cudaError_t launch_xnorm2(const float4* X, int64_t n, int m4, float* out, cudaStream_t s);
cudaError_t launch_to_bf16(const float* X, int64_t n, int m_pad, int m8, __nv_bfloat16* out,
                           cudaStream_t s);

}  // namespace fg

// The index object behind the opaque handle.
struct finger_index {
    int device = 0;
    int num_sms = 0;
    int64_t n = 0;
    int m = 0, m_pad = 0, m4 = 0, m8 = 0;
    float* X = nullptr;
    float* xnorm2 = nullptr;
    __nv_bfloat16* xs_hi = nullptr;   // BF16 high / low parts of X (tensor-core kNN), lazily
    __nv_bfloat16* xs_lo = nullptr;
    // graph
    int deg0 = 0, M = 0, maxlevel = 0, entry = 0;
    int64_t up_rows = 0;
    uint32_t* adj0 = nullptr;
    int64_t* up_off = nullptr;
    uint32_t* up_adj = nullptr;
    std::vector<int32_t> h_level;
    // FINGER tables
    int r = 0, r_pad = 0;
    float* P = nullptr;
    float* Pc = nullptr;
    float* edge_u = nullptr;
    float2* edge_s = nullptr;
    double stats[5] = {0, 0, 0, 0, 0};
    double corr = 0.0 / 0.0;
    // eigen-decomposition of the D_res Gram matrix (diagonalised G and its
    // eigenvectors), kept for rebuilds at another rank with the same draw
    double* eig_G = nullptr;
    double* eig_V = nullptr;
    uint64_t eig_seed = 0;
    int eig_spn = 0;
    // LP tables
    __nv_bfloat16* Xh = nullptr;  // BF16 rows (mode LP)
    uint8_t* edge_q = nullptr;   // fragment-order FP8 codes (modes LP and FINGER_F8, see DevIndex)
    // FP16 codes (fragment order, see DevIndex)
    uint16_t* edge_h = nullptr;
    int hks = 0;
    uint32_t* adj_t = nullptr;    // tagged layer-0 adjacency (see DevIndex)
    float code_scale = 256.0f;
    // learned predictor
    int has_mlp = 0;
    int mlp_kp = 0;
    uint2* W1f = nullptr;         // fragment-major BF16 (see DevIndex)
    uint2* W2f = nullptr;
    float* w3 = nullptr;
    float* b1 = nullptr;
    float* b2 = nullptr;
    float b3 = 0.f, mlp_eps = 0.f;
    float mlp_delta = -1.f;       // see DevIndex
    std::vector<float> h_mlp;     // FP32 master copy (W1, b1, W2, b2, w3, b3)
    // search state
    int mode = FINGER_MODE_PLAIN;
    int warmup = 5;
    int max_expansions = 0;       // 0 = n + 16
    int visited_bits = 0;         // visited-hash slots: 0 = 16-bit where they fit, 32 = always 32-bit
    int32_t* cnt_q = nullptr;
    // scratch
    uint32_t* work = nullptr;     // 4 words
    int* err = nullptr;
    unsigned long long* cnt = nullptr;
    uint32_t* bitmap = nullptr;
    int64_t bitmap_slots = 0, words = 0;
    uint32_t* spill = nullptr;
    int spill_cap = 0;
    // staging for host-buffer search
    float* stage_q = nullptr;
    int64_t* stage_ids = nullptr;
    float* stage_d = nullptr;
    int64_t stage_cap_q = 0, stage_cap_o = 0;
    std::map<int, fg::SearchPlan> tuned;     // autotuned plans keyed by ef bucket
    std::map<int, float> tuned_ms;           // their best sample-batch time
    int64_t searches = 0;
    double build_ms = 0;
    int64_t device_bytes = 0;
    std::vector<void*> allocs;
};

fg::DevIndex make_dev(const finger_index* ix);

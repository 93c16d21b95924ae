// Uneven query batches (per-query K and ef) in one persistent launch, replayed
// from captured CUDA graphs, with launch shapes chosen by an autotuner.
//
// A batch runs the same search kernel as finger_search with the per-query K /
// ef arrays and output offsets.  The launch is sized for the batch's bound on
// ef (bucketed to a power of two): result-list capacity, visited-hash size and
// warps per block come from the tuned plan of that bucket if the autotuner ran
// for it, else from the default heuristic.  The first call for an (nq bucket,
// ef bucket) shape (powers of two) captures the work-counter reset and the
// kernel into a CUDA graph; later calls of that shape update the kernel node's
// arguments (queries, sizes, outputs) and replay the graph.
#include <string.h>

#include <algorithm>
#include <chrono>
#include <mutex>
#include <vector>

#include "internal.cuh"

using namespace fg;

finger_status fg_make_plan(finger_index* ix, int mode, int ef_max, int64_t nq, SearchPlan* p,
                           int wpb, int H, int occ = 0, int shape = 0);
finger_status fg_run_search(finger_index* ix, const SearchPlan& p, SearchArgs& a, cudaStream_t s);
SearchArgs fg_base_args(finger_index* ix, const SearchPlan& p);
finger_status fg_check_mode_ready(const finger_index* ix, int mode);
finger_status fg_ensure_scratch(finger_index* ix, int64_t slots);

namespace {

int bucket_of(int ef) {
    int b = 16;
    while (b < ef) b <<= 1;
    return b;
}

struct Captured {
    cudaGraph_t graph = nullptr;        // kept: its kernel node is updated per call
    cudaGraphExec_t exec = nullptr;
    cudaGraphNode_t knode = nullptr;
    cudaKernelNodeParams kp{};
};

using CaptureMap = std::map<std::pair<int64_t, int>, Captured>;

// Captured graphs of every index, keyed by index.  The outer map is shared by
// all indices, so every lookup, insertion and removal of an index's entry
// holds the mutex; the inner map of one index is touched only by calls on
// that index (which callers serialise) and std::map keeps its node in place
// while other indices come and go.
std::map<const finger_index*, CaptureMap>& captures() {
    static std::map<const finger_index*, CaptureMap> c;
    return c;
}
std::mutex& captures_mutex() {
    static std::mutex mu;
    return mu;
}
CaptureMap& captures_of(const finger_index* ix) {
    std::lock_guard<std::mutex> lock(captures_mutex());
    return captures()[ix];
}

}  // namespace

void fg_drop_captures(const finger_index* ix) {
    std::lock_guard<std::mutex> lock(captures_mutex());
    auto it = captures().find(ix);
    if (it == captures().end()) return;
    for (auto& kv : it->second) {
        if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
        if (kv.second.graph) cudaGraphDestroy(kv.second.graph);
    }
    captures().erase(it);
}

extern "C" {

finger_status finger_search_batch(finger_index* ix, const float* queries, int64_t nq,
                                  const int32_t* K, const int32_t* ef, int max_ef,
                                  const int64_t* out_off, int64_t* out_ids, float* out_dists,
                                  void* stream) {
    if (!ix || nq < 0 || max_ef < 1 || max_ef > MAX_EF) return FINGER_ERR_INVALID_ARG;
    if (nq == 0) return FINGER_OK;
    if (!queries || !K || !ef || !out_off || !out_ids || !out_dists) return FINGER_ERR_INVALID_ARG;
    finger_status st = fg_check_mode_ready(ix, ix->mode);
    if (st != FINGER_OK) return st;
    int prev = 0;
    cudaGetDevice(&prev);
    if (prev != ix->device) cudaSetDevice(ix->device);
    cudaStream_t s = (cudaStream_t)stream;
    const int bucket = std::min(bucket_of(max_ef), MAX_EF);
    // launch shapes are keyed by power-of-two buckets of nq and ef, so one
    // captured graph serves every batch of its bucket (surplus warps exit)
    int64_t nqb = 1;
    while (nqb < nq) nqb <<= 1;
    SearchPlan p;
    auto tit = ix->tuned.find(bucket);
    if (tit != ix->tuned.end() && tit->second.mode == ix->mode) {
        p = tit->second;
        st = fg_make_plan(ix, ix->mode, bucket, nqb, &p, p.wpb, p.H, p.occ, p.shape);
        if (st != FINGER_OK) {   // (not expected: the tuner ran this shape)
            cudaGetLastError();
            st = fg_make_plan(ix, ix->mode, bucket, nqb, &p, 4, 0);
        }
    } else {
        st = fg_make_plan(ix, ix->mode, bucket, nqb, &p, 4, 0);
    }
    if (st != FINGER_OK) {
        if (prev != ix->device) cudaSetDevice(prev);
        return st;
    }
    st = fg_ensure_scratch(ix, (int64_t)p.blocks * p.wpb);
    if (st != FINGER_OK) {
        if (prev != ix->device) cudaSetDevice(prev);
        return st;
    }
    SearchArgs a = fg_base_args(ix, p);
    a.Q = queries;
    a.nq = nq;
    a.K = 0;
    a.ef = bucket;
    a.K_arr = K;
    a.ef_arr = ef;
    a.out_off = out_off;
    a.out_ids = out_ids;
    a.out_d = out_dists;
    a.rerank = 32;
    const DevIndex d = make_dev(ix);
    const auto key = std::make_pair(nqb, bucket * 4 + ix->mode);
    auto& caps = captures_of(ix);
    auto it = caps.find(key);
    finger_status ret = FINGER_OK;
    if (it == caps.end()) {
        // capture: reset the work counter, launch the kernel
        cudaGraph_t graph = nullptr;
        Captured c;
        cudaStream_t cs = nullptr;
        if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            ret = FINGER_ERR_CUDA;
        } else {
            bool ok = cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed) == cudaSuccess;
            ok = ok && cudaMemsetAsync(ix->work, 0, sizeof(uint32_t), cs) == cudaSuccess;
            ok = ok && launch_search(d, a, p, cs) == cudaSuccess;
            ok = (cudaStreamEndCapture(cs, &graph) == cudaSuccess) && ok;
            if (ok) {
                size_t nn = 0;
                cudaGraphGetNodes(graph, nullptr, &nn);
                std::vector<cudaGraphNode_t> nodes(nn);
                cudaGraphGetNodes(graph, nodes.data(), &nn);
                for (auto n : nodes) {
                    cudaGraphNodeType t;
                    cudaGraphNodeGetType(n, &t);
                    if (t == cudaGraphNodeTypeKernel) {
                        c.knode = n;
                        cudaGraphKernelNodeGetParams(n, &c.kp);
                    }
                }
                ok = c.knode && cudaGraphInstantiate(&c.exec, graph, 0) == cudaSuccess;
            }
            cudaStreamDestroy(cs);
            if (!ok) {
                if (c.exec) cudaGraphExecDestroy(c.exec);
                if (graph) cudaGraphDestroy(graph);
                cudaGetLastError();
                ret = FINGER_ERR_CUDA;
            } else {
                c.graph = graph;
                it = caps.emplace(key, c).first;
            }
        }
    }
    if (ret == FINGER_OK) {
        Captured& c = it->second;
        DevIndex dd = d;
        SearchArgs aa = a;
        void* args[] = {&dd, &aa};
        cudaKernelNodeParams kp = c.kp;
        kp.kernelParams = args;
        kp.extra = nullptr;
        if (cudaGraphExecKernelNodeSetParams(c.exec, c.knode, &kp) != cudaSuccess ||
            cudaGraphLaunch(c.exec, s) != cudaSuccess) {
            cudaGetLastError();
            ret = FINGER_ERR_CUDA;
        } else {
            ix->searches += nq;
        }
    }
    if (prev != ix->device) cudaSetDevice(prev);
    return ret;
}

// Autotuner: time the candidate launch shapes of an ef bucket on a sample batch
// (device queries, uniform K/ef) and keep the fastest for finger_search_batch.
// Candidates: warps per block {2, 4, 8} x visited-hash slots {H/2, H, 2H}
// around the default H x the kernel's register variants (the one with the
// most resident warps that shared memory admits, and each one the mode has
// with fewer: 64 / 80 / 96 registers, compiled for 32 / 24 / 20 resident
// warps) x the exact-row shape (the default groups of lanes per row, and rows
// on all 32 lanes: fewer rows in flight per warp, the staging depth).
// Returns the best time in *best_ms (may be NULL); finger_get_tuned reads
// the pick back.
finger_status finger_autotune(finger_index* ix, const float* queries, int64_t nq, int K, int ef,
                              int64_t* scratch_ids, float* scratch_dists, float* best_ms,
                              void* stream) {
    if (!ix || !queries || nq < 1 || K < 1 || ef < K || ef > MAX_EF || !scratch_ids ||
        !scratch_dists)
        return FINGER_ERR_INVALID_ARG;
    finger_status st = fg_check_mode_ready(ix, ix->mode);
    if (st != FINGER_OK) return st;
    int prev = 0;
    cudaGetDevice(&prev);
    if (prev != ix->device) cudaSetDevice(ix->device);
    cudaStream_t s = (cudaStream_t)stream;
    const int bucket = std::min(bucket_of(ef), MAX_EF);
    // planned at the sample's ef: the shape a uniform search at that ef uses
    SearchPlan def;
    st = fg_make_plan(ix, ix->mode, ef, nq, &def, 4, 0);
    if (st != FINGER_OK) {
        if (prev != ix->device) cudaSetDevice(prev);
        return st;
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    SearchPlan bestp = def;
    const int Hs[3] = {std::max(256, def.H / 2), def.H, std::min(16384, def.H * 2)};
    const int Ws[3] = {2, 4, 8};
    const int Os[4] = {0, 8, 6, 5};   // 0: the largest variant that fits
    for (int wi = 0; wi < 3; ++wi)
        for (int hi = 0; hi < 3; ++hi)
            for (int oi = 0; oi < 4; ++oi)
                for (int sh = 0; sh < 2; ++sh) {
            SearchPlan p;
            if (fg_make_plan(ix, ix->mode, ef, nq, &p, Ws[wi], Hs[hi], Os[oi], sh) != FINGER_OK) {
                cudaGetLastError();
                continue;
            }
            if (oi > 0) {
                // a forced variant only when it is smaller than the automatic one
                SearchPlan a0;
                if (fg_make_plan(ix, ix->mode, ef, nq, &a0, Ws[wi], Hs[hi], 0) == FINGER_OK &&
                    Os[oi] >= a0.occ)
                    continue;
            }
            SearchArgs a = fg_base_args(ix, p);
            a.Q = queries;
            a.nq = nq;
            a.K = K;
            a.ef = ef;
            a.out_ids = scratch_ids;
            a.out_d = scratch_dists;
            a.rerank = std::min(ef, 2 * K);
            float tbest = 1e30f;
            for (int rep = 0; rep < 3; ++rep) {
                cudaEventRecord(e0, s);
                if (fg_run_search(ix, p, a, s) != FINGER_OK) break;
                cudaEventRecord(e1, s);
                cudaEventSynchronize(e1);
                float ms = 0;
                cudaEventElapsedTime(&ms, e0, e1);
                if (rep > 0) tbest = std::min(tbest, ms);
            }
            if (tbest < best) {
                best = tbest;
                bestp = p;
            }
                }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ix->tuned[bucket] = bestp;
    ix->tuned_ms[bucket] = best;
    fg_drop_captures(ix);
    if (best_ms) *best_ms = best;
    if (prev != ix->device) cudaSetDevice(prev);
    return cudaGetLastError() == cudaSuccess ? FINGER_OK : FINGER_ERR_CUDA;
}

finger_status finger_get_tuned(const finger_index* ix, int ef, int* warps_per_block,
                               int* hash_slots, int* resident_warps, int* rows_per_warp,
                               float* best_ms) {
    if (!ix || ef < 1 || ef > MAX_EF) return FINGER_ERR_INVALID_ARG;
    const int bucket = std::min(bucket_of(ef), MAX_EF);
    auto it = ix->tuned.find(bucket);
    if (it == ix->tuned.end() || it->second.mode != ix->mode) return FINGER_ERR_NOT_BUILT;
    if (warps_per_block) *warps_per_block = it->second.wpb;
    if (hash_slots) *hash_slots = it->second.H;
    if (resident_warps) *resident_warps = it->second.bps * it->second.wpb;
    if (rows_per_warp) *rows_per_warp = rows_in_flight(it->second.G, it->second.VPL);
    if (best_ms) {
        auto mt = ix->tuned_ms.find(bucket);
        *best_ms = mt == ix->tuned_ms.end() ? 0.f : mt->second;
    }
    return FINGER_OK;
}

}  // extern "C"

// finger_search_noalloc: the same search as finger_search, for callers that
// must not allocate device memory while they run.
//
// finger_search keeps per-warp scratch for its exact visited set (a bitmap of
// n bits per resident warp plus a list of the ids it set, used once a query's
// shared-memory hash is 3/4 full) and allocates or grows that scratch on
// first use and whenever a launch needs more resident warps than before.
// Some callers cannot accept an allocation inside a query call: serving
// processes that reserve their whole device-memory budget at start-up (a
// caching allocator already owns the rest of HBM, so a late cudaMalloc can fail
// or force the cache to release memory), and latency-critical loops for which
// cudaMalloc/cudaFree, which may synchronise the device and take unbounded
// time, are not allowed on the query path.  This entry point takes its scratch
// from one fixed array in device memory instead.
//
// The array is a file-scope __device__ array of NOALLOC_SCRATCH_BYTES (64 MiB).
// The CUDA runtime reserves it on every device that loads this library and it
// stays reserved until the process exits.  Host code cannot use the array's
// name as a device address, so the first call on each device (with that device
// current) looks the address up with cudaGetSymbolAddress and caches it; that
// first call should come before any stream capture.  Every call shares the
// array and the array keeps the previous call's contents.  What must start at
// zero is the work counter and every visited bitmap.  Each call clears the
// counter (the array's first 256 bytes).  The bitmaps need no clear per call:
// the kernel sets a bitmap bit only for an id it also appends to the query's
// spill list, and before the query ends (also when it stops at a limit) it
// zeroes every word the list names, so a launch that runs to completion leaves
// its bitmap region zero.  The spill lists follow that region and keep ids, so
// the library remembers, per device, where the zeroed region ends: a call
// whose bitmaps reach beyond it (the first call on a device, a larger n or
// more warps than the call before, or any call after one whose launch failed
// to enqueue) clears its whole bitmap region first.  Two calls whose kernels
// overlap on the GPU (on different streams, or from several host threads)
// race on the array; callers must serialise them.
//
// Capacity: a launch needs, per resident warp, ceil(n / 32) words of bitmap
// (padded to 16 bytes) and a spill list of min(max(n, 64), 65536) ids, the
// same list length as finger_search, so a query ends with the same results and
// status as there.  The launch uses as many warps as fit: at n = 1M about 176
// (finger_search runs several thousand), at n = 200k about 233; below four
// warps the block shrinks (n above roughly 1.3e8); if not even one warp fits
// (n above roughly 5e8) the call returns FINGER_ERR_UNSUPPORTED.
#include <algorithm>
#include <mutex>

#include "internal.cuh"

using namespace fg;

finger_status fg_make_plan(finger_index* ix, int mode, int ef_max, int64_t nq, SearchPlan* p,
                           int wpb, int H, int occ = 0, int shape = 0);
SearchArgs fg_base_args(finger_index* ix, const SearchPlan& p);
finger_status fg_check_mode_ready(const finger_index* ix, int mode);

namespace {

constexpr size_t NOALLOC_SCRATCH_BYTES = size_t(64) << 20;
constexpr size_t NOALLOC_HEADER = 256;     // work counter, padded
constexpr int NOALLOC_MAX_DEVICES = 64;
constexpr int NOALLOC_SPILL_CAP = 1 << 16;   // as in finger_search

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

void* g_scratch_addr[NOALLOC_MAX_DEVICES] = {};
// end (byte offset) of the bitmap region known to be zero after the last call
size_t g_zero_end[NOALLOC_MAX_DEVICES] = {};
std::mutex g_scratch_mu;

// device address of the scratch array on the current device (looked up once)
cudaError_t scratch_address(int device, void** out) {
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[device]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        if (!p) return cudaErrorInvalidSymbol;
        g_scratch_addr[device] = p;
    }
    *out = g_scratch_addr[device];
    return cudaSuccess;
}

size_t zero_end(int device) {
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    return g_zero_end[device];
}

void set_zero_end(int device, size_t end) {
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    g_zero_end[device] = end;
}

}  // namespace

extern "C" finger_status finger_search_noalloc(finger_index* ix, const float* queries, int64_t nq,
                                               int K, int ef, int64_t* out_ids, float* out_dists,
                                               void* stream) {
    if (!ix || nq < 0 || K < 1 || ef < K || ef > MAX_EF) return FINGER_ERR_INVALID_ARG;
    if (nq == 0) return FINGER_OK;
    if (!queries || !out_ids || !out_dists) return FINGER_ERR_INVALID_ARG;
    finger_status st = fg_check_mode_ready(ix, ix->mode);
    if (st != FINGER_OK) return st;
    if (ix->device < 0 || ix->device >= NOALLOC_MAX_DEVICES) return FINGER_ERR_UNSUPPORTED;
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != ix->device) cudaSetDevice(ix->device);
    finger_status ret = FINGER_OK;
    void* base = nullptr;
    SearchPlan p;
    if (scratch_address(ix->device, &base) != cudaSuccess) {
        cudaGetLastError();
        ret = FINGER_ERR_CUDA;
    } else if ((st = fg_make_plan(ix, ix->mode, ef, nq, &p, 4, 0)) != FINGER_OK) {
        ret = st;
    } else {
        const int64_t words = ((ix->n + 31) / 32 + 3) & ~int64_t(3);
        const int spill_cap = (int)std::min<int64_t>(std::max<int64_t>(ix->n, 64), NOALLOC_SPILL_CAP);
        const int64_t per_slot = words * 4 + (int64_t)spill_cap * 4;
        const int64_t max_slots = (int64_t)(NOALLOC_SCRATCH_BYTES - NOALLOC_HEADER) / per_slot;
        if (max_slots < 1) {
            ret = FINGER_ERR_UNSUPPORTED;
        } else {
            if ((int64_t)p.blocks * p.wpb > max_slots) {
                if (max_slots >= p.wpb) {
                    p.blocks = (int)(max_slots / p.wpb);
                } else {
                    p.wpb = (int)max_slots;
                    p.blocks = 1;
                }
            }
            const int64_t slots = (int64_t)p.blocks * p.wpb;
            unsigned char* b = static_cast<unsigned char*>(base);
            uint32_t* work = reinterpret_cast<uint32_t*>(b);
            uint32_t* bitmap = reinterpret_cast<uint32_t*>(b + NOALLOC_HEADER);
            uint32_t* spill = bitmap + slots * words;
            cudaStream_t s = (cudaStream_t)stream;
            // the array keeps the last call's contents: the work counter is
            // cleared on every call, this call's bitmap region only where it
            // reaches beyond the region known to be zero (see the file comment)
            const size_t need = NOALLOC_HEADER + (size_t)(slots * words * 4);
            const size_t clear = need <= zero_end(ix->device) ? NOALLOC_HEADER : need;
            if (cudaMemsetAsync(b, 0, clear, s) != cudaSuccess) {
                cudaGetLastError();
                set_zero_end(ix->device, 0);
                ret = FINGER_ERR_CUDA;
            } else {
                SearchArgs a = fg_base_args(ix, p);
                a.Q = queries;
                a.nq = nq;
                a.K = K;
                a.ef = ef;
                a.out_ids = out_ids;
                a.out_d = out_dists;
                a.rerank = std::min(ef, 2 * K);
                a.work = work;
                a.bitmap = bitmap;
                a.words = words;
                a.spill = spill;
                a.spill_cap = spill_cap;
                if (launch_search(make_dev(ix), a, p, s) != cudaSuccess) {
                    cudaGetLastError();
                    set_zero_end(ix->device, 0);
                    ret = FINGER_ERR_CUDA;
                } else {
                    set_zero_end(ix->device, need);
                    ix->searches += nq;
                }
            }
        }
    }
    if (prev >= 0 && prev != ix->device) cudaSetDevice(prev);
    return ret;
}

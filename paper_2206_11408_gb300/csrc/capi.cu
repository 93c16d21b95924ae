// C ABI of libfinger.so (declared in include/finger.h): index management,
// search planning and launches, file I/O.  Host code only; kernels live in
// search_m*.cu, knn.cu, graph.cu and tables.cu.
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <vector>

#include "internal.cuh"

namespace fg {
cudaError_t launch_mode0(const DevIndex&, const SearchArgs&, const SearchPlan&, cudaStream_t);
cudaError_t launch_mode1(const DevIndex&, const SearchArgs&, const SearchPlan&, cudaStream_t);
cudaError_t launch_lp_k2(const DevIndex&, const SearchArgs&, const SearchPlan&, cudaStream_t);
cudaError_t launch_lp_k4(const DevIndex&, const SearchArgs&, const SearchPlan&, cudaStream_t);
cudaError_t launch_mode3(const DevIndex&, const SearchArgs&, const SearchPlan&, cudaStream_t);
cudaError_t occupancy_mode0(const SearchPlan&, int*);
cudaError_t occupancy_mode1(const SearchPlan&, int*);
cudaError_t occupancy_lp_k2(const SearchPlan&, int*);
cudaError_t occupancy_lp_k4(const SearchPlan&, int*);
cudaError_t occupancy_mode3(const SearchPlan&, int*);
cudaError_t launch_f16_k2(const DevIndex&, const SearchArgs&, const SearchPlan&, cudaStream_t);
cudaError_t launch_f16_k4(const DevIndex&, const SearchArgs&, const SearchPlan&, cudaStream_t);
cudaError_t occupancy_f16_k2(const SearchPlan&, int*);
cudaError_t occupancy_f16_k4(const SearchPlan&, int*);
cudaError_t launch_f8_k2(const DevIndex&, const SearchArgs&, const SearchPlan&, cudaStream_t);
cudaError_t launch_f8_k4(const DevIndex&, const SearchArgs&, const SearchPlan&, cudaStream_t);
cudaError_t occupancy_f8_k2(const SearchPlan&, int*);
cudaError_t occupancy_f8_k4(const SearchPlan&, int*);
cudaError_t launch_mode_harvest(const DevIndex&, const SearchArgs&, const SearchPlan&,
                                cudaStream_t);
cudaError_t occupancy_mode_harvest(const SearchPlan&, int*);

void choose_groups(int nchunks, int* G, int* VPL) {
    if (nchunks <= 8) {
        *G = 8;
        *VPL = 1;
    } else if (nchunks <= 16) {
        *G = 16;
        *VPL = 1;
    } else if (nchunks <= 32) {
        // two chunks per lane, two rows per warp pass: eight rows in flight
        *G = 16;
        *VPL = 2;
    } else {
        *G = 32;
        const int v = (nchunks + 31) / 32;
        *VPL = v <= 1 ? 1 : v <= 2 ? 2 : v <= 4 ? 4 : 8;
    }
}

// the modes whose estimates are a tensor-core product with FP16 or FP8 codes
bool code_mode(int mode) {
    return mode == FINGER_MODE_FINGER_F16 || mode == FINGER_MODE_FINGER_LP ||
           mode == FINGER_MODE_FINGER_F8;
}

// length (floats) of the unit query-residual projection u_q in shared memory:
// the code modes hold its B fragments there, 16 words per k step
int search_uq_len(const DevIndex& ix, int mode) {
    const int r_pad = ix.r4 * 4;
    return code_mode(mode) ? std::max(r_pad, 16 * ix.hks) : r_pad;
}

int search_smem_per_warp(const DevIndex& ix, int mode, int ef_cap, int H, int NPL, int h16) {
    const int r_pad = ix.r4 * 4;
    const int uq_len = search_uq_len(ix, mode);
    const int qs_len = mode == FINGER_MODE_FINGER_LP ? ix.m8 * 8 : ix.m4 * 4;
    // the code modes keep the staged query in a region of its own
    const bool own_qs = code_mode(mode);
    const int qs_bytes = own_qs ? 4 * ((qs_len + 3) & ~3) : 0;
    const int tile = mode == FINGER_MODE_FINGER_MLP ? 2 * 16 * (ix.mlp_kp + MLP_PAD) : 0;
    int b = 8 * ef_cap + (h16 ? 2 : 4) * H + 4 * (uq_len + r_pad) + qs_bytes + 32 * 32 * NPL +
            32 + tile;
    return (b + 15) & ~15;
}

cudaError_t launch_search(const DevIndex& ix, const SearchArgs& a, const SearchPlan& p,
                          cudaStream_t s) {
    switch (p.mode) {
        case 0: return launch_mode0(ix, a, p, s);
        case 1: return launch_mode1(ix, a, p, s);
        case 2: return ix.hks == 2 ? launch_lp_k2(ix, a, p, s) : launch_lp_k4(ix, a, p, s);
        case 3: return launch_mode3(ix, a, p, s);
        case 4: return ix.hks == 2 ? launch_f16_k2(ix, a, p, s) : launch_f16_k4(ix, a, p, s);
        case 5: return ix.hks == 2 ? launch_f8_k2(ix, a, p, s) : launch_f8_k4(ix, a, p, s);
        case MODE_HARVEST: return launch_mode_harvest(ix, a, p, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t search_occupancy(const DevIndex& ix, const SearchPlan& p, int* bps) {
    switch (p.mode) {
        case 0: return occupancy_mode0(p, bps);
        case 1: return occupancy_mode1(p, bps);
        case 2: return ix.hks == 2 ? occupancy_lp_k2(p, bps) : occupancy_lp_k4(p, bps);
        case 3: return occupancy_mode3(p, bps);
        case 4: return ix.hks == 2 ? occupancy_f16_k2(p, bps) : occupancy_f16_k4(p, bps);
        case 5: return ix.hks == 2 ? occupancy_f8_k2(p, bps) : occupancy_f8_k4(p, bps);
        case MODE_HARVEST: return occupancy_mode_harvest(p, bps);
    }
    return cudaErrorInvalidValue;
}

}  // namespace fg

using namespace fg;

void fg_drop_captures(const finger_index* ix);

fg::DevIndex make_dev(const finger_index* ix) {
    DevIndex d{};
    d.n = ix->n;
    d.m = ix->m;
    d.m4 = ix->m4;
    d.m8 = ix->m8;
    d.deg0 = ix->deg0;
    d.Mup = ix->M;
    d.maxlevel = ix->maxlevel;
    d.entry = ix->entry;
    d.X = reinterpret_cast<const float4*>(ix->X);
    d.xnorm2 = ix->xnorm2;
    d.adj0 = ix->adj0;
    d.up_off = ix->up_off;
    d.up_adj = ix->up_adj;
    d.r = ix->r;
    d.r4 = ix->r_pad / 4;
    d.P = reinterpret_cast<const float4*>(ix->P);
    d.Pc = reinterpret_cast<const float4*>(ix->Pc);
    d.edge_u = reinterpret_cast<const float4*>(ix->edge_u);
    d.edge_s = ix->edge_s;
    const double mu = ix->stats[0], sigma = ix->stats[1], muh = ix->stats[2],
                 sigmah = ix->stats[3], eps = ix->stats[4];
    const double alpha = sigmah > 0 ? sigma / sigmah : 0.0;
    d.alpha = (float)alpha;
    d.beta = (float)(mu + eps - muh * alpha);
    d.Xh = reinterpret_cast<const uint4*>(ix->Xh);
    d.edge_q = reinterpret_cast<const uint4*>(ix->edge_q);
    d.code_inv = 1.0f / ix->code_scale;
    d.edge_h = reinterpret_cast<const uint4*>(ix->edge_h);
    d.hks = ix->hks;
    d.adj_t = ix->adj_t;
    d.W1f = ix->W1f;
    d.W2f = ix->W2f;
    d.w3 = ix->w3;
    d.b1 = ix->b1;
    d.b2 = ix->b2;
    d.b3 = ix->b3;
    d.mlp_eps = ix->mlp_eps;
    d.mlp_delta = ix->mlp_delta;
    d.mlp_kp = ix->mlp_kp;
    return d;
}

namespace {

#define CUDA_OK(x)                                  \
    do {                                            \
        if ((x) != cudaSuccess) {                   \
            return FINGER_ERR_CUDA;                 \
        }                                           \
    } while (0)

template <class T>
finger_status dmalloc(T** p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    if (cudaMalloc((void**)p, count * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        return FINGER_ERR_OOM;
    }
    return FINGER_OK;
}

int pow2ceil(int v) {
    int p = 1;
    while (p < v) p <<= 1;
    return p;
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

// default launch plan for a mode and a bound on ef
// default launch plan for a mode and a bound on ef; occ_force > 0 takes that
// resident-block variant (the autotuner's choice) instead of the largest one
// shared memory admits
// shape 0: the row shape choose_groups picks; shape 1: rows on all 32 lanes
// (fewer rows in flight, more chunks per load round), when that differs
finger_status make_plan(finger_index* ix, int mode, int ef_max, int64_t nq, SearchPlan* p,
                        int wpb = 4, int H = 0, int occ_force = 0, int shape = 0) {
    const DevIndex d = make_dev(ix);
    p->mode = mode;
    const int nchunks = mode == FINGER_MODE_FINGER_LP ? ix->m8 : ix->m4;
    choose_groups(nchunks, &p->G, &p->VPL);
    if (shape == 1) {
        if (p->G == 32) return FINGER_ERR_UNSUPPORTED;   // already the widest
        const int v = (nchunks + 31) / 32;
        p->G = 32;
        p->VPL = v <= 1 ? 1 : v <= 2 ? 2 : v <= 4 ? 4 : 8;
    } else if (shape != 0) {
        return FINGER_ERR_INVALID_ARG;
    }
    p->NPL = ix->deg0 > 32 ? 2 : 1;
    p->ef_cap = (ef_max + 3) & ~3;
    if (H <= 0) H = pow2ceil(std::min(std::max(16 * ef_max, 512), 2048));
    if (mode == FINGER_MODE_FINGER_LP) H = std::max(H, pow2ceil(2 * p->ef_cap));
    else H = std::max(H, pow2ceil(ix->m_pad));   // the query is staged in the hash region
    p->H = H;
    // 16-bit visited slots: ids must fit the bucket index plus 15 bits
    // (n <= 4096 H), and what reuses the table's H / 2 words must fit there:
    // the staged query (m_pad words) outside LP mode, the re-rank buffer
    // (2 ef_cap words) in LP mode
    p->h16 = ix->visited_bits != 32 && ix->n <= 4096 * (int64_t)H &&
             (mode == FINGER_MODE_FINGER_LP ? H >= 4 * p->ef_cap : H >= 2 * ix->m_pad);
    p->wpb = wpb;
    p->smem_per_warp = search_smem_per_warp(d, mode, p->ef_cap, p->H, p->NPL, p->h16);
    p->blk_smem = 0;
    if (p->blk_smem + (int64_t)p->smem_per_warp * wpb > 227 * 1024) return FINGER_ERR_UNSUPPORTED;
    // the kernel variant with the most resident blocks that shared memory admits:
    // 8 blocks (64 registers, plain mode), 6 (80 registers, plain, FP32 FINGER,
    // LP and FP16 codes), else 5 (96 registers)
    int bps = 0;
    p->occ = 5;
    if (occ_force > 0) {
        // the forced variant, at as many blocks as it admits
        SearchPlan t = *p;
        t.occ = occ_force;
        int b = 0;
        if (search_occupancy(d, t, &b) != cudaSuccess || b < 1) {
            cudaGetLastError();
            return FINGER_ERR_UNSUPPORTED;
        }
        p->occ = occ_force;
        bps = b;
    } else {
        for (int occ : {8, 6}) {
            SearchPlan t = *p;
            t.occ = occ;
            int b = 0;
            if (search_occupancy(d, t, &b) == cudaSuccess && b >= occ) {
                p->occ = occ;
                bps = b;
                break;
            }
            cudaGetLastError();
        }
    }
    if (p->occ == 5 && (search_occupancy(d, *p, &bps) != cudaSuccess || bps < 1)) {
        cudaGetLastError();
        return FINGER_ERR_UNSUPPORTED;
    }
    p->bps = bps;
    p->shape = shape;
    int64_t blocks = (int64_t)ix->num_sms * bps;
    blocks = std::min<int64_t>(blocks, (nq + wpb - 1) / wpb);
    p->blocks = (int)std::max<int64_t>(blocks, 1);
    return FINGER_OK;
}

// The plan of a uniform search: the autotuner's launch shape when one was
// kept for this mode and the power-of-two ef bucket of ef (finger_autotune),
// else the default.
finger_status make_search_plan(finger_index* ix, int ef, int64_t nq, SearchPlan* p) {
    int bucket = 16;
    while (bucket < ef) bucket <<= 1;
    bucket = std::min(bucket, MAX_EF);
    auto it = ix->tuned.find(bucket);
    if (it != ix->tuned.end() && it->second.mode == ix->mode) {
        SearchPlan t = it->second;
        if (make_plan(ix, ix->mode, ef, nq, &t, t.wpb, t.H, t.occ, t.shape) == FINGER_OK) {
            *p = t;
            return FINGER_OK;
        }
        cudaGetLastError();
    }
    return make_plan(ix, ix->mode, ef, nq, p);
}

finger_status ensure_scratch(finger_index* ix, int64_t slots) {
    const int64_t words = (ix->n + 31) / 32;
    if (slots <= ix->bitmap_slots && ix->bitmap) return FINGER_OK;
    cudaFree(ix->bitmap);
    cudaFree(ix->spill);
    ix->bitmap = nullptr;
    ix->spill = nullptr;
    ix->bitmap_slots = 0;
    const int spill_cap = (int)std::min<int64_t>(std::max<int64_t>(ix->n, 64), 1 << 16);
    finger_status st = dmalloc(&ix->bitmap, (size_t)(slots * words));
    if (st != FINGER_OK) return st;
    st = dmalloc(&ix->spill, (size_t)(slots * spill_cap));
    if (st != FINGER_OK) {
        cudaFree(ix->bitmap);
        ix->bitmap = nullptr;
        return st;
    }
    CUDA_OK(cudaMemset(ix->bitmap, 0, sizeof(uint32_t) * slots * words));
    ix->bitmap_slots = slots;
    ix->words = words;
    ix->spill_cap = spill_cap;
    return FINGER_OK;
}

finger_status check_mode_ready(const finger_index* ix, int mode) {
    if (!ix->adj0) return FINGER_ERR_NOT_BUILT;
    if (mode != FINGER_MODE_PLAIN && !ix->edge_u) return FINGER_ERR_NOT_BUILT;
    if (mode == FINGER_MODE_FINGER_LP && (!ix->Xh || !ix->edge_q || !ix->adj_t))
        return FINGER_ERR_NOT_BUILT;
    if (mode == FINGER_MODE_FINGER_F8 && (!ix->edge_q || !ix->adj_t)) return FINGER_ERR_NOT_BUILT;
    if (mode == FINGER_MODE_FINGER_F16 && (!ix->edge_h || !ix->adj_t)) return FINGER_ERR_NOT_BUILT;
    if (mode == FINGER_MODE_FINGER_MLP && !ix->has_mlp) return FINGER_ERR_NOT_BUILT;
    return FINGER_OK;
}

SearchArgs base_args(finger_index* ix, const SearchPlan& p) {
    SearchArgs a{};
    a.warmup = ix->warmup;
    a.ef_cap = p.ef_cap;
    a.H = p.H;
    a.h16 = p.h16;
    a.rerank = 0;
    a.max_expansions = ix->max_expansions > 0 ? ix->max_expansions
                                              : (int)std::min<int64_t>(ix->n + 16, 1 << 30);
    a.work = ix->work;
    a.err = ix->err;
    a.cnt = ix->cnt;
    a.cnt_q = ix->cnt_q;
    a.bitmap = ix->bitmap;
    a.words = ix->words;
    a.spill = ix->spill;
    a.spill_cap = ix->spill_cap;
    a.warp_smem = p.smem_per_warp;
    a.blk_smem = p.blk_smem;
    return a;
}

finger_status run_search(finger_index* ix, const SearchPlan& p, SearchArgs& a, cudaStream_t s) {
    finger_status st = ensure_scratch(ix, (int64_t)p.blocks * p.wpb);
    if (st != FINGER_OK) return st;
    a.bitmap = ix->bitmap;
    a.words = ix->words;
    a.spill = ix->spill;
    a.spill_cap = ix->spill_cap;
    CUDA_OK(cudaMemsetAsync(ix->work, 0, sizeof(uint32_t), s));
    const DevIndex d = make_dev(ix);
    if (launch_search(d, a, p, s) != cudaSuccess) {
        cudaGetLastError();
        return FINGER_ERR_CUDA;
    }
    ix->searches += a.nq;
    return FINGER_OK;
}

uint64_t wsum64(const void* p, size_t bytes) {
    const unsigned char* c = static_cast<const unsigned char*>(p);
    uint64_t h = 1469598103934665603ULL, s = 0;
    size_t i = 0;
    for (; i + 8 <= bytes; i += 8) {
        uint64_t v;
        memcpy(&v, c + i, 8);
        s += v * 0x9E3779B97F4A7C15ULL + (s >> 29);
    }
    for (; i < bytes; ++i) s = (s ^ c[i]) * 1099511628211ULL;
    return s ^ h ^ (uint64_t)bytes;
}

}  // namespace

// entry points shared with batch.cu
finger_status fg_make_plan(finger_index* ix, int mode, int ef_max, int64_t nq, SearchPlan* p,
                           int wpb, int H, int occ, int shape) {
    return make_plan(ix, mode, ef_max, nq, p, wpb, H, occ, shape);
}
finger_status fg_run_search(finger_index* ix, const SearchPlan& p, SearchArgs& a, cudaStream_t s) {
    return run_search(ix, p, a, s);
}
SearchArgs fg_base_args(finger_index* ix, const SearchPlan& p) { return base_args(ix, p); }
finger_status fg_check_mode_ready(const finger_index* ix, int mode) {
    return check_mode_ready(ix, mode);
}
finger_status fg_ensure_scratch(finger_index* ix, int64_t slots) {
    return ensure_scratch(ix, slots);
}

extern "C" {

const char* finger_status_str(finger_status s) {
    switch (s) {
        case FINGER_OK: return "ok";
        case FINGER_ERR_INVALID_ARG: return "invalid argument";
        case FINGER_ERR_IO: return "i/o error";
        case FINGER_ERR_FORMAT: return "bad index file format";
        case FINGER_ERR_OOM: return "out of memory";
        case FINGER_ERR_CUDA: return "CUDA error";
        case FINGER_ERR_NOT_BUILT: return "graph or tables not built";
        case FINGER_ERR_LIMIT: return "kernel iteration or capacity limit reached";
        case FINGER_ERR_UNSUPPORTED: return "unsupported size";
    }
    return "unknown status";
}

int64_t finger_table_bytes(int64_t n, int deg0, int r, int lp) {
    if (n < 0 || deg0 < 0 || r < 0) return -1;
    if (!lp) return (int64_t)(r + 2) * n * deg0 * (int64_t)sizeof(float);
    // FP8 codes: per node 32 (deg0 <= 32) or 64 slots x 32 or 64 codes, plus
    // the FP32 edge scalars of every slot
    const int64_t slots = deg0 > 32 ? 64 : 32, codes = r > 32 ? 64 : 32;
    return n * slots * codes + 8 * n * deg0;
}

finger_status finger_index_create(int device, int64_t n, int m, const float* vectors_host,
                                  finger_index** out) {
    if (!out || !vectors_host || n < 1 || n >= (1LL << 31) - 1 || m < 1) return FINGER_ERR_INVALID_ARG;
    if (m > MAX_M) return FINGER_ERR_UNSUPPORTED;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return FINGER_ERR_CUDA;
    }
    DeviceGuard g(device);
    finger_index* ix = new finger_index();
    ix->device = device;
    cudaDeviceGetAttribute(&ix->num_sms, cudaDevAttrMultiProcessorCount, device);
    ix->n = n;
    ix->m = m;
    ix->m_pad = (m + 7) & ~7;
    ix->m4 = ix->m_pad / 4;
    ix->m8 = ix->m_pad / 8;
    finger_status st = dmalloc(&ix->X, (size_t)n * ix->m_pad);
    if (st == FINGER_OK) st = dmalloc(&ix->xnorm2, (size_t)n);
    if (st == FINGER_OK) st = dmalloc(&ix->work, 4);
    if (st == FINGER_OK) st = dmalloc(&ix->err, 1);
    if (st == FINGER_OK) st = dmalloc(&ix->cnt, 16);
    if (st != FINGER_OK) {
        finger_index_free(ix);
        return st;
    }
    if (cudaMemset(ix->X, 0, sizeof(float) * n * ix->m_pad) != cudaSuccess ||
        cudaMemcpy2D(ix->X, sizeof(float) * ix->m_pad, vectors_host, sizeof(float) * m,
                     sizeof(float) * m, (size_t)n, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(ix->err, 0, sizeof(int)) != cudaSuccess ||
        cudaMemset(ix->cnt, 0, sizeof(unsigned long long) * 16) != cudaSuccess ||
        launch_xnorm2(reinterpret_cast<const float4*>(ix->X), n, ix->m4, ix->xnorm2, 0) !=
            cudaSuccess ||
        cudaDeviceSynchronize() != cudaSuccess) {
        cudaGetLastError();
        finger_index_free(ix);
        return FINGER_ERR_CUDA;
    }
    *out = ix;
    return FINGER_OK;
}

void finger_index_free(finger_index* ix) {
    if (!ix) return;
    DeviceGuard g(ix->device);
    fg_drop_captures(ix);
    void* ptrs[] = {ix->X, ix->xnorm2, ix->adj0, ix->up_off, ix->up_adj, ix->P, ix->Pc,
                    ix->edge_u, ix->edge_s, ix->Xh, ix->edge_q, ix->W1f, ix->W2f, ix->w3,
                    ix->b1, ix->b2, ix->work, ix->err, ix->cnt, ix->bitmap, ix->spill,
                    ix->stage_q, ix->stage_ids, ix->stage_d, ix->eig_G, ix->eig_V, ix->xs_hi,
                    ix->xs_lo, ix->edge_h, ix->adj_t};
    for (void* p : ptrs) cudaFree(p);
    delete ix;
}

static void drop_tables(finger_index* ix) {
    void* ptrs[] = {ix->P, ix->Pc, ix->edge_u, ix->edge_s, ix->Xh, ix->edge_q,
                    ix->W1f, ix->W2f, ix->w3, ix->b1, ix->b2, ix->eig_G, ix->eig_V,
                    ix->edge_h, ix->adj_t};
    for (void* p : ptrs) cudaFree(p);
    ix->eig_G = ix->eig_V = nullptr;
    ix->corr = 0.0 / 0.0;
    ix->P = ix->Pc = ix->edge_u = nullptr;
    ix->edge_s = nullptr;
    ix->Xh = nullptr;
    ix->edge_q = nullptr;
    ix->edge_h = nullptr;
    ix->adj_t = nullptr;
    ix->hks = 0;
    ix->W1f = ix->W2f = nullptr;
    ix->w3 = ix->b1 = ix->b2 = nullptr;
    ix->r = ix->r_pad = 0;
    ix->has_mlp = 0;
    ix->h_mlp.clear();
    ix->tuned.clear();
    ix->tuned_ms.clear();
    fg_drop_captures(ix);
}

finger_status finger_index_set_graph(finger_index* ix, int deg0, const int32_t* adj0,
                                     const int32_t* level, const int64_t* up_off, int64_t up_rows,
                                     int M, const int32_t* up_adj, int32_t entry,
                                     int32_t maxlevel) {
    if (!ix || !adj0 || !level || !up_off || deg0 < 1 || deg0 > MAX_DEG0 || M < 1 ||
        M > MAX_MUP || up_rows < 0 || (up_rows > 0 && !up_adj) || entry < 0 || entry >= ix->n ||
        maxlevel < 0)
        return FINGER_ERR_INVALID_ARG;
    const int64_t n = ix->n;
    // host-side validation: ids in range, rows packed, no duplicates, no self-loops
    std::vector<int32_t> seen(n, -1);
    int64_t rows_needed = 0;
    for (int64_t v = 0; v < n; ++v) {
        if (level[v] < 0 || level[v] > maxlevel) return FINGER_ERR_INVALID_ARG;
        if (level[v] > 0) {
            if (up_off[v] < 0 || up_off[v] + level[v] > up_rows) return FINGER_ERR_INVALID_ARG;
        }
        rows_needed += level[v];
        bool ended = false;
        for (int j = 0; j < deg0; ++j) {
            const int32_t u = adj0[v * deg0 + j];
            if (u < 0) {
                ended = true;
                continue;
            }
            if (ended || u >= n || u == v || seen[u] == (int32_t)v) return FINGER_ERR_INVALID_ARG;
            seen[u] = (int32_t)v;
        }
    }
    if (level[entry] != maxlevel) return FINGER_ERR_INVALID_ARG;
    // upper rows: ids in range, and a neighbour listed on level l has level >= l
    for (int64_t v = 0; v < n; ++v)
        for (int l = 1; l <= level[v]; ++l) {
            const int32_t* row = up_adj + (up_off[v] + l - 1) * M;
            for (int j = 0; j < M; ++j) {
                const int32_t u = row[j];
                if (u < 0) continue;
                if (u >= n || u == v || level[u] < l) return FINGER_ERR_INVALID_ARG;
            }
        }
    DeviceGuard g(ix->device);
    drop_tables(ix);
    cudaFree(ix->adj0);
    cudaFree(ix->up_off);
    cudaFree(ix->up_adj);
    ix->adj0 = nullptr;
    ix->up_off = nullptr;
    ix->up_adj = nullptr;
    finger_status st = dmalloc(&ix->adj0, (size_t)n * deg0);
    if (st == FINGER_OK) st = dmalloc(&ix->up_off, (size_t)n);
    if (st == FINGER_OK) st = dmalloc(&ix->up_adj, (size_t)std::max<int64_t>(up_rows, 1) * M);
    if (st != FINGER_OK) return st;
    CUDA_OK(cudaMemcpy(ix->adj0, adj0, sizeof(int32_t) * n * deg0, cudaMemcpyHostToDevice));
    CUDA_OK(cudaMemcpy(ix->up_off, up_off, sizeof(int64_t) * n, cudaMemcpyHostToDevice));
    if (up_rows > 0)
        CUDA_OK(cudaMemcpy(ix->up_adj, up_adj, sizeof(int32_t) * up_rows * M,
                           cudaMemcpyHostToDevice));
    ix->deg0 = deg0;
    ix->M = M;
    ix->up_rows = up_rows;
    ix->entry = entry;
    ix->maxlevel = maxlevel;
    ix->h_level.assign(level, level + n);
    (void)rows_needed;
    return FINGER_OK;
}

finger_status finger_build_graph(finger_index* ix, const finger_graph_params* p, void* stream) {
    if (!ix || !p) return FINGER_ERR_INVALID_ARG;
    DeviceGuard g(ix->device);
    drop_tables(ix);
    return build_graph(ix, p, (cudaStream_t)stream);
}

finger_status finger_get_graph(const finger_index* ix, int32_t* adj0, int32_t* level,
                               int64_t* up_off, int32_t* up_adj, int32_t* entry,
                               int32_t* maxlevel) {
    if (!ix) return FINGER_ERR_INVALID_ARG;
    if (!ix->adj0) return FINGER_ERR_NOT_BUILT;
    DeviceGuard g(ix->device);
    if (adj0)
        CUDA_OK(cudaMemcpy(adj0, ix->adj0, sizeof(int32_t) * ix->n * ix->deg0,
                           cudaMemcpyDeviceToHost));
    if (level) memcpy(level, ix->h_level.data(), sizeof(int32_t) * ix->n);
    if (up_off)
        CUDA_OK(cudaMemcpy(up_off, ix->up_off, sizeof(int64_t) * ix->n, cudaMemcpyDeviceToHost));
    if (up_adj && ix->up_rows > 0)
        CUDA_OK(cudaMemcpy(up_adj, ix->up_adj, sizeof(int32_t) * ix->up_rows * ix->M,
                           cudaMemcpyDeviceToHost));
    if (entry) *entry = ix->entry;
    if (maxlevel) *maxlevel = ix->maxlevel;
    return FINGER_OK;
}

finger_status finger_get_info(const finger_index* ix, finger_info* out) {
    if (!ix || !out) return FINGER_ERR_INVALID_ARG;
    out->n = ix->n;
    out->m = ix->m;
    out->deg0 = ix->deg0;
    out->M = ix->M;
    out->maxlevel = ix->maxlevel;
    out->entry = ix->entry;
    out->up_rows = ix->up_rows;
    out->r = ix->r;
    out->has_lp = ix->Xh != nullptr && ix->edge_q != nullptr;
    out->has_half_codes = ix->edge_h != nullptr;
    out->has_fp8_codes = ix->edge_q != nullptr;
    out->has_mlp = ix->has_mlp;
    int64_t b = ix->n * (ix->m_pad + 1) * 4;
    if (ix->adj0) b += ix->n * ix->deg0 * 4 + ix->n * 8 + ix->up_rows * ix->M * 4;
    if (ix->edge_u) b += ix->n * ix->r_pad * 4 + finger_table_bytes(ix->n, ix->deg0, ix->r_pad, 0);
    const int64_t tiles = ix->deg0 > 32 ? 4 : 2;
    if (ix->Xh) b += ix->n * ix->m8 * 16;
    if (ix->edge_q) b += ix->n * tiles * ix->hks * 256;
    if (ix->edge_h) b += ix->n * tiles * ix->hks * 512;
    if (ix->adj_t) b += ix->n * ix->deg0 * 4;
    b += ix->bitmap_slots * ix->words * 4 + ix->bitmap_slots * ix->spill_cap * 4;
    out->device_bytes = b;
    return FINGER_OK;
}

finger_status finger_build_tables(finger_index* ix, const finger_build_params* p, void* stream) {
    if (!ix || !p) return FINGER_ERR_INVALID_ARG;
    DeviceGuard g(ix->device);
    fg_drop_captures(ix);
    ix->tuned.clear();
    ix->tuned_ms.clear();
    ix->has_mlp = 0;
    ix->h_mlp.clear();
    return build_tables(ix, p, (cudaStream_t)stream);
}

finger_status finger_select_rank(finger_index* ix, const finger_build_params* p, double threshold,
                                 int r_step, int r_max, int* r_out, double* corr_trace,
                                 void* stream) {
    if (!ix || !p) return FINGER_ERR_INVALID_ARG;
    DeviceGuard g(ix->device);
    fg_drop_captures(ix);
    ix->tuned.clear();
    ix->tuned_ms.clear();
    ix->has_mlp = 0;
    ix->h_mlp.clear();
    return select_rank(ix, p, threshold, r_step, r_max, r_out, corr_trace, (cudaStream_t)stream);
}

finger_status finger_get_tables(const finger_index* ix, float* P, double* stats, float* node_proj,
                                float* edge_u, float* edge_s) {
    if (!ix) return FINGER_ERR_INVALID_ARG;
    if (!ix->edge_u) return FINGER_ERR_NOT_BUILT;
    DeviceGuard g(ix->device);
    const int r = ix->r, rp = ix->r_pad, m = ix->m;
    if (P)
        CUDA_OK(cudaMemcpy2D(P, sizeof(float) * m, ix->P, sizeof(float) * ix->m_pad,
                             sizeof(float) * m, r, cudaMemcpyDeviceToHost));
    if (stats)
        for (int i = 0; i < 5; ++i) stats[i] = ix->stats[i];
    if (node_proj)
        CUDA_OK(cudaMemcpy2D(node_proj, sizeof(float) * r, ix->Pc, sizeof(float) * rp,
                             sizeof(float) * r, ix->n, cudaMemcpyDeviceToHost));
    const int64_t ne = ix->n * ix->deg0;
    if (edge_u)
        CUDA_OK(cudaMemcpy2D(edge_u, sizeof(float) * r, ix->edge_u, sizeof(float) * rp,
                             sizeof(float) * r, ne, cudaMemcpyDeviceToHost));
    if (edge_s)
        CUDA_OK(cudaMemcpy(edge_s, ix->edge_s, sizeof(float2) * ne, cudaMemcpyDeviceToHost));
    return FINGER_OK;
}

finger_status finger_set_mode(finger_index* ix, int mode, int warmup) {
    if (!ix || mode < 0 || mode > FINGER_MODE_FINGER_F8) return FINGER_ERR_INVALID_ARG;
    ix->mode = mode;
    if (warmup >= 0) ix->warmup = warmup;
    return FINGER_OK;
}

finger_status finger_set_limit(finger_index* ix, int max_expansions) {
    if (!ix || max_expansions < 0) return FINGER_ERR_INVALID_ARG;
    ix->max_expansions = max_expansions;
    return FINGER_OK;
}

finger_status finger_set_visited_slots(finger_index* ix, int bits) {
    if (!ix || (bits != 0 && bits != 32)) return FINGER_ERR_INVALID_ARG;
    if (ix->visited_bits != bits) fg_drop_captures(ix);   // captured launches hold the plan
    ix->visited_bits = bits;
    return FINGER_OK;
}

finger_status finger_set_counters(finger_index* ix, int32_t* counters_device) {
    if (!ix) return FINGER_ERR_INVALID_ARG;
    ix->cnt_q = counters_device;
    return FINGER_OK;
}

finger_status finger_search(finger_index* ix, const float* queries, int64_t nq, int K, int ef,
                            int64_t* out_ids, float* out_dists, void* stream) {
    if (!ix || nq < 0 || K < 1 || ef < K || ef > MAX_EF) return FINGER_ERR_INVALID_ARG;
    if (nq == 0) return FINGER_OK;
    if (!queries || !out_ids || !out_dists) return FINGER_ERR_INVALID_ARG;
    finger_status st = check_mode_ready(ix, ix->mode);
    if (st != FINGER_OK) return st;
    DeviceGuard g(ix->device);
    SearchPlan p;
    st = make_search_plan(ix, ef, nq, &p);
    if (st != FINGER_OK) return st;
    SearchArgs a = base_args(ix, p);
    a.Q = queries;
    a.nq = nq;
    a.K = K;
    a.ef = ef;
    a.out_ids = out_ids;
    a.out_d = out_dists;
    a.rerank = std::min(ef, 2 * K);
    return run_search(ix, p, a, (cudaStream_t)stream);
}

finger_status finger_search_host(finger_index* ix, const float* queries_host, int64_t nq, int K,
                                 int ef, int64_t* out_ids_host, float* out_dists_host,
                                 void* stream) {
    if (!ix || nq < 0 || K < 1 || ef < K || ef > MAX_EF) return FINGER_ERR_INVALID_ARG;
    if (nq == 0) return FINGER_OK;
    if (!queries_host || !out_ids_host || !out_dists_host) return FINGER_ERR_INVALID_ARG;
    DeviceGuard g(ix->device);
    cudaStream_t s = (cudaStream_t)stream;
    if (ix->stage_cap_q < nq * ix->m) {
        cudaFree(ix->stage_q);
        ix->stage_q = nullptr;
        ix->stage_cap_q = 0;
        finger_status st = dmalloc(&ix->stage_q, (size_t)(nq * ix->m));
        if (st != FINGER_OK) return st;
        ix->stage_cap_q = nq * ix->m;
    }
    if (ix->stage_cap_o < nq * K) {
        cudaFree(ix->stage_ids);
        cudaFree(ix->stage_d);
        ix->stage_ids = nullptr;
        ix->stage_d = nullptr;
        ix->stage_cap_o = 0;
        finger_status st = dmalloc(&ix->stage_ids, (size_t)(nq * K));
        if (st == FINGER_OK) st = dmalloc(&ix->stage_d, (size_t)(nq * K));
        if (st != FINGER_OK) return st;
        ix->stage_cap_o = nq * K;
    }
    CUDA_OK(cudaMemcpyAsync(ix->stage_q, queries_host, sizeof(float) * nq * ix->m,
                            cudaMemcpyHostToDevice, s));
    finger_status st = finger_search(ix, ix->stage_q, nq, K, ef, ix->stage_ids, ix->stage_d, stream);
    if (st != FINGER_OK) return st;
    CUDA_OK(cudaMemcpyAsync(out_ids_host, ix->stage_ids, sizeof(int64_t) * nq * K,
                            cudaMemcpyDeviceToHost, s));
    CUDA_OK(cudaMemcpyAsync(out_dists_host, ix->stage_d, sizeof(float) * nq * K,
                            cudaMemcpyDeviceToHost, s));
    CUDA_OK(cudaStreamSynchronize(s));
    return FINGER_OK;
}

finger_status finger_knn(finger_index* ix, const float* queries, int64_t nq, int K,
                         int64_t* out_ids, float* out_dists, void* stream) {
    if (!ix || nq < 0 || K < 1 || K > 256) return FINGER_ERR_INVALID_ARG;
    if (nq == 0) return FINGER_OK;
    if (!queries || !out_ids || !out_dists) return FINGER_ERR_INVALID_ARG;
    DeviceGuard g(ix->device);
    cudaError_t e;
    if (K <= knn_tc_max_k())
        e = launch_knn_tc(ix, queries, nq, K, out_ids, out_dists, (cudaStream_t)stream);
    else
        e = launch_knn(reinterpret_cast<const float4*>(ix->X), ix->n, ix->m4, queries, ix->m, ix->m,
                       nq, K, false, nullptr, out_ids, out_dists, (cudaStream_t)stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? FINGER_ERR_OOM : FINGER_ERR_CUDA;
    }
    return FINGER_OK;
}

finger_status finger_sync(finger_index* ix) {
    if (!ix) return FINGER_ERR_INVALID_ARG;
    DeviceGuard g(ix->device);
    if (cudaDeviceSynchronize() != cudaSuccess) {
        cudaGetLastError();
        return FINGER_ERR_CUDA;
    }
    int e = 0;
    CUDA_OK(cudaMemcpy(&e, ix->err, sizeof(int), cudaMemcpyDeviceToHost));
    return e ? (finger_status)e : FINGER_OK;
}

finger_status finger_get_stats(finger_index* ix, finger_stats* out) {
    if (!ix || !out) return FINGER_ERR_INVALID_ARG;
    DeviceGuard g(ix->device);
    if (cudaDeviceSynchronize() != cudaSuccess) {
        cudaGetLastError();
        return FINGER_ERR_CUDA;
    }
    unsigned long long c[9];
    int e = 0;
    CUDA_OK(cudaMemcpy(c, ix->cnt, sizeof(c), cudaMemcpyDeviceToHost));
    CUDA_OK(cudaMemcpy(&e, ix->err, sizeof(int), cudaMemcpyDeviceToHost));
    out->searches = ix->searches;
    for (int i = 0; i < 8; ++i) out->counters[i] = (int64_t)c[i];
    out->device_error = e;
    out->mu = ix->stats[0];
    out->sigma = ix->stats[1];
    out->mu_hat = ix->stats[2];
    out->sigma_hat = ix->stats[3];
    out->eps = ix->stats[4];
    out->build_ms = ix->build_ms;
    out->corr = ix->corr;
    // bytes of FP16 / FP8 code blocks read (the kernel counts them per half block)
    out->code_bytes = (int64_t)c[8];
    return FINGER_OK;
}

finger_status finger_reset_stats(finger_index* ix) {
    if (!ix) return FINGER_ERR_INVALID_ARG;
    DeviceGuard g(ix->device);
    CUDA_OK(cudaMemset(ix->cnt, 0, sizeof(unsigned long long) * 16));
    CUDA_OK(cudaMemset(ix->err, 0, sizeof(int)));
    ix->searches = 0;
    return FINGER_OK;
}

}  // extern "C"

// Exact K-nearest-neighbour ground truth on the 5th-generation tensor cores.
//
// The distance matrix is a dense contraction: ||q - x||^2 = ||q||^2 + ||x||^2
// - 2 q.x.  q.x runs on tcgen05.mma (kind::f16, BF16 operands, FP32
// accumulators in tensor memory) with each FP32 operand split into a BF16 high
// part and a BF16 low part: q.x ~ qh.xh + qh.xl + ql.xh (the dropped ql.xl and
// the rounding of the parts are ~2^-17 of |q||x|).  Every query row keeps the
// K' smallest approximate distances of its base segment; a second kernel then
// recomputes the candidates' distances exactly in FP32 (sum of (q - x)^2) and
// returns the K best by (distance, id), so the result is the exact kNN unless
// more than K' - K rows lie within the approximation error of the K-th
// distance.
//
// k_knn_tc is persistent (one CTA per SM) and warp-specialised:
//   warp 0     TMA producer: 64-column (128-byte, SWIZZLE_128B) chunks of the
//              query tile (hi, lo) and the base tile (hi, lo) into a 2-stage ring
//   warp 1     MMA issuer (one elected lane): 3 products x 4 K-steps per chunk
//              into one of two 128x128 FP32 accumulators in tensor memory
//   warps 2-5  epilogue: tcgen05.ld of the accumulator (thread = query row),
//              distances and their per-row minimum against the row's K'-th
//              distance; the few rows with a smaller one are transposed
//              through shared memory and their new candidates inserted into
//              the row's sorted K' list by the whole warp (ballot for the
//              position, shuffle for the shift); the accumulator is handed
//              back through an mbarrier
// Work items are (query tile of 128, segment of base tiles), so small query
// batches still fill the GPU.  Every mbarrier wait is bounded: on a timeout the
// kernel raises an error flag, every role leaves its loop, and tensor memory is
// released.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <vector>

#include "internal.cuh"

namespace fg {

namespace {

constexpr int TQ = 128;                      // query rows per tile (MMA M)
constexpr int TB = 128;                      // base rows per tile (MMA N)
constexpr int KCH = 64;                      // K elements per chunk (128 bytes of BF16)
constexpr int STAGES = 2;
constexpr int PART = TQ * 128;               // one 128-row x 128-byte operand part: 16 KB
constexpr int STAGE_BYTES = 4 * PART;        // qh, ql, xh, xl
constexpr int TC_THREADS = 192;
constexpr long WAIT_TRIES = 1L << 21;

struct TcArgs {
    int64_t nq, n;
    int nchunk;           // ceil(m / 64)
    int nbt;              // base tiles
    int nseg;             // base segments per query tile; segment s holds the base
                          // tiles s, s + nseg, s + 2 nseg, ... (interleaved)
    int nqt;              // query tiles
    int causal;           // 1: queries are the base rows, row i sees base rows < i
    const float* qn;      // ||q||^2 (FP32), nq
    const float* xn;      // ||x||^2 (FP32), n
    int32_t* cand;        // nq x nseg x KP candidate ids (-1 = none)
    float* cand_d;        // optional: their approximate distances
    int* err;             // device status word (FINGER_ERR_LIMIT on a wait timeout)
};

// work item -> (query tile, segment): the largest causal items first
__device__ __forceinline__ void item_of(const TcArgs& a, int item, int& qt, int& seg, int& bt_end) {
    qt = a.causal ? a.nqt - 1 - item / a.nseg : item / a.nseg;
    seg = item % a.nseg;
    bt_end = a.causal ? min(a.nbt, qt + 1) : a.nbt;
}

__device__ __forceinline__ uint32_t s32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// bounded parity wait; false (and the abort flag raised) on timeout
__device__ __forceinline__ bool wait_bar(uint32_t bar, uint32_t parity, volatile int* abort_flag,
                                         int* err) {
    for (long it = 0; it < WAIT_TRIES; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok) return true;
        if (*abort_flag) return false;
    }
    *abort_flag = 1;
    atomicOr(err, (int)FINGER_ERR_LIMIT);
    return false;
}

// shared-memory matrix descriptor: K-major operand, 128-byte swizzle, 8-row
// atoms of 1024 bytes stacked along M/N
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
    return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

__device__ __forceinline__ void mma_bf16_tc(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc,
                                            uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
        "l"(ad), "l"(bd), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void tma_2d(uint32_t dst, const CUtensorMap* map, int x, int y,
                                       uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            dst),
        "l"((uint64_t)map), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
        "%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
          "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
          "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

template <int KP>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_knn_tc(const __grid_constant__ CUtensorMap tqh, const __grid_constant__ CUtensorMap tql,
             const __grid_constant__ CUtensorMap txh, const __grid_constant__ CUtensorMap txl,
             TcArgs a) {
    static_assert(KP == 32 || KP == 64, "candidate lists of 32 or 64");
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* sm = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char* stages = sm;                                   // STAGES x 64 KB
    float* Ld = reinterpret_cast<float*>(sm + STAGES * STAGE_BYTES);   // 128 x KP (row-major)
    int32_t* Li = reinterpret_cast<int32_t*>(Ld + KP * TQ);
    float* Bs = reinterpret_cast<float*>(Li + KP * TQ);                // 4 x 32 x 33
    uint64_t* bars = reinterpret_cast<uint64_t*>(Bs + 4 * 32 * 33);   // full[2] empty[2] accf[2] acce[2]
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 8);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t full0 = s32(bars), empty0 = s32(bars + 2), accf0 = s32(bars + 4),
                   acce0 = s32(bars + 6);

    if (threadIdx.x == 0) {
        for (int i = 0; i < 2; ++i) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(full0 + 8 * i));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(empty0 + 8 * i));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(accf0 + 8 * i));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 128;" ::"r"(acce0 + 8 * i));
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(
            s32(tmem_slot)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    const int items = a.nqt * a.nseg;

    if (warp == 0) {
        if (lane == 0) {
            uint32_t it = 0;
            for (int item = blockIdx.x; item < items && !*abort_flag; item += gridDim.x) {
                int qt, seg, bt_end;
                item_of(a, item, qt, seg, bt_end);
                for (int bt = seg; bt < bt_end && !*abort_flag; bt += a.nseg)
                    for (int c = 0; c < a.nchunk; ++c, ++it) {
                        const int s = it % STAGES;
                        const uint32_t ph = (it / STAGES) & 1u;
                        if (!wait_bar(empty0 + 8 * s, ph ^ 1u, abort_flag, a.err)) break;
                        const uint32_t fb = full0 + 8 * s;
                        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb),
                                     "r"(STAGE_BYTES)
                                     : "memory");
                        const uint32_t dst = s32(stages + (size_t)s * STAGE_BYTES);
                        tma_2d(dst, &tqh, c * KCH, qt * TQ, fb);
                        tma_2d(dst + PART, &tql, c * KCH, qt * TQ, fb);
                        tma_2d(dst + 2 * PART, &txh, c * KCH, bt * TB, fb);
                        tma_2d(dst + 3 * PART, &txl, c * KCH, bt * TB, fb);
                    }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // D F32, A BF16, B BF16, K-major A and B, N = 128, M = 128
            const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TB >> 3) << 17) |
                                   ((uint32_t)(TQ >> 4) << 24);
            uint32_t it = 0, tile = 0;
            for (int item = blockIdx.x; item < items && !*abort_flag; item += gridDim.x) {
                int qt, seg, bt_end;
                item_of(a, item, qt, seg, bt_end);
                for (int bt = seg; bt < bt_end && !*abort_flag; bt += a.nseg, ++tile) {
                    const uint32_t b = tile & 1u, tph = (tile >> 1) & 1u;
                    if (!wait_bar(acce0 + 8 * b, tph ^ 1u, abort_flag, a.err)) break;
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t d = tmem + b * TB;
                    for (int c = 0; c < a.nchunk; ++c, ++it) {
                        const int s = it % STAGES;
                        const uint32_t ph = (it / STAGES) & 1u;
                        if (!wait_bar(full0 + 8 * s, ph, abort_flag, a.err)) break;
                        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                        const uint32_t base = s32(stages + (size_t)s * STAGE_BYTES);
#pragma unroll
                        for (int k = 0; k < KCH / 16; ++k) {
                            const uint64_t qh = sdesc(base + 32 * k), ql = sdesc(base + PART + 32 * k);
                            const uint64_t xh = sdesc(base + 2 * PART + 32 * k),
                                           xl = sdesc(base + 3 * PART + 32 * k);
                            mma_bf16_tc(d, qh, xh, idesc, (c | k) != 0);
                            mma_bf16_tc(d, qh, xl, idesc, 1u);
                            mma_bf16_tc(d, ql, xh, idesc, 1u);
                        }
                        asm volatile(
                            "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                empty0 + 8 * s)
                            : "memory");
                    }
                    asm volatile(
                        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                            accf0 + 8 * b)
                        : "memory");
                }
            }
        }
    } else {
        // epilogue: warp w owns the query rows 32 (w % 4) + lane of every tile
        // (the tensor-memory lanes it may read).  Per 32-column block a thread
        // forms its row's 32 distances and their minimum; only rows whose
        // minimum beats their K'-th distance go on, through a transpose in
        // shared memory, to a warp-wide insertion into the row's sorted list.
        const int quarter = warp & 3;
        const int row = 32 * quarter + lane;
        float* B = Bs + (warp - 2) * 32 * 33;               // 32 x 32 transpose, padded
        float* Lw = Ld + (size_t)quarter * 32 * KP;          // this warp's 32 lists, row-major
        int32_t* Lwi = Li + (size_t)quarter * 32 * KP;
        uint32_t tile = 0;
        for (int item = blockIdx.x; item < items && !*abort_flag; item += gridDim.x) {
            int qt, seg, bt_end;
            item_of(a, item, qt, seg, bt_end);
            const int64_t q0 = (int64_t)qt * TQ;
            const int64_t qi = q0 + row;
            const int64_t id_end = a.causal ? min(qi, a.n) : a.n;   // ids below this count
            const int64_t lim = a.causal ? min(q0, a.n) : a.n;      // smallest id_end of the tile
            const float qn = qi < a.nq ? a.qn[qi] : 0.f;
            float thr = qi < a.nq ? INFINITY : -INFINITY;            // K'-th distance of the row
            for (int k = lane; k < 32 * KP; k += 32) {
                Lw[k] = INFINITY;
                Lwi[k] = -1;
            }
            __syncwarp();
            for (int bt = seg; bt < bt_end; bt += a.nseg, ++tile) {
                const uint32_t b = tile & 1u, tph = (tile >> 1) & 1u;
                if (!wait_bar(accf0 + 8 * b, tph, abort_flag, a.err)) break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t tbase = tmem + ((uint32_t)(32 * quarter) << 16) + b * TB;
                const bool masked = (int64_t)(bt + 1) * TB > lim;
                for (int c0 = 0; c0 < TB; c0 += 32) {
                    float v[32];
                    tmem_ld32(tbase + c0, v);
                    const int64_t id0 = (int64_t)bt * TB + c0;
                    if (!masked) {
                        const float4* x4 = reinterpret_cast<const float4*>(a.xn + id0);
#pragma unroll
                        for (int j4 = 0; j4 < 8; ++j4) {
                            const float4 x = __ldg(x4 + j4);
                            v[4 * j4] = fmaf(-2.f, v[4 * j4], qn + x.x);
                            v[4 * j4 + 1] = fmaf(-2.f, v[4 * j4 + 1], qn + x.y);
                            v[4 * j4 + 2] = fmaf(-2.f, v[4 * j4 + 2], qn + x.z);
                            v[4 * j4 + 3] = fmaf(-2.f, v[4 * j4 + 3], qn + x.w);
                        }
                    } else {
#pragma unroll
                        for (int j = 0; j < 32; ++j) {
                            const int64_t id = id0 + j;
                            v[j] = id < id_end ? fmaf(-2.f, v[j], qn + __ldg(a.xn + id)) : INFINITY;
                        }
                    }
                    float mn = v[0];
#pragma unroll
                    for (int j = 1; j < 32; ++j) mn = fminf(mn, v[j]);
                    unsigned rows = __ballot_sync(0xffffffffu, mn < thr);
                    if (!rows) continue;
#pragma unroll
                    for (int j = 0; j < 32; ++j) B[j * 33 + lane] = v[j];
                    __syncwarp();
                    while (rows) {
                        const int r = __ffs(rows) - 1;
                        rows &= rows - 1;
                        float t = __shfl_sync(0xffffffffu, thr, r);
                        const float dj = B[lane * 33 + r];           // column lane of row r
                        unsigned hit = __ballot_sync(0xffffffffu, dj < t);
                        float* Lr = Lw + r * KP;
                        int32_t* Lir = Lwi + r * KP;
                        float d0 = Lr[lane], d1 = INFINITY;
                        int32_t i0 = Lir[lane], i1 = -1;
                        if (KP == 64) {
                            d1 = Lr[lane + 32];
                            i1 = Lir[lane + 32];
                        }
                        while (hit) {
                            const int c = __ffs(hit) - 1;
                            hit &= hit - 1;
                            const float cd = __shfl_sync(0xffffffffu, dj, c);
                            if (!(cd < t)) continue;
                            const int32_t cid = (int32_t)(id0 + c);
                            // ids grow along the scan, so equal distances already
                            // in the list come first: position = #entries <= cd
                            int pos = __popc(__ballot_sync(0xffffffffu, d0 <= cd));
                            if (KP == 64) pos += __popc(__ballot_sync(0xffffffffu, d1 <= cd));
                            const float u0 = __shfl_up_sync(0xffffffffu, d0, 1);
                            const int32_t ui0 = __shfl_up_sync(0xffffffffu, i0, 1);
                            if (KP == 64) {
                                float u1 = __shfl_up_sync(0xffffffffu, d1, 1);
                                int32_t ui1 = __shfl_up_sync(0xffffffffu, i1, 1);
                                const float t31 = __shfl_sync(0xffffffffu, d0, 31);
                                const int32_t ti31 = __shfl_sync(0xffffffffu, i0, 31);
                                if (lane == 0) {
                                    u1 = t31;
                                    ui1 = ti31;
                                }
                                if (lane + 32 > pos) {
                                    d1 = u1;
                                    i1 = ui1;
                                } else if (lane + 32 == pos) {
                                    d1 = cd;
                                    i1 = cid;
                                }
                            }
                            if (lane > pos) {
                                d0 = u0;
                                i0 = ui0;
                            } else if (lane == pos) {
                                d0 = cd;
                                i0 = cid;
                            }
                            t = __shfl_sync(0xffffffffu, KP == 64 ? d1 : d0, 31);
                        }
                        Lr[lane] = d0;
                        Lir[lane] = i0;
                        if (KP == 64) {
                            Lr[lane + 32] = d1;
                            Lir[lane + 32] = i1;
                        }
                        if (lane == r) thr = t;
                    }
                    __syncwarp();
                }
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(acce0 + 8 * b) : "memory");
            }
            __syncwarp();
            for (int r = 0; r < 32; ++r) {
                const int64_t qr = q0 + 32 * quarter + r;
                if (qr >= a.nq) break;
                const size_t o = ((size_t)qr * a.nseg + seg) * KP;
                for (int k = lane; k < KP; k += 32) {
                    a.cand[o + k] = Lwi[r * KP + k];
                    if (a.cand_d) a.cand_d[o + k] = Lw[r * KP + k];
                }
            }
            __syncwarp();
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(tmem));
}

// FP32 rows -> BF16 high and low parts (row stride ms, zero padded) and the
// FP32 squared norm of every row; one warp per row
__global__ void k_split_bf16(const float* __restrict__ X, int64_t rows, int m, int64_t x_stride,
                             int ms, __nv_bfloat16* hi, __nv_bfloat16* lo, float* norm2) {
    const int lane = threadIdx.x & 31;
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (w >= rows) return;
    float acc = 0.f;
    for (int k = lane; k < ms; k += 32) {
        const float x = k < m ? X[w * x_stride + k] : 0.f;
        const __nv_bfloat16 h = __float2bfloat16_rn(x);
        hi[w * ms + k] = h;
        lo[w * ms + k] = __float2bfloat16_rn(x - __bfloat162float(h));
        acc = fmaf(x, x, acc);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (norm2 && lane == 0) norm2[w] = acc;
}

// exact FP32 distances of every query's candidates and the K best by
// (distance, id); one warp per query
__global__ void k_rerank(const float4* __restrict__ X, int m4, const float* __restrict__ Q, int m,
                         int64_t nq, const int32_t* __restrict__ cand, int nc, int K,
                         int64_t* out_ids, float* out_d) {
    extern __shared__ float rr_s[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int64_t q = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib;
    if (q >= nq) return;
    float* cd = rr_s + (size_t)wib * 2 * nc;
    int32_t* ci = reinterpret_cast<int32_t*>(cd + nc);
    const float* qr = Q + (size_t)q * m;
    for (int i = 0; i < nc; ++i) {
        const int32_t id = cand[(size_t)q * nc + i];
        float acc = 0.f;
        if (id >= 0) {
            const float4* xr = X + (size_t)id * m4;
            for (int k = lane; k < m4; k += 32) {
                const float4 x = __ldg(xr + k);
                const int e = 4 * k;
                float dlt;
                if (e < m) { dlt = qr[e] - x.x; acc = fmaf(dlt, dlt, acc); }
                if (e + 1 < m) { dlt = qr[e + 1] - x.y; acc = fmaf(dlt, dlt, acc); }
                if (e + 2 < m) { dlt = qr[e + 2] - x.z; acc = fmaf(dlt, dlt, acc); }
                if (e + 3 < m) { dlt = qr[e + 3] - x.w; acc = fmaf(dlt, dlt, acc); }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        }
        if (lane == 0) {
            cd[i] = id >= 0 ? acc : INFINITY;
            ci[i] = id;
        }
    }
    __syncwarp();
    // rank of every candidate among the valid ones by (distance, id)
    for (int i = lane; i < nc; i += 32) {
        const float di = cd[i];
        const int32_t ii = ci[i];
        if (ii < 0) continue;
        int rank = 0;
        for (int j = 0; j < nc; ++j) {
            const int32_t ij = ci[j];
            if (ij < 0) continue;
            rank += cd[j] < di || (cd[j] == di && ij < ii);
        }
        if (rank < K) {
            out_ids[(size_t)q * K + rank] = ii;
            out_d[(size_t)q * K + rank] = di;
        }
    }
    __syncwarp();
    // pad when fewer than K valid candidates
    int valid = 0;
    for (int j = lane; j < nc; j += 32) valid += ci[j] >= 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) valid += __shfl_xor_sync(0xffffffffu, valid, o);
    for (int k = valid + lane; k < K; k += 32) {
        out_ids[(size_t)q * K + k] = -1;
        out_d[(size_t)q * K + k] = INFINITY;
    }
}

// Merge of the segments' candidate lists by approximate distance: the K
// smallest (distance, id) of every row, int64 ids (-1 padded); one warp per row
__global__ void k_merge_topk(const int32_t* __restrict__ cand, const float* __restrict__ cand_d,
                             int64_t rows, int nc, int K, int64_t* out_ids, float* out_d) {
    const int lane = threadIdx.x & 31;
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (w >= rows) return;
    const int32_t* ci = cand + (size_t)w * nc;
    const float* cd = cand_d + (size_t)w * nc;
    int valid = 0;
    for (int i = lane; i < nc; i += 32) {
        const int32_t ii = ci[i];
        if (ii < 0) continue;
        valid++;
        const float di = cd[i];
        int rank = 0;
        for (int j = 0; j < nc; ++j) {
            const int32_t ij = ci[j];
            if (ij < 0) continue;
            const float dj = cd[j];
            rank += dj < di || (dj == di && ij < ii);
        }
        if (rank < K) {
            out_ids[(size_t)w * K + rank] = ii;
            out_d[(size_t)w * K + rank] = di;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) valid += __shfl_xor_sync(0xffffffffu, valid, o);
    for (int k = valid + lane; k < K; k += 32) {
        out_ids[(size_t)w * K + k] = -1;
        out_d[(size_t)w * K + k] = INFINITY;
    }
}

PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        cudaDriverEntryPointQueryResult q;
        void* p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

bool make_map(CUtensorMap* map, const void* base, int64_t rows, int m, int ms) {
    auto enc = get_encode();
    if (!enc) return false;
    cuuint64_t dims[2] = {(cuuint64_t)m, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)ms * 2};
    cuuint32_t box[2] = {KCH, TQ};
    cuuint32_t es[2] = {1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides,
               box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int KP>
size_t tc_smem() {
    return 1024 + (size_t)STAGES * STAGE_BYTES + (size_t)KP * TQ * 8 + 4 * 32 * 33 * 4 + 8 * 8 + 16;
}

template <int KP>
cudaError_t run_tc(const CUtensorMap* maps, TcArgs a, int grid, cudaStream_t s) {
    const size_t smem = tc_smem<KP>();
    cudaError_t e = cudaFuncSetAttribute(k_knn_tc<KP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    k_knn_tc<KP><<<grid, TC_THREADS, smem, s>>>(maps[0], maps[1], maps[2], maps[3], a);
    return cudaGetLastError();
}

}  // namespace

// Largest K the tensor-core path serves (its candidate lists hold 32 or 64).
int knn_tc_max_k() { return 40; }

namespace {

// BF16 split of the base rows, made once per index
cudaError_t ensure_split(finger_index* ix, cudaStream_t s) {
    if (ix->xs_hi) return cudaSuccess;
    const int m = ix->m, ms = (m + 7) & ~7;
    const int64_t n = ix->n;
    if (cudaMalloc(&ix->xs_hi, sizeof(__nv_bfloat16) * (size_t)n * ms) != cudaSuccess ||
        cudaMalloc(&ix->xs_lo, sizeof(__nv_bfloat16) * (size_t)n * ms) != cudaSuccess) {
        cudaFree(ix->xs_hi);
        ix->xs_hi = nullptr;
        ix->xs_lo = nullptr;
        cudaGetLastError();
        return cudaErrorMemoryAllocation;
    }
    k_split_bf16<<<(unsigned)((n * 32 + 255) / 256), 256, 0, s>>>(ix->X, n, m, ix->m_pad, ms,
                                                                  ix->xs_hi, ix->xs_lo, nullptr);
    return cudaGetLastError();
}

// one launch of k_knn_tc over nq query rows (BF16 parts qh/ql) against the base
cudaError_t run_items(finger_index* ix, const __nv_bfloat16* qh, const __nv_bfloat16* ql,
                      const float* qn, int64_t nq, int KP, int nseg, bool causal, int32_t* cand,
                      float* cand_d, cudaStream_t s) {
    const int m = ix->m, ms = (m + 7) & ~7;
    const int64_t n = ix->n;
    CUtensorMap maps[4];
    if (!make_map(&maps[0], qh, nq, m, ms) || !make_map(&maps[1], ql, nq, m, ms) ||
        !make_map(&maps[2], ix->xs_hi, n, m, ms) || !make_map(&maps[3], ix->xs_lo, n, m, ms))
        return cudaErrorInvalidValue;
    TcArgs a;
    a.nq = nq;
    a.n = n;
    a.nchunk = (m + KCH - 1) / KCH;
    a.nbt = (int)((n + TB - 1) / TB);
    a.nseg = nseg;
    a.nqt = (int)((nq + TQ - 1) / TQ);
    a.causal = causal ? 1 : 0;
    a.qn = qn;
    a.xn = ix->xnorm2;
    a.cand = cand;
    a.cand_d = cand_d;
    a.err = ix->err;
    const int grid = (int)std::min<int64_t>(ix->num_sms, (int64_t)a.nqt * nseg);
    return KP == 32 ? run_tc<32>(maps, a, grid, s) : run_tc<64>(maps, a, grid, s);
}

}  // namespace

cudaError_t launch_knn_tc(finger_index* ix, const float* Q, int64_t nq, int K, int64_t* out_ids,
                          float* out_d, cudaStream_t s) {
    if (nq <= 0) return cudaSuccess;
    const int m = ix->m, ms = (m + 7) & ~7;
    const int64_t n = ix->n;
    cudaError_t e = ensure_split(ix, s);
    if (e != cudaSuccess) return e;
    const int KP = K <= 16 ? 32 : 64;
    const int nqt = (int)((nq + TQ - 1) / TQ);
    const int nbt = (int)((n + TB - 1) / TB);
    // enough (query tile, base segment) items for two per SM, at most 64
    // segments; any segmentation is exact here because K <= KP
    const int nseg = std::max(1, std::min({nbt, 64, (2 * ix->num_sms + nqt - 1) / nqt}));
    const int nc = nseg * KP;
    __nv_bfloat16 *qh = nullptr, *ql = nullptr;
    float* qn = nullptr;
    int32_t* cand = nullptr;
    if (cudaMallocAsync(&qh, sizeof(__nv_bfloat16) * (size_t)nq * ms, s) != cudaSuccess ||
        cudaMallocAsync(&ql, sizeof(__nv_bfloat16) * (size_t)nq * ms, s) != cudaSuccess ||
        cudaMallocAsync(&qn, sizeof(float) * (size_t)nq, s) != cudaSuccess ||
        cudaMallocAsync(&cand, sizeof(int32_t) * (size_t)nq * nc, s) != cudaSuccess) {
        e = cudaErrorMemoryAllocation;
        goto done;
    }
    k_split_bf16<<<(unsigned)((nq * 32 + 255) / 256), 256, 0, s>>>(Q, nq, m, m, ms, qh, ql, qn);
    if ((e = cudaGetLastError()) != cudaSuccess) goto done;
    if ((e = run_items(ix, qh, ql, qn, nq, KP, nseg, false, cand, nullptr, s)) != cudaSuccess)
        goto done;
    {
        const int wpb = nc > 1024 ? 1 : 4;
        const size_t smem = (size_t)wpb * 2 * nc * sizeof(float);
        if (smem > 48 * 1024 &&
            (e = cudaFuncSetAttribute(k_rerank, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem)) != cudaSuccess)
            goto done;
        k_rerank<<<(unsigned)((nq + wpb - 1) / wpb), 32 * wpb, smem, s>>>(
            reinterpret_cast<const float4*>(ix->X), ix->m4, Q, m, nq, cand, nc, K, out_ids, out_d);
        e = cudaGetLastError();
    }
done:
    // stream-ordered frees: the temporaries live until the kernels above finish
    if (qh) cudaFreeAsync(qh, s);
    if (ql) cudaFreeAsync(ql, s);
    if (qn) cudaFreeAsync(qn, s);
    if (cand) cudaFreeAsync(cand, s);
    return e;
}

// Causal candidates of the graph builder on the tensor cores: for every base
// row i, the K (<= 256) smallest approximate distances to the rows j < i,
// ascending by (distance, id), int64 ids padded with -1.  Eight interleaved
// base segments keep 64 each: with random ids a node's K nearest spread over
// the segments (for K = 256, 32 per segment on average), so the merged lists
// are its K nearest; only the first rows (fewer than 8 x 128 predecessors)
// can lose candidates beyond 64 of one tile.  Distances carry the BF16-split
// error (~1e-5 relative), which candidate selection tolerates.
cudaError_t launch_knn_tc_causal(finger_index* ix, int K, int64_t* out_ids, float* out_d,
                                 cudaStream_t s) {
    const int64_t n = ix->n;
    if (n <= 1) return cudaSuccess;
    cudaError_t e = ensure_split(ix, s);
    if (e != cudaSuccess) return e;
    constexpr int KP = 64, NSEG = 8;
    const int nc = NSEG * KP;
    int32_t* cand = nullptr;
    float* cand_d = nullptr;
    if (cudaMallocAsync(&cand, sizeof(int32_t) * (size_t)n * nc, s) != cudaSuccess ||
        cudaMallocAsync(&cand_d, sizeof(float) * (size_t)n * nc, s) != cudaSuccess) {
        e = cudaErrorMemoryAllocation;
        goto done;
    }
    if ((e = run_items(ix, ix->xs_hi, ix->xs_lo, ix->xnorm2, n, KP, NSEG, true, cand, cand_d, s)) !=
        cudaSuccess)
        goto done;
    k_merge_topk<<<(unsigned)((n * 32 + 255) / 256), 256, 0, s>>>(cand, cand_d, n, nc, K, out_ids,
                                                                 out_d);
    e = cudaGetLastError();
done:
    if (cand) cudaFreeAsync(cand, s);
    if (cand_d) cudaFreeAsync(cand_d, s);
    return e;
}

}  // namespace fg

// Persistent greedy-search kernel: one warp per query.
//
// Layer 0 follows Algorithm 1 (PLAIN) or Algorithm 4 (FINGER modes) of
// arXiv 2206.11408 with these readings of the paper:
//   * keys are (distance, id) compared lexicographically;
//   * a neighbour is admitted iff |T| < ef or its key is below the key of the
//     worst entry of T (Algorithm 1's admission test read together with the
//     eviction that keeps |T| <= ef); entries evicted from T are never
//     expanded, so the candidate queue C is exactly the unexpanded part of T
//     and one sorted array holds both;
//   * a neighbour is marked visited before it is evaluated, so one skipped by
//     the estimate is never examined again;
//   * from the (warmup+1)-th expansion on, while |T| = ef, a new neighbour
//     whose estimate (Algorithm 3) exceeds the current ub is skipped; ub is the
//     distance of the worst entry of T at that moment (neighbours are taken in
//     adjacency order, so ub can fall between two neighbours of one centre).
//
// GB300 mapping.  A warp owns one query from an atomic work counter until the
// batch is drained (grid = SMs x resident blocks).  Per warp in shared memory:
// the result list T (keys and ids, the EXP bit marks expanded entries), an
// exact visited hash (16-bit slots, one bucket of eight per id, where the ids
// fit; else 32-bit slots in probed buckets of four) that spills to a per-warp
// global bitmap once 3/4 full, the unit residual projection of the query, and
// staging.  An expansion gathers the adjacency row (coalesced, lane j <-
// neighbour j), in FP32 FINGER then the per-edge rows of the new neighbours
// (compacted, r/4 lanes per row, eight 16-byte loads per lane in flight,
// butterfly sums) -- the FP16 / FP8 code modes instead read the centre's
// whole code block with the adjacency row and form all estimates as one
// tensor-core product -- and last the full rows of the neighbours whose
// estimate passes (groups of G lanes per row, 16-byte loads, shuffle
// reduction).  Estimates are formed for every new neighbour against the ub
// at the start of the expansion; the sequential gate is then replayed on the
// whole warp in adjacency order (the running ub read from a 32-deep pool of
// T's tail and the admitted keys), so the traversal is exactly the
// per-neighbour one of Algorithm 4, and the admitted keys are merged into T
// once.
#pragma once

#include "internal.cuh"

namespace fg {

#define FULLMASK 0xffffffffu

// Debug builds (-DFG_CHECKED=1) validate every shared/global index of the
// search kernel: the first violation's site code is latched into the status
// word and the index is clamped to 0, so a faulty traversal reports instead of
// faulting.  Release builds compile the checks away.
#ifndef FG_CHECKED
#define FG_CHECKED 0
#endif
__device__ int* g_chk_err;
__device__ __forceinline__ int64_t chk(int64_t i, int64_t lim, int code) {
    if (FG_CHECKED && (i < 0 || i >= lim)) {
        atomicCAS(g_chk_err, 0, code);
        return 0;
    }
    return i;
}
#define CK(i, lim, code) chk((int64_t)(i), (int64_t)(lim), (code))

__device__ __forceinline__ bool key_lt(float da, uint32_t ia, float db, uint32_t ib) {
    return da < db || (da == db && ia < ib);
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULLMASK, v, o);
    return v;
}

template <bool LP, int VPL>
struct QRegs {
    float v[VPL][LP ? 8 : 4];
};

template <bool LP, int G, int VPL>
__device__ __forceinline__ void load_qregs(QRegs<LP, VPL>& q, const float* qs, int nchunks,
                                           int kin) {
    constexpr int W = LP ? 8 : 4;
#pragma unroll
    for (int v = 0; v < VPL; ++v) {
        const int ch = kin + G * v;
#pragma unroll
        for (int e = 0; e < W; ++e) q.v[v][e] = ch < nchunks ? qs[ch * W + e] : 0.f;
    }
}

__device__ __forceinline__ void bf16x8(const uint4& x, float* f) {
    const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&x);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        float2 t = __bfloat1622float2(h[i]);
        f[2 * i] = t.x;
        f[2 * i + 1] = t.y;
    }
}

// partial sum of (q - x)^2 over this lane's chunks of row `id`
template <bool LP, int G, int VPL>
__device__ __forceinline__ float row_partial(const QRegs<LP, VPL>& q, const DevIndex& ix,
                                             uint32_t id, int kin) {
    float acc = 0.f;
    if constexpr (!LP) {
        const float4* row = ix.X + (size_t)id * ix.m4;
        float4 x[VPL];
#pragma unroll
        for (int v = 0; v < VPL; ++v) {
            const int ch = kin + G * v;
            x[v] = ch < ix.m4 ? __ldg(row + ch) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int v = 0; v < VPL; ++v) {
            float d;
            d = q.v[v][0] - x[v].x; acc = fmaf(d, d, acc);
            d = q.v[v][1] - x[v].y; acc = fmaf(d, d, acc);
            d = q.v[v][2] - x[v].z; acc = fmaf(d, d, acc);
            d = q.v[v][3] - x[v].w; acc = fmaf(d, d, acc);
        }
    } else {
        const uint4* row = ix.Xh + (size_t)id * ix.m8;
        uint4 x[VPL];
#pragma unroll
        for (int v = 0; v < VPL; ++v) {
            const int ch = kin + G * v;
            x[v] = ch < ix.m8 ? __ldg(row + ch) : make_uint4(0u, 0u, 0u, 0u);
        }
#pragma unroll
        for (int v = 0; v < VPL; ++v) {
            float f[8];
            bf16x8(x[v], f);
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const float d = q.v[v][e] - f[e];
                acc = fmaf(d, d, acc);
            }
        }
    }
    return acc;
}

// exact distances of the rows nbs[lst[i]], i < nlist, into xb[lst[i]].  With
// QS the lane's query chunks are read from the staged query qs (shared
// memory) for this call only instead of living in registers for the whole
// search (the FP16-code mode, whose code block needs the registers).
template <bool LP, int G, int VPL, bool QS = false>
__device__ __forceinline__ void exact_list(const QRegs<LP, VPL>& qr, const float* qs,
                                           const DevIndex& ix, const uint32_t* nbs,
                                           const int* lst, int nlist, float* xb, int lane,
                                           uint32_t idm = 0xFFFFFFFFu) {
    QRegs<LP, VPL> qt;
    if constexpr (QS) load_qregs<LP, G, VPL>(qt, qs, LP ? ix.m8 : ix.m4, lane % G);
    const QRegs<LP, VPL>& q = QS ? qt : qr;
    constexpr int RPW = 32 / G;
    constexpr int U = rows_per_group(VPL);   // rows per group in flight
    const int grp = lane / G, kin = lane % G;
    for (int base = 0; base < nlist; base += U * RPW) {
        int o[U];
        float p[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int i = base + u * RPW + grp;
            o[u] = i < nlist ? lst[i] : -1;
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
            p[u] = o[u] >= 0 ? row_partial<LP, G, VPL>(q, ix, (uint32_t)CK(nbs[CK(o[u], 64, 1018)] & idm, ix.n, 1019), kin) : 0.f;
#pragma unroll
        for (int off = G / 2; off > 0; off >>= 1)
#pragma unroll
            for (int u = 0; u < U; ++u) p[u] += __shfl_xor_sync(FULLMASK, p[u], off);
        if (kin == 0)
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (o[u] >= 0) xb[o[u]] = p[u];
    }
    __syncwarp();
}

// L2 prefetch of one full row (issued by the lane that owns the neighbour, so
// every row of an expansion is requested at once)
template <bool LP>
__device__ __forceinline__ void prefetch_row(const DevIndex& ix, uint32_t id) {
    const char* base = LP ? reinterpret_cast<const char*>(ix.Xh + (size_t)id * ix.m8)
                          : reinterpret_cast<const char*>(ix.X + (size_t)id * ix.m4);
    const int bytes = LP ? ix.m8 * 16 : ix.m4 * 16;
    for (int off = 0; off < bytes; off += 128)
        asm volatile("prefetch.global.L2 [%0];" ::"l"(base + off));
}

// exact FP32 distance of one row, whole warp (used for the FP32 re-rank)
__device__ __forceinline__ float exact_f32_row(const float* qs, const DevIndex& ix, uint32_t id,
                                               int lane) {
    const float4* row = ix.X + (size_t)id * ix.m4;
    const float4* q4 = reinterpret_cast<const float4*>(qs);
    float acc = 0.f;
    for (int k = lane; k < ix.m4; k += 32) {
        const float4 x = __ldg(row + k);
        const float4 y = q4[k];
        float d;
        d = y.x - x.x; acc = fmaf(d, d, acc);
        d = y.y - x.y; acc = fmaf(d, d, acc);
        d = y.z - x.z; acc = fmaf(d, d, acc);
        d = y.w - x.w; acc = fmaf(d, d, acc);
    }
    return warp_sum(acc);
}

// first unexpanded entry of T at or after `from` (sz if none), with the entry
// itself (id as stored, distance) taken from the lane that loaded it
__device__ __forceinline__ int find_next_entry(const float* Tk, const uint32_t* Ti, int sz,
                                               int from, int lane, uint32_t& raw, float& d) {
    for (int b = from; b < sz; b += 32) {
        const int i = b + lane;
        uint32_t v = EXP;
        float kd = 0.f;
        if (i < sz) {
            v = Ti[i];
            kd = Tk[i];
        }
        const unsigned m = __ballot_sync(FULLMASK, !(v & EXP));
        if (m) {
            const int src = __ffs(m) - 1;
            raw = __shfl_sync(FULLMASK, v, src);
            d = __shfl_sync(FULLMASK, kd, src);
            return b + src;
        }
    }
    return sz;
}

// Merge the sorted list A (ak / ai, na <= 32 NPL entries) into the sorted
// T[0..tk): T[0..tk + na) afterwards (tk + na <= ef).  Each key of A finds its
// rank in T by binary search; the entries of T above the smallest of those
// ranks move up by the number of keys of A below them (the ranks at or below
// their position), 32 at a time from the top; then the keys of A are written
// at rank + index.  The scan cursor moves
// back to the first position that changed.
template <int NPL>
__device__ __forceinline__ void t_merge(float* Tk, uint32_t* Ti, int tk, const float* ak,
                                        const uint32_t* ai, int na, int ef, uint32_t idm,
                                        int& cursor, int lane) {
    int apt[NPL];         // rank of each key of A among T[0..tk)
    float akd[NPL];
    uint32_t aki[NPL];
#pragma unroll
    for (int t = 0; t < NPL; ++t) {
        const int k = lane + 32 * t;
        apt[t] = 0;
        akd[t] = 0.f;
        aki[t] = 0u;
        if (k < na) {
            akd[t] = ak[k];
            aki[t] = ai[k];
            int lo = 0, hi = tk;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (key_lt(Tk[mid], Ti[mid] & idm, akd[t], aki[t] & idm)) lo = mid + 1;
                else hi = mid;
            }
            apt[t] = lo;
        }
    }
    const int pmin = __shfl_sync(FULLMASK, apt[0], 0);   // A is sorted
    for (int top = tk - 1; top >= pmin; top -= 32) {
        const int i = top - lane;
        const bool act = i >= pmin;
        float kd = 0.f;
        uint32_t ki = 0;
        if (act) {
            kd = Tk[i];
            ki = Ti[i];
        }
        // the keys of A below T[i] are those whose rank in T is at most i
        int sh = 0;
        if (na == 1) {
            sh = act ? 1 : 0;
        } else {
            for (int k = 0; k < na; ++k) {
                const int r = __shfl_sync(FULLMASK, k < 32 ? apt[0] : apt[NPL - 1], k & 31);
                sh += act && r <= i;
            }
        }
        __syncwarp();
        if (act && sh) {
            Tk[CK(i + sh, ef, 1014)] = kd;
            Ti[i + sh] = ki;
        }
        __syncwarp();
    }
#pragma unroll
    for (int t = 0; t < NPL; ++t) {
        const int k = lane + 32 * t;
        if (k < na) {
            Tk[CK(apt[t] + k, ef, 1015)] = akd[t];
            Ti[apt[t] + k] = aki[t];
        }
    }
    __syncwarp();
    if (pmin < cursor) cursor = pmin;
}

enum { V_SEEN = 0, V_NEW = 1, V_NEW_SPILL = 2, V_PENDING = 3 };

// The visited hash in shared memory is bucketed: H slots form H/4 buckets of
// four (one 16-byte load per probe), buckets are probed linearly from the one
// the multiplicative hash picks.  Short probe chains up to a high load let the
// table take 3/4 of its slots before the warp switches to spill mode.
__device__ __forceinline__ uint32_t hbucket(uint32_t id, int logNB) {
    return (id * 2654435769u) >> (32 - logNB);
}

// exact test-and-set of the visited set.  Once the shared-memory table is 3/4
// full (spill mode) ids not found in it are test-and-set in the warp's global
// bitmap; the call then returns V_PENDING with the old bitmap word in `oldw`
// (its value is only waited for where the caller first reads it).  Lanes of the
// warp insert distinct ids concurrently: a lost compare-and-swap means another
// lane filled that slot, and the bucket is read again.
__device__ __forceinline__ int visit(uint32_t* hash, int H, int logNB, uint32_t id, bool spill_mode,
                                     uint32_t* bitmap, uint32_t& oldw) {
    const uint32_t mask = (uint32_t)(H >> 2) - 1u;
    uint32_t b = hbucket(id, logNB);
    int retries = 0;
    for (int probe = 0; probe <= (int)mask; ++probe) {
        uint4 v;   // a fresh read: other lanes may have filled slots since
        asm volatile("ld.volatile.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                     : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                     : "r"((uint32_t)__cvta_generic_to_shared(hash + 4 * CK(b, H >> 2, 1020))));
        if (v.x == id || v.y == id || v.z == id || v.w == id) return V_SEEN;
        const int e = v.x == PAD ? 0 : v.y == PAD ? 1 : v.z == PAD ? 2 : v.w == PAD ? 3 : -1;
        if (e < 0) {
            b = (b + 1) & mask;
            continue;
        }
        // the id is in no bucket of its probe sequence
        if (spill_mode) {
            oldw = atomicOr(&bitmap[id >> 5], 1u << (id & 31));
            return V_PENDING;
        }
        const uint32_t old = atomicCAS(&hash[4 * b + e], PAD, id);
        if (old == PAD) return V_NEW;
        if (old == id) return V_SEEN;
        if (++retries <= 4) --probe;   // re-read this bucket (bounded)
        else b = (b + 1) & mask;
    }
    return V_SEEN;  // unreachable: the table never fills (3/4 plus one batch < 1)
}

// The same visited set in 16-bit slots, for ids below 2^B with B = logNB + 15
// (logNB = log2 of the bucket count; buckets of eight slots, one 16-byte
// load).  h = id * 0x9E3779B1 mod 2^B is a bijection, so the bucket h >> 15
// and the 15 low bits identify the id; a slot holds those 15 bits, hence never
// the empty value 0xFFFF.  Each id has a single bucket: one probe measured
// faster than probe sequences of two, four or eight buckets.  An id whose
// bucket is full goes to the bitmap (V_PENDING) on every visit, since slots
// are never freed.  A lost compare-and-swap means another lane took a slot of
// the bucket, so after eight the bucket is full.
__device__ __forceinline__ int visit16(uint16_t* hash, int logNB, uint32_t id, bool spill_mode,
                                       uint32_t* bitmap, uint32_t& oldw) {
    const uint32_t h = (id * 0x9E3779B1u) & ((1u << (logNB + 15)) - 1u);
    const uint32_t want = h & 0x7FFFu, w2 = want * 0x10001u;
    uint16_t* bucket = hash + 8 * CK(h >> 15, 1u << logNB, 1023);
    const uint32_t saddr = (uint32_t)__cvta_generic_to_shared(bucket);
    for (int tries = 0; tries <= 8; ++tries) {
        uint4 v;   // a fresh read: other lanes may have filled slots since
        asm volatile("ld.volatile.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                     : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                     : "r"(saddr));
        if (__vcmpeq2(v.x, w2) | __vcmpeq2(v.y, w2) | __vcmpeq2(v.z, w2) | __vcmpeq2(v.w, w2))
            return V_SEEN;
        const uint32_t em = (__vcmpeq2(v.x, 0xFFFFFFFFu) & 0x00010001u) |
                            ((__vcmpeq2(v.y, 0xFFFFFFFFu) & 0x00010001u) << 1) |
                            ((__vcmpeq2(v.z, 0xFFFFFFFFu) & 0x00010001u) << 2) |
                            ((__vcmpeq2(v.w, 0xFFFFFFFFu) & 0x00010001u) << 3);
        if (!em || spill_mode) break;   // not in the table: the bitmap decides
        // first empty slot: word k = bit k of the low half, low/high half
        const int lo = __ffs(em & 0xFu), hi = __ffs(em >> 16);
        const int e = lo && (!hi || lo <= hi) ? 2 * (lo - 1) : 2 * (hi - 1) + 1;
        const unsigned short old = atomicCAS(reinterpret_cast<unsigned short*>(bucket + e),
                                             (unsigned short)0xFFFFu, (unsigned short)want);
        if (old == 0xFFFFu) return V_NEW;
        if (old == want) return V_SEEN;
    }
    oldw = atomicOr(&bitmap[id >> 5], 1u << (id & 31));
    return V_PENDING;
}

// t_hat for one edge: r-dot of the stored unit residual projection with uq
// (harvest of the learned predictor's training data)
__device__ __forceinline__ float edge_cos(const DevIndex& ix, size_t e, const float* uq) {
    float acc = 0.f;
    const float4* u = ix.edge_u + e * ix.r4;
    const float4* v = reinterpret_cast<const float4*>(uq);
    // r <= 64: two halves of up to eight 16-byte loads, each half issued
    // before its products (same summation order as a plain loop)
#pragma unroll
    for (int h = 0; h < 16; h += 8) {
        float4 x[8];
#pragma unroll
        for (int k = 0; k < 8; ++k)
            if (h + k < ix.r4) x[k] = __ldg(u + h + k);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            if (h + k < ix.r4) {
                const float4 y = v[h + k];
                acc = fmaf(x[k].x, y.x, acc);
                acc = fmaf(x[k].y, y.y, acc);
                acc = fmaf(x[k].z, y.z, acc);
                acc = fmaf(x[k].w, y.w, acc);
            }
        }
    }
    return acc;
}

// ---- FP16 codes (mode FINGER_F16).  The estimates of one expansion are the
// matrix-vector product t_hat = A u_q of the centre's code rows A (rows =
// slots, FP16) with the unit residual projection of the query u_q, run on the
// tensor cores as m16n8k16 MMAs with FP32 accumulation.  The table holds A in
// the MMA's A-fragment order: for centre c, tile T (slots 16T .. 16T+15, NT =
// 32 NPL slots per node, zero rows beyond deg0) and k step ks (codes 16ks ..
// 16ks+15, KS = 2 or 4 steps), 32 lanes x 16 bytes, lane l = 4g + t holding
// rows 16T+g and 16T+g+8 at codes 16ks+2t, +1, +8, +9.  A centre's block is
// contiguous and its address depends on c alone, so it is requested in the
// same round trip as c's adjacency row, one 16-byte load per lane per (tile,
// k step), at most eight per round.  u_q is split into FP16 high and low parts
// (hi = fp16(u), lo = fp16(u - hi)) for the even and odd columns of B, so
// columns 2t and 2t+1 of the product sum to A u_q with u_q kept to about 22
// bits; the codes are exact FP16 values.  KS and NT are compile-time, so the
// whole product is straight-line code.  The reduced-precision mode (LP) keeps
// the same fragments as FP8-e4m3 codes of 256 u: one 16-byte load per lane
// holds two k steps of a tile, and each FP8 pair becomes one FP16 pair of the A
// operand by a single conversion (e4m3 values are exact in FP16).
__device__ __forceinline__ void mma_f16(float* d, const uint4& a, uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a.x), "r"(a.y), "r"(a.z), "r"(a.w), "r"(b0), "r"(b1));
}

// D += A B for one m16n8k32 tile with FP8-e4m3 operands, FP32 accumulation
__device__ __forceinline__ void mma_e4m3(float* d, const uint4& a, uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k32.row.col.f32.e4m3.e4m3.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a.x), "r"(a.y), "r"(a.z), "r"(a.w), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t pack_half2(float lo, float hi) {
    __half2 v = __floats2half2_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&v);
}

// one round: tiles t0 .. t0 + TPR - 1 (TPR = min(NT, 8 / KS)) into hx[T KS + ks].
// The second half of the block (tiles NT/2 ..) holds slots 16 NT/2 .. and is
// all zero rows for a centre of at most that degree; it is read only when
// `full` (the centre's tag) says the centre has more neighbours, else zeros.
template <int KS, int NT, bool W8 = false>
__device__ __forceinline__ void wb_load(const DevIndex& ix, uint32_t c, int t0, bool full,
                                        uint4 (&hx)[8], int lane) {
    if constexpr (W8) {   // FP8 storage: KS / 2 loads per tile, every tile in one round
        constexpr int KP = KS / 2;
        const uint4* base = ix.edge_q + (size_t)c * NT * KP * 32 + lane;
#pragma unroll
        for (int T = 0; T < NT; ++T)
#pragma unroll
            for (int p = 0; p < KP; ++p) {
                const bool need = T < NT / 2 || full;
                hx[T * KP + p] = need ? __ldg(base + (T * KP + p) * 32) : make_uint4(0u, 0u, 0u, 0u);
            }
        return;
    }
    constexpr int TPR = NT * KS <= 8 ? NT : 8 / KS;
    const uint4* base = ix.edge_h + ((size_t)c * NT + t0) * KS * 32 + lane;
#pragma unroll
    for (int T = 0; T < TPR; ++T)
#pragma unroll
        for (int ks = 0; ks < KS; ++ks) {
            const bool need = TPR < NT || T < NT / 2 || full;   // (compile-time unless split)
            hx[T * KS + ks] = need ? __ldg(base + (T * KS + ks) * 32) : make_uint4(0u, 0u, 0u, 0u);
        }
}

// The B fragments live in shared memory as packed half2 words in fragment
// order: word ((ks * 2 + p) * 4 + t) * 2 + w holds codes 16ks + 2t + 8w, +1 of
// u_q's high (p = 0) or low (p = 1) part, so lane 4g + t reads its two words
// of step ks (column g takes part g & 1) with one 8-byte load.  wb_bfrag_store
// writes them from u_q's entries 2l, 2l + 1 formed by lane l.
__device__ __forceinline__ void wb_bfrag_store(uint32_t* bsm, float u0, float u1, int ks_n, int lane) {
    const __half2 h = __floats2half2_rn(u0, u1);
    const float2 hf = __half22float2(h);
    const __half2 l = __floats2half2_rn(u0 - hf.x, u1 - hf.y);
    const int ks = lane >> 3, t = lane & 3, w = (lane >> 2) & 1;
    if (ks < ks_n) {
        bsm[((ks * 2 + 0) * 4 + t) * 2 + w] = *reinterpret_cast<const uint32_t*>(&h);
        bsm[((ks * 2 + 1) * 4 + t) * 2 + w] = *reinterpret_cast<const uint32_t*>(&l);
    }
}

// FP8 codes (modes LP and FINGER_F8): the codes are 256 u_d in the 8-bit
// A-fragment order of mma.m16n8k32, and 256 u_q enters as an e4m3 high part
// (even B columns) plus the e4m3 rounding of the remainder (odd columns), so
// the product needs no conversion.  Byte j of word ((kk * 2 + p) * 4 + t) * 2
// + w of the B region holds code 32kk + 16w + 4t + j of part p, so lane 4g + t
// reads its two words of step kk (column g takes part g & 1) with one 8-byte
// load; lane l forms codes 2l and 2l + 1.
__device__ __forceinline__ float e4m3_value(uint32_t code) {
    const __half_raw h = __nv_cvt_fp8_to_halfraw((__nv_fp8_storage_t)code, __NV_E4M3);
    return __half2float(__half(h));
}

__device__ __forceinline__ void wb_bfrag_store8(uint32_t* bsm, float u0, float u1, int kp_n,
                                                int lane) {
    const float s0 = 256.f * u0, s1 = 256.f * u1;
    const uint32_t h0 = __nv_cvt_float_to_fp8(s0, __NV_SATFINITE, __NV_E4M3);
    const uint32_t h1 = __nv_cvt_float_to_fp8(s1, __NV_SATFINITE, __NV_E4M3);
    const uint32_t l0 = __nv_cvt_float_to_fp8(s0 - e4m3_value(h0), __NV_SATFINITE, __NV_E4M3);
    const uint32_t l1 = __nv_cvt_float_to_fp8(s1 - e4m3_value(h1), __NV_SATFINITE, __NV_E4M3);
    const int kk = lane >> 4, w = (lane >> 3) & 1, t = (lane >> 1) & 3, j = 2 * (lane & 1);
    if (kk < kp_n) {
        uint16_t* b16 = reinterpret_cast<uint16_t*>(bsm);
        b16[((((kk * 2 + 0) * 4 + t) * 2 + w) * 4 + j) >> 1] = (uint16_t)(h0 | h1 << 8);
        b16[((((kk * 2 + 1) * 4 + t) * 2 + w) * 4 + j) >> 1] = (uint16_t)(l0 | l1 << 8);
    }
}

// A block with more than four FP8 products per expansion (64 slots and r > 32)
// measured faster the other way: its codes follow the FP16 fragment order of
// m16n8k16, two k steps per 16 bytes, each FP8 pair becomes one FP16 pair of
// the A operand by a single conversion (exact), and u_q takes the FP16 high /
// low split of the FP16-code mode.
__device__ __forceinline__ uint32_t e4m3x2_to_half2(uint32_t pair) {
    const __half2_raw h = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)pair, __NV_E4M3);
    return (uint32_t)h.x | ((uint32_t)h.y << 16);
}

// the A fragment of k step (2p + h) from a 16-byte FP8 load (h: which half)
__device__ __forceinline__ uint4 e4m3_frag(const uint4& x, int h) {
    const uint32_t lo = h ? x.z : x.x, hi = h ? x.w : x.y;
    return make_uint4(e4m3x2_to_half2(lo & 0xFFFFu), e4m3x2_to_half2(lo >> 16),
                      e4m3x2_to_half2(hi & 0xFFFFu), e4m3x2_to_half2(hi >> 16));
}

// whether a code block of NT tiles and KS k steps of 16 is multiplied in FP8
template <int NT, int KS>
__host__ __device__ constexpr bool fp8_product() { return NT * (KS / 2) <= 4; }

// t_hat of rows 16(t0+T)+g (v[2(t0+T)]) and +8 (v[2(t0+T)+1]) for the round's
// tiles; k step outer, so each code register dies at its MMA.

template <int KS, int NT, bool W8 = false>
__device__ __forceinline__ void wb_mma(const uint4 (&hx)[8], const uint32_t* bsm, int t0,
                                       float (&v)[8], int lane) {
    if constexpr (W8) {   // every tile
        constexpr int KP = KS / 2;
        const uint2* bf = reinterpret_cast<const uint2*>(bsm) + ((lane >> 2) & 1) * 4 + (lane & 3);
        float acc[NT][4];
#pragma unroll
        for (int T = 0; T < NT; ++T) acc[T][0] = acc[T][1] = acc[T][2] = acc[T][3] = 0.f;
        if constexpr (fp8_product<NT, KS>()) {   // 32 FP8 codes per MMA
#pragma unroll
            for (int kk = 0; kk < KP; ++kk) {
                const uint2 b = bf[kk * 8];
#pragma unroll
                for (int T = 0; T < NT; ++T) mma_e4m3(acc[T], hx[T * KP + kk], b.x, b.y);
            }
        } else {   // FP8 pairs converted to FP16 pairs, 16 codes per MMA
#pragma unroll
            for (int ks = 0; ks < KS; ++ks) {
                const uint2 b = bf[ks * 8];
#pragma unroll
                for (int T = 0; T < NT; ++T)
                    mma_f16(acc[T], e4m3_frag(hx[T * KP + ks / 2], ks & 1), b.x, b.y);
            }
        }
#pragma unroll
        for (int T = 0; T < NT; ++T) {
            v[2 * T] = acc[T][0] + acc[T][1];
            v[2 * T + 1] = acc[T][2] + acc[T][3];
        }
        return;
    }
    constexpr int TPR = NT * KS <= 8 ? NT : 8 / KS;
    const uint2* bf = reinterpret_cast<const uint2*>(bsm) + ((lane >> 2) & 1) * 4 + (lane & 3);
    float acc[TPR][4];
#pragma unroll
    for (int T = 0; T < TPR; ++T) acc[T][0] = acc[T][1] = acc[T][2] = acc[T][3] = 0.f;
#pragma unroll
    for (int ks = 0; ks < KS; ++ks) {
        const uint2 b = bf[ks * 8];
#pragma unroll
        for (int T = 0; T < TPR; ++T) mma_f16(acc[T], hx[T * KS + ks], b.x, b.y);
    }
#pragma unroll
    for (int T = 0; T < TPR; ++T) {
        v[2 * (t0 + T)] = acc[T][0] + acc[T][1];
        v[2 * (t0 + T) + 1] = acc[T][2] + acc[T][3];
    }
}

// lane j of slot block s receives t_hat of row 32s + j: lane 4g + t offers
// row 32s + 8t + g
template <int NPL>
__device__ __forceinline__ void wb_route(const float (&v)[8], float* th, int lane) {
    const int t = lane & 3;
    const int src = 4 * (lane & 7) + (lane >> 3);
#pragma unroll
    for (int s = 0; s < NPL; ++s) {
        const float e = t == 0 ? v[4 * s] : t == 1 ? v[4 * s + 1] : t == 2 ? v[4 * s + 2] : v[4 * s + 3];
        th[s] = __shfl_sync(FULLMASK, e, src);
    }
}

// Features of one (q, c, d) triple for the learned angle predictor (an
// extension; the paper has no learned predictor): f = [u_q * u_d (r values),
// t_hat, ||q_res|| / ||q||, ||d_res|| / ||d||, a / (|a| + |b| + 1e-6)], with
// ||d||^2 = b^2 ||c||^2 + ||d_res||^2, written as FP32 into a global row
// (harvest).  Returns t_hat, summed in the same order as edge_cos.
__device__ __forceinline__ float features_row(const DevIndex& ix, size_t e, const float* uq,
                                              float2 sc, float cc, float ac, float qres_n,
                                              float qn2, float* grow) {
    const float4* ud = ix.edge_u + e * ix.r4;
    float th = 0.f;
    for (int k = 0; k < ix.r4; ++k) {
        const float4 x = __ldg(ud + k);
        const float p[4] = {x.x * uq[4 * k], x.y * uq[4 * k + 1], x.z * uq[4 * k + 2],
                            x.w * uq[4 * k + 3]};
        th = fmaf(x.x, uq[4 * k], th);
        th = fmaf(x.y, uq[4 * k + 1], th);
        th = fmaf(x.z, uq[4 * k + 2], th);
        th = fmaf(x.w, uq[4 * k + 3], th);
#pragma unroll
        for (int i = 0; i < 4; ++i)
            if (4 * k + i < ix.r) grow[4 * k + i] = p[i];
    }
    const float dnorm = sqrtf(sc.y * sc.y * cc + sc.x * sc.x);
    grow[ix.r] = th;
    grow[ix.r + 1] = qn2 > 0.f ? qres_n * rsqrtf(qn2) : 0.f;
    grow[ix.r + 2] = dnorm > 0.f ? sc.x / dnorm : 0.f;
    grow[ix.r + 3] = ac / (fabsf(ac) + fabsf(sc.y) + 1e-6f);
    return th;
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&v);
}

// The same features as features_row, written as one BF16 row of the predictor
// tile in a single pass over the edge row: each 16-byte chunk of u_d gives four
// products (one 8-byte store) and four terms of t_hat; then the four tail
// features and the zero padding up to kp.  Returns t_hat, summed in edge_cos
// order.  (Entries r..r_pad-1 of u_d are 0, so their products are 0 before the
// tail overwrites them.)
__device__ __forceinline__ float features_tile(const DevIndex& ix, size_t e, const float* uq,
                                              float2 sc, float cc, float ac, float qres_n,
                                              float qn2, __nv_bfloat16* xrow) {
    const float4* ud = ix.edge_u + e * ix.r4;
    const float4* uq4 = reinterpret_cast<const float4*>(uq);
    uint2* out = reinterpret_cast<uint2*>(xrow);
    float th = 0.f;
    for (int k = 0; k < ix.r4; ++k) {
        const float4 x = __ldg(ud + k);
        const float4 y = uq4[k];
        th = fmaf(x.x, y.x, th);
        th = fmaf(x.y, y.y, th);
        th = fmaf(x.z, y.z, th);
        th = fmaf(x.w, y.w, th);
        out[k] = make_uint2(pack_bf16x2(x.x * y.x, x.y * y.y), pack_bf16x2(x.z * y.z, x.w * y.w));
    }
    const float dnorm = sqrtf(sc.y * sc.y * cc + sc.x * sc.x);
    const int r = ix.r;
    xrow[r] = __float2bfloat16_rn(th);
    xrow[r + 1] = __float2bfloat16_rn(qn2 > 0.f ? qres_n * rsqrtf(qn2) : 0.f);
    xrow[r + 2] = __float2bfloat16_rn(dnorm > 0.f ? sc.x / dnorm : 0.f);
    xrow[r + 3] = __float2bfloat16_rn(ac / (fabsf(ac) + fabsf(sc.y) + 1e-6f));
    for (int j = r + 4; j < ix.mlp_kp; ++j) xrow[j] = __float2bfloat16_rn(0.f);
    return th;
}

// D += A B for one m16n8k16 tile, BF16 operands, FP32 accumulators
__device__ __forceinline__ void mma_bf16(float* d, const uint32_t* a, uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// The predictor r+4 -> 64 -> 64 -> 1 on one 16-row tile of feature rows with
// warp-level BF16 tensor-core MMAs (m16n8k16, FP32 accumulation).  Layer 1's
// accumulators are turned into the A operand of layer 2 in registers (the C
// layout of two n8 tiles is the A layout of one k16 step); layer 3 is an FP32
// dot reduced over the lane quad.  The B operands are stored fragment-major
// (one 8-byte word pair per lane per (n8 tile, k16 step)), so each fragment is
// one coalesced load that stays in L1; biases and w3 are FP32 in global memory.
__device__ __forceinline__ void mlp_tile(const __nv_bfloat16* xt, int kp, const uint2* W1f,
                                         const uint2* W2f, const float* b1, const float* b2,
                                         const float* w3, float b3, float* yout, int lane) {
    const int g = lane >> 2, t = lane & 3;
    const int nks = kp >> 4;
    const int xs = kp + MLP_PAD;
    const int r0 = g, r1 = g + 8;
    float acc[8][4];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
        const float c0 = __ldg(b1 + 8 * nt + 2 * t), c1 = __ldg(b1 + 8 * nt + 2 * t + 1);
        acc[nt][0] = c0;
        acc[nt][1] = c1;
        acc[nt][2] = c0;
        acc[nt][3] = c1;
    }
    for (int ks = 0; ks < nks; ++ks) {
        const uint32_t* X0 = reinterpret_cast<const uint32_t*>(xt + r0 * xs + 16 * ks);
        const uint32_t* X1 = reinterpret_cast<const uint32_t*>(xt + r1 * xs + 16 * ks);
        const uint32_t a[4] = {X0[t], X1[t], X0[t + 4], X1[t + 4]};
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            const uint2 w = __ldg(W1f + (nt * nks + ks) * 32 + lane);
            mma_bf16(acc[nt], a, w.x, w.y);
        }
    }
    uint32_t h[4][4];
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
        h[kk][0] = pack_bf16x2(fmaxf(acc[2 * kk][0], 0.f), fmaxf(acc[2 * kk][1], 0.f));
        h[kk][1] = pack_bf16x2(fmaxf(acc[2 * kk][2], 0.f), fmaxf(acc[2 * kk][3], 0.f));
        h[kk][2] = pack_bf16x2(fmaxf(acc[2 * kk + 1][0], 0.f), fmaxf(acc[2 * kk + 1][1], 0.f));
        h[kk][3] = pack_bf16x2(fmaxf(acc[2 * kk + 1][2], 0.f), fmaxf(acc[2 * kk + 1][3], 0.f));
    }
    float p0 = 0.f, p1 = 0.f;
    // layer 2 as a rolled loop over the eight n8 tiles: its accumulators live
    // only inside one iteration, and the kernel's code stays small enough for
    // the instruction cache
#pragma unroll 1
    for (int nt = 0; nt < 8; ++nt) {
        float cacc[4];
        cacc[0] = cacc[2] = __ldg(b2 + 8 * nt + 2 * t);
        cacc[1] = cacc[3] = __ldg(b2 + 8 * nt + 2 * t + 1);
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
            const uint2 w = __ldg(W2f + (nt * 4 + kk) * 32 + lane);
            mma_bf16(cacc, h[kk], w.x, w.y);
        }
        const float wa = __ldg(w3 + 8 * nt + 2 * t), wb = __ldg(w3 + 8 * nt + 2 * t + 1);
        p0 = fmaf(fmaxf(cacc[0], 0.f), wa, fmaf(fmaxf(cacc[1], 0.f), wb, p0));
        p1 = fmaf(fmaxf(cacc[2], 0.f), wa, fmaf(fmaxf(cacc[3], 0.f), wb, p1));
    }
    p0 += __shfl_xor_sync(FULLMASK, p0, 1);
    p0 += __shfl_xor_sync(FULLMASK, p0, 2);
    p1 += __shfl_xor_sync(FULLMASK, p1, 1);
    p1 += __shfl_xor_sync(FULLMASK, p1, 2);
    if (t == 0) {
        yout[r0] = p0 + b3;
        yout[r1] = p1 + b3;
    }
}

template <int MODE, int G, int VPL, int NPL, int OCC>
__global__ void __launch_bounds__(128, OCC) k_search(DevIndex ix, SearchArgs a) {
    constexpr bool LP = MODE == MODE_LP_K2 || MODE == MODE_LP_K4;   // BF16 rows, FP8 codes
    constexpr bool W8 = LP || MODE == MODE_F8_K2 || MODE == MODE_F8_K4;   // FP8 codes
    constexpr bool EST = MODE != FINGER_MODE_PLAIN;
    constexpr bool MLP = MODE == FINGER_MODE_FINGER_MLP;
    constexpr bool HARV = MODE == MODE_HARVEST;
    // FP16 (FINGER_F16) or FP8 (LP, FINGER_F8) codes, product on the tensor cores; k steps
    constexpr bool WB = MODE == MODE_F16_K2 || MODE == MODE_F16_K4 || W8;
    constexpr int WKS = MODE == MODE_F16_K2 || MODE == MODE_LP_K2 || MODE == MODE_F8_K2 ? 2 : 4;
    // bytes of half a code block (the slots 16 NPL .. of a centre are the other half)
    constexpr int HALF_BYTES = NPL * WKS * 512 / (W8 ? 2 : 1);
    constexpr int WNT = 2 * NPL;                            // tiles per node
    // ids in T: FP16-code mode ids carry the tag TAG (the node has more than
    // 16 NPL neighbours, so its code block's second half is needed) below EXP
    constexpr uint32_t TAG = 0x40000000u;
    constexpr uint32_t IDM = WB ? ~(EXP | TAG) : ~EXP;        // id without flags
    extern __shared__ __align__(16) unsigned char sm[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int wpb = blockDim.x >> 5;
    const unsigned ltmask = (1u << lane) - 1u;
    const int r_pad = ix.r4 * 4;
    const int nchunks = LP ? ix.m8 : ix.m4;
    const int qs_len = LP ? ix.m8 * 8 : ix.m4 * 4;

    unsigned char* wb = sm + a.blk_smem + (size_t)wib * a.warp_smem;
    // Per-warp region: first the fixed-size staging of one expansion (compile-
    // time offsets from wb, so its addresses need no pointer registers), then
    // the regions whose sizes depend on the launch (result list, visited hash,
    // projections, staged query, predictor tile).
    uint32_t* nbs = reinterpret_cast<uint32_t*>(wb);           // neighbour of each slot
    float* es = reinterpret_cast<float*>(nbs + 32 * NPL);      // estimate of each slot
    float* xb = es + 32 * NPL;                                 // exact distance / t_hat
    int* lst = reinterpret_cast<int*>(xb + 32 * NPL);          // compacted slot lists
    float* ak = reinterpret_cast<float*>(lst + 32 * NPL);      // admitted keys (sorted)
    uint32_t* ai = reinterpret_cast<uint32_t*>(ak + 32 * NPL);
    int* apos = reinterpret_cast<int*>(ai + 32 * NPL);         // slot of each admission
    float* aub = reinterpret_cast<float*>(apos + 32 * NPL);    // ub after it
    int* meta = reinterpret_cast<int*>(aub + 32 * NPL);        // replay results (8 ints)
    float* Tk = reinterpret_cast<float*>(meta + 8);
    uint32_t* Ti = reinterpret_cast<uint32_t*>(Tk + a.ef_cap);
    uint32_t* hash = Ti + a.ef_cap;
    const int hwords = a.h16 ? a.H >> 1 : a.H;   // 32-bit words of the visited hash
    float* uq = reinterpret_cast<float*>(hash + hwords);
    // FP16 codes: the region holds u_q's B fragments, 16 KS packed words
    const int uq_len = WB ? max(r_pad, 16 * WKS) : r_pad;
    float* pq = uq + uq_len;
    // the query staging buffer is only read before the visited hash is cleared,
    // so outside the LP mode (which re-reads it for the FP32 re-rank) and the
    // FP16-code mode (whose exact distances read it) it lives inside the hash
    // region (the plan keeps its words >= m_pad)
    constexpr bool QSM = LP || WB;   // query kept in its own region
    float* qs = QSM ? pq + r_pad : reinterpret_cast<float*>(hash);
    __nv_bfloat16* xt = reinterpret_cast<__nv_bfloat16*>(QSM ? qs + ((qs_len + 3) & ~3) : pq + r_pad);   // predictor input tile
    if (FG_CHECKED) g_chk_err = a.err;   // same value from every thread
    const int64_t slot = (int64_t)blockIdx.x * wpb + wib;
    uint32_t* bitmap = a.bitmap + slot * a.words;
    uint32_t* spl = a.spill + slot * a.spill_cap;
    const int logNB = 31 - __clz(a.H >> (a.h16 ? 3 : 2));   // buckets of the visited hash

    for (;;) {
        int qi = 0;
        if (lane == 0) qi = (int)atomicAdd(a.work, 1u);
        qi = __shfl_sync(FULLMASK, qi, 0);
        if (qi >= a.nq) break;
        const int K = a.K_arr ? a.K_arr[qi] : a.K;
        const int ef = min(max(a.ef_arr ? a.ef_arr[qi] : a.ef, 1), a.ef_cap);
        const int64_t ooff = a.out_off ? a.out_off[qi] : (int64_t)qi * K;

        // ---- stage the query (a1: ||q||^2 and P q)
        const float* qg = a.Q + (size_t)qi * ix.m;
        for (int i = lane; i < qs_len; i += 32) qs[i] = i < ix.m ? qg[i] : 0.f;
        __syncwarp();
        QRegs<LP, VPL> q;
        if constexpr (!WB) load_qregs<LP, G, VPL>(q, qs, nchunks, lane % G);
        float qn2 = 0.f;
        for (int i = lane; i < ix.m; i += 32) qn2 = fmaf(qs[i], qs[i], qn2);
        qn2 = warp_sum(qn2);
        if constexpr (EST) {
            for (int i = lane; i < r_pad; i += 32) {
                const float4* prow = ix.P + (size_t)i * ix.m4;
                const float4* q4 = reinterpret_cast<const float4*>(qs);
                float acc = 0.f;
                for (int k = 0; k < ix.m4; ++k) {
                    const float4 p = __ldg(prow + k);
                    const float4 y = q4[k];
                    acc = fmaf(p.x, y.x, acc);
                    acc = fmaf(p.y, y.y, acc);
                    acc = fmaf(p.z, y.z, acc);
                    acc = fmaf(p.w, y.w, acc);
                }
                pq[i] = acc;
            }
            __syncwarp();
        }
        int c_exp = 0, c_exa = 0, c_est = 0, c_skip = 0, c_exact = 0, c_adm = 0, c_up = 0,
            c_gath = 0, c_half = 0;   // c_half: code-block halves read (FP16 codes)
        bool fail = false;

        // ---- a2: greedy descent through levels maxlevel..1 (exact distances)
        uint32_t cur = (uint32_t)ix.entry;
        if (lane == 0) {
            nbs[0] = cur;
            lst[0] = 0;
        }
        __syncwarp();
        exact_list<LP, G, VPL, WB>(q, qs, ix, nbs, lst, 1, xb, lane);
        float dcur = xb[0];
        c_up++;
        c_gath++;
        __syncwarp();
        for (int l = ix.maxlevel; l >= 1; --l) {
            for (int it = 0;; ++it) {
                if (it >= a.max_expansions) {
                    fail = true;
                    break;
                }
                const uint32_t* row = ix.up_adj + (size_t)CK(ix.up_off[CK(cur, ix.n, 1006)] + l - 1, 1LL << 40, 1007) * ix.Mup;
                const uint32_t id = lane < ix.Mup ? row[lane] : PAD;
                const bool v = id != PAD;
                const unsigned bm = __ballot_sync(FULLMASK, v);
                nbs[lane] = id;
                if (v) lst[__popc(bm & ltmask)] = lane;
                __syncwarp();
                const int cv = __popc(bm);
                exact_list<LP, G, VPL, WB>(q, qs, ix, nbs, lst, cv, xb, lane);
                c_up += cv;
                c_gath += cv;
                float bd = v ? xb[lane] : INFINITY;
                uint32_t bi = v ? id : PAD;
                if (key_lt(dcur, cur, bd, bi)) {
                    bd = dcur;
                    bi = cur;
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const float od = __shfl_xor_sync(FULLMASK, bd, o);
                    const uint32_t oi = __shfl_xor_sync(FULLMASK, bi, o);
                    if (key_lt(od, oi, bd, bi)) {
                        bd = od;
                        bi = oi;
                    }
                }
                __syncwarp();
                if (bi == cur) break;
                cur = bi;
                dcur = bd;
            }
        }

        // ---- a3..a6: layer 0
        for (int i = lane; i < hwords; i += 32) hash[i] = PAD;
        __syncwarp();
        if (lane == 0) {
            Tk[0] = dcur;
            Ti[0] = WB ? cur | TAG : cur;   // (its degree is not looked up: read both halves)
            if (a.h16) {   // the table is empty: distance 0, first slot
                const uint32_t h = (cur * 0x9E3779B1u) & ((1u << (logNB + 15)) - 1u);
                reinterpret_cast<uint16_t*>(hash)[8 * (h >> 15)] = (uint16_t)(h & 0x7FFFu);
            } else {
                hash[4 * hbucket(cur, logNB)] = cur;
            }
        }
        __syncwarp();
        int sz = 1, cursor = 0, hcount = 1, nspill = 0;
        bool spill_mode = false;
        int expansions = 0;
        while (!fail) {
            uint32_t craw = 0u;
            float dc = 0.f;
            cursor = find_next_entry(Tk, Ti, sz, cursor, lane, craw, dc);
            if (cursor >= sz) break;
            if (expansions >= a.max_expansions || nspill + 32 * NPL > a.spill_cap) {
                fail = true;
                break;
            }
            (void)CK(cursor, ef, 1001);
            const uint32_t c = craw & IDM;
            const bool cfull = craw & TAG;   // FP16 codes: second half of the block needed
            __syncwarp();
            if (lane == 0) Ti[cursor] = craw | EXP;
            expansions++;
            const bool use_est = EST && expansions > a.warmup;

            uint32_t nb[NPL], nbt[NPL];   // neighbour ids; as stored (FP16 codes: tagged)
#pragma unroll
            for (int s = 0; s < NPL; ++s) {
                const int j = s * 32 + lane;
                nbt[s] = j < ix.deg0 ? __ldg((WB ? ix.adj_t : ix.adj0) +
                                             CK((size_t)c * ix.deg0 + j, ix.n * ix.deg0, 1003))
                                     : PAD;
                nb[s] = WB && nbt[s] != PAD ? nbt[s] & IDM : nbt[s];
            }
            float cc = 0.f, pc0 = 0.f, pc1 = 0.f;
            if (use_est) {
                cc = __ldg(ix.xnorm2 + c);
                const float* pcr = reinterpret_cast<const float*>(ix.Pc) + (size_t)c * r_pad;
                if constexpr (WB) {   // entries 2 lane, 2 lane + 1
                    if (2 * lane < r_pad) {
                        const float2 p2 = __ldg(reinterpret_cast<const float2*>(pcr) + lane);
                        pc0 = p2.x;
                        pc1 = p2.y;
                    }
                } else {
                    if (lane < r_pad) pc0 = __ldg(pcr + lane);
                    if (lane + 32 < r_pad) pc1 = __ldg(pcr + lane + 32);
                }
            }
            // FP16 codes: c's code block and edge scalars, requested in the same
            // round trip as the adjacency row
            uint4 hx[8];
            float2 scw[NPL];
            float th[NPL];
            float wac = 0.f, wqres2 = 0.f;   // a and ||q_res||^2 of this centre
            if constexpr (WB) {
                if (use_est) {
#pragma unroll
                    for (int s = 0; s < NPL; ++s) {
                        const int j = s * 32 + lane;
                        scw[s] = j < ix.deg0 ? __ldg(ix.edge_s + (size_t)c * ix.deg0 + j)
                                             : make_float2(0.f, 0.f);
                    }
                    wb_load<WKS, WNT, W8>(ix, c, 0, cfull, hx, lane);
                    c_half += cfull ? 2 : 1;
                    // per-centre prep (Sec. 3.2 identity for q^T c, Supplementary G),
                    // then the product: the codes arrive with the adjacency row
                    // and are consumed before the visited test
                    const float qc = 0.5f * (qn2 + cc - dc);
                    wac = cc > 0.f ? qc / cc : 0.f;
                    wqres2 = fmaxf(qn2 - wac * qc, 0.f);
                    // this lane's entries 2 lane, 2 lane + 1 of P q_res = P q - a P c
                    float u0 = 0.f, u1 = 0.f;
                    if (2 * lane < r_pad) {
                        const float2 q2 = reinterpret_cast<const float2*>(pq)[lane];
                        u0 = q2.x - wac * pc0;
                        u1 = q2.y - wac * pc1;
                    }
                    const float nrm = warp_sum(u0 * u0 + u1 * u1);
                    const float inv = nrm > 0.f ? rsqrtf(nrm) : 0.f;
                    uint32_t* bsm = reinterpret_cast<uint32_t*>(uq);
                    if constexpr (W8 && fp8_product<WNT, WKS>())
                        wb_bfrag_store8(bsm, u0 * inv, u1 * inv, WKS / 2, lane);
                    else
                        wb_bfrag_store(bsm, u0 * inv, u1 * inv, WKS, lane);
                    __syncwarp();
                    float v[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                    wb_mma<WKS, WNT, W8>(hx, bsm, 0, v, lane);
                    if constexpr (!W8 && WNT * WKS > 8) {   // second round: tiles 2, 3
                        if (cfull) {
                            wb_load<WKS, WNT>(ix, c, 2, true, hx, lane);
                            wb_mma<WKS, WNT>(hx, bsm, 2, v, lane);
                        }
                    }
                    wb_route<NPL>(v, th, lane);
                    if constexpr (W8) {   // codes of 256 u_d (times parts of 256 u_q)
                        const float sc = fp8_product<WNT, WKS>() ? ix.code_inv * (1.f / 256.f)
                                                                : ix.code_inv;
#pragma unroll
                        for (int s = 0; s < NPL; ++s) th[s] *= sc;
                    }
                }
            }
            // In FINGER mode a bitmap test-and-set is resolved only after the
            // neighbour's edge row has been requested, so the two round trips
            // overlap; a neighbour that turns out visited just drops its estimate.
            constexpr bool DEFER = MODE == FINGER_MODE_FINGER || WB;
            bool isnew[NPL], pend[NPL];
            uint32_t pold[NPL];
#pragma unroll
            for (int s = 0; s < NPL; ++s) {
                int res = V_SEEN;
                uint32_t oldw = 0u;
                if (nb[s] != PAD)
                    res = a.h16 ? visit16(reinterpret_cast<uint16_t*>(hash), logNB,
                                          (uint32_t)CK(nb[s], ix.n, 1004), spill_mode, bitmap, oldw)
                                : visit(hash, a.H, logNB, (uint32_t)CK(nb[s], ix.n, 1004), spill_mode,
                                        bitmap, oldw);
                if (!DEFER && res == V_PENDING)
                    res = (oldw & (1u << (nb[s] & 31))) ? V_SEEN : V_NEW_SPILL;
                pend[s] = res == V_PENDING;
                pold[s] = oldw;
                isnew[s] = res != V_SEEN;
                if (!DEFER) {
                    const unsigned sb = __ballot_sync(FULLMASK, res == V_NEW_SPILL);
                    if (res == V_NEW_SPILL) spl[CK(nspill + __popc(sb & ltmask), a.spill_cap, 1005)] = nb[s];
                    nspill += __popc(sb);
                }
                hcount += __popc(__ballot_sync(FULLMASK, res == V_NEW));
                nbs[s * 32 + lane] = nbt[s];
            }
            if (hcount > a.H - (a.H >> 2)) spill_mode = true;

            // a4: per-centre prep (Sec. 3.2 identity for q^T c, Supplementary G)
            float ac = 0.f, qres2 = 0.f, qres_n = 0.f;
            if (WB && use_est) {   // formed at the pop
                ac = wac;
                qres2 = wqres2;
                qres_n = sqrtf(qres2);
            } else if (use_est) {
                const float qc = 0.5f * (qn2 + cc - dc);
                ac = cc > 0.f ? qc / cc : 0.f;
                qres2 = fmaxf(qn2 - ac * qc, 0.f);
                qres_n = sqrtf(qres2);
                {
                    const float u0 = lane < r_pad ? pq[lane] - ac * pc0 : 0.f;
                    const float u1 = lane + 32 < r_pad ? pq[lane + 32] - ac * pc1 : 0.f;
                    const float nrm = warp_sum(u0 * u0 + u1 * u1);
                    const float inv = nrm > 0.f ? rsqrtf(nrm) : 0.f;
                    if (lane < r_pad) uq[lane] = u0 * inv;
                    if (lane + 32 < r_pad) uq[lane + 32] = u1 * inv;
                    __syncwarp();
                }
            }

            // a5: estimates of the new neighbours against ub at expansion start
            const bool full0 = sz == ef;
            const float ub0 = full0 ? Tk[ef - 1] : INFINITY;
            float tr[NPL];          // distribution-matched cosine per slot
            int64_t hpos[NPL];      // harvest record of each slot (-1: none)
#pragma unroll
            for (int s = 0; s < NPL; ++s) {
                tr[s] = 0.f;
                hpos[s] = -1;
            }
            int crow[NPL];          // MLP: compact feature row of each predicted slot (-1: none)
#pragma unroll
            for (int s = 0; s < NPL; ++s) crow[s] = -1;
            if constexpr (HARV) {
                if (use_est) {
#pragma unroll
                    for (int s = 0; s < NPL; ++s) {
                        const int o = s * 32 + lane;
                        int64_t pos = -1;
                        const bool rec = isnew[s] && full0;
                        const unsigned bm = __ballot_sync(FULLMASK, rec);
                        unsigned long long base = 0;
                        if (lane == 0 && bm) base = atomicAdd(a.hv_count, (unsigned long long)__popc(bm));
                        base = __shfl_sync(FULLMASK, base, 0);
                        if (rec) pos = (int64_t)base + __popc(bm & ltmask);
                        if (pos >= a.hv_cap) pos = -1;
                        hpos[s] = pos;
                        if (isnew[s]) {
                            const size_t e = (size_t)c * ix.deg0 + o;
                            const float2 sc = __ldg(ix.edge_s + e);
                            const float th =
                                pos >= 0 ? features_row(ix, e, uq, sc, cc, ac, qres_n, qn2,
                                                        a.hv_feat + pos * (ix.r + 4))
                                         : edge_cos(ix, e, uq);
                            tr[s] = fmaf(th, ix.alpha, ix.beta);
                        }
                    }
                }
            }
            // FP32 FINGER: t_hat of every new neighbour by one balanced gather.
            // The new neighbours are compacted and lpr lanes share an edge row
            // (lpr = r/4 rounded up to a power of two, at most 16), so one
            // 16-byte load per lane covers 32 / lpr rows and eight loads per
            // lane are in flight at once; the row sums come from a
            // transpose-reduce over the row's lanes (a butterfly for lpr = 4).
            constexpr bool BAL = MODE == FINGER_MODE_FINGER || MLP;
            constexpr int GS = 8;
            float2 scv[NPL];
            if constexpr (BAL) {
                if (use_est) {
                    int nn = 0;
#pragma unroll
                    for (int s = 0; s < NPL; ++s) {
                        const int o = s * 32 + lane;
                        scv[s] = isnew[s] ? __ldg(ix.edge_s + (size_t)c * ix.deg0 + o)
                                          : make_float2(0.f, 0.f);
                        const unsigned bm = __ballot_sync(FULLMASK, isnew[s]);
                        if (isnew[s]) lst[nn + __popc(bm & ltmask)] = o;
                        nn += __popc(bm);
                    }
                    __syncwarp();
                    const int llpr = ix.r4 <= 4 ? 2 : ix.r4 <= 8 ? 3 : 4;
                    const int lpr = 1 << llpr, rps = 32 >> llpr;
                    const int sub = lane >> llpr, k4 = lane & (lpr - 1);
                    const float4 y = k4 < ix.r4 ? reinterpret_cast<const float4*>(uq)[k4]
                                                : make_float4(0.f, 0.f, 0.f, 0.f);
                    const float4* eb = ix.edge_u + (size_t)c * ix.deg0 * ix.r4;
                    for (int base = 0; base < nn; base += GS * rps) {
                        float4 x[GS];
#pragma unroll
                        for (int g = 0; g < GS; ++g) {
                            const int i = base + g * rps + sub;
                            x[g] = (i < nn && k4 < ix.r4)
                                       ? __ldg(eb + (size_t)lst[CK(i, 32 * NPL, 1021)] * ix.r4 + k4)
                                       : make_float4(0.f, 0.f, 0.f, 0.f);
                        }
                        float pg[GS];
#pragma unroll
                        for (int g = 0; g < GS; ++g) {
                            pg[g] = x[g].x * y.x;
                            pg[g] = fmaf(x[g].y, y.y, pg[g]);
                            pg[g] = fmaf(x[g].z, y.z, pg[g]);
                            pg[g] = fmaf(x[g].w, y.w, pg[g]);
                        }
                        if (lpr >= 8) {
                            // transpose-reduce over the row's lanes: each step hands the
                            // partner lane half of the remaining slots, so the eight
                            // sums take 8 shuffles instead of 8 x log2(lpr)
                            const bool hi8 = lpr == 16;
                            const int kb = hi8 ? k4 >> 1 : k4;   // slot this lane ends with
                            const int o0 = lpr >> 1;
                            float q4[4], q2[2];
#pragma unroll
                            for (int j = 0; j < 4; ++j) {
                                const bool b = kb & 4;
                                const float sd = b ? pg[j] : pg[j + 4];
                                q4[j] = (b ? pg[j + 4] : pg[j]) + __shfl_xor_sync(FULLMASK, sd, o0);
                            }
#pragma unroll
                            for (int j = 0; j < 2; ++j) {
                                const bool b = kb & 2;
                                const float sd = b ? q4[j] : q4[j + 2];
                                q2[j] = (b ? q4[j + 2] : q4[j]) + __shfl_xor_sync(FULLMASK, sd, o0 >> 1);
                            }
                            const bool b1 = kb & 1;
                            float t = (b1 ? q2[1] : q2[0]) +
                                      __shfl_xor_sync(FULLMASK, b1 ? q2[0] : q2[1], o0 >> 2);
                            if (hi8) t += __shfl_xor_sync(FULLMASK, t, 1);
                            const int i = base + kb * rps + sub;
                            if ((!hi8 || !(k4 & 1)) && i < nn) xb[lst[CK(i, 32 * NPL, 1022)]] = t;
                        } else {
#pragma unroll
                            for (int g = 0; g < GS; ++g) {
                                float p = pg[g];
                                for (int o = lpr >> 1; o > 0; o >>= 1) p += __shfl_xor_sync(FULLMASK, p, o);
                                const int i = base + g * rps + sub;
                                if (k4 == 0 && i < nn) xb[lst[CK(i, 32 * NPL, 1022)]] = p;
                            }
                        }
                    }
                    __syncwarp();
                }
            }
            if constexpr (MLP) {
                // learned predictor (an extension): the matched estimate of every
                // new slot from the gather above; a slot whose matched estimate lies
                // within the margin mlp_delta * ub of the ub at the expansion start
                // (every slot when mlp_delta < 0) gets the predictor.  Its feature
                // rows go through the network 16 at a time (one m16 tile per
                // round); outputs land in `ak` (free until the admission replay)
                // at the slot's compact row.
                if (use_est) {
                    int nunc = 0;
#pragma unroll
                    for (int s = 0; s < NPL; ++s) {
                        bool unc = false;
                        if (isnew[s]) {
                            tr[s] = fmaf(xb[s * 32 + lane], ix.alpha, ix.beta);
                            const float dd = ac - scv[s].y;
                            const float est_m = dd * dd * cc + qres2 + scv[s].x * scv[s].x -
                                                2.f * qres_n * scv[s].x * tr[s];
                            unc = ix.mlp_delta < 0.f ||
                                  (full0 && fabsf(est_m - ub0) <= ix.mlp_delta * ub0);
                        }
                        const unsigned bm = __ballot_sync(FULLMASK, unc);
                        if (unc) crow[s] = nunc + __popc(bm & ltmask);
                        nunc += __popc(bm);
                    }
                    uint32_t* xw = reinterpret_cast<uint32_t*>(xt);
                    const int xs = ix.mlp_kp + MLP_PAD;
                    const int wpr = xs >> 1;
                    for (int base = 0; base < nunc; base += 16) {
#pragma unroll
                        for (int s = 0; s < NPL; ++s) {
                            if (crow[s] >= base && crow[s] < base + 16) {
                                const size_t e = (size_t)c * ix.deg0 + s * 32 + lane;
                                features_tile(ix, e, uq, scv[s], cc, ac, qres_n, qn2,
                                              xt + (size_t)(crow[s] - base) * xs);
                            }
                        }
                        const int rows = min(16, nunc - base);
                        for (int i = rows * wpr + lane; i < 16 * wpr; i += 32) xw[i] = 0u;
                        __syncwarp();
                        mlp_tile(xt, ix.mlp_kp, ix.W1f, ix.W2f, ix.b1, ix.b2, ix.w3, ix.b3,
                                 ak + base, lane);
                        __syncwarp();
                    }
                }
            }
            int nl = 0;
            bool needr[NPL];
#pragma unroll
            for (int s = 0; s < NPL; ++s) {
                float est = -INFINITY;
                if (use_est && isnew[s]) {
                    const size_t e = (size_t)c * ix.deg0 + s * 32 + lane;
                    const float2 sc = BAL ? scv[s] : WB ? scw[s] : __ldg(ix.edge_s + e);
                    float t;
                    if constexpr (MLP) {
                        // the predictor's cosine where it ran (the matched cosine is
                        // the fallback for a non-finite output), else the matched one
                        t = tr[s];
                        if (crow[s] >= 0) {
                            const float y = ak[crow[s]];
                            if (isfinite(y)) t = y + ix.mlp_eps;
                        }
                    } else if constexpr (BAL) {
                        t = fmaf(xb[s * 32 + lane], ix.alpha, ix.beta);
                    } else if constexpr (WB) {
                        t = fmaf(th[s], ix.alpha, ix.beta);
                    } else if constexpr (HARV) {
                        t = tr[s];
                    } else {
                        t = fmaf(edge_cos(ix, e, uq), ix.alpha, ix.beta);
                    }
                    const float dd = ac - sc.y;
                    est = dd * dd * cc + qres2 + sc.x * sc.x - 2.f * qres_n * sc.x * t;
                }
                if (DEFER) {
                    // resolve the deferred bitmap test-and-set of this slot
                    if (pend[s]) isnew[s] = !(pold[s] & (1u << (nb[s] & 31)));
                    const bool sp = pend[s] && isnew[s];
                    const unsigned sb = __ballot_sync(FULLMASK, sp);
                    if (sp) spl[CK(nspill + __popc(sb & ltmask), a.spill_cap, 1005)] = nb[s];
                    nspill += __popc(sb);
                }
                bool need = isnew[s] && (!use_est || !full0 || !(est > ub0));
                if (HARV && hpos[s] >= 0) need = true;   // the record needs the exact distance
                needr[s] = need;
                if (need) prefetch_row<LP>(ix, nb[s]);
                es[s * 32 + lane] = est;
                const unsigned bm = __ballot_sync(FULLMASK, need);
                if (need) lst[CK(nl + __popc(bm & ltmask), 32 * NPL, 1017)] = s * 32 + lane;
                nl += __popc(bm);
            }
            __syncwarp();
            // a6: exact distances of the survivors
            exact_list<LP, G, VPL, WB>(q, qs, ix, nbs, lst, nl, xb, lane, IDM);
            c_gath += nl;
            if constexpr (HARV) {
                // target cos(q_res, d_res) = (q^T d - a b ||c||^2) / (||q_res|| ||d_res||),
                // q^T d from the exact distance, ||d||^2 = b^2 ||c||^2 + ||d_res||^2
#pragma unroll
                for (int s = 0; s < NPL; ++s) {
                    if (hpos[s] < 0) continue;
                    const int o = s * 32 + lane;
                    const float2 sc = __ldg(ix.edge_s + (size_t)c * ix.deg0 + o);
                    const float dn2 = sc.y * sc.y * cc + sc.x * sc.x;
                    const float qd = 0.5f * (qn2 + dn2 - xb[o]);
                    const float den = qres_n * sc.x;
                    a.hv_target[hpos[s]] = den > 0.f ? (qd - ac * sc.y * cc) / den : 0.f;
                    int32_t* tp = a.hv_trip + hpos[s] * 3;
                    tp[0] = qi;
                    tp[1] = (int32_t)c;
                    tp[2] = (int32_t)nb[s];
                }
            }

            // New neighbours met while T is below ef are admitted with no gate:
            // the first ef - |T| of them in slot order are rank-sorted into
            // ak / ai and merged at once.  The rest, met once T is full (all of
            // them when it was full at the start), go through the gate replay.
            bool gate[NPL];
            bool replay = full0;
#pragma unroll
            for (int s = 0; s < NPL; ++s) gate[s] = isnew[s];
            if (!full0) {
                unsigned bnew[NPL], bfill[NPL];
                int nnew = 0;
#pragma unroll
                for (int s = 0; s < NPL; ++s) {
                    bnew[s] = __ballot_sync(FULLMASK, isnew[s]);
                    nnew += __popc(bnew[s]);
                }
                const int f = min(nnew, ef - sz);
                bool fill[NPL];
                int before = 0;
#pragma unroll
                for (int s = 0; s < NPL; ++s) {
                    const int idx = before + __popc(bnew[s] & ltmask);
                    fill[s] = isnew[s] && idx < f;
                    gate[s] = isnew[s] && idx >= f;
                    bfill[s] = __ballot_sync(FULLMASK, fill[s]);
                    before += __popc(bnew[s]);
                }
#pragma unroll
                for (int s = 0; s < NPL; ++s) {
                    const float md = xb[s * 32 + lane];
                    const uint32_t mi = nb[s];
                    int rk = 0;
#pragma unroll
                    for (int s2 = 0; s2 < NPL; ++s2) {
                        unsigned bits = bfill[s2];
                        while (bits) {
                            const int j = __ffs(bits) - 1;
                            bits &= bits - 1;
                            const int o = s2 * 32 + j;
                            rk += key_lt(xb[o], nbs[o] & IDM, md, mi);
                        }
                    }
                    if (fill[s]) {
                        ak[rk] = md;
                        ai[rk] = nbt[s];   // as stored in T
                    }
                }
                __syncwarp();
                c_exa += f;
                c_exact += f;
                c_adm += f;
                if (f > 0) t_merge<NPL>(Tk, Ti, sz, ak, ai, f, ef, IDM, cursor, lane);
                sz += f;
                replay = nnew > f;   // T is full now and new neighbours remain
            }
            if (replay) {
                // T is full and stays full.  Only neighbours evaluated exactly and
                // below the starting ub can be admitted; replay the sequential gate
                // over them with a running model of ub (top-ef of T and the admitted
                // set A), then merge A into T once.
                const float u0d = Tk[ef - 1];
                const uint32_t u0i = Ti[ef - 1] & IDM;
                unsigned cb[NPL], cskip[NPL];
                float xd[NPL];     // exact distance of each slot
                float estv[NPL];   // estimate of each slot (read back: no register across the gathers)
                int ncand = 0;
#pragma unroll
                for (int s = 0; s < NPL; ++s) {
                    const int o = s * 32 + lane;
                    xd[s] = xb[o];
                    estv[s] = es[o];
                    const bool cand = gate[s] && needr[s] && key_lt(xd[s], nb[s], u0d, u0i);
                    cb[s] = __ballot_sync(FULLMASK, cand);
                    cskip[s] = 0u;
                    ncand += __popc(cb[s]);
                }
                int tk, na, nadm;
                float myub[NPL];   // the running ub (distance) when the scan reaches each slot
                if (ncand == 0) {
                    tk = ef;
                    na = 0;
                    nadm = 0;
#pragma unroll
                    for (int t = 0; t < NPL; ++t) myub[t] = u0d;
                } else if (ncand == 1) {
                    // The first candidate in slot order is always admitted (its
                    // estimate and key are below the starting ub); it pushes out
                    // T's last entry, and ub becomes the larger of it and T[ef - 2].
                    int s1 = 0;
#pragma unroll
                    for (int s = NPL - 1; s >= 0; --s)
                        if (cb[s]) s1 = s;
                    float xs = xd[0];
                    uint32_t ns = nbt[0];
                    unsigned bs = cb[0];
#pragma unroll
                    for (int s = 1; s < NPL; ++s)
                        if (s == s1) {
                            xs = xd[s];
                            ns = nbt[s];
                            bs = cb[s];
                        }
                    const int jj = __ffs(bs) - 1;
                    const int o1 = s1 * 32 + jj;
                    const float cd = __shfl_sync(FULLMASK, xs, jj);
                    const uint32_t craw2 = __shfl_sync(FULLMASK, ns, jj);   // as stored in T
                    float ubd = cd;
                    uint32_t ubi = craw2 & IDM;
                    if (ef >= 2) {
                        const float td = Tk[ef - 2];
                        const uint32_t ti = Ti[ef - 2] & IDM;
                        if (key_lt(ubd, ubi, td, ti)) {
                            ubd = td;
                            ubi = ti;
                        }
                    }
#pragma unroll
                    for (int t = 0; t < NPL; ++t) myub[t] = t * 32 + lane <= o1 ? u0d : ubd;
                    tk = ef - 1;
                    na = 1;
                    nadm = 1;
                    if (lane == 0) {
                        ak[0] = cd;
                        ai[0] = craw2;
                    }
                    __syncwarp();
                } else if (ncand < 32) {
                    // Warp-parallel replay.  After j admissions the top ef is the
                    // ef smallest keys of T and the admitted set A, so ub is the
                    // (j+1)-th largest key of T's tail and A: lane p holds the
                    // p-th largest of them (the pool, 32 deep, enough for j < 32),
                    // lane j the j-th admission (the log).  Candidates are taken
                    // in slot order as the sequential scan meets them.
                    float pd = lane < ef ? Tk[ef - 1 - lane] : -1.f;   // -1: below any distance
                    uint32_t pi = lane < ef ? Ti[ef - 1 - lane] & IDM : 0u;
                    float ld = 0.f;
                    uint32_t li = 0u;
                    float ubd = u0d;
                    uint32_t ubi = u0i;
                    int j = 0, prev = -1;
#pragma unroll
                    for (int s = 0; s < NPL; ++s) {
                        unsigned bits = cb[s];
                        unsigned skm = 0u;
                        while (bits) {
                            const int jj = __ffs(bits) - 1;
                            bits &= bits - 1;
                            const int o = s * 32 + jj;
#pragma unroll
                            for (int t = 0; t < NPL; ++t) {
                                const int so = t * 32 + lane;
                                if (so > prev && so <= o) myub[t] = ubd;
                            }
                            prev = o;
                            const float ce = __shfl_sync(FULLMASK, estv[s], jj);
                            const float cd = __shfl_sync(FULLMASK, xd[s], jj);
                            const uint32_t craw2 = __shfl_sync(FULLMASK, nbt[s], jj);   // as stored in T
                            const uint32_t cid = craw2 & IDM;
                            if (use_est && ce > ubd) {
                                skm |= 1u << jj;
                                continue;
                            }
                            if (!key_lt(cd, cid, ubd, ubi)) continue;
                            // admit: log it, insert it into the descending pool
                            if (lane == j) {
                                ld = cd;
                                li = craw2;
                            }
                            const int pos = __popc(__ballot_sync(FULLMASK, key_lt(cd, cid, pd, pi)));
                            const float sd = __shfl_up_sync(FULLMASK, pd, 1);
                            const uint32_t si = __shfl_up_sync(FULLMASK, pi, 1);
                            if (lane > pos) {
                                pd = sd;
                                pi = si;
                            } else if (lane == pos) {
                                pd = cd;
                                pi = cid;
                            }
                            ++j;
                            ubd = __shfl_sync(FULLMASK, pd, j);
                            ubi = __shfl_sync(FULLMASK, pi, j);
                        }
                        cskip[s] = skm;
                    }
#pragma unroll
                    for (int t = 0; t < NPL; ++t)
                        if (t * 32 + lane > prev) myub[t] = ubd;
                    nadm = j;
                    // the j largest keys left the top ef; an admitted key stays iff
                    // it is below the smallest of them, pool[j - 1]
                    const float thd = __shfl_sync(FULLMASK, pd, j > 0 ? j - 1 : 0);
                    const uint32_t thi = __shfl_sync(FULLMASK, pi, j > 0 ? j - 1 : 0);
                    const bool kept = lane < j && key_lt(ld, li & IDM, thd, thi);
                    const unsigned bk = __ballot_sync(FULLMASK, kept);
                    na = __popc(bk);
                    tk = ef - na;
                    // the kept admissions, ascending, into ak / ai for the merge
                    int rk = 0;
                    for (int t = 0; t < j; ++t) {
                        const float od = __shfl_sync(FULLMASK, ld, t);
                        const uint32_t oi = __shfl_sync(FULLMASK, li, t);
                        rk += ((bk >> t) & 1u) && key_lt(od, oi & IDM, ld, li & IDM);
                    }
                    if (kept) {
                        ak[rk] = ld;
                        ai[rk] = li;
                    }
                    __syncwarp();
                } else {
                    // 32 or more candidates: the serial replay on lane 0, results
                    // through shared memory
                    if (lane == 0) {
                        float ubd = u0d;
                        uint32_t ubi = u0i;
                        int tk = ef, na = 0, nadm = 0;
#pragma unroll
                        for (int s = 0; s < NPL; ++s) {
                            unsigned bits = cb[s];
                            unsigned skm = 0u;
                            while (bits) {
                                const int j = __ffs(bits) - 1;
                                bits &= bits - 1;
                                const int o = s * 32 + j;
                                if (use_est && es[o] > ubd) {
                                    skm |= 1u << j;
                                    continue;
                                }
                                const float d = xb[CK(o, 32 * NPL, 1008)];
                                const uint32_t idt = nbs[o];   // as stored in T
                                const uint32_t id = idt & IDM;
                                if (!key_lt(d, id, ubd, ubi)) continue;
                                // the current worst of the top ef leaves it
                                if (tk == 0 ||
                                    (na > 0 && key_lt(Tk[CK(tk - 1, ef, 1009)], Ti[tk - 1] & IDM,
                                                      ak[CK(na - 1, 32 * NPL, 1010)], ai[na - 1] & IDM)))
                                    na--;
                                else
                                    tk--;
                                // insert (d, id) into the sorted admitted list
                                int p = na;
                                while (p > 0 && key_lt(d, id, ak[p - 1], ai[p - 1] & IDM)) {
                                    ak[CK(p, 32 * NPL, 1011)] = ak[p - 1];
                                    ai[p] = ai[p - 1];
                                    --p;
                                }
                                ak[CK(p, 32 * NPL, 1012)] = d;
                                ai[p] = idt;
                                na++;
                                // new ub: the larger of T[tk-1] and max(A)
                                ubd = ak[na - 1];
                                ubi = ai[na - 1] & IDM;
                                if (tk > 0 && key_lt(ubd, ubi, Tk[tk - 1], Ti[tk - 1] & IDM)) {
                                    ubd = Tk[tk - 1];
                                    ubi = Ti[tk - 1] & IDM;
                                }
                                apos[CK(nadm, 32 * NPL, 1013)] = o;
                                aub[nadm] = ubd;
                                nadm++;
                            }
                            meta[3 + s] = (int)skm;
                        }
                        meta[0] = tk;
                        meta[1] = na;
                        meta[2] = nadm;
                    }
                    __syncwarp();
                    tk = meta[0];
                    na = meta[1];
                    nadm = meta[2];
#pragma unroll
                    for (int s = 0; s < NPL; ++s) {
                        cskip[s] = (unsigned)meta[3 + s];
                        const int o = s * 32 + lane;
                        float ubt = u0d;
                        for (int k = 0; k < nadm; ++k)
                            if (apos[k] < o) ubt = aub[k];
                        myub[s] = ubt;
                    }
                }
                // counters of every new neighbour under the sequential semantics
#pragma unroll
                for (int s = 0; s < NPL; ++s) {
                    bool skipped = false;
                    if (gate[s]) {
                        if ((cb[s] >> lane) & 1u) skipped = (cskip[s] >> lane) & 1u;
                        else if (use_est) skipped = estv[s] > myub[s];
                    }
                    const int nnew = __popc(__ballot_sync(FULLMASK, gate[s]));
                    const int nsk = __popc(__ballot_sync(FULLMASK, skipped));
                    c_exa += nnew;
                    if (use_est) c_est += nnew;
                    c_skip += nsk;
                    c_exact += nnew - nsk;
                }
                c_adm += nadm;
                // merge A (sorted, na entries) into T[0..tk) -> T[0..ef)
                if (na > 0) t_merge<NPL>(Tk, Ti, tk, ak, ai, na, ef, IDM, cursor, lane);
            }
            __syncwarp();
        }
        c_exp = expansions;

        // ---- LP: re-rank the head of T with FP32 rows
        if constexpr (LP) {
            const int R = min(sz, max(K, a.rerank));
            float* rk = reinterpret_cast<float*>(hash);
            uint32_t* ri = hash + a.ef_cap;   // the plan keeps 2 ef_cap words in the table
            for (int i = 0; i < R; ++i) {
                const float d = exact_f32_row(qs, ix, Ti[i] & IDM, lane);
                if (lane == 0) Tk[i] = d;
            }
            __syncwarp();
            for (int i = lane; i < R; i += 32) {
                const float d = Tk[i];
                const uint32_t id = Ti[i] & IDM;
                int rank = 0;
                for (int j = 0; j < R; ++j) rank += key_lt(Tk[j], Ti[j] & IDM, d, id);
                rk[rank] = d;
                ri[rank] = id;
            }
            __syncwarp();
            for (int i = lane; i < R; i += 32) {
                Tk[i] = rk[i];
                Ti[i] = ri[i];
            }
            __syncwarp();
        }

        // ---- a7: output
        for (int k = lane; k < K; k += 32) {
            a.out_ids[ooff + k] = k < sz ? (int64_t)(Ti[k] & IDM) : (int64_t)-1;
            a.out_d[ooff + k] = k < sz ? Tk[k] : INFINITY;
        }
        for (int i = lane; i < nspill; i += 32) bitmap[spl[i] >> 5] = 0u;
        if (lane == 0) {
            if (fail) atomicOr(a.err, (int)FINGER_ERR_LIMIT);
            unsigned long long* g = a.cnt;
            atomicAdd(g + 0, (unsigned long long)c_exp);
            atomicAdd(g + 1, (unsigned long long)c_exa);
            atomicAdd(g + 2, (unsigned long long)c_est);
            atomicAdd(g + 3, (unsigned long long)c_skip);
            atomicAdd(g + 4, (unsigned long long)c_exact);
            atomicAdd(g + 5, (unsigned long long)c_adm);
            atomicAdd(g + 6, (unsigned long long)c_up);
            atomicAdd(g + 7, (unsigned long long)c_gath);
            if (WB) atomicAdd(g + 8, (unsigned long long)c_half * HALF_BYTES);
            if (a.cnt_q) {
                int32_t* cq = a.cnt_q + (size_t)qi * 8;
                cq[0] = c_exp;
                cq[1] = c_exa;
                cq[2] = c_est;
                cq[3] = c_skip;
                cq[4] = c_exact;
                cq[5] = c_adm;
                cq[6] = c_up;
                cq[7] = c_gath;
            }
        }
        __syncwarp();
    }
}

// instantiate and dispatch one mode over the (G, VPL, NPL) variants and the
// resident-block target: 5 blocks of 4 warps (96 registers) everywhere, 6 (80
// registers) for the plain, FINGER, LP and FP16/FP8-code modes, 8 (64 registers)
// for the plain mode.  The FINGER modes keep their gathers in flight in
// registers and are fastest at 6 (the FP16-code mode measured slower at 7,
// where it spills); plain search at 8.
#define LP_MODE(m) ((m) == MODE_LP_K2 || (m) == MODE_LP_K4 || (m) == MODE_F8_K2 || (m) == MODE_F8_K4)

template <int MODE, int OCC>
cudaError_t launch_occ(const DevIndex& ix, const SearchArgs& a, const SearchPlan& p,
                       cudaStream_t s) {
    const int smem = p.blk_smem + p.smem_per_warp * p.wpb;
    const dim3 grid(p.blocks), block(p.wpb * 32);
#define FG_CASE(G_, V_, N_)                                                                    \
    if (p.G == G_ && p.VPL == V_ && p.NPL == N_) {                                           \
        auto k = k_search<MODE, G_, V_, N_, OCC>;                                              \
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem); \
        if (e != cudaSuccess) return e;                                                       \
        k<<<grid, block, smem, s>>>(ix, a);                                                   \
        return cudaGetLastError();                                                            \
    }
#define FG_NPL(N_)                                                                             \
    FG_CASE(8, 1, N_) FG_CASE(16, 1, N_) FG_CASE(16, 2, N_) FG_CASE(32, 1, N_) FG_CASE(32, 2, N_)               \
    FG_CASE(32, 4, N_) FG_CASE(32, 8, N_)
    FG_NPL(1)
    FG_NPL(2)
#undef FG_NPL
#undef FG_CASE
    return cudaErrorInvalidValue;
}

template <int MODE, int OCC>
cudaError_t occupancy_occ(const SearchPlan& p, int* blocks) {
    const int smem = p.blk_smem + p.smem_per_warp * p.wpb;
#define FG_CASE(G_, V_, N_)                                                                    \
    if (p.G == G_ && p.VPL == V_ && p.NPL == N_) {                                           \
        auto k = k_search<MODE, G_, V_, N_, OCC>;                                              \
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem); \
        if (e != cudaSuccess) return e;                                                       \
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, k, p.wpb * 32, smem);     \
    }
#define FG_NPL(N_)                                                                             \
    FG_CASE(8, 1, N_) FG_CASE(16, 1, N_) FG_CASE(16, 2, N_) FG_CASE(32, 1, N_) FG_CASE(32, 2, N_)               \
    FG_CASE(32, 4, N_) FG_CASE(32, 8, N_)
    FG_NPL(1)
    FG_NPL(2)
#undef FG_NPL
#undef FG_CASE
    return cudaErrorInvalidValue;
}

#define F8_MODE(m) ((m) == MODE_F8_K2 || (m) == MODE_F8_K4)

template <int MODE>
cudaError_t launch_mode(const DevIndex& ix, const SearchArgs& a, const SearchPlan& p,
                        cudaStream_t s) {
    if constexpr (MODE == FINGER_MODE_PLAIN || F8_MODE(MODE))
        if (p.occ == 8) return launch_occ<MODE, 8>(ix, a, p, s);
    if constexpr (MODE == FINGER_MODE_PLAIN || MODE == FINGER_MODE_FINGER ||
                  LP_MODE(MODE) || MODE == MODE_F16_K2 || MODE == MODE_F16_K4)
        if (p.occ == 6) return launch_occ<MODE, 6>(ix, a, p, s);
    if (p.occ != 5) return cudaErrorInvalidValue;
    return launch_occ<MODE, 5>(ix, a, p, s);
}

// resident blocks per SM of the variant the plan names; 0 for a variant the
// mode does not have
template <int MODE>
cudaError_t occupancy_mode(const SearchPlan& p, int* blocks) {
    if constexpr (MODE == FINGER_MODE_PLAIN || F8_MODE(MODE))
        if (p.occ == 8) return occupancy_occ<MODE, 8>(p, blocks);
    if constexpr (MODE == FINGER_MODE_PLAIN || MODE == FINGER_MODE_FINGER ||
                  LP_MODE(MODE) || MODE == MODE_F16_K2 || MODE == MODE_F16_K4)
        if (p.occ == 6) return occupancy_occ<MODE, 6>(p, blocks);
    if (p.occ != 5) {
        *blocks = 0;
        return cudaSuccess;
    }
    return occupancy_occ<MODE, 5>(p, blocks);
}

}  // namespace fg

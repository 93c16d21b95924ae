// Index files and uneven-batch search (C ABI, see include/finger.h).
//
// File layout (little endian): a 128-byte header
//   magic "FINGERIX", u32 version, u32 flags (1 = graph, 2 = tables, 4 = LP, 8 = MLP,
//   16 = FP16 codes, 32 = FP8 codes without the LP rows),
//   i64 n, i32 m, i32 deg0, i32 M, i32 maxlevel, i32 entry, i32 r, i64 up_rows,
//   f64 stats[5], u64 checksum of the payload, zero padding
// followed by the sections, each written only when its flag is set:
//   vectors n*m f32 | level n i32, up_off n i64, adj0 n*deg0 i32, up_adj up_rows*M i32 |
//   P r*m f32, node_proj n*r f32, edge_u (n*deg0)*r f32, edge_s (n*deg0)*2 f32 |
//   mlp master weights (f32, count u64 first) and mlp_eps.
// The LP tables and the FP16 / FP8 codes are rebuilt from the FP32 tables on load.
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "internal.cuh"

using namespace fg;

finger_status finger_load_mlp_internal(finger_index* ix, const float* w, int64_t count, float eps);
cudaError_t lp_rebuild(finger_index* ix);
cudaError_t half_rebuild(finger_index* ix);
cudaError_t fp8_rebuild(finger_index* ix);

namespace {

constexpr uint32_t VERSION = 1;

struct Header {
    char magic[8];
    uint32_t version, flags;
    int64_t n;
    int32_t m, deg0, M, maxlevel, entry, r;
    int64_t up_rows;
    double stats[5];
    uint64_t checksum;
};
static_assert(sizeof(Header) <= 128, "header size");

struct Sum {
    uint64_t s = 0x243F6A8885A308D3ULL;
    void add(const void* p, size_t bytes) {
        const unsigned char* c = static_cast<const unsigned char*>(p);
        size_t i = 0;
        for (; i + 8 <= bytes; i += 8) {
            uint64_t v;
            memcpy(&v, c + i, 8);
            s = (s ^ v) * 0x100000001B3ULL + (s >> 31);
        }
        for (; i < bytes; ++i) s = (s ^ c[i]) * 0x100000001B3ULL;
    }
};

struct Writer {
    FILE* f;
    Sum sum;
    bool ok = true;
    void put(const void* p, size_t bytes) {
        if (!ok) return;
        sum.add(p, bytes);
        ok = fwrite(p, 1, bytes, f) == bytes;
    }
};

struct Reader {
    FILE* f;
    Sum sum;
    bool ok = true;
    void get(void* p, size_t bytes) {
        if (!ok) return;
        ok = fread(p, 1, bytes, f) == bytes;
        if (ok) sum.add(p, bytes);
    }
};

template <class T>
std::vector<T> d2h_rows(const void* d, int64_t rows, int width, int pitch) {
    std::vector<T> h((size_t)rows * width);
    if (rows > 0 && width > 0)
        cudaMemcpy2D(h.data(), sizeof(T) * width, d, sizeof(T) * pitch, sizeof(T) * width, rows,
                     cudaMemcpyDeviceToHost);
    return h;
}

}  // namespace

extern "C" {

finger_status finger_index_save(const finger_index* ix, const char* path) {
    if (!ix || !path) return FINGER_ERR_INVALID_ARG;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(ix->device);
    FILE* f = fopen(path, "wb");
    if (!f) {
        cudaSetDevice(prev);
        return FINGER_ERR_IO;
    }
    Header h{};
    memcpy(h.magic, "FINGERIX", 8);
    h.version = VERSION;
    h.flags = (ix->adj0 ? 1u : 0u) | (ix->edge_u ? 2u : 0u) | (ix->Xh && ix->edge_q ? 4u : 0u) |
              (ix->has_mlp ? 8u : 0u) | (ix->edge_h ? 16u : 0u) |
              (!ix->Xh && ix->edge_q ? 32u : 0u);
    h.n = ix->n;
    h.m = ix->m;
    h.deg0 = ix->deg0;
    h.M = ix->M;
    h.maxlevel = ix->maxlevel;
    h.entry = ix->entry;
    h.r = ix->r;
    h.up_rows = ix->up_rows;
    for (int i = 0; i < 5; ++i) h.stats[i] = ix->stats[i];
    unsigned char pad[128] = {0};
    fwrite(pad, 1, 128, f);   // placeholder, rewritten with the checksum
    Writer w{f};
    const int64_t chunk = 1 << 16;
    for (int64_t r0 = 0; r0 < ix->n && w.ok; r0 += chunk) {
        const int64_t rows = std::min(chunk, ix->n - r0);
        auto v = d2h_rows<float>(ix->X + r0 * ix->m_pad, rows, ix->m, ix->m_pad);
        w.put(v.data(), v.size() * 4);
    }
    if (h.flags & 1u) {
        w.put(ix->h_level.data(), sizeof(int32_t) * ix->n);
        auto uo = d2h_rows<int64_t>(ix->up_off, 1, (int)ix->n, (int)ix->n);
        w.put(uo.data(), uo.size() * 8);
        auto a0 = d2h_rows<int32_t>(ix->adj0, ix->n, ix->deg0, ix->deg0);
        w.put(a0.data(), a0.size() * 4);
        if (ix->up_rows > 0) {
            auto ua = d2h_rows<int32_t>(ix->up_adj, ix->up_rows, ix->M, ix->M);
            w.put(ua.data(), ua.size() * 4);
        }
    }
    if (h.flags & 2u) {
        auto P = d2h_rows<float>(ix->P, ix->r, ix->m, ix->m_pad);
        w.put(P.data(), P.size() * 4);
        auto Pc = d2h_rows<float>(ix->Pc, ix->n, ix->r, ix->r_pad);
        w.put(Pc.data(), Pc.size() * 4);
        const int64_t ne = ix->n * ix->deg0;
        for (int64_t e0 = 0; e0 < ne && w.ok; e0 += chunk * 16) {
            const int64_t rows = std::min(chunk * 16, ne - e0);
            auto u = d2h_rows<float>(ix->edge_u + e0 * ix->r_pad, rows, ix->r, ix->r_pad);
            w.put(u.data(), u.size() * 4);
        }
        auto es = d2h_rows<float>(ix->edge_s, ne, 2, 2);
        w.put(es.data(), es.size() * 4);
    }
    if (h.flags & 8u) {
        const uint64_t cnt = ix->h_mlp.size();
        w.put(&cnt, 8);
        w.put(ix->h_mlp.data(), cnt * 4);
        w.put(&ix->mlp_eps, 4);
    }
    h.checksum = w.sum.s;
    bool ok = w.ok && cudaGetLastError() == cudaSuccess;
    if (ok) {
        fseek(f, 0, SEEK_SET);
        memcpy(pad, &h, sizeof(h));
        ok = fwrite(pad, 1, 128, f) == 128;
    }
    ok = (fclose(f) == 0) && ok;
    cudaSetDevice(prev);
    return ok ? FINGER_OK : FINGER_ERR_IO;
}

finger_status finger_index_load(const char* path, int device, finger_index** out) {
    if (!path || !out) return FINGER_ERR_INVALID_ARG;
    *out = nullptr;
    FILE* f = fopen(path, "rb");
    if (!f) return FINGER_ERR_IO;
    unsigned char buf[128];
    Header h{};
    if (fread(buf, 1, 128, f) != 128) {
        fclose(f);
        return FINGER_ERR_FORMAT;
    }
    memcpy(&h, buf, sizeof(h));
    if (memcmp(h.magic, "FINGERIX", 8) != 0 || h.version != VERSION || h.n < 1 || h.m < 1 ||
        h.m > MAX_M || h.deg0 < 0 || h.deg0 > MAX_DEG0 || h.M < 0 || h.M > MAX_MUP ||
        h.r < 0 || h.r > MAX_R || h.up_rows < 0 || h.entry < 0 || h.entry >= h.n) {
        fclose(f);
        return FINGER_ERR_FORMAT;
    }
    Reader rd{f};
    std::vector<float> X((size_t)h.n * h.m);
    rd.get(X.data(), X.size() * 4);
    std::vector<int32_t> level, adj0, up_adj;
    std::vector<int64_t> up_off;
    std::vector<float> P, Pc, eu, es, mlp;
    float mlp_eps = 0.f;
    if (h.flags & 1u) {
        level.resize(h.n);
        up_off.resize(h.n);
        adj0.resize((size_t)h.n * h.deg0);
        up_adj.resize((size_t)h.up_rows * h.M);
        rd.get(level.data(), level.size() * 4);
        rd.get(up_off.data(), up_off.size() * 8);
        rd.get(adj0.data(), adj0.size() * 4);
        if (h.up_rows > 0) rd.get(up_adj.data(), up_adj.size() * 4);
    }
    if (h.flags & 2u) {
        const int64_t ne = h.n * h.deg0;
        P.resize((size_t)h.r * h.m);
        Pc.resize((size_t)h.n * h.r);
        eu.resize((size_t)ne * h.r);
        es.resize((size_t)ne * 2);
        rd.get(P.data(), P.size() * 4);
        rd.get(Pc.data(), Pc.size() * 4);
        rd.get(eu.data(), eu.size() * 4);
        rd.get(es.data(), es.size() * 4);
    }
    if (h.flags & 8u) {
        uint64_t cnt = 0;
        rd.get(&cnt, 8);
        if (!rd.ok || cnt > (1u << 24)) {
            fclose(f);
            return FINGER_ERR_FORMAT;
        }
        mlp.resize(cnt);
        rd.get(mlp.data(), cnt * 4);
        rd.get(&mlp_eps, 4);
    }
    fclose(f);
    if (!rd.ok) return FINGER_ERR_FORMAT;
    if (rd.sum.s != h.checksum) return FINGER_ERR_FORMAT;
    finger_index* ix = nullptr;
    finger_status st = finger_index_create(device, h.n, h.m, X.data(), &ix);
    if (st != FINGER_OK) return st;
    if (h.flags & 1u) {
        st = finger_index_set_graph(ix, h.deg0, adj0.data(), level.data(), up_off.data(),
                                    h.up_rows, h.M, up_adj.data(), h.entry, h.maxlevel);
        if (st != FINGER_OK) {
            finger_index_free(ix);
            return st == FINGER_ERR_INVALID_ARG ? FINGER_ERR_FORMAT : st;
        }
    }
    if (h.flags & 2u) {
        int prev = 0;
        cudaGetDevice(&prev);
        cudaSetDevice(device);
        const int r = h.r, rp = (r + 3) & ~3;
        const int64_t ne = h.n * h.deg0;
        bool ok = cudaMalloc(&ix->P, sizeof(float) * rp * ix->m_pad) == cudaSuccess &&
                  cudaMalloc(&ix->Pc, sizeof(float) * h.n * rp) == cudaSuccess &&
                  cudaMalloc(&ix->edge_u, sizeof(float) * ne * rp) == cudaSuccess &&
                  cudaMalloc(&ix->edge_s, sizeof(float2) * ne) == cudaSuccess;
        ok = ok && cudaMemset(ix->P, 0, sizeof(float) * rp * ix->m_pad) == cudaSuccess &&
             cudaMemset(ix->Pc, 0, sizeof(float) * h.n * rp) == cudaSuccess &&
             cudaMemset(ix->edge_u, 0, sizeof(float) * ne * rp) == cudaSuccess;
        ok = ok &&
             cudaMemcpy2D(ix->P, sizeof(float) * ix->m_pad, P.data(), sizeof(float) * h.m,
                          sizeof(float) * h.m, r, cudaMemcpyHostToDevice) == cudaSuccess &&
             cudaMemcpy2D(ix->Pc, sizeof(float) * rp, Pc.data(), sizeof(float) * r,
                          sizeof(float) * r, h.n, cudaMemcpyHostToDevice) == cudaSuccess &&
             cudaMemcpy2D(ix->edge_u, sizeof(float) * rp, eu.data(), sizeof(float) * r,
                          sizeof(float) * r, ne, cudaMemcpyHostToDevice) == cudaSuccess &&
             cudaMemcpy(ix->edge_s, es.data(), sizeof(float) * 2 * ne, cudaMemcpyHostToDevice) ==
                 cudaSuccess;
        ix->r = r;
        ix->r_pad = rp;
        for (int i = 0; i < 5; ++i) ix->stats[i] = h.stats[i];
        if (ok && (h.flags & 4u)) ok = lp_rebuild(ix) == cudaSuccess;
        if (ok && (h.flags & 16u)) ok = half_rebuild(ix) == cudaSuccess;
        if (ok && (h.flags & 32u)) ok = fp8_rebuild(ix) == cudaSuccess;
        cudaSetDevice(prev);
        if (!ok) {
            cudaGetLastError();
            finger_index_free(ix);
            return FINGER_ERR_CUDA;
        }
    }
    if (h.flags & 8u) {
        st = finger_load_mlp_internal(ix, mlp.data(), (int64_t)mlp.size(), mlp_eps);
        if (st != FINGER_OK) {
            finger_index_free(ix);
            return st;
        }
    }
    *out = ix;
    return FINGER_OK;
}

}  // extern "C"

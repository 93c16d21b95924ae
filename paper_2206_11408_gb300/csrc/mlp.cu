// Learned angle predictor (an extension of FINGER; the paper has no learned
// predictor): training data harvest, training kernels and weight upload.
//
// The predictor maps the r + 4 features of a (q, c, d) triple (see
// features_row in search_impl.cuh) to cos(q_res, d_res) with a 64-64 ReLU MLP
// and replaces the distribution matching of Algorithm 3 in the MLP search mode.
// Weights are stored in BF16 (W1, W2, w3) with FP32 biases; training keeps FP32
// master weights and runs the forward pass exactly as inference does (BF16
// weights, hidden-layer inputs rounded to BF16, FP32 accumulation), with the
// roundings passed straight through in the backward pass.
//
// Kernels (one mini-batch of B rows per step):
//   k_quant     BF16-rounded copies of the master weights
//   k_fwd       thread per row: x~, h1~ = bf16(relu(W1 x~ + b1)), h2 = relu(W2 h1~ + b2),
//               y = w3 . h2 + b3, residual y - t
//   k_bwd       thread per row: dy = 2 (y - t) / B, dz2 = dy w3 [h2 > 0],
//               dz1 = W2^T dz2 [h1 > 0]
//   k_wgrad     thread per weight: sums of dz1 x~, dz2 h1~, dy h2 over the batch
//   k_adam      Adam on the FP32 masters
#include <math.h>
#include <string.h>

#include <algorithm>
#include <numeric>
#include <random>
#include <vector>

#include "internal.cuh"

using namespace fg;

finger_status fg_make_plan(finger_index* ix, int mode, int ef_max, int64_t nq, SearchPlan* p,
                           int wpb, int H, int occ = 0, int shape = 0);
finger_status fg_run_search(finger_index* ix, const SearchPlan& p, SearchArgs& a, cudaStream_t s);
SearchArgs fg_base_args(finger_index* ix, const SearchPlan& p);
void fg_drop_captures(const finger_index* ix);

namespace {

constexpr int HID = MLP_H;

__host__ __device__ inline int64_t wcount(int nf) { return (int64_t)HID * nf + HID + HID * HID + HID + HID + 1; }

struct Off {
    int64_t W1, b1, W2, b2, w3, b3;
    __host__ __device__ explicit Off(int nf) {
        W1 = 0;
        b1 = W1 + (int64_t)HID * nf;
        W2 = b1 + HID;
        b2 = W2 + HID * HID;
        w3 = b2 + HID;
        b3 = w3 + HID;
    }
};

__device__ __forceinline__ float bf(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

__global__ void k_quant(const float* w, int64_t n, int64_t b1, int64_t W2, int64_t b2, int64_t w3,
                        int64_t b3, float* q) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const bool is_bias = (i >= b1 && i < W2) || (i >= b2 && i < w3) || i == b3;
    q[i] = is_bias ? w[i] : bf(w[i]);
}

// forward: rows idx[0..B) of X (N x nf); stores x~ (B x nf), h1~ (B x H), h2 (B x H), res (B)
__global__ void k_fwd(const float* wq, int nf, const float* X, const float* T, const int64_t* idx,
                      int B, float* xs, float* h1s, float* h2s, float* res, float* y_out) {
    extern __shared__ float sw[];
    const Off o(nf);
    const int64_t nw = wcount(nf);
    for (int64_t i = threadIdx.x; i < nw; i += blockDim.x) sw[i] = wq[i];
    __syncthreads();
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const int64_t row = idx ? idx[b] : b;
    float x[96];
    for (int i = 0; i < nf; ++i) {
        x[i] = bf(X[row * nf + i]);
        if (xs) xs[(int64_t)b * nf + i] = x[i];
    }
    float z2[HID];
    for (int k = 0; k < HID; ++k) z2[k] = sw[o.b2 + k];
    for (int j = 0; j < HID; ++j) {
        float z = sw[o.b1 + j];
        for (int i = 0; i < nf; ++i) z = fmaf(sw[o.W1 + (int64_t)j * nf + i], x[i], z);
        const float h = bf(fmaxf(z, 0.f));
        if (h1s) h1s[(int64_t)b * HID + j] = h;
        for (int k = 0; k < HID; ++k) z2[k] = fmaf(sw[o.W2 + k * HID + j], h, z2[k]);
    }
    float y = sw[o.b3];
    for (int k = 0; k < HID; ++k) {
        const float h2 = fmaxf(z2[k], 0.f);
        if (h2s) h2s[(int64_t)b * HID + k] = h2;
        y = fmaf(sw[o.w3 + k], h2, y);
    }
    if (res) res[b] = y - (T ? T[row] : 0.f);
    if (y_out) y_out[b] = y;
}

__global__ void k_bwd(const float* wq, int nf, const float* h1s, const float* h2s, const float* res,
                      int B, float* dys, float* dz1s, float* dz2s) {
    extern __shared__ float sw[];
    const Off o(nf);
    for (int64_t i = threadIdx.x; i < HID * HID; i += blockDim.x) sw[i] = wq[o.W2 + i];
    for (int i = threadIdx.x; i < HID; i += blockDim.x) sw[HID * HID + i] = wq[o.w3 + i];
    __syncthreads();
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const float dy = 2.f * res[b] / (float)B;
    dys[b] = dy;
    float dz2[HID];
    for (int k = 0; k < HID; ++k) {
        dz2[k] = h2s[(int64_t)b * HID + k] > 0.f ? dy * sw[HID * HID + k] : 0.f;
        dz2s[(int64_t)b * HID + k] = dz2[k];
    }
    for (int j = 0; j < HID; ++j) {
        float s = 0.f;
        for (int k = 0; k < HID; ++k) s = fmaf(sw[k * HID + j], dz2[k], s);
        dz1s[(int64_t)b * HID + j] = h1s[(int64_t)b * HID + j] > 0.f ? s : 0.f;
    }
}

// one thread per weight: gradient summed over the batch
__global__ void k_wgrad(int nf, int B, const float* xs, const float* h1s, const float* h2s,
                        const float* dys, const float* dz1s, const float* dz2s, float* g) {
    const Off o(nf);
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= wcount(nf)) return;
    float s = 0.f;
    if (i < o.b1) {
        const int j = (int)(i / nf), k = (int)(i % nf);
        for (int b = 0; b < B; ++b) s = fmaf(dz1s[(int64_t)b * HID + j], xs[(int64_t)b * nf + k], s);
    } else if (i < o.W2) {
        const int j = (int)(i - o.b1);
        for (int b = 0; b < B; ++b) s += dz1s[(int64_t)b * HID + j];
    } else if (i < o.b2) {
        const int k = (int)((i - o.W2) / HID), j = (int)((i - o.W2) % HID);
        for (int b = 0; b < B; ++b) s = fmaf(dz2s[(int64_t)b * HID + k], h1s[(int64_t)b * HID + j], s);
    } else if (i < o.w3) {
        const int k = (int)(i - o.b2);
        for (int b = 0; b < B; ++b) s += dz2s[(int64_t)b * HID + k];
    } else if (i < o.b3) {
        const int k = (int)(i - o.w3);
        for (int b = 0; b < B; ++b) s = fmaf(dys[b], h2s[(int64_t)b * HID + k], s);
    } else {
        for (int b = 0; b < B; ++b) s += dys[b];
    }
    g[i] = s;
}

__global__ void k_adam(float* w, const float* g, float* m, float* v, int64_t n, float lr, float b1,
                       float b2, float c1, float c2) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    m[i] = b1 * m[i] + (1.f - b1) * gi;
    v[i] = b2 * v[i] + (1.f - b2) * gi * gi;
    const float mh = m[i] / c1, vh = v[i] / c2;
    w[i] -= lr * mh / (sqrtf(vh) + 1e-8f);
}

__global__ void k_abs_sum(const float* res, int n, double* out) {
    __shared__ double s[256];
    double a = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        a += fabs((double)res[i]);
    s[threadIdx.x] = a;
    __syncthreads();
    for (int k = 128; k > 0; k >>= 1) {
        if ((int)threadIdx.x < k) s[threadIdx.x] += s[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(out, s[0]);
}

__global__ void k_sq_sum(const float* res, int n, double* out) {
    __shared__ double s[256];
    double a = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        a += (double)res[i] * res[i];
    s[threadIdx.x] = a;
    __syncthreads();
    for (int k = 128; k > 0; k >>= 1) {
        if ((int)threadIdx.x < k) s[threadIdx.x] += s[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(out, s[0]);
}

struct Buf {
    std::vector<void*> ptrs;
    template <class T>
    T* get(size_t count) {
        void* p = nullptr;
        if (cudaMalloc(&p, std::max<size_t>(count, 1) * sizeof(T)) != cudaSuccess) return nullptr;
        ptrs.push_back(p);
        return static_cast<T*>(p);
    }
    ~Buf() {
        for (void* p : ptrs) cudaFree(p);
    }
};

cudaError_t fwd_bwd(const float* wq, int nf, const float* X, const float* T, const int64_t* idx,
                    int B, float* xs, float* h1s, float* h2s, float* res, float* dys, float* dz1s,
                    float* dz2s, float* g, cudaStream_t s) {
    const size_t smw = sizeof(float) * wcount(nf);
    cudaFuncSetAttribute(k_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smw);
    k_fwd<<<(B + 127) / 128, 128, smw, s>>>(wq, nf, X, T, idx, B, xs, h1s, h2s, res, nullptr);
    const size_t smb = sizeof(float) * (HID * HID + HID);
    k_bwd<<<(B + 127) / 128, 128, smb, s>>>(wq, nf, h1s, h2s, res, B, dys, dz1s, dz2s);
    const int64_t nw = wcount(nf);
    k_wgrad<<<(unsigned)((nw + 127) / 128), 128, 0, s>>>(nf, B, xs, h1s, h2s, dys, dz1s, dz2s, g);
    return cudaGetLastError();
}

}  // namespace

// upload a flat FP32 predictor (the order of finger.h) as the inference copy
finger_status finger_load_mlp_internal(finger_index* ix, const float* w, int64_t count, float eps) {
    if (!ix || !w || ix->r < 1) return ix && ix->r < 1 ? FINGER_ERR_NOT_BUILT : FINGER_ERR_INVALID_ARG;
    const int nf = ix->r + 4;
    if (count != wcount(nf)) return FINGER_ERR_INVALID_ARG;
    const Off o(nf);
    const int kp = (nf + 15) & ~15;
    std::vector<__nv_bfloat16> W1((size_t)HID * kp), W2((size_t)HID * HID);
    for (int j = 0; j < HID; ++j)
        for (int i = 0; i < kp; ++i)
            W1[(size_t)j * kp + i] = __float2bfloat16_rn(i < nf ? w[o.W1 + (int64_t)j * nf + i] : 0.f);
    for (int i = 0; i < HID * HID; ++i) W2[i] = __float2bfloat16_rn(w[o.W2 + i]);
    // fragment-major B operands of m16n8k16 (row n = 8 nt + g of the weight
    // matrix, k pairs 16 ks + 2t and 16 ks + 2t + 8 of that row; g = lane / 4,
    // t = lane % 4): one uint2 per lane per (nt, ks)
    auto frag = [](const std::vector<__nv_bfloat16>& Wm, int K) {
        const int nk = K / 16;
        std::vector<uint2> f((size_t)8 * nk * 32);
        auto bits = [&](int row, int col) {
            __nv_bfloat16 v = Wm[(size_t)row * K + col];
            uint16_t u;
            memcpy(&u, &v, 2);
            return (uint32_t)u;
        };
        for (int nt = 0; nt < 8; ++nt)
            for (int ks = 0; ks < nk; ++ks)
                for (int lane = 0; lane < 32; ++lane) {
                    const int n = 8 * nt + (lane >> 2), c = 16 * ks + 2 * (lane & 3);
                    f[((size_t)nt * nk + ks) * 32 + lane] =
                        make_uint2(bits(n, c) | bits(n, c + 1) << 16,
                                   bits(n, c + 8) | bits(n, c + 9) << 16);
                }
        return f;
    };
    const std::vector<uint2> W1f = frag(W1, kp), W2f = frag(W2, HID);
    std::vector<float> w3(HID), b1(w + o.b1, w + o.b1 + HID), b2(w + o.b2, w + o.b2 + HID);
    for (int k = 0; k < HID; ++k) w3[k] = __bfloat162float(__float2bfloat16_rn(w[o.w3 + k]));
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(ix->device);
    cudaFree(ix->W1f);
    cudaFree(ix->W2f);
    cudaFree(ix->w3);
    cudaFree(ix->b1);
    cudaFree(ix->b2);
    ix->W1f = ix->W2f = nullptr;
    ix->w3 = ix->b1 = ix->b2 = nullptr;
    bool ok = cudaMalloc(&ix->W1f, W1f.size() * sizeof(uint2)) == cudaSuccess &&
              cudaMalloc(&ix->W2f, W2f.size() * sizeof(uint2)) == cudaSuccess &&
              cudaMalloc(&ix->w3, HID * 4) == cudaSuccess &&
              cudaMalloc(&ix->b1, HID * 4) == cudaSuccess &&
              cudaMalloc(&ix->b2, HID * 4) == cudaSuccess;
    ok = ok &&
         cudaMemcpy(ix->W1f, W1f.data(), W1f.size() * sizeof(uint2), cudaMemcpyHostToDevice) ==
             cudaSuccess &&
         cudaMemcpy(ix->W2f, W2f.data(), W2f.size() * sizeof(uint2), cudaMemcpyHostToDevice) ==
             cudaSuccess &&
         cudaMemcpy(ix->w3, w3.data(), HID * 4, cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(ix->b1, b1.data(), HID * 4, cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(ix->b2, b2.data(), HID * 4, cudaMemcpyHostToDevice) == cudaSuccess;
    cudaSetDevice(prev);
    if (!ok) {
        cudaGetLastError();
        return FINGER_ERR_OOM;
    }
    ix->b3 = w[o.b3];
    ix->mlp_eps = eps;
    ix->mlp_kp = kp;
    ix->h_mlp.assign(w, w + count);
    ix->has_mlp = 1;
    fg_drop_captures(ix);
    return FINGER_OK;
}

extern "C" {

int64_t finger_mlp_size(int r) { return r < 1 ? -1 : wcount(r + 4); }

finger_status finger_set_predictor(finger_index* ix, const float* weights, int64_t count,
                                   float eps) {
    return finger_load_mlp_internal(ix, weights, count, eps);
}

finger_status finger_set_predictor_gate(finger_index* ix, float delta) {
    if (!ix || !(delta == delta)) return FINGER_ERR_INVALID_ARG;
    if (ix->mlp_delta != delta) fg_drop_captures(ix);   // captured launches hold the index view
    ix->mlp_delta = delta;
    return FINGER_OK;
}

finger_status finger_get_predictor(const finger_index* ix, float* weights, float* eps) {
    if (!ix) return FINGER_ERR_INVALID_ARG;
    if (!ix->has_mlp) return FINGER_ERR_NOT_BUILT;
    if (weights) memcpy(weights, ix->h_mlp.data(), ix->h_mlp.size() * sizeof(float));
    if (eps) *eps = ix->mlp_eps;
    return FINGER_OK;
}

finger_status finger_harvest(finger_index* ix, const float* queries, int64_t nq, int ef,
                             int64_t cap, float* feat, float* target, int32_t* triples,
                             int64_t* count, void* stream) {
    if (!ix || !queries || nq < 1 || ef < 1 || ef > MAX_EF || cap < 1 || !feat || !target ||
        !triples || !count)
        return FINGER_ERR_INVALID_ARG;
    if (!ix->adj0 || !ix->edge_u) return FINGER_ERR_NOT_BUILT;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(ix->device);
    cudaStream_t s = (cudaStream_t)stream;
    finger_status st;
    SearchPlan p;
    Buf buf;
    int64_t* ids = buf.get<int64_t>((size_t)nq);
    float* ds = buf.get<float>((size_t)nq);
    unsigned long long* cnt = buf.get<unsigned long long>(1);
    if (!ids || !ds || !cnt) {
        cudaSetDevice(prev);
        return FINGER_ERR_OOM;
    }
    st = fg_make_plan(ix, MODE_HARVEST, ef, nq, &p, 4, 0);
    if (st == FINGER_OK) {
        SearchArgs a = fg_base_args(ix, p);
        a.Q = queries;
        a.nq = nq;
        a.K = 1;
        a.ef = ef;
        a.out_ids = ids;
        a.out_d = ds;
        a.hv_feat = feat;
        a.hv_target = target;
        a.hv_trip = triples;
        a.hv_count = cnt;
        a.hv_cap = cap;
        if (cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), s) != cudaSuccess) st = FINGER_ERR_CUDA;
        else st = fg_run_search(ix, p, a, s);
        unsigned long long h = 0;
        if (st == FINGER_OK &&
            (cudaMemcpyAsync(&h, cnt, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
             cudaStreamSynchronize(s) != cudaSuccess))
            st = FINGER_ERR_CUDA;
        *count = (int64_t)std::min<unsigned long long>(h, (unsigned long long)cap);
    }
    cudaGetLastError();
    cudaSetDevice(prev);
    return st;
}

finger_status finger_mlp_loss_grad(finger_index* ix, int nf, const float* weights,
                                   const float* feat, const float* target, int64_t n, float* grad,
                                   double* loss, void* stream) {
    if (!ix || nf < 1 || nf > 96 || !weights || !feat || !target || n < 1 || n > (1 << 24) || !grad)
        return FINGER_ERR_INVALID_ARG;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(ix->device);
    cudaStream_t s = (cudaStream_t)stream;
    const int B = (int)n;
    const int64_t nw = wcount(nf);
    Buf buf;
    float* w = buf.get<float>(nw);
    float* wq = buf.get<float>(nw);
    float* g = buf.get<float>(nw);
    float* xs = buf.get<float>((size_t)B * nf);
    float* h1s = buf.get<float>((size_t)B * HID);
    float* h2s = buf.get<float>((size_t)B * HID);
    float* res = buf.get<float>(B);
    float* dys = buf.get<float>(B);
    float* dz1s = buf.get<float>((size_t)B * HID);
    float* dz2s = buf.get<float>((size_t)B * HID);
    double* acc = buf.get<double>(1);
    finger_status st = FINGER_OK;
    if (!w || !wq || !g || !xs || !h1s || !h2s || !res || !dys || !dz1s || !dz2s || !acc) {
        st = FINGER_ERR_OOM;
    } else {
        const Off o(nf);
        double h = 0;
        bool ok = cudaMemcpyAsync(w, weights, nw * 4, cudaMemcpyHostToDevice, s) == cudaSuccess;
        k_quant<<<(unsigned)((nw + 255) / 256), 256, 0, s>>>(w, nw, o.b1, o.W2, o.b2, o.w3, o.b3, wq);
        ok = ok && fwd_bwd(wq, nf, feat, target, nullptr, B, xs, h1s, h2s, res, dys, dz1s, dz2s, g,
                           s) == cudaSuccess;
        ok = ok && cudaMemsetAsync(acc, 0, 8, s) == cudaSuccess;
        k_sq_sum<<<64, 256, 0, s>>>(res, B, acc);
        ok = ok && cudaMemcpyAsync(grad, g, nw * 4, cudaMemcpyDeviceToHost, s) == cudaSuccess;
        ok = ok && cudaMemcpyAsync(&h, acc, 8, cudaMemcpyDeviceToHost, s) == cudaSuccess;
        ok = ok && cudaStreamSynchronize(s) == cudaSuccess;
        if (!ok) st = FINGER_ERR_CUDA;
        if (loss) *loss = h / B;
    }
    cudaGetLastError();
    cudaSetDevice(prev);
    return st;
}

finger_status finger_mlp_predict(finger_index* ix, const float* feat, int64_t n, float* out,
                                 void* stream) {
    if (!ix || !feat || !out || n < 0) return FINGER_ERR_INVALID_ARG;
    if (!ix->has_mlp) return FINGER_ERR_NOT_BUILT;
    if (n == 0) return FINGER_OK;
    const int nf = ix->r + 4;
    const int64_t nw = wcount(nf);
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(ix->device);
    cudaStream_t s = (cudaStream_t)stream;
    Buf buf;
    float* w = buf.get<float>(nw);
    float* wq = buf.get<float>(nw);
    finger_status st = FINGER_OK;
    if (!w || !wq) {
        st = FINGER_ERR_OOM;
    } else {
        const Off o(nf);
        bool ok = cudaMemcpyAsync(w, ix->h_mlp.data(), nw * 4, cudaMemcpyHostToDevice, s) == cudaSuccess;
        k_quant<<<(unsigned)((nw + 255) / 256), 256, 0, s>>>(w, nw, o.b1, o.W2, o.b2, o.w3, o.b3, wq);
        const size_t smw = sizeof(float) * nw;
        cudaFuncSetAttribute(k_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smw);
        for (int64_t lo = 0; lo < n && ok; lo += 1 << 20) {
            const int B = (int)std::min<int64_t>(n - lo, 1 << 20);
            k_fwd<<<(B + 127) / 128, 128, smw, s>>>(wq, nf, feat + lo * nf, nullptr, nullptr, B,
                                                    nullptr, nullptr, nullptr, nullptr, out + lo);
        }
        ok = ok && cudaGetLastError() == cudaSuccess && cudaStreamSynchronize(s) == cudaSuccess;
        if (!ok) st = FINGER_ERR_CUDA;
    }
    cudaGetLastError();
    cudaSetDevice(prev);
    return st;
}

finger_status finger_train_predictor(finger_index* ix, const finger_train_params* p, float* losses,
                                     void* stream) {
    if (!ix || !p || !p->feat || !p->target || p->n_train < 1 || p->n_val < 0 || p->epochs < 1 ||
        p->batch < 1 || p->batch > (1 << 20) || !(p->lr > 0))
        return FINGER_ERR_INVALID_ARG;
    if (ix->r < 1) return FINGER_ERR_NOT_BUILT;
    const int nf = ix->r + 4;
    const int64_t nw = wcount(nf);
    const Off o(nf);
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(ix->device);
    cudaStream_t s = (cudaStream_t)stream;
    const int B = p->batch;
    Buf buf;
    float* w = buf.get<float>(nw);
    float* wq = buf.get<float>(nw);
    float* g = buf.get<float>(nw);
    float* m1 = buf.get<float>(nw);
    float* m2 = buf.get<float>(nw);
    float* xs = buf.get<float>((size_t)B * nf);
    float* h1s = buf.get<float>((size_t)B * HID);
    float* h2s = buf.get<float>((size_t)B * HID);
    float* res = buf.get<float>(B);
    float* dys = buf.get<float>(B);
    float* dz1s = buf.get<float>((size_t)B * HID);
    float* dz2s = buf.get<float>((size_t)B * HID);
    int64_t* idx = buf.get<int64_t>((size_t)p->n_train);
    double* acc = buf.get<double>(1);
    if (!w || !wq || !g || !m1 || !m2 || !xs || !h1s || !h2s || !res || !dys || !dz1s || !dz2s ||
        !idx || !acc) {
        cudaSetDevice(prev);
        return FINGER_ERR_OOM;
    }
    // He-uniform initialisation of the masters (seeded), zero biases
    std::vector<float> hw((size_t)nw, 0.f);
    std::mt19937_64 rng(p->seed);
    std::uniform_real_distribution<float> U(-1.f, 1.f);
    const float s1 = sqrtf(6.f / nf), s2 = sqrtf(6.f / HID);
    for (int64_t i = 0; i < (int64_t)HID * nf; ++i) hw[o.W1 + i] = U(rng) * s1;
    for (int64_t i = 0; i < HID * HID; ++i) hw[o.W2 + i] = U(rng) * s2;
    for (int64_t i = 0; i < HID; ++i) hw[o.w3 + i] = U(rng) * s2;
    bool ok = cudaMemcpyAsync(w, hw.data(), nw * 4, cudaMemcpyHostToDevice, s) == cudaSuccess &&
              cudaMemsetAsync(m1, 0, nw * 4, s) == cudaSuccess &&
              cudaMemsetAsync(m2, 0, nw * 4, s) == cudaSuccess;
    std::vector<int64_t> perm((size_t)p->n_train);
    std::iota(perm.begin(), perm.end(), 0);
    int64_t step = 0;
    const float b1 = 0.9f, b2 = 0.999f;
    for (int ep = 0; ep < p->epochs && ok; ++ep) {
        std::shuffle(perm.begin(), perm.end(), rng);
        ok = cudaMemcpyAsync(idx, perm.data(), perm.size() * 8, cudaMemcpyHostToDevice, s) == cudaSuccess &&
             cudaStreamSynchronize(s) == cudaSuccess;
        double sq = 0;
        ok = ok && cudaMemsetAsync(acc, 0, 8, s) == cudaSuccess;
        for (int64_t lo = 0; lo + B <= p->n_train && ok; lo += B) {
            step++;
            k_quant<<<(unsigned)((nw + 255) / 256), 256, 0, s>>>(w, nw, o.b1, o.W2, o.b2, o.w3, o.b3, wq);
            ok = fwd_bwd(wq, nf, p->feat, p->target, idx + lo, B, xs, h1s, h2s, res, dys, dz1s,
                         dz2s, g, s) == cudaSuccess;
            k_sq_sum<<<16, 256, 0, s>>>(res, B, acc);
            const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
            k_adam<<<(unsigned)((nw + 255) / 256), 256, 0, s>>>(w, g, m1, m2, nw, p->lr, b1, b2, c1, c2);
        }
        ok = ok && cudaMemcpyAsync(&sq, acc, 8, cudaMemcpyDeviceToHost, s) == cudaSuccess &&
             cudaStreamSynchronize(s) == cudaSuccess;
        if (losses) losses[ep] = (float)(sq / std::max<int64_t>(1, (p->n_train / B) * B));
    }
    // eps' = mean |prediction - target| on the held-out rows (inference semantics)
    float eps = 0.f;
    if (ok) {
        k_quant<<<(unsigned)((nw + 255) / 256), 256, 0, s>>>(w, nw, o.b1, o.W2, o.b2, o.w3, o.b3, wq);
        ok = cudaMemsetAsync(acc, 0, 8, s) == cudaSuccess;
        const int64_t v0 = p->n_train, nv = p->n_val;
        const size_t smw = sizeof(float) * nw;
        cudaFuncSetAttribute(k_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smw);
        for (int64_t lo = 0; lo < nv && ok; lo += B) {
            const int nb = (int)std::min<int64_t>(B, nv - lo);
            k_fwd<<<(nb + 127) / 128, 128, smw, s>>>(wq, nf, p->feat + (v0 + lo) * nf,
                                                     p->target + v0 + lo, nullptr, nb, nullptr,
                                                     nullptr, nullptr, res, nullptr);
            k_abs_sum<<<16, 256, 0, s>>>(res, nb, acc);
        }
        double sa = 0;
        ok = ok && cudaMemcpyAsync(&sa, acc, 8, cudaMemcpyDeviceToHost, s) == cudaSuccess &&
             cudaStreamSynchronize(s) == cudaSuccess;
        eps = nv > 0 ? (float)(sa / nv) : 0.f;
    }
    if (ok) ok = cudaMemcpy(hw.data(), w, nw * 4, cudaMemcpyDeviceToHost) == cudaSuccess;
    cudaGetLastError();
    cudaSetDevice(prev);
    if (!ok) return FINGER_ERR_CUDA;
    return finger_load_mlp_internal(ix, hw.data(), nw, eps);
}

}  // extern "C"

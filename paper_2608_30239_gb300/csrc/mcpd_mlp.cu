// Learned scan weights and initial marginals: per-clone features, a 16-64-64-2 MLP with bf16
// parameters and fp32 accumulation, its loss, backward pass and Adam update, and the two heads.
//
// Not in the paper.  The paper proves that any fixed positive scan weights leave pi invariant
// (Proposition 1) and that the coupled estimator is unbiased from any initial distribution
// (Theorem 1), so scan weights w and initial marginals nu predicted from the observed design are
// admissible inputs of the method: w = (1 - a) softmax(o_1) + a / n (a = 0.5 keeps every site's
// weight >= 0.5 / n) and nu = clamp(sigmoid(o_2), 1e-6, 1 - 1e-6).
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "mcpd_internal.h"

namespace mcpd {
namespace {

constexpr int F = 16, H = 64, O = 2;
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + H * F, OFF_W2 = OFF_B1 + H, OFF_B2 = OFF_W2 + H * H;
constexpr int OFF_W3 = OFF_B2 + H, OFF_B3 = OFF_W3 + O * H, NPARAM = OFF_B3 + O;   // 5378

__device__ __forceinline__ void stage_params(const __nv_bfloat16 *W, float *sW) {
    for (int i = threadIdx.x; i < NPARAM; i += blockDim.x) sW[i] = __bfloat162float(W[i]);
    __syncthreads();
}

// Z1 = W1 x + b1, H1 = relu(Z1), Z2 = W2 H1 + b2, H2 = relu(Z2), out = W3 H2 + b3 (one row).
__device__ __forceinline__ void row_forward(const float *sW, const float *x, float *z1, float *z2,
                                            float *out) {
#pragma unroll 4
    for (int a = 0; a < H; ++a) {
        float acc = sW[OFF_B1 + a];
#pragma unroll
        for (int c = 0; c < F; ++c) acc = fmaf(sW[OFF_W1 + a * F + c], x[c], acc);
        z1[a] = acc;
    }
#pragma unroll 2
    for (int a = 0; a < H; ++a) {
        float acc = sW[OFF_B2 + a];
#pragma unroll
        for (int b = 0; b < H; ++b) acc = fmaf(sW[OFF_W2 + a * H + b], fmaxf(z1[b], 0.f), acc);
        z2[a] = acc;
    }
#pragma unroll
    for (int o = 0; o < O; ++o) {
        float acc = sW[OFF_B3 + o];
#pragma unroll
        for (int b = 0; b < H; ++b) acc = fmaf(sW[OFF_W3 + o * H + b], fmaxf(z2[b], 0.f), acc);
        out[o] = acc;
    }
}

__global__ void mlp_forward_kernel(long long n, const float *X, const __nv_bfloat16 *W, float *Out) {
    __shared__ float sW[NPARAM];
    stage_params(W, sW);
    for (long long r = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; r < n;
         r += static_cast<long long>(gridDim.x) * blockDim.x) {
        float x[F], z1[H], z2[H], out[O];
#pragma unroll
        for (int c = 0; c < F; ++c) x[c] = X[r * F + c];
        row_forward(sW, x, z1, z2, out);
        Out[r * O] = out[0];
        Out[r * O + 1] = out[1];
    }
}

// Per row: recompute the activations and back-propagate dOut to dZ2 and dZ1.
__global__ void mlp_rows_backward_kernel(long long n, const float *X, const __nv_bfloat16 *W,
                                         const float *dOut, float *H1, float *H2, float *DZ1,
                                         float *DZ2) {
    __shared__ float sW[NPARAM];
    stage_params(W, sW);
    for (long long r = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; r < n;
         r += static_cast<long long>(gridDim.x) * blockDim.x) {
        float x[F], z1[H], z2[H], out[O];
#pragma unroll
        for (int c = 0; c < F; ++c) x[c] = X[r * F + c];
        row_forward(sW, x, z1, z2, out);
        const float d0 = dOut[r * O], d1 = dOut[r * O + 1];
        float dz2[H];
#pragma unroll
        for (int b = 0; b < H; ++b) {
            const float dh = fmaf(sW[OFF_W3 + b], d0, sW[OFF_W3 + H + b] * d1);
            dz2[b] = z2[b] > 0.f ? dh : 0.f;
            H2[r * H + b] = fmaxf(z2[b], 0.f);
            DZ2[r * H + b] = dz2[b];
        }
#pragma unroll 2
        for (int b = 0; b < H; ++b) {
            float dh = 0.f;
#pragma unroll
            for (int a = 0; a < H; ++a) dh = fmaf(sW[OFF_W2 + a * H + b], dz2[a], dh);
            DZ1[r * H + b] = z1[b] > 0.f ? dh : 0.f;
            H1[r * H + b] = fmaxf(z1[b], 0.f);
        }
    }
}

// Partial parameter gradients of one chunk of rows (fixed chunking, so the sum is reproducible):
// gW1 = DZ1^T X, gb1 = sum DZ1, gW2 = DZ2^T H1, gb2 = sum DZ2, gW3 = dOut^T H2, gb3 = sum dOut.
__global__ void mlp_param_partials_kernel(long long n, long long chunk, const float *X,
                                          const float *dOut, const float *H1, const float *H2,
                                          const float *DZ1, const float *DZ2, float *partials) {
    const long long r0 = static_cast<long long>(blockIdx.x) * chunk;
    const long long r1 = min(n, r0 + chunk);
    for (int k = threadIdx.x; k < NPARAM; k += blockDim.x) {
        float acc = 0.f;
        if (k < OFF_B1) {
            const int a = k / F, c = k % F;
            for (long long r = r0; r < r1; ++r) acc = fmaf(DZ1[r * H + a], X[r * F + c], acc);
        } else if (k < OFF_W2) {
            const int a = k - OFF_B1;
            for (long long r = r0; r < r1; ++r) acc += DZ1[r * H + a];
        } else if (k < OFF_B2) {
            const int a = (k - OFF_W2) / H, b = (k - OFF_W2) % H;
            for (long long r = r0; r < r1; ++r) acc = fmaf(DZ2[r * H + a], H1[r * H + b], acc);
        } else if (k < OFF_W3) {
            const int a = k - OFF_B2;
            for (long long r = r0; r < r1; ++r) acc += DZ2[r * H + a];
        } else if (k < OFF_B3) {
            const int o = (k - OFF_W3) / H, b = (k - OFF_W3) % H;
            for (long long r = r0; r < r1; ++r) acc = fmaf(dOut[r * O + o], H2[r * H + b], acc);
        } else {
            const int o = k - OFF_B3;
            for (long long r = r0; r < r1; ++r) acc += dOut[r * O + o];
        }
        partials[static_cast<long long>(blockIdx.x) * NPARAM + k] = acc;
    }
}

__global__ void mlp_reduce_partials_kernel(int chunks, const float *partials, float *grad) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= NPARAM) return;
    float acc = 0.f;
    for (int c = 0; c < chunks; ++c) acc += partials[static_cast<long long>(c) * NPARAM + k];
    grad[k] = acc;
}

// Loss per segment (instance) and dOut: cross-entropy of softmax(o_1) to target_w plus the mean
// binary cross-entropy of sigmoid(o_2) to target_p, each segment weighted 1 / n_seg.
__global__ void mlp_loss_kernel(int n_seg, const long long *seg, const float *Out,
                                const float *target_w, const float *target_p, float *dOut,
                                double *loss_seg) {
    const int s = blockIdx.x;
    const long long a = seg[s], b = seg[s + 1];
    __shared__ float red[256];
    __shared__ double redd[256];
    float mx = -3.0e38f;
    for (long long r = a + threadIdx.x; r < b; r += blockDim.x) mx = fmaxf(mx, Out[r * O]);
    red[threadIdx.x] = mx;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] = fmaxf(red[threadIdx.x], red[threadIdx.x + w]);
        __syncthreads();
    }
    mx = red[0];
    __syncthreads();
    float se = 0.f, st = 0.f;
    for (long long r = a + threadIdx.x; r < b; r += blockDim.x) { se += __expf(Out[r * O] - mx); st += target_w[r]; }
    red[threadIdx.x] = se;
    redd[threadIdx.x] = st;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) { red[threadIdx.x] += red[threadIdx.x + w]; redd[threadIdx.x] += redd[threadIdx.x + w]; }
        __syncthreads();
    }
    const float lse = mx + __logf(red[0]);
    const float tsum = static_cast<float>(redd[0]);
    __syncthreads();
    const float inv_seg = 1.f / n_seg, inv_len = 1.f / static_cast<float>(b - a);
    double part = 0.0;
    for (long long r = a + threadIdx.x; r < b; r += blockDim.x) {
        const float o1 = Out[r * O], z = Out[r * O + 1], t = target_w[r], p = target_p[r];
        const float sm = __expf(o1 - lse);
        dOut[r * O] = (sm * tsum - t) * inv_seg;
        const float sig = 1.f / (1.f + __expf(-z));
        dOut[r * O + 1] = (sig - p) * inv_len * inv_seg;
        const float softplus = z > 0.f ? z + log1pf(__expf(-z)) : log1pf(__expf(z));
        part += static_cast<double>(-t * (o1 - lse)) + static_cast<double>((softplus - p * z) * inv_len);
    }
    redd[threadIdx.x] = part;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) redd[threadIdx.x] += redd[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) loss_seg[s] = redd[0] / n_seg;
}

__global__ void mlp_adam_kernel(int step, float lr, float b1, float b2, float eps, float *master,
                                float *m, float *v, const float *grad, __nv_bfloat16 *W) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= NPARAM) return;
    const float g = grad[k];
    const float mk = b1 * m[k] + (1.f - b1) * g;
    const float vk = b2 * v[k] + (1.f - b2) * g * g;
    m[k] = mk;
    v[k] = vk;
    const float mhat = mk / (1.f - powf(b1, static_cast<float>(step)));
    const float vhat = vk / (1.f - powf(b2, static_cast<float>(step)));
    master[k] -= lr * mhat / (sqrtf(vhat) + eps);
    W[k] = __float2bfloat16_rn(master[k]);
}

__global__ void mlp_cast_kernel(const float *master, __nv_bfloat16 *W) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < NPARAM) W[k] = __float2bfloat16_rn(master[k]);
}

// Heads per segment: w = 0.5 softmax(o_1) + 0.5 / n, nu = clamp(sigmoid(o_2)).
__global__ void mlp_heads_kernel(const long long *seg, const float *Out, double *w, double *nu) {
    const int s = blockIdx.x;
    const long long a = seg[s], b = seg[s + 1];
    __shared__ double red[256];
    double mx = -1e300;
    for (long long r = a + threadIdx.x; r < b; r += blockDim.x) mx = fmax(mx, static_cast<double>(Out[r * O]));
    red[threadIdx.x] = mx;
    __syncthreads();
    for (int k = blockDim.x / 2; k > 0; k >>= 1) {
        if (threadIdx.x < k) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + k]);
        __syncthreads();
    }
    mx = red[0];
    __syncthreads();
    double se = 0.0;
    for (long long r = a + threadIdx.x; r < b; r += blockDim.x) se += exp(static_cast<double>(Out[r * O]) - mx);
    red[threadIdx.x] = se;
    __syncthreads();
    for (int k = blockDim.x / 2; k > 0; k >>= 1) {
        if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
        __syncthreads();
    }
    const double tot = red[0];
    const double n = static_cast<double>(b - a);
    for (long long r = a + threadIdx.x; r < b; r += blockDim.x) {
        w[r] = 0.5 * (exp(static_cast<double>(Out[r * O]) - mx) / tot) + 0.5 / n;
        const double sg = 1.0 / (1.0 + exp(-static_cast<double>(Out[r * O + 1])));
        nu[r] = fmin(fmax(sg, 1e-6), 1.0 - 1e-6);
    }
}

// Features, pass 1 (per clone): degree, positive pools, all-positive flag; pool sizes.
__global__ void feat_pass1(long long n, const int32_t *ptr, const int32_t *pools, const uint8_t *y,
                           const int64_t *clone_pool_base, int32_t *deg, int32_t *npos,
                           int32_t *allpos, int32_t *psize, int32_t *nap, const int32_t *clone_inst) {
    const long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const long long base = clone_pool_base[i];
    int d = 0, p = 0;
    for (int e = ptr[i]; e < ptr[i + 1]; ++e) {
        const long long j = base + pools[e];
        p += y[j];
        ++d;
        atomicAdd(&psize[j], 1);
    }
    deg[i] = d;
    npos[i] = p;
    const int ap = (d > 0 && p == d) ? 1 : 0;
    allpos[i] = ap;
    if (ap) atomicAdd(&nap[clone_inst[i]], 1);
}

__global__ void feat_pass2(long long n, const int32_t *ptr, const int32_t *pools,
                           const int64_t *clone_pool_base, const int32_t *allpos, int32_t *ap_pool) {
    const long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n || !allpos[i]) return;
    for (int e = ptr[i]; e < ptr[i + 1]; ++e) atomicAdd(&ap_pool[clone_pool_base[i] + pools[e]], 1);
}

__global__ void feat_pass3(long long n, const int32_t *ptr, const int32_t *pools, const uint8_t *y,
                           const int64_t *clone_pool_base, const int32_t *deg, const int32_t *npos,
                           const int32_t *allpos, const int32_t *psize, const int32_t *ap_pool,
                           const int32_t *nap, const int32_t *clone_inst, const double *consts,
                           float *Fout) {
    const long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int s = clone_inst[i];
    const double lam = consts[4 * s], a_pos = consts[4 * s + 1], a_neg = consts[4 * s + 2], dbar = consts[4 * s + 3];
    const long long base = clone_pool_base[i];
    const int d = deg[i], p = npos[i], nn = d - p, ap = allpos[i];
    double sum_d = 0.0, sum_dpos = 0.0, sum_inv = 0.0;
    int min_ap = 1 << 30, sole = 0, unexplained = 0;
    for (int e = ptr[i]; e < ptr[i + 1]; ++e) {
        const long long j = base + pools[e];
        sum_d += psize[j];
        if (y[j]) {
            sum_dpos += psize[j];
            min_ap = min(min_ap, ap_pool[j]);
            sum_inv += 1.0 / max(ap_pool[j], 1);
            if (ap && ap_pool[j] == 1) ++sole;
            if (ap_pool[j] == 0) ++unexplained;
        }
    }
    float *f = Fout + i * 16;
    f[0] = d / 8.0f;
    f[1] = p / 8.0f;
    f[2] = nn / 8.0f;
    f[3] = static_cast<float>(p) / static_cast<float>(max(d, 1));
    f[4] = static_cast<float>((lam + p * a_pos + nn * a_neg) / 10.0);
    f[5] = d ? static_cast<float>(sum_d / d / dbar) : 0.f;
    f[6] = p ? static_cast<float>(sum_dpos / p / dbar) : 0.f;
    f[7] = static_cast<float>(ap);
    f[8] = p ? min_ap / 10.0f : 0.f;
    f[9] = p ? static_cast<float>(sum_inv / p) : 0.f;
    f[10] = sole / 8.0f;
    f[11] = unexplained / 8.0f;
    f[12] = nap[s] / 100.0f;
    f[13] = static_cast<float>(lam / 10.0);
    f[14] = static_cast<float>(a_pos / 10.0);
    f[15] = static_cast<float>(a_neg / 10.0);
}

int grid_for(long long n, int block) {
    long long g = (n + block - 1) / block;
    return static_cast<int>(g < 1 ? 1 : (g > 65535LL * 64 ? 65535LL * 64 : g));
}

}  // namespace
}  // namespace mcpd

namespace {
int fail_m(mcpd_ctx *ctx, int code, const std::string &msg) {
    if (ctx) ctx->err = msg;
    return code;
}
}  // namespace

#define CUM(call)                                                                                 \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess) return fail_m(ctx, MCPD_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

extern "C" {

int mcpd_mlp_num_params(void) { return mcpd::NPARAM; }

int mcpd_features_batch(mcpd_ctx *ctx, int32_t n_inst, const mcpd_design *designs,
                        const uint8_t *const *ys, const double *rates, float *feat_dev) {
    using namespace mcpd;
    if (!ctx || n_inst < 1 || !designs || !ys || !rates || !feat_dev) return MCPD_EINVAL;
    // Concatenate the designs: clone rows keep their local pool ids plus a per-clone pool base.
    std::vector<int32_t> ptr(1, 0), pools, cinst;
    std::vector<int64_t> pbase;
    std::vector<uint8_t> y;
    std::vector<double> consts(4 * static_cast<size_t>(n_inst));
    long long pool_off = 0;
    for (int32_t s = 0; s < n_inst; ++s) {
        const mcpd_design &d = designs[s];
        if (d.n_clones < 1 || d.n_pools < 1 || !d.clone_ptr) return fail_m(ctx, MCPD_EINVAL, "bad design");
        const double fp = rates[3 * s], fn = rates[3 * s + 1], q = rates[3 * s + 2];
        if (!(fp > 0 && fp < 1 && fn > 0 && fn < 1 && q > 0 && q < 1)) return fail_m(ctx, MCPD_EINVAL, "rates out of (0,1)");
        consts[4 * s] = std::log(q) - std::log(1.0 - q);
        consts[4 * s + 1] = std::log(1.0 - fn) - std::log(fp);
        consts[4 * s + 2] = std::log(fn) - std::log(1.0 - fp);
        consts[4 * s + 3] = static_cast<double>(d.clone_ptr[d.n_clones]) / d.n_pools;
        for (int32_t i = 0; i < d.n_clones; ++i) {
            for (int32_t e = d.clone_ptr[i]; e < d.clone_ptr[i + 1]; ++e) {
                if (d.clone_pools[e] < 0 || d.clone_pools[e] >= d.n_pools) return fail_m(ctx, MCPD_EINVAL, "pool id");
                pools.push_back(d.clone_pools[e]);
            }
            ptr.push_back(static_cast<int32_t>(pools.size()));
            pbase.push_back(pool_off);
            cinst.push_back(s);
        }
        for (int32_t j = 0; j < d.n_pools; ++j) y.push_back(ys[s][j] ? 1 : 0);
        pool_off += d.n_pools;
    }
    const long long n = static_cast<long long>(cinst.size());
    CUM(cudaSetDevice(ctx->device));
    cudaStream_t st = ctx->stream;
    void *buf = nullptr;
    const size_t nb = ptr.size() * 4 + pools.size() * 4 + y.size() + pbase.size() * 8 + cinst.size() * 4 +
                      consts.size() * 8 + 4 * n * 4 + 2 * pool_off * 4 + n_inst * 4 + 1024;
    CUM(cudaMalloc(&buf, nb));
    char *p = static_cast<char *>(buf);
    auto take = [&](size_t bytes) { char *at = p; p += (bytes + 15) / 16 * 16; return at; };
    int32_t *d_ptr = reinterpret_cast<int32_t *>(take(ptr.size() * 4));
    int32_t *d_pools = reinterpret_cast<int32_t *>(take(pools.size() * 4 + 4));
    uint8_t *d_y = reinterpret_cast<uint8_t *>(take(y.size()));
    int64_t *d_pbase = reinterpret_cast<int64_t *>(take(pbase.size() * 8));
    int32_t *d_cinst = reinterpret_cast<int32_t *>(take(cinst.size() * 4));
    double *d_consts = reinterpret_cast<double *>(take(consts.size() * 8));
    int32_t *d_deg = reinterpret_cast<int32_t *>(take(n * 4));
    int32_t *d_npos = reinterpret_cast<int32_t *>(take(n * 4));
    int32_t *d_allpos = reinterpret_cast<int32_t *>(take(n * 4));
    int32_t *d_psize = reinterpret_cast<int32_t *>(take(pool_off * 4));
    int32_t *d_ap = reinterpret_cast<int32_t *>(take(pool_off * 4));
    int32_t *d_nap = reinterpret_cast<int32_t *>(take(n_inst * 4));
    int rc = MCPD_OK;
    do {
        if (cudaMemcpyAsync(d_ptr, ptr.data(), ptr.size() * 4, cudaMemcpyHostToDevice, st) != cudaSuccess ||
            (!pools.empty() && cudaMemcpyAsync(d_pools, pools.data(), pools.size() * 4, cudaMemcpyHostToDevice, st) != cudaSuccess) ||
            cudaMemcpyAsync(d_y, y.data(), y.size(), cudaMemcpyHostToDevice, st) != cudaSuccess ||
            cudaMemcpyAsync(d_pbase, pbase.data(), pbase.size() * 8, cudaMemcpyHostToDevice, st) != cudaSuccess ||
            cudaMemcpyAsync(d_cinst, cinst.data(), cinst.size() * 4, cudaMemcpyHostToDevice, st) != cudaSuccess ||
            cudaMemcpyAsync(d_consts, consts.data(), consts.size() * 8, cudaMemcpyHostToDevice, st) != cudaSuccess ||
            cudaMemsetAsync(d_psize, 0, pool_off * 4, st) != cudaSuccess ||
            cudaMemsetAsync(d_ap, 0, pool_off * 4, st) != cudaSuccess ||
            cudaMemsetAsync(d_nap, 0, n_inst * 4, st) != cudaSuccess) { rc = MCPD_ECUDA; break; }
        const int g = grid_for(n, 256);
        feat_pass1<<<g, 256, 0, st>>>(n, d_ptr, d_pools, d_y, d_pbase, d_deg, d_npos, d_allpos, d_psize, d_nap, d_cinst);
        feat_pass2<<<g, 256, 0, st>>>(n, d_ptr, d_pools, d_pbase, d_allpos, d_ap);
        feat_pass3<<<g, 256, 0, st>>>(n, d_ptr, d_pools, d_y, d_pbase, d_deg, d_npos, d_allpos, d_psize, d_ap,
                                      d_nap, d_cinst, d_consts, feat_dev);
        if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess) rc = MCPD_ECUDA;
    } while (0);
    cudaFree(buf);
    return rc == MCPD_OK ? MCPD_OK : fail_m(ctx, rc, "features kernels");
}

int mcpd_mlp_forward(mcpd_ctx *ctx, int64_t n_rows, const float *X, const uint16_t *W, float *Out) {
    if (!ctx || n_rows < 0 || (n_rows && (!X || !W || !Out))) return MCPD_EINVAL;
    CUM(cudaSetDevice(ctx->device));
    if (n_rows == 0) return MCPD_OK;
    const int g = std::min(mcpd::grid_for(n_rows, 256), ctx->sm_count * 8);
    mcpd::mlp_forward_kernel<<<g, 256, 0, ctx->stream>>>(n_rows, X, reinterpret_cast<const __nv_bfloat16 *>(W), Out);
    CUM(cudaGetLastError());
    return MCPD_OK;
}

int mcpd_mlp_loss(mcpd_ctx *ctx, int32_t n_seg, const int64_t *seg_dev, const float *Out,
                  const float *target_w, const float *target_p, float *dOut, double *loss_seg_dev) {
    if (!ctx || n_seg < 1 || !seg_dev || !Out || !target_w || !target_p || !dOut || !loss_seg_dev) return MCPD_EINVAL;
    CUM(cudaSetDevice(ctx->device));
    mcpd::mlp_loss_kernel<<<n_seg, 256, 0, ctx->stream>>>(n_seg, reinterpret_cast<const long long *>(seg_dev), Out,
                                                           target_w, target_p, dOut, loss_seg_dev);
    CUM(cudaGetLastError());
    return MCPD_OK;
}

int mcpd_mlp_backward(mcpd_ctx *ctx, int64_t n_rows, const float *X, const uint16_t *W,
                      const float *dOut, float *work, int64_t work_floats, float *grad) {
    using namespace mcpd;
    if (!ctx || n_rows < 1 || !X || !W || !dOut || !work || !grad) return MCPD_EINVAL;
    const long long chunk = 1024;
    const long long chunks = (n_rows + chunk - 1) / chunk;
    const long long need = 4 * H * n_rows + chunks * NPARAM;
    if (work_floats < need) return fail_m(ctx, MCPD_EINVAL, "backward workspace too small");
    CUM(cudaSetDevice(ctx->device));
    float *H1 = work, *H2 = H1 + H * n_rows, *DZ1 = H2 + H * n_rows, *DZ2 = DZ1 + H * n_rows;
    float *partials = DZ2 + H * n_rows;
    const int g = std::min(grid_for(n_rows, 128), ctx->sm_count * 8);
    mlp_rows_backward_kernel<<<g, 128, 0, ctx->stream>>>(n_rows, X, reinterpret_cast<const __nv_bfloat16 *>(W),
                                                         dOut, H1, H2, DZ1, DZ2);
    mlp_param_partials_kernel<<<static_cast<unsigned>(chunks), 256, 0, ctx->stream>>>(n_rows, chunk, X, dOut, H1, H2,
                                                                                        DZ1, DZ2, partials);
    mlp_reduce_partials_kernel<<<(NPARAM + 255) / 256, 256, 0, ctx->stream>>>(static_cast<int>(chunks), partials, grad);
    CUM(cudaGetLastError());
    return MCPD_OK;
}

int64_t mcpd_mlp_backward_workspace(int64_t n_rows) {
    const long long chunks = (n_rows + 1023) / 1024;
    return 4LL * 64 * n_rows + chunks * mcpd::NPARAM;
}

int mcpd_mlp_adam(mcpd_ctx *ctx, int32_t step, float lr, float beta1, float beta2, float eps,
                  float *master, float *m, float *v, const float *grad, uint16_t *W) {
    if (!ctx || step < 1 || !master || !m || !v || !grad || !W) return MCPD_EINVAL;
    CUM(cudaSetDevice(ctx->device));
    mcpd::mlp_adam_kernel<<<(mcpd::NPARAM + 255) / 256, 256, 0, ctx->stream>>>(
        step, lr, beta1, beta2, eps, master, m, v, grad, reinterpret_cast<__nv_bfloat16 *>(W));
    CUM(cudaGetLastError());
    return MCPD_OK;
}

int mcpd_mlp_cast(mcpd_ctx *ctx, const float *master, uint16_t *W) {
    if (!ctx || !master || !W) return MCPD_EINVAL;
    CUM(cudaSetDevice(ctx->device));
    mcpd::mlp_cast_kernel<<<(mcpd::NPARAM + 255) / 256, 256, 0, ctx->stream>>>(master, reinterpret_cast<__nv_bfloat16 *>(W));
    CUM(cudaGetLastError());
    return MCPD_OK;
}

int mcpd_mlp_heads(mcpd_ctx *ctx, int32_t n_seg, const int64_t *seg_dev, const float *Out,
                   double *w_dev, double *nu_dev) {
    if (!ctx || n_seg < 1 || !seg_dev || !Out || !w_dev || !nu_dev) return MCPD_EINVAL;
    CUM(cudaSetDevice(ctx->device));
    mcpd::mlp_heads_kernel<<<n_seg, 256, 0, ctx->stream>>>(reinterpret_cast<const long long *>(seg_dev), Out, w_dev, nu_dev);
    CUM(cudaGetLastError());
    return MCPD_OK;
}

}  // extern "C"

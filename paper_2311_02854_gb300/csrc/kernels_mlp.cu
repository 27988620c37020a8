// Kernels of the learned Davidson preconditioner (see mlp.h): features,
// forward (FP32 or bf16 weights), per-sample backward, reductions of the
// parameter gradient, Adam, the scaled correction and the collection of
// training pairs.
#include <cmath>

#include "engine.h"
#include "mlp.h"

namespace dmrg {
namespace {

constexpr int NT = 128;

__device__ __forceinline__ float tanh_f(float z) { return tanhf(z); }

// parameters into shared memory (FP32, or converted from the bf16 copy)
__device__ __forceinline__ void load_params(float* sw, const float* w, const __nv_bfloat16* wb, bool bf16) {
    for (int i = threadIdx.x; i < kMlpParams; i += blockDim.x)
        sw[i] = bf16 ? __bfloat162float(wb[i]) : w[i];
    __syncthreads();
}

// g(x) for one feature row; optionally writes h1 / h2 (64 each)
__device__ __forceinline__ float mlp_eval(const float* sw, const float* x, float* h1, float* h2) {
    float a[kMlpHid];
#pragma unroll
    for (int i = 0; i < kMlpHid; ++i) {
        float z = sw[kMlpOffB1 + i];
#pragma unroll
        for (int k = 0; k < kMlpIn; ++k) z = fmaf(sw[kMlpOffW1 + i * kMlpIn + k], x[k], z);
        a[i] = tanh_f(z);
        if (h1) h1[i] = a[i];
    }
    float g = sw[kMlpOffB3];
    for (int j = 0; j < kMlpHid; ++j) {
        float z = sw[kMlpOffB2 + j];
        const float* w2 = sw + kMlpOffW2 + j * kMlpHid;
#pragma unroll
        for (int i = 0; i < kMlpHid; ++i) z = fmaf(w2[i], a[i], z);
        const float h = tanh_f(z);
        if (h2) h2[j] = h;
        g = fmaf(sw[kMlpOffW3 + j], h, g);
    }
    return g;
}

__global__ void __launch_bounds__(NT) features_kernel(const double* __restrict__ hd, const double* __restrict__ r,
                                                      double theta, double s, double rmax, int64_t n,
                                                      const int64_t* __restrict__ sec_off,
                                                      const float* __restrict__ sec_q, int nsec,
                                                      float* __restrict__ x) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int lo = 0, hi = nsec - 1;  // sector holding element i
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (sec_off[mid] <= i) lo = mid;
            else hi = mid - 1;
        }
        float* xi = x + i * kMlpIn;
        xi[0] = (float)((hd[i] - theta) / s);
        xi[1] = (float)(theta / s);
        xi[2] = (float)(r[i] / rmax);
        xi[3] = sec_q[2 * lo];
        xi[4] = sec_q[2 * lo + 1];
    }
}

__global__ void __launch_bounds__(NT) forward_kernel(const float* __restrict__ w, const __nv_bfloat16* __restrict__ wb,
                                                     bool bf16, const float* __restrict__ x, int64_t n,
                                                     float* __restrict__ g) {
    __shared__ float sw[kMlpParams];
    load_params(sw, w, wb, bf16);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        float xi[kMlpIn];
#pragma unroll
        for (int k = 0; k < kMlpIn; ++k) xi[k] = x[i * kMlpIn + k];
        g[i] = mlp_eval(sw, xi, nullptr, nullptr);
    }
}

__device__ __forceinline__ uint64_t mix64(uint64_t z) {  // splitmix64 finaliser
    z += 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

// Per sample b of a batch (row idx(b) of the set; identity when seed == 0):
// forward, then dg = 2 w (g - y)/B (w = 1 without weights), dz2 = dg W3 (1 - h2^2),
// dz1 = (W2^T dz2)(1 - h1^2).
// work rows: [h1 (64) | h2 (64) | dz1 (64) | dz2 (64) | dg | x (5)]
constexpr int kWorkRow = 4 * kMlpHid + 1 + kMlpIn;

__global__ void __launch_bounds__(NT) backward_kernel(const float* __restrict__ w, const float* __restrict__ x,
                                                      const float* __restrict__ y, const float* __restrict__ wt,
                                                      int64_t n_set, int64_t B, uint64_t seed,
                                                      float* __restrict__ work, float* __restrict__ loss) {
    __shared__ float sw[kMlpParams];
    __shared__ float red[NT];
    load_params(sw, w, nullptr, false);
    float lsum = 0.f;
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < B; b += (int64_t)gridDim.x * blockDim.x) {
        const int64_t idx = seed ? (int64_t)(mix64(seed ^ (uint64_t)b * 0x2545f4914f6cdd1dull) % (uint64_t)n_set) : b;
        float* row = work + b * kWorkRow;
        float* h1 = row;
        float* h2 = row + kMlpHid;
        float* dz1 = row + 2 * kMlpHid;
        float* dz2 = row + 3 * kMlpHid;
        float xi[kMlpIn];
#pragma unroll
        for (int k = 0; k < kMlpIn; ++k) {
            xi[k] = x[idx * kMlpIn + k];
            row[4 * kMlpHid + 1 + k] = xi[k];
        }
        const float g = mlp_eval(sw, xi, h1, h2);
        const float e = g - y[idx];
        const float wi = wt ? wt[idx] : 1.f;
        lsum += wi * e * e;
        const float dg = 2.f * wi * e / (float)B;
        row[4 * kMlpHid] = dg;
        for (int j = 0; j < kMlpHid; ++j) dz2[j] = dg * sw[kMlpOffW3 + j] * (1.f - h2[j] * h2[j]);
        for (int i = 0; i < kMlpHid; ++i) {
            float s = 0.f;
            for (int j = 0; j < kMlpHid; ++j) s = fmaf(sw[kMlpOffW2 + j * kMlpHid + i], dz2[j], s);
            dz1[i] = s * (1.f - h1[i] * h1[i]);
        }
    }
    red[threadIdx.x] = lsum;
    __syncthreads();
    for (int s = NT / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(loss, red[0] / (float)B);
}

// grad[out_off + j*ni + i] += sum_b work[b][aoff + j] * work[b][boff + i]   (i < ni)
// and, for i == ni (bias column), grad[bias_off + j] += sum_b work[b][aoff + j]
__global__ void outer_kernel(const float* __restrict__ work, int64_t B, int aoff, int boff, int ni, int out_off,
                             int bias_off, int64_t chunk, float* __restrict__ grad) {
    const int j = blockIdx.x, i = threadIdx.x;
    if (i > ni) return;
    const int64_t b0 = blockIdx.y * chunk, b1 = min(B, b0 + chunk);
    float s = 0.f;
    for (int64_t b = b0; b < b1; ++b) {
        const float* row = work + b * kWorkRow;
        s = fmaf(row[aoff + j], i < ni ? row[boff + i] : 1.f, s);
    }
    if (i < ni) atomicAdd(grad + out_off + j * ni + i, s);
    else if (bias_off >= 0) atomicAdd(grad + bias_off + j, s);
}

__global__ void adam_kernel(float* __restrict__ w, float* __restrict__ m, float* __restrict__ v,
                            const float* __restrict__ g, int n, float lr, float c1, float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = 0.9f * m[i] + 0.1f * gi;
    const float vi = 0.999f * v[i] + 0.001f * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + 1e-8f);
}

__global__ void to_bf16_kernel(const float* __restrict__ w, __nv_bfloat16* __restrict__ wb, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) wb[i] = __float2bfloat16_rn(w[i]);
}

__global__ void apply_kernel(const double* __restrict__ r, const double* __restrict__ hd, double theta,
                             const float* __restrict__ g, double* __restrict__ t, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double d = hd[i] - theta;
        if (fabs(d) < 1e-8) d = d < 0.0 ? -1e-8 : 1e-8;
        float gi = g[i];
        if (!(gi == gi) || isinf(gi)) gi = 1.f;  // non-finite output: the Jacobi step
        gi = fminf(fmaxf(gi, -10.f), 10.f);
        t[i] = -(double)gi * r[i] / d;
    }
}

// sample k at element i = k * stride: flag, features and target
__global__ void collect_kernel(const double* __restrict__ hd, const double* __restrict__ r,
                               const double* __restrict__ t, double theta, double s, double rmax, int64_t n,
                               int64_t stride, int64_t take, const int64_t* __restrict__ sec_off,
                               const float* __restrict__ sec_q, int nsec, int* __restrict__ flag,
                               float* __restrict__ xs, float* __restrict__ ys, float* __restrict__ ws) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= take) return;
    const int64_t i = k * stride;
    const double d = hd[i] - theta;
    const bool ok = i < n && fabs(r[i]) > 1e-12 * rmax && fabs(d) > 1e-8;
    flag[k] = ok ? 1 : 0;
    if (!ok) return;
    int lo = 0, hi = nsec - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (sec_off[mid] <= i) lo = mid;
        else hi = mid - 1;
    }
    xs[k * kMlpIn + 0] = (float)(d / s);
    xs[k * kMlpIn + 1] = (float)(theta / s);
    xs[k * kMlpIn + 2] = (float)(r[i] / rmax);
    xs[k * kMlpIn + 3] = sec_q[2 * lo];
    xs[k * kMlpIn + 4] = sec_q[2 * lo + 1];
    const double g = -t[i] * d / r[i];
    ys[k] = (float)fmin(fmax(g, -10.0), 10.0);
    // weight of the pair: an error dg in g moves the correction by dg r_i / (H_ii - theta)
    const double q = r[i] / d;
    ws[k] = (float)fmin(q * q, 1e30);
}

__global__ void compact_kernel(const int* __restrict__ pos, const int* __restrict__ flag, int64_t take,
                               const float* __restrict__ xs, const float* __restrict__ ys,
                               const float* __restrict__ ws, float wscale, float* __restrict__ x,
                               float* __restrict__ y, float* __restrict__ w) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= take || !flag[k]) return;
    const int64_t p = pos[k];
    for (int c = 0; c < kMlpIn; ++c) x[p * kMlpIn + c] = xs[k * kMlpIn + c];
    y[p] = ys[k];
    w[p] = ws[k] * wscale;
}

uint64_t mix64_host(uint64_t z) {
    z += 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

__global__ void absmax_kernel(const double* __restrict__ x, double shift, int64_t n, double* __restrict__ part) {
    __shared__ double red[256];
    double m = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        m = fmax(m, fabs(x[i] - shift));
    red[threadIdx.x] = m;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + s]);
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

int grid_n(int64_t n) {
    int64_t g = (n + NT - 1) / NT;
    return (int)std::max<int64_t>(1, std::min<int64_t>(g, 152 * 16));
}

}  // namespace

void Mlp::release() {
    for (void* p : {(void*)d_w, (void*)d_wb, (void*)d_adam, (void*)d_grad, (void*)d_x, (void*)d_y, (void*)d_wt,
                    (void*)d_work, (void*)d_sec_off, (void*)d_sec_q})
        if (p) cudaFree(p);
    d_w = nullptr;
    d_wb = nullptr;
    d_adam = d_grad = d_x = d_y = d_wt = d_work = d_sec_q = nullptr;
    d_sec_off = nullptr;
    n_set = cap_set = cap_work = 0;
    n_sec = 0;
    trained = false;
}

void mlp_init(Mlp& m, uint32_t seed, cudaStream_t st) {
    if (!m.d_w) {
        DMRG_CHECK_CUDA(cudaMalloc(&m.d_w, kMlpParams * sizeof(float)));
        DMRG_CHECK_CUDA(cudaMalloc(&m.d_wb, kMlpParams * sizeof(__nv_bfloat16)));
        DMRG_CHECK_CUDA(cudaMalloc(&m.d_adam, 2 * kMlpParams * sizeof(float)));
        DMRG_CHECK_CUDA(cudaMalloc(&m.d_grad, (kMlpParams + 1) * sizeof(float)));
    }
    // uniform draws from a counter-based generator (splitmix64 of seed and index)
    std::vector<float> w(kMlpParams, 0.f);
    auto u01 = [&](uint64_t i) {
        uint64_t z = ((uint64_t)seed << 32) + i + 0x9e3779b97f4a7c15ull;
        z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
        z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
        z ^= z >> 31;
        return (double)(z >> 11) * (1.0 / 9007199254740992.0);
    };
    const double a1 = 1.0 / std::sqrt((double)kMlpIn), a2 = 1.0 / std::sqrt((double)kMlpHid);
    for (int i = 0; i < kMlpHid * kMlpIn; ++i) w[kMlpOffW1 + i] = (float)(a1 * (2.0 * u01(i) - 1.0));
    for (int i = 0; i < kMlpHid * kMlpHid; ++i) w[kMlpOffW2 + i] = (float)(a2 * (2.0 * u01(1000 + i) - 1.0));
    for (int i = 0; i < kMlpHid; ++i) w[kMlpOffW3 + i] = (float)(1e-2 * (2.0 * u01(9000 + i) - 1.0));
    w[kMlpOffB3] = 1.f;  // g ~ 1: starts as the Jacobi preconditioner
    DMRG_CHECK_CUDA(cudaMemcpyAsync(m.d_w, w.data(), kMlpParams * sizeof(float), cudaMemcpyHostToDevice, st));
    DMRG_CHECK_CUDA(cudaMemsetAsync(m.d_adam, 0, 2 * kMlpParams * sizeof(float), st));
    m.adam_t = 0;
    mlp_publish(m, st);
}

void mlp_features(const Mlp& m, const double* hd, const double* r, double theta, double s, double rmax, int64_t n,
                  float* x, cudaStream_t st) {
    DMRG_REQUIRE(m.d_sec_off && m.n_sec > 0, DMRG_EINVAL, "MLP features need the bond's sector table");
    features_kernel<<<grid_n(n), NT, 0, st>>>(hd, r, theta, s > 0 ? s : 1.0, rmax > 0 ? rmax : 1.0, n, m.d_sec_off,
                                             m.d_sec_q, m.n_sec, x);
    ++launch_counter();
    DMRG_CHECK_CUDA(cudaGetLastError());
}

void mlp_forward(const Mlp& m, const float* x, int64_t n, float* g, bool bf16, cudaStream_t st) {
    if (n <= 0) return;
    forward_kernel<<<grid_n(n), NT, 0, st>>>(m.d_w, m.d_wb, bf16, x, n, g);
    ++launch_counter();
    DMRG_CHECK_CUDA(cudaGetLastError());
}

namespace {
void ensure_work(Mlp& m, int64_t B) {
    if (B <= m.cap_work) return;
    cudaFree(m.d_work);
    m.cap_work = B;
    DMRG_CHECK_CUDA(cudaMalloc(&m.d_work, (size_t)B * kWorkRow * sizeof(float)));
}

void gradient_batch(Mlp& m, const float* x, const float* y, const float* wt, int64_t n_set, int64_t B,
                    uint64_t seed, float* grad, float* loss, cudaStream_t st) {
    ensure_work(m, B);
    DMRG_CHECK_CUDA(cudaMemsetAsync(grad, 0, kMlpParams * sizeof(float), st));
    DMRG_CHECK_CUDA(cudaMemsetAsync(loss, 0, sizeof(float), st));
    backward_kernel<<<grid_n(B), NT, 0, st>>>(m.d_w, x, y, wt, n_set, B, seed, m.d_work, loss);
    const int64_t chunk = 1024;
    const unsigned nch = (unsigned)((B + chunk - 1) / chunk);
    // W3 / b3: dg (column 256) x h2 (columns 64..127)
    outer_kernel<<<dim3(1, nch), kMlpHid + 1, 0, st>>>(m.d_work, B, 4 * kMlpHid, kMlpHid, kMlpHid, kMlpOffW3, kMlpOffB3,
                                                 chunk, grad);
    // W2 / b2: dz2 (192..255) x h1 (0..63)
    outer_kernel<<<dim3(kMlpHid, nch), kMlpHid + 1, 0, st>>>(m.d_work, B, 3 * kMlpHid, 0, kMlpHid, kMlpOffW2,
                                                             kMlpOffB2, chunk, grad);
    // W1 / b1: dz1 (128..191) x x (257..261)
    outer_kernel<<<dim3(kMlpHid, nch), kMlpIn + 1, 0, st>>>(m.d_work, B, 2 * kMlpHid, 4 * kMlpHid + 1, kMlpIn,
                                                            kMlpOffW1, kMlpOffB1, chunk, grad);
    launch_counter() += 4;
    DMRG_CHECK_CUDA(cudaGetLastError());
}
}  // namespace

void mlp_gradient(Mlp& m, const float* x, const float* y, const float* w, int64_t n, float* grad, float* loss,
                  cudaStream_t st) {
    gradient_batch(m, x, y, w, n, n, 0, grad, loss, st);
}

void mlp_adam(Mlp& m, float lr, cudaStream_t st) {
    ++m.adam_t;
    const float c1 = 1.f - std::pow(0.9f, (float)m.adam_t), c2 = 1.f - std::pow(0.999f, (float)m.adam_t);
    adam_kernel<<<(kMlpParams + 255) / 256, 256, 0, st>>>(m.d_w, m.d_adam, m.d_adam + kMlpParams, m.d_grad,
                                                          kMlpParams, lr, c1, c2);
    ++launch_counter();
    DMRG_CHECK_CUDA(cudaGetLastError());
}

void mlp_publish(Mlp& m, cudaStream_t st) {
    to_bf16_kernel<<<(kMlpParams + 255) / 256, 256, 0, st>>>(m.d_w, m.d_wb, kMlpParams);
    ++launch_counter();
    DMRG_CHECK_CUDA(cudaGetLastError());
}

double dev_absmax(const double* x, double shift, int64_t n, double* work, cudaStream_t st) {
    if (n <= 0) return 0.0;
    const int blocks = (int)std::min<int64_t>(512, (n + 255) / 256);
    absmax_kernel<<<blocks, 256, 0, st>>>(x, shift, n, work);
    ++launch_counter();
    std::vector<double> h(blocks);
    DMRG_CHECK_CUDA(cudaMemcpyAsync(h.data(), work, blocks * sizeof(double), cudaMemcpyDeviceToHost, st));
    DMRG_CHECK_CUDA(cudaStreamSynchronize(st));
    double m = 0.0;
    for (double v : h) m = std::max(m, v);
    return m;
}

void mlp_apply(const double* r, const double* hd, double theta, const float* g, double* t, int64_t n,
               cudaStream_t st) {
    apply_kernel<<<grid_n(n), NT, 0, st>>>(r, hd, theta, g, t, n);
    ++launch_counter();
    DMRG_CHECK_CUDA(cudaGetLastError());
}

int64_t mlp_collect(Mlp& m, const double* hd, const double* r, const double* t, double theta, double s, double rmax,
                    int64_t n, int64_t max_take, cudaStream_t st) {
    DMRG_REQUIRE(m.d_sec_off && m.n_sec > 0, DMRG_EINVAL, "MLP pairs need the bond's sector table");
    const int64_t take = std::min<int64_t>(max_take, n);
    if (take <= 0) return 0;
    const int64_t stride = std::max<int64_t>(1, n / take);
    if (m.n_set + take > m.cap_set) {  // grow the set
        const int64_t cap = std::max<int64_t>(2 * m.cap_set, m.n_set + take);
        float *nx = nullptr, *ny = nullptr, *nw = nullptr;
        DMRG_CHECK_CUDA(cudaMalloc(&nx, (size_t)cap * kMlpIn * sizeof(float)));
        DMRG_CHECK_CUDA(cudaMalloc(&ny, (size_t)cap * sizeof(float)));
        DMRG_CHECK_CUDA(cudaMalloc(&nw, (size_t)cap * sizeof(float)));
        if (m.n_set > 0) {
            DMRG_CHECK_CUDA(cudaMemcpyAsync(nx, m.d_x, (size_t)m.n_set * kMlpIn * sizeof(float),
                                            cudaMemcpyDeviceToDevice, st));
            DMRG_CHECK_CUDA(cudaMemcpyAsync(ny, m.d_y, (size_t)m.n_set * sizeof(float), cudaMemcpyDeviceToDevice, st));
            DMRG_CHECK_CUDA(cudaMemcpyAsync(nw, m.d_wt, (size_t)m.n_set * sizeof(float), cudaMemcpyDeviceToDevice, st));
        }
        DMRG_CHECK_CUDA(cudaStreamSynchronize(st));
        cudaFree(m.d_x);
        cudaFree(m.d_y);
        if (m.d_wt) cudaFree(m.d_wt);
        m.d_x = nx;
        m.d_y = ny;
        m.d_wt = nw;
        m.cap_set = cap;
    }
    int* flag = nullptr;
    float *xs = nullptr, *ys = nullptr, *ws = nullptr;
    DMRG_CHECK_CUDA(cudaMalloc(&flag, (size_t)take * 2 * sizeof(int)));
    DMRG_CHECK_CUDA(cudaMalloc(&xs, (size_t)take * (kMlpIn + 2) * sizeof(float)));
    ys = xs + (size_t)take * kMlpIn;
    ws = ys + take;
    const int blocks = (int)((take + NT - 1) / NT);
    collect_kernel<<<blocks, NT, 0, st>>>(hd, r, t, theta, s > 0 ? s : 1.0, rmax > 0 ? rmax : 1.0, n, stride, take,
                                          m.d_sec_off, m.d_sec_q, m.n_sec, flag, xs, ys, ws);
    ++launch_counter();
    std::vector<int> hf(take), pos(take);
    std::vector<float> hw(take);
    DMRG_CHECK_CUDA(cudaMemcpyAsync(hf.data(), flag, take * sizeof(int), cudaMemcpyDeviceToHost, st));
    DMRG_CHECK_CUDA(cudaMemcpyAsync(hw.data(), ws, take * sizeof(float), cudaMemcpyDeviceToHost, st));
    DMRG_CHECK_CUDA(cudaStreamSynchronize(st));
    int64_t cnt = 0;
    double wsum = 0.0;
    for (int64_t k = 0; k < take; ++k) {
        pos[k] = (int)(m.n_set + cnt);
        cnt += hf[k];
        if (hf[k]) wsum += hw[k];
    }
    // every solve's pairs carry weights of mean 1, so each correction equation
    // counts alike whatever the scale of its residual
    const float wscale = (cnt > 0 && wsum > 0.0) ? (float)((double)cnt / wsum) : 1.f;
    DMRG_CHECK_CUDA(cudaMemcpyAsync(flag + take, pos.data(), take * sizeof(int), cudaMemcpyHostToDevice, st));
    compact_kernel<<<blocks, NT, 0, st>>>(flag + take, flag, take, xs, ys, ws, wscale, m.d_x, m.d_y, m.d_wt);
    ++launch_counter();
    DMRG_CHECK_CUDA(cudaStreamSynchronize(st));
    cudaFree(flag);
    cudaFree(xs);
    m.n_set += cnt;
    return cnt;
}

// Training entry used by the C-ABI: epochs over the set in batches of B rows
// drawn by the counter-based generator; returns the first and last batch losses.
void mlp_train(Mlp& m, int steps, int64_t B, float lr, uint64_t seed, float* loss_first, float* loss_last,
               float* held_first, float* held_last, cudaStream_t st) {
    DMRG_REQUIRE(m.n_set > 0, DMRG_EINVAL, "no training pairs collected");
    DMRG_REQUIRE(m.d_w, DMRG_EINVAL, "MLP not initialised");
    float* d_loss = m.d_grad + kMlpParams;
    // the last tenth of the set (the latest solves) is held out of training
    const int64_t n_hold = m.n_set >= 20 ? m.n_set / 10 : 0;
    const int64_t n_train = m.n_set - n_hold;
    auto held = [&](float* out) {
        if (!out) return;
        *out = 0.f;
        if (n_hold == 0) return;
        gradient_batch(m, m.d_x + n_train * kMlpIn, m.d_y + n_train, m.d_wt + n_train, n_hold, n_hold, 0, m.d_grad,
                       d_loss, st);
        DMRG_CHECK_CUDA(cudaMemcpyAsync(out, d_loss, sizeof(float), cudaMemcpyDeviceToHost, st));
        DMRG_CHECK_CUDA(cudaStreamSynchronize(st));
    };
    held(held_first);
    for (int s = 0; s < steps; ++s) {
        gradient_batch(m, m.d_x, m.d_y, m.d_wt, n_train, B, mix64_host(seed + 1 + (uint64_t)s), m.d_grad, d_loss, st);
        if (s == 0 || s == steps - 1) {
            float l = 0.f;
            DMRG_CHECK_CUDA(cudaMemcpyAsync(&l, d_loss, sizeof(float), cudaMemcpyDeviceToHost, st));
            DMRG_CHECK_CUDA(cudaStreamSynchronize(st));
            if (s == 0 && loss_first) *loss_first = l;
            if (s == steps - 1 && loss_last) *loss_last = l;
        }
        mlp_adam(m, lr, st);
    }
    held(held_last);
    mlp_publish(m, st);
    DMRG_CHECK_CUDA(cudaStreamSynchronize(st));
    m.trained = true;
}

}  // namespace dmrg

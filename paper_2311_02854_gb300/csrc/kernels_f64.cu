// FP64 kernels of libdmrg: the segmented grouped GEMM (every block product of
// the sigma step, the renormalisation, the intermediates and the density
// matrices; Sec. 2.2 "GEMM step" with the "reduction" fused into the
// accumulator) and the vector / Jacobi kernels of Davidson and decimation.
#include <cuda_bf16.h>

#include <cmath>

#include "engine.h"

namespace dmrg {

int64_t& launch_counter() {
    static int64_t c = 0;
    return c;
}

// ---------------------------------------------------------------------------
// Work lists
// ---------------------------------------------------------------------------

void WorkList::add_block(int64_t c_off, int c_buf, int m, int n, int ldc, const std::vector<Seg>& s,
                         uint8_t mode, int64_t kchunk, int tile, float alpha) {
    if (m <= 0 || n <= 0) return;
    // split segments into K-chunks (only for atomically accumulated blocks)
    std::vector<std::pair<int, int>> chunks;
    const bool atomic = (mode == TILE_ATOMIC || mode == 2 || mode == 4);
    if (atomic && kchunk > 0) {
        int beg = 0;
        int64_t acc = 0;
        for (int i = 0; i < (int)s.size(); ++i) {
            if (acc > 0 && acc + s[i].k > kchunk) {
                chunks.push_back({beg, i});
                beg = i;
                acc = 0;
            }
            acc += s[i].k;
        }
        chunks.push_back({beg, (int)s.size()});
    } else {
        chunks.push_back({0, (int)s.size()});
    }
    for (auto& ch : chunks) {
        int sb = (int)segs.size();
        for (int i = ch.first; i < ch.second; ++i) {
            segs.push_back(s[i]);
            flops += 2.0 * m * n * (double)s[i].k;
        }
        int se = (int)segs.size();
        const int tm = tile_m > 0 ? tile_m : tile, tn = tile_n > 0 ? tile_n : tile;
        for (int m0 = 0; m0 < m; m0 += tm)
            for (int n0 = 0; n0 < n; n0 += tn) {
                Tile t{};
                t.alpha = alpha;
                t.c_off = c_off;
                t.ldc = ldc;
                t.m = m;
                t.n = n;
                t.m0 = m0;
                t.n0 = n0;
                t.seg_beg = sb;
                t.seg_end = se;
                t.c_buf = (uint8_t)c_buf;
                t.mode = mode;
                tiles.push_back(t);
            }
    }
}

void WorkList::upload(cudaStream_t st) {
    if (tile_m == oz_tile_rows() && tiles.size() > 1) {
        // the tensor-core engine's persistent CTAs take tiles round-robin: longest
        // first (stable counting sort on the stage count), so that short tiles
        // fill in at the end instead of a few long ones trailing
        const int tk = oz_stage_depth();
        std::vector<int> nst(tiles.size());
        int maxn = 0;
        for (size_t i = 0; i < tiles.size(); ++i) {
            int64_t n = 0;
            for (int s = tiles[i].seg_beg; s < tiles[i].seg_end; ++s) n += (segs[s].k + tk - 1) / tk;
            nst[i] = (int)std::min<int64_t>(n, 1 << 20);
            maxn = std::max(maxn, nst[i]);
        }
        std::vector<size_t> pos((size_t)maxn + 2, 0);
        for (int n : nst) ++pos[(size_t)(maxn - n) + 1];
        for (size_t i = 1; i < pos.size(); ++i) pos[i] += pos[i - 1];
        std::vector<Tile> sorted(tiles.size());
        for (size_t i = 0; i < tiles.size(); ++i) sorted[pos[(size_t)(maxn - nst[i])]++] = tiles[i];
        tiles.swap(sorted);
    }
    if (tiles.size() > cap_tiles) {
        if (d_tiles) cudaFree(d_tiles);
        cap_tiles = tiles.size() + tiles.size() / 4 + 16;
        DMRG_CHECK_CUDA(cudaMalloc(&d_tiles, cap_tiles * sizeof(Tile)));
    }
    if (segs.size() > cap_segs) {
        if (d_segs) cudaFree(d_segs);
        cap_segs = segs.size() + segs.size() / 4 + 16;
        DMRG_CHECK_CUDA(cudaMalloc(&d_segs, cap_segs * sizeof(Seg)));
    }
    if (!tiles.empty())
        DMRG_CHECK_CUDA(cudaMemcpyAsync(d_tiles, tiles.data(), tiles.size() * sizeof(Tile),
                                        cudaMemcpyHostToDevice, st));
    if (!segs.empty())
        DMRG_CHECK_CUDA(cudaMemcpyAsync(d_segs, segs.data(), segs.size() * sizeof(Seg),
                                        cudaMemcpyHostToDevice, st));
}

void WorkList::release() {
    if (d_tiles) cudaFree(d_tiles);
    if (d_segs) cudaFree(d_segs);
    d_tiles = nullptr;
    d_segs = nullptr;
    cap_tiles = cap_segs = 0;
}

// ---------------------------------------------------------------------------
// Segmented grouped GEMM, FP64 (64x64 tile, 256 threads, 4x4 per thread)
// ---------------------------------------------------------------------------

namespace {
constexpr int BM = 64, BN = 64, BK = 16, NT = 256;

// element idx of buffer buf (FP64, or bf16 pieces read as hi + lo)
__device__ __forceinline__ double ld_elem(const BufTable& bt, int buf, int64_t idx) {
    if (bt.pmask & (1u << buf)) {
        const __nv_bfloat16* h = (const __nv_bfloat16*)bt.p[buf];
        double x = (double)__bfloat162float(h[idx]);
        if (bt.lo[buf]) {
            const __nv_bfloat16* l = (const __nv_bfloat16*)bt.lo[buf];
            x += (double)__bfloat162float(l[idx]);
            if (bt.pstride[buf]) x += (double)__bfloat162float(l[bt.pstride[buf] + idx]);
        }
        return x;
    }
    return bt.p[buf][idx];
}

__global__ void __launch_bounds__(NT) seg_gemm_f64_kernel(const Tile* __restrict__ tiles,
                                                          const Seg* __restrict__ segs, BufTable bt) {
    const Tile T = tiles[blockIdx.x];
    const int v = blockIdx.y;
    __shared__ double As[BK][BM + 1];
    __shared__ double Bs[BK][BN + 1];
    const int tid = threadIdx.x;
    const int tx = tid % 16, ty = tid / 16;
    double acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
    const int mrem = T.m - T.m0, nrem = T.n - T.n0;
    for (int s = T.seg_beg; s < T.seg_end; ++s) {
        const Seg S = segs[s];
        int64_t A = S.a_off + (int64_t)v * bt.vstride[S.a_buf];
        int64_t B = S.b_off + (int64_t)v * bt.vstride[S.b_buf];
        A += S.a_tr ? (int64_t)T.m0 : (int64_t)T.m0 * S.lda;
        B += S.b_tr ? (int64_t)T.n0 * S.ldb : (int64_t)T.n0;
        for (int k0 = 0; k0 < S.k; k0 += BK) {
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                int m, kk;
                if (!S.a_tr) {
                    kk = tid % BK;
                    m = tid / BK + 16 * i;
                } else {
                    m = tid % BM;
                    kk = tid / BM + 4 * i;
                }
                double x = 0.0;
                if (m < mrem && k0 + kk < S.k)
                    x = ld_elem(bt, S.a_buf,
                                A + (S.a_tr ? (int64_t)(k0 + kk) * S.lda + m : (int64_t)m * S.lda + k0 + kk));
                As[kk][m] = x * S.alpha;
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                int n, kk;
                if (!S.b_tr) {
                    n = tid % BN;
                    kk = tid / BN + 4 * i;
                } else {
                    kk = tid % BK;
                    n = tid / BK + 16 * i;
                }
                double x = 0.0;
                if (n < nrem && k0 + kk < S.k)
                    x = ld_elem(bt, S.b_buf,
                                B + (S.b_tr ? (int64_t)n * S.ldb + k0 + kk : (int64_t)(k0 + kk) * S.ldb + n));
                Bs[kk][n] = x;
            }
            __syncthreads();
#pragma unroll
            for (int kk = 0; kk < BK; ++kk) {
                double a[4], b[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
                for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
            }
            __syncthreads();
        }
    }
    double* C = bt.p[T.c_buf] + T.c_off + (int64_t)v * bt.vstride[T.c_buf];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int r = T.m0 + ty + 16 * i;
        if (r >= T.m) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int c = T.n0 + tx + 16 * j;
            if (c >= T.n) continue;
            double* dst = C + (int64_t)r * T.ldc + c;
            if (T.mode == TILE_ATOMIC)
                atomicAdd(dst, acc[i][j]);
            else
                *dst = acc[i][j];
        }
    }
}
// The same product for lists whose segments all have K = 1 (rank-1 updates,
// e.g. the diagonal of H_eff as sums of diag(O_L) diag(O_R)^T): each thread
// reads its 4 + 4 operand elements straight from global memory (they stay in
// L1 across the segments of a tile), no shared-memory staging or barriers.
// Same accumulation order per element as seg_gemm_f64_kernel.
__global__ void __launch_bounds__(NT) seg_outer_f64_kernel(const Tile* __restrict__ tiles,
                                                           const Seg* __restrict__ segs, BufTable bt) {
    const Tile T = tiles[blockIdx.x];
    const int v = blockIdx.y;
    const int tid = threadIdx.x;
    const int tx = tid % 16, ty = tid / 16;
    double acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
    const int mrem = T.m - T.m0, nrem = T.n - T.n0;
    for (int s = T.seg_beg; s < T.seg_end; ++s) {
        const Seg S = segs[s];
        int64_t A = S.a_off + (int64_t)v * bt.vstride[S.a_buf];
        int64_t B = S.b_off + (int64_t)v * bt.vstride[S.b_buf];
        A += S.a_tr ? (int64_t)T.m0 : (int64_t)T.m0 * S.lda;
        B += S.b_tr ? (int64_t)T.n0 * S.ldb : (int64_t)T.n0;
        double a[4], b[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int m = ty + 16 * i;
            a[i] = m < mrem ? ld_elem(bt, S.a_buf, A + (S.a_tr ? (int64_t)m : (int64_t)m * S.lda)) * S.alpha : 0.0;
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int n = tx + 16 * j;
            b[j] = n < nrem ? ld_elem(bt, S.b_buf, B + (S.b_tr ? (int64_t)n * S.ldb : (int64_t)n)) : 0.0;
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    double* C = bt.p[T.c_buf] + T.c_off + (int64_t)v * bt.vstride[T.c_buf];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int r = T.m0 + ty + 16 * i;
        if (r >= T.m) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int c = T.n0 + tx + 16 * j;
            if (c >= T.n) continue;
            double* dst = C + (int64_t)r * T.ldc + c;
            if (T.mode == TILE_ATOMIC)
                atomicAdd(dst, acc[i][j]);
            else
                *dst = acc[i][j];
        }
    }
}
}  // namespace

void launch_seg_gemm_f64(const WorkList& w, const BufTable& bt, int nvec, cudaStream_t st) {
    if (w.tiles.empty()) return;
    if (w.tile_m == oz_tile_rows() && !w.rank1) {
        launch_seg_gemm_oz(w, bt, nvec, oz_error_word(), st);
        return;
    }
    DMRG_REQUIRE(w.tile_m == 0 || w.tile_m == BM, DMRG_EINVAL, "work list tile shape not runnable on the FP64 engine");
    const int64_t n = (int64_t)w.tiles.size();
    const int64_t maxg = 2147483647LL;
    DMRG_REQUIRE(n <= maxg && nvec <= 65535, DMRG_EINVAL, "work list too large for one launch");
    dim3 grid((unsigned)n, (unsigned)nvec);
    if (w.rank1)
        seg_outer_f64_kernel<<<grid, NT, 0, st>>>(w.d_tiles, w.d_segs, bt);
    else
        seg_gemm_f64_kernel<<<grid, NT, 0, st>>>(w.d_tiles, w.d_segs, bt);
    ++launch_counter();
    DMRG_CHECK_CUDA(cudaGetLastError());
}

void launch_seg_gemm_f64_lists(const Tile* d_tiles, int64_t ntiles, const Seg* d_segs, const BufTable& bt,
                               cudaStream_t st) {
    if (ntiles <= 0) return;
    DMRG_REQUIRE(ntiles <= 2147483647LL, DMRG_EINVAL, "work list too large for one launch");
    seg_gemm_f64_kernel<<<dim3((unsigned)ntiles, 1), NT, 0, st>>>(d_tiles, d_segs, bt);
    ++launch_counter();
    DMRG_CHECK_CUDA(cudaGetLastError());
}

// ---------------------------------------------------------------------------
// Vector kernels
// ---------------------------------------------------------------------------

namespace {

__device__ double block_sum(double x, double* sh) {
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[wid] = x;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += sh[i];
    return t;  // valid in thread 0
}

__global__ void dots_stage1(const double* __restrict__ X, int64_t ldx, const double* __restrict__ y,
                            int64_t n, double* __restrict__ part, int nblk) {
    __shared__ double sh[32];
    const int i = blockIdx.y;
    double acc = 0.0;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)nblk * blockDim.x)
        acc = fma(X[(int64_t)i * ldx + k], y[k], acc);
    double t = block_sum(acc, sh);
    if (threadIdx.x == 0) part[(int64_t)i * nblk + blockIdx.x] = t;
}

__global__ void dots_stage2(const double* __restrict__ part, int nblk, double* __restrict__ out) {
    __shared__ double sh[32];
    const int i = blockIdx.x;
    double acc = 0.0;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) acc += part[(int64_t)i * nblk + b];
    double t = block_sum(acc, sh);
    if (threadIdx.x == 0) out[i] = t;
}

__global__ void combine_kernel(const double* __restrict__ X, int64_t ldx, int m, const double* __restrict__ c,
                               int64_t n, double* __restrict__ y) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int i = 0; i < m; ++i) acc = fma(c[i], X[(int64_t)i * ldx + k], acc);
        y[k] = acc;
    }
}

__global__ void axpby_kernel(double a, const double* __restrict__ x, double b, double* __restrict__ y, int64_t n) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        y[k] = a * x[k] + b * y[k];
}

__global__ void precond_kernel(const double* __restrict__ r, const double* __restrict__ d, double theta,
                               double* __restrict__ t, int64_t n) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        double den = d[k] - theta;
        if (fabs(den) < 1e-8) den = (den < 0.0) ? -1e-8 : 1e-8;
        t[k] = -r[k] / den;
    }
}

__global__ void fill_kernel(double* x, double v, int64_t n) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        x[k] = v;
}

__global__ void perturb_kernel(double* x, int64_t n, uint32_t seed, double amp) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        uint32_t h = (uint32_t)k * 2654435761u ^ (seed * 2246822519u);
        h ^= h >> 15;
        h *= 2246822519u;
        h ^= h >> 13;
        h *= 3266489917u;
        h ^= h >> 16;
        x[k] += amp * ((double)h * (1.0 / 4294967296.0) - 0.5);
    }
}

__global__ void identity_kernel(double* x, int n) {
    const int64_t nn = (int64_t)n * n;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nn; k += (int64_t)gridDim.x * blockDim.x)
        x[k] = (k / n == k % n) ? 1.0 : 0.0;
}

int grid_for(int64_t n, int threads = 256) {
    int64_t g = (n + threads - 1) / threads;
    if (g > 152 * 32) g = 152 * 32;
    return (int)(g < 1 ? 1 : g);
}

}  // namespace

void dev_dots(const double* X, int64_t ldx, int m, const double* y, int64_t n, double* out, double* work,
              cudaStream_t st) {
    if (m <= 0) return;
    int nblk = (int)((n + 256 * 8 - 1) / (256 * 8));
    if (nblk > 256) nblk = 256;
    if (nblk < 1) nblk = 1;
    dots_stage1<<<dim3(nblk, m), 256, 0, st>>>(X, ldx, y, n, work, nblk);
    dots_stage2<<<m, 256, 0, st>>>(work, nblk, out);
    launch_counter() += 2;
    DMRG_CHECK_CUDA(cudaGetLastError());
}

void dev_combine(const double* X, int64_t ldx, int m, const double* c, int64_t n, double* y, cudaStream_t st) {
    combine_kernel<<<grid_for(n), 256, 0, st>>>(X, ldx, m, c, n, y);
    ++launch_counter();
    DMRG_CHECK_CUDA(cudaGetLastError());
}

void dev_axpby(double a, const double* x, double b, double* y, int64_t n, cudaStream_t st) {
    axpby_kernel<<<grid_for(n), 256, 0, st>>>(a, x, b, y, n);
    ++launch_counter();
    DMRG_CHECK_CUDA(cudaGetLastError());
}

void dev_jacobi_precond(const double* r, const double* d, double theta, double* t, int64_t n, cudaStream_t st) {
    precond_kernel<<<grid_for(n), 256, 0, st>>>(r, d, theta, t, n);
    ++launch_counter();
    DMRG_CHECK_CUDA(cudaGetLastError());
}

void dev_fill(double* x, double v, int64_t n, cudaStream_t st) {
    if (n <= 0) return;
    fill_kernel<<<grid_for(n), 256, 0, st>>>(x, v, n);
    ++launch_counter();
    DMRG_CHECK_CUDA(cudaGetLastError());
}

void dev_perturb(double* x, int64_t n, uint32_t seed, double amp, cudaStream_t st) {
    perturb_kernel<<<grid_for(n), 256, 0, st>>>(x, n, seed, amp);
    ++launch_counter();
    DMRG_CHECK_CUDA(cudaGetLastError());
}

void dev_identity(double* x, int n, cudaStream_t st) {
    identity_kernel<<<grid_for((int64_t)n * n), 256, 0, st>>>(x, n);
    ++launch_counter();
    DMRG_CHECK_CUDA(cudaGetLastError());
}

// ---------------------------------------------------------------------------
// Batched cyclic Jacobi eigensolver (round-robin ordering), one CTA per matrix
// (Golub & Van Loan, Alg. 8.4.3 with parallel ordering).
// ---------------------------------------------------------------------------

namespace {
constexpr int kJacThreads = 512;

__global__ void __launch_bounds__(kJacThreads) jacobi_eigh_kernel(const EigJob* __restrict__ jobs, int max_sweeps) {
    const EigJob J = jobs[blockIdx.x];
    const int n = J.n, lda = J.lda;
    double* __restrict__ A = J.A;
    double* __restrict__ V = J.V;
    extern __shared__ double sm[];
    const int ne = n + (n & 1);
    const int np = ne / 2;
    double* cs = sm;            // np
    double* sn = sm + np;       // np
    int* pp = (int*)(sm + 2 * np);
    int* qq = pp + np;
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int64_t idx = tid; idx < (int64_t)n * n; idx += nt) {
        int i = (int)(idx / n), j = (int)(idx % n);
        V[(int64_t)i * lda + j] = (i == j) ? 1.0 : 0.0;
    }
    __syncthreads();
    if (n <= 1) {
        if (tid == 0 && n == 1) J.w[0] = A[0];
        return;
    }
    // threshold Jacobi: a pair is rotated only if |a_pq| > eps * sqrt(|a_pp a_qq|)
    // (relative accuracy of small eigenvalues); stop after a sweep without rotations
    __shared__ int rotated;
    for (int sweep = 0; sweep < max_sweeps; ++sweep) {
        if (tid == 0) rotated = 0;
        __syncthreads();
        for (int r = 0; r < ne - 1; ++r) {
            for (int t = tid; t < np; t += nt) {
                int a, b;
                if (t == 0) {
                    a = r % (ne - 1);
                    b = ne - 1;
                } else {
                    a = (r + t) % (ne - 1);
                    b = (r + ne - 1 - t) % (ne - 1);
                }
                int p = a < b ? a : b, q = a < b ? b : a;
                double c = 1.0, s = 0.0;
                if (q < n) {
                    const double apq = A[(int64_t)p * lda + q];
                    const double app = A[(int64_t)p * lda + p], aqq = A[(int64_t)q * lda + q];
                    if (fabs(apq) > 1e-15 * sqrt(fabs(app * aqq)) && fabs(apq) > 1e-300) {
                        double tau = (aqq - app) / (2.0 * apq);
                        double tt = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                        c = 1.0 / sqrt(1.0 + tt * tt);
                        s = tt * c;
                        rotated = 1;
                    }
                }
                cs[t] = c;
                sn[t] = s;
                pp[t] = p;
                qq[t] = (q < n) ? q : -1;
            }
            __syncthreads();
            // rows: A <- J^T A
            for (int64_t idx = tid; idx < (int64_t)np * n; idx += nt) {
                int t = (int)(idx / n), k = (int)(idx % n);
                int q = qq[t];
                double s = sn[t];
                if (q < 0 || s == 0.0) continue;
                int p = pp[t];
                double c = cs[t];
                double x = A[(int64_t)p * lda + k], y = A[(int64_t)q * lda + k];
                A[(int64_t)p * lda + k] = c * x - s * y;
                A[(int64_t)q * lda + k] = s * x + c * y;
            }
            __syncthreads();
            // columns: A <- A J, V <- V J
            for (int64_t idx = tid; idx < (int64_t)np * n; idx += nt) {
                int t = (int)(idx / n), k = (int)(idx % n);
                int q = qq[t];
                double s = sn[t];
                if (q < 0 || s == 0.0) continue;
                int p = pp[t];
                double c = cs[t];
                double x = A[(int64_t)k * lda + p], y = A[(int64_t)k * lda + q];
                A[(int64_t)k * lda + p] = c * x - s * y;
                A[(int64_t)k * lda + q] = s * x + c * y;
                x = V[(int64_t)k * lda + p];
                y = V[(int64_t)k * lda + q];
                V[(int64_t)k * lda + p] = c * x - s * y;
                V[(int64_t)k * lda + q] = s * x + c * y;
            }
            __syncthreads();
        }
        if (!rotated) break;
        __syncthreads();
    }
    for (int i = tid; i < n; i += nt) J.w[i] = A[(int64_t)i * lda + i];
}
}  // namespace

void dev_jacobi_eigh_batched(const EigJob* d_jobs, int njobs, int max_sweeps, cudaStream_t st) {
    if (njobs <= 0) return;
    // shared memory sized for matrices up to 4096
    const int maxn = 4096;
    size_t smem = (size_t)(maxn / 2) * (2 * sizeof(double) + 2 * sizeof(int));
    static bool attr = false;
    if (!attr) {
        DMRG_CHECK_CUDA(cudaFuncSetAttribute(jacobi_eigh_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem));
        attr = true;
    }
    jacobi_eigh_kernel<<<njobs, kJacThreads, smem, st>>>(d_jobs, max_sweeps);
    ++launch_counter();
    DMRG_CHECK_CUDA(cudaGetLastError());
}

}  // namespace dmrg

// Block Jacobi eigensolver for the reduced density matrices of the
// decimation step (Sec. 2.1).
//
// Each matrix is padded to a multiple of BB and cut into BB x BB blocks.  A
// sweep pairs the blocks round-robin; in every round each pair (I, J) has its
// 2BB x 2BB diagonal subproblem diagonalised approximately (cyclic Jacobi
// sweeps in shared memory, giving an orthogonal Q), after which A <- Q^T A Q
// and V <- V Q are applied to the block rows and columns I, J as 2BB-wide
// products by many CTAs.  Traffic per sweep is O(n^3 / BB) instead of the
// O(n^3) of the element-wise Jacobi, and a round keeps nb/2 x n/(2BB) CTAs
// busy instead of one.  Rotations below an absolute floor (a small multiple
// of |A|) are skipped: they cannot change any eigenvalue by more than the
// rounding error of the FP64 result.
#include <algorithm>
#include <cmath>

#include "eig.h"

namespace dmrg {
namespace {

constexpr int BB = 32;      // block size
constexpr int SB = 2 * BB;  // subproblem size
constexpr int LD = SB + 1;  // padded shared-memory row
constexpr int NT = 256;
// two-stage solve (FP32 sweeps, then FP64) for batches whose largest matrix has
// at least this many rows; FP32 stage: stop at off/|A| <= kTol32, when a sweep
// below off/|A| = kStallFrom32 no longer halves it, or after kMaxSweeps32 sweeps
constexpr int kTwoStageMin = 256;
constexpr double kTol32 = 1e-5, kStall32 = 0.5, kStallFrom32 = 1e-3;
constexpr int kMaxSweeps32 = 30;
// FP64 sweeps: below off/|A| = kStallFrom64 a sweep that does not halve it ends
// the solve (the rounding floor of a large matrix lies near 1e-14 .. 1e-13)
constexpr double kStall64 = 0.5, kStallFrom64 = 1e-10;
// two-stage FP64 sweeps: couplings between two states below kTau |A|_F are
// left alone (they only mix weights no truncation can keep)
constexpr double kTau = 1e-12;
// cyclic sweeps at most per 2BB x 2BB subproblem (FP32 stage, FP64 sweeps).
// One: solving the subproblems further (3 / 4 sweeps) made the K = 73
// decimations slower (more outer FP64 sweeps, 2.1 -> 3.2 s per call)
constexpr int kInner32 = 1, kInner64 = 1;

template <typename T>
struct BJMat {
    T* A;  // n x n, padded copy
    T* V;  // n x n
    int n, nb;
    double floor;
    // pairs whose two diagonal entries are both below tau are neither rotated
    // nor counted in off(A): states that far below every kept weight may stay
    // mixed among themselves (0: every pair counts)
    double tau;
};

// rotations whose |a_pq| is below this multiple of sqrt|a_pp a_qq| are skipped
// (the rounding level of the arithmetic type)
template <typename T>
struct RelSkip;
template <>
struct RelSkip<double> {
    static constexpr double v = 1e-15;
};
template <>
struct RelSkip<float> {
    static constexpr double v = 1e-7;
};

// pair t of round r among ne (even) players, a < b
__device__ __forceinline__ void rr_pair(int r, int t, int ne, int& a, int& b) {
    int x, y;
    if (t == 0) {
        x = r % (ne - 1);
        y = ne - 1;
    } else {
        x = (r + t) % (ne - 1);
        y = (r + ne - 1 - t) % (ne - 1);
    }
    a = min(x, y);
    b = max(x, y);
}

// matrix of a batched job index: jobs of matrix g are [job_off[g], job_off[g+1])
__device__ __forceinline__ int find_mat(const int* job_off, int nmat, int job) {
    int lo = 0, hi = nmat - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (job_off[mid] <= job) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

template <typename T>
struct PairRef {
    BJMat<T> M;
    int I, J;
    bool live;
};

template <typename T>
__device__ __forceinline__ PairRef<T> pair_of(const BJMat<T>* mats, const int* job_off, int nmat, int round, int job) {
    PairRef<T> r;
    const int g = find_mat(job_off, nmat, job);
    r.M = mats[g];
    const int ne = r.M.nb + (r.M.nb & 1);
    rr_pair(round % (ne - 1), job - job_off[g], ne, r.I, r.J);
    r.live = r.J < r.M.nb;  // J == nb: the padding player of an odd block count
    return r;
}

// global index of row a (0 <= a < SB) of the pair's subproblem
template <typename T>
__device__ __forceinline__ int sub_index(const PairRef<T>& p, int a) {
    return a < BB ? p.I * BB + a : p.J * BB + a - BB;
}

// Q of each job (SB x SB, row-major) from cyclic Jacobi sweeps over its
// subproblem: up to max_inner sweeps, fewer once a sweep rotates nothing
template <typename T>
__global__ void __launch_bounds__(NT) bj_solve(const BJMat<T>* __restrict__ mats, const int* __restrict__ job_off,
                                              int nmat, int round, T* __restrict__ Qall, int max_inner) {
    extern __shared__ __align__(16) unsigned char sm_raw[];
    T* S = reinterpret_cast<T*>(sm_raw);  // SB x LD
    T* Qs = S + SB * LD;                   // SB x LD
    __shared__ T cs[BB], sn[BB];
    __shared__ int pp[BB], qq[BB];
    __shared__ int rotated;
    const PairRef<T> pr = pair_of(mats, job_off, nmat, round, blockIdx.x);
    T* Q = Qall + (int64_t)blockIdx.x * SB * SB;
    const int tid = threadIdx.x;
    for (int e = tid; e < SB * SB; e += NT) {
        const int a = e / SB, b = e % SB;
        S[a * LD + b] = pr.live ? pr.M.A[(int64_t)sub_index(pr, a) * pr.M.n + sub_index(pr, b)] : T(0);
        Qs[a * LD + b] = (a == b) ? T(1) : T(0);
    }
    __syncthreads();
    for (int sw = 0; pr.live && sw < max_inner; ++sw) {
        if (tid == 0) rotated = 0;
        __syncthreads();
        for (int r = 0; r < SB - 1; ++r) {
            if (tid < BB) {
                int p, q;
                rr_pair(r, tid, SB, p, q);
                T c = T(1), s = T(0);
                const T apq = S[p * LD + q], app = S[p * LD + p], aqq = S[q * LD + q];
                if (fabs((double)apq) > pr.M.floor &&
                    fabs((double)apq) > RelSkip<T>::v * sqrt(fabs((double)app * (double)aqq)) &&
                    (fabs((double)app) >= pr.M.tau || fabs((double)aqq) >= pr.M.tau)) {
                    const T tau = (aqq - app) / (T(2) * apq);
                    const T t = (tau >= T(0) ? T(1) : T(-1)) / (fabs(tau) + sqrt(T(1) + tau * tau));
                    c = T(1) / sqrt(T(1) + t * t);
                    s = t * c;
                    if (s != T(0)) rotated = 1;
                }
                cs[tid] = c;
                sn[tid] = s;
                pp[tid] = p;
                qq[tid] = q;
            }
            __syncthreads();
            for (int e = tid; e < BB * SB; e += NT) {  // rows p, q of S
                const int u = e / SB, k = e % SB;
                const T s = sn[u];
                if (s == T(0)) continue;
                const int p = pp[u], q = qq[u];
                const T c = cs[u], x = S[p * LD + k], y = S[q * LD + k];
                S[p * LD + k] = c * x - s * y;
                S[q * LD + k] = s * x + c * y;
            }
            __syncthreads();
            for (int e = tid; e < BB * SB; e += NT) {  // columns p, q of S and Q
                const int u = e / SB, k = e % SB;
                const T s = sn[u];
                if (s == T(0)) continue;
                const int p = pp[u], q = qq[u];
                const T c = cs[u];
                T x = S[k * LD + p], y = S[k * LD + q];
                S[k * LD + p] = c * x - s * y;
                S[k * LD + q] = s * x + c * y;
                x = Qs[k * LD + p];
                y = Qs[k * LD + q];
                Qs[k * LD + p] = c * x - s * y;
                Qs[k * LD + q] = s * x + c * y;
            }
            __syncthreads();
        }
        const int any = rotated;  // read by every thread before the next reset
        __syncthreads();
        if (!any) break;
    }
    for (int e = tid; e < SB * SB; e += NT) Q[e] = Qs[(e / SB) * LD + e % SB];
}

// A[rows I u J, column tile] <- Q^T A[rows I u J, column tile]; one CTA per (job, tile)
template <typename T>
__global__ void __launch_bounds__(NT) bj_rows(const BJMat<T>* __restrict__ mats, const int* __restrict__ job_off,
                                             int nmat, int round, const T* __restrict__ Qall, int ntile) {
    extern __shared__ __align__(16) unsigned char sm_raw[];
    T* Qs = reinterpret_cast<T*>(sm_raw);
    T* As = Qs + SB * LD;
    const int job = blockIdx.x / ntile, tile = blockIdx.x % ntile;
    const PairRef<T> pr = pair_of(mats, job_off, nmat, round, job);
    if (!pr.live || tile * SB >= pr.M.n) return;
    const T* Q = Qall + (int64_t)job * SB * SB;
    const int n = pr.M.n, tid = threadIdx.x;
    for (int e = tid; e < SB * SB; e += NT) {
        const int a = e / SB, b = e % SB, col = tile * SB + b;
        Qs[a * LD + b] = Q[e];
        As[a * LD + b] = (col < n) ? pr.M.A[(int64_t)sub_index(pr, a) * n + col] : T(0);
    }
    __syncthreads();
    // 4 x 4 outputs per thread (rows ty + 16u, columns tx + 16w): 16 independent
    // FMA chains and 8 shared loads per 16 FMAs
    const int ty = tid / 16, tx = tid % 16;
    T acc[4][4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int w = 0; w < 4; ++w) acc[u][w] = T(0);
#pragma unroll 4
    for (int k = 0; k < SB; ++k) {
        T qa[4], ab[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            qa[u] = Qs[k * LD + ty + 16 * u];
            ab[u] = As[k * LD + tx + 16 * u];
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int w = 0; w < 4; ++w) acc[u][w] = fma(qa[u], ab[w], acc[u][w]);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            const int a = ty + 16 * u, col = tile * SB + tx + 16 * w;
            if (col < n) pr.M.A[(int64_t)sub_index(pr, a) * n + col] = acc[u][w];
        }
}

// Double-float arithmetic for the FP64 sweeps of large matrices: GB300's FP32
// units run ~64x its FP64 rate, and a pair (h, l) of floats with x = h + l
// carries ~48 significant bits.  Products by Dekker's splitting through fma
// (TwoProd), sums by Knuth's TwoSum; the _rn intrinsics keep the compiler
// from contracting the error-free steps into fused operations.
struct F2 {
    float h, l;
};
__device__ __forceinline__ F2 f2_split(double x) {
    const float h = (float)x;
    return {h, (float)(x - (double)h)};
}
__device__ __forceinline__ double f2_join(F2 a) { return (double)a.h + (double)a.l; }
// acc += a * b
__device__ __forceinline__ void f2_fma(F2& acc, F2 a, F2 b) {
    const float p = __fmul_rn(a.h, b.h);
    float e = fmaf(a.h, b.h, -p);
    e = fmaf(a.h, b.l, e);
    e = fmaf(a.l, b.h, e);
    const float s = __fadd_rn(acc.h, p);
    const float v = __fsub_rn(s, acc.h);
    const float t = __fadd_rn(__fsub_rn(acc.h, __fsub_rn(s, v)), __fsub_rn(p, v));
    const float lo = __fadd_rn(__fadd_rn(t, e), acc.l);
    const float hi = __fadd_rn(s, lo);
    acc.l = __fsub_rn(lo, __fsub_rn(hi, s));
    acc.h = hi;
}

// bj_rows for FP64 matrices in double-float arithmetic (same tiling)
__global__ void __launch_bounds__(NT) bj_rows_df(const BJMat<double>* __restrict__ mats,
                                                 const int* __restrict__ job_off, int nmat, int round,
                                                 const double* __restrict__ Qall, int ntile) {
    extern __shared__ __align__(16) unsigned char sm_raw[];
    F2* Qs = reinterpret_cast<F2*>(sm_raw);
    F2* As = Qs + SB * LD;
    const int job = blockIdx.x / ntile, tile = blockIdx.x % ntile;
    const PairRef<double> pr = pair_of(mats, job_off, nmat, round, job);
    if (!pr.live || tile * SB >= pr.M.n) return;
    const double* Q = Qall + (int64_t)job * SB * SB;
    const int n = pr.M.n, tid = threadIdx.x;
    for (int e = tid; e < SB * SB; e += NT) {
        const int a = e / SB, b = e % SB, col = tile * SB + b;
        Qs[a * LD + b] = f2_split(Q[e]);
        As[a * LD + b] = f2_split((col < n) ? pr.M.A[(int64_t)sub_index(pr, a) * n + col] : 0.0);
    }
    __syncthreads();
    const int ty = tid / 16, tx = tid % 16;
    F2 acc[4][4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int w = 0; w < 4; ++w) acc[u][w] = {0.f, 0.f};
#pragma unroll 2
    for (int k = 0; k < SB; ++k) {
        F2 qa[4], ab[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            qa[u] = Qs[k * LD + ty + 16 * u];
            ab[u] = As[k * LD + tx + 16 * u];
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int w = 0; w < 4; ++w) f2_fma(acc[u][w], qa[u], ab[w]);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            const int a = ty + 16 * u, col = tile * SB + tx + 16 * w;
            if (col < n) pr.M.A[(int64_t)sub_index(pr, a) * n + col] = f2_join(acc[u][w]);
        }
}

// bj_cols for FP64 matrices in double-float arithmetic (same tiling)
__global__ void __launch_bounds__(NT) bj_cols_df(const BJMat<double>* __restrict__ mats,
                                                 const int* __restrict__ job_off, int nmat, int round,
                                                 const double* __restrict__ Qall, int ntile) {
    extern __shared__ __align__(16) unsigned char sm_raw[];
    F2* Qs = reinterpret_cast<F2*>(sm_raw);
    F2* As = Qs + SB * LD;
    const int job = blockIdx.x / ntile, tile = blockIdx.x % ntile;
    const PairRef<double> pr = pair_of(mats, job_off, nmat, round, job);
    if (!pr.live || tile * SB >= pr.M.n) return;
    const double* Q = Qall + (int64_t)job * SB * SB;
    const int n = pr.M.n, tid = threadIdx.x;
    for (int e = tid; e < SB * SB; e += NT) Qs[(e / SB) * LD + e % SB] = f2_split(Q[e]);
    for (int which = 0; which < 2; ++which) {
        double* X = which ? pr.M.V : pr.M.A;
        for (int e = tid; e < SB * SB; e += NT) {
            const int a = e / SB, b = e % SB, row = tile * SB + a;
            As[a * LD + b] = f2_split((row < n) ? X[(int64_t)row * n + sub_index(pr, b)] : 0.0);
        }
        __syncthreads();
        const int ty = tid / 16, tx = tid % 16;
        F2 acc[4][4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int w = 0; w < 4; ++w) acc[u][w] = {0.f, 0.f};
#pragma unroll 2
        for (int k = 0; k < SB; ++k) {
            F2 xa[4], qb[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                xa[u] = As[(ty + 16 * u) * LD + k];
                qb[u] = Qs[k * LD + tx + 16 * u];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int w = 0; w < 4; ++w) f2_fma(acc[u][w], xa[u], qb[w]);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int w = 0; w < 4; ++w) {
                const int row = tile * SB + ty + 16 * u;
                if (row < n) X[(int64_t)row * n + sub_index(pr, tx + 16 * w)] = f2_join(acc[u][w]);
            }
        __syncthreads();
    }
}

// X[row tile, columns I u J] <- X[row tile, columns I u J] Q for X = A, then X = V
template <typename T>
__global__ void __launch_bounds__(NT) bj_cols(const BJMat<T>* __restrict__ mats, const int* __restrict__ job_off,
                                             int nmat, int round, const T* __restrict__ Qall, int ntile) {
    extern __shared__ __align__(16) unsigned char sm_raw[];
    T* Qs = reinterpret_cast<T*>(sm_raw);
    T* As = Qs + SB * LD;
    const int job = blockIdx.x / ntile, tile = blockIdx.x % ntile;
    const PairRef<T> pr = pair_of(mats, job_off, nmat, round, job);
    if (!pr.live || tile * SB >= pr.M.n) return;
    const T* Q = Qall + (int64_t)job * SB * SB;
    const int n = pr.M.n, tid = threadIdx.x;
    for (int e = tid; e < SB * SB; e += NT) Qs[(e / SB) * LD + e % SB] = Q[e];
    for (int which = 0; which < 2; ++which) {
        T* X = which ? pr.M.V : pr.M.A;
        for (int e = tid; e < SB * SB; e += NT) {
            const int a = e / SB, b = e % SB, row = tile * SB + a;
            As[a * LD + b] = (row < n) ? X[(int64_t)row * n + sub_index(pr, b)] : T(0);
        }
        __syncthreads();
        // 4 x 4 outputs per thread, as in bj_rows
        const int ty = tid / 16, tx = tid % 16;
        T acc[4][4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int w = 0; w < 4; ++w) acc[u][w] = T(0);
#pragma unroll 4
        for (int k = 0; k < SB; ++k) {
            T xa[4], qb[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                xa[u] = As[(ty + 16 * u) * LD + k];
                qb[u] = Qs[k * LD + tx + 16 * u];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int w = 0; w < 4; ++w) acc[u][w] = fma(xa[u], qb[w], acc[u][w]);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int w = 0; w < 4; ++w) {
                const int row = tile * SB + ty + 16 * u;
                if (row < n) X[(int64_t)row * n + sub_index(pr, tx + 16 * w)] = acc[u][w];
            }
        __syncthreads();
    }
}

// out[2g] = |off(A_g)|_F^2, out[2g+1] = |A_g|_F^2 (accumulated in FP64)
template <typename T>
__global__ void __launch_bounds__(NT) bj_norms(const BJMat<T>* __restrict__ mats, double* __restrict__ out) {
    const BJMat<T> M = mats[blockIdx.x];
    __shared__ double s_off[NT], s_all[NT];
    double off = 0.0, all = 0.0;
    const int64_t nn = (int64_t)M.n * M.n;
    for (int64_t e = threadIdx.x; e < nn; e += NT) {
        const double x = (double)M.A[e];
        all += x * x;
        const int i = (int)(e / M.n), j = (int)(e % M.n);
        if (i != j && (M.tau == 0.0 || fabs((double)M.A[(int64_t)i * M.n + i]) >= M.tau ||
                       fabs((double)M.A[(int64_t)j * M.n + j]) >= M.tau))
            off += x * x;
    }
    s_off[threadIdx.x] = off;
    s_all[threadIdx.x] = all;
    __syncthreads();
    for (int w = NT / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            s_off[threadIdx.x] += s_off[threadIdx.x + w];
            s_all[threadIdx.x] += s_all[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[2 * blockIdx.x] = s_off[0];
        out[2 * blockIdx.x + 1] = s_all[0];
    }
}

// padded FP64 copy of A_g, V_g <- identity; with a32 (optional) also the FP32
// copies A32 = A, V32 = identity
__global__ void __launch_bounds__(NT) bj_load(const BJMat<double>* __restrict__ mats,
                                             const BJMat<float>* __restrict__ m32, const EigJob* __restrict__ jobs) {
    const BJMat<double> M = mats[blockIdx.y];
    const EigJob J = jobs[blockIdx.y];
    const int64_t nn = (int64_t)M.n * M.n;
    for (int64_t e = blockIdx.x * (int64_t)NT + threadIdx.x; e < nn; e += (int64_t)gridDim.x * NT) {
        const int i = (int)(e / M.n), j = (int)(e % M.n);
        const double a = (i < J.n && j < J.n) ? J.A[(int64_t)i * J.lda + j] : 0.0;
        M.A[e] = a;
        M.V[e] = (i == j) ? 1.0 : 0.0;
        if (m32) {
            m32[blockIdx.y].A[e] = (float)a;
            m32[blockIdx.y].V[e] = (i == j) ? 1.f : 0.f;
        }
    }
}

// V64_g <- V32_g (widened)
__global__ void __launch_bounds__(NT) bj_widen(const BJMat<double>* __restrict__ mats,
                                              const BJMat<float>* __restrict__ m32) {
    const BJMat<double> M = mats[blockIdx.y];
    const float* v = m32[blockIdx.y].V;
    const int64_t nn = (int64_t)M.n * M.n;
    for (int64_t e = blockIdx.x * (int64_t)NT + threadIdx.x; e < nn; e += (int64_t)gridDim.x * NT) M.V[e] = (double)v[e];
}

// One FP64 product per matrix g: C = alpha op(X) Y + beta Z (op(X) = X or X^T;
// Z optional), all n x n row-major.  64 x 64 output tiles, 32-deep K steps
// staged in shared memory, 4 x 4 outputs per thread.
struct GemmJob {
    const double* X;
    const double* Y;
    const double* Z;
    double* C;
    int n, xt;
    double alpha, beta;
};
constexpr int GT = 64, GK = 32;
__global__ void __launch_bounds__(NT) bj_gemm(const GemmJob* __restrict__ jobs) {
    const GemmJob G = jobs[blockIdx.y];
    const int nt = (G.n + GT - 1) / GT;
    if ((int)blockIdx.x >= nt * nt) return;
    const int i0 = (blockIdx.x / nt) * GT, j0 = (blockIdx.x % nt) * GT;
    __shared__ double Xs[GT][GK + 1];
    __shared__ double Ys[GK][GT + 1];
    const int tid = threadIdx.x, ty = tid / 16, tx = tid % 16;
    double acc[4][4] = {};
    for (int k0 = 0; k0 < G.n; k0 += GK) {
        for (int e = tid; e < GT * GK; e += NT) {
            int i, k;
            if (G.xt) {  // X^T(i, k) = X[k][i]: consecutive threads along i
                i = e % GT;
                k = e / GT;
            } else {
                i = e / GK;
                k = e % GK;
            }
            const int gi = i0 + i, gk = k0 + k;
            Xs[i][k] = (gi < G.n && gk < G.n) ? (G.xt ? G.X[(int64_t)gk * G.n + gi] : G.X[(int64_t)gi * G.n + gk]) : 0.0;
        }
        for (int e = tid; e < GK * GT; e += NT) {
            const int k = e / GT, j = e % GT, gk = k0 + k, gj = j0 + j;
            Ys[k][j] = (gk < G.n && gj < G.n) ? G.Y[(int64_t)gk * G.n + gj] : 0.0;
        }
        __syncthreads();
#pragma unroll 8
        for (int k = 0; k < GK; ++k) {
            double a[4], b[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                a[u] = Xs[ty * 4 + u][k];
                b[u] = Ys[k][tx * 4 + u];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int w = 0; w < 4; ++w) acc[u][w] = fma(a[u], b[w], acc[u][w]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            const int gi = i0 + ty * 4 + u, gj = j0 + tx * 4 + w;
            if (gi < G.n && gj < G.n) {
                const int64_t o = (int64_t)gi * G.n + gj;
                G.C[o] = G.alpha * acc[u][w] + (G.Z ? G.beta * G.Z[o] : 0.0);
            }
        }
}

// eigenvectors (the leading n x n of V) and eigenvalues out
__global__ void __launch_bounds__(NT) bj_store(const BJMat<double>* __restrict__ mats, const EigJob* __restrict__ jobs) {
    const BJMat<double> M = mats[blockIdx.y];
    const EigJob J = jobs[blockIdx.y];
    const int64_t nn = (int64_t)J.n * J.n;
    for (int64_t e = blockIdx.x * (int64_t)NT + threadIdx.x; e < nn; e += (int64_t)gridDim.x * NT) {
        const int i = (int)(e / J.n), j = (int)(e % J.n);
        J.V[(int64_t)i * J.lda + j] = M.V[(int64_t)i * M.n + j];
        if (i == j) J.w[i] = M.A[(int64_t)i * M.n + i];
    }
}

// sweeps of the block Jacobi method in type T until max over matrices of
// off/|A| <= tol, or the decrease of a sweep is below `stall` (factor), or
// max_sweeps; returns the sweeps run; hist gets off/|A| before each sweep
template <typename T>
int bj_sweeps(const BJMat<T>* d_mats, const int* d_off, int nmat, int njob,
              int ne_max, int ntile, T* Qall, double* d_norm, int max_sweeps, double tol, double stall,
              double stall_from, int max_inner, cudaStream_t st, std::vector<double>* hist, double* final_worst,
              bool df = false) {
    const size_t smem = 2 * SB * LD * sizeof(T);
    static bool attr = false;
    if (!attr) {
        DMRG_CHECK_CUDA(cudaFuncSetAttribute(bj_solve<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        DMRG_CHECK_CUDA(cudaFuncSetAttribute(bj_rows<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        DMRG_CHECK_CUDA(cudaFuncSetAttribute(bj_cols<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        if constexpr (sizeof(T) == 8) {
            static_assert(sizeof(F2) == sizeof(T), "double-float tiles take the shared memory of FP64 tiles");
            DMRG_CHECK_CUDA(cudaFuncSetAttribute(bj_rows_df, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            DMRG_CHECK_CUDA(cudaFuncSetAttribute(bj_cols_df, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        }
        attr = true;
    }
    std::vector<double> nrm(2 * nmat);
    double prev = -1.0;
    int sweeps = 0;
    for (;;) {
        bj_norms<T><<<nmat, NT, 0, st>>>(d_mats, d_norm);
        ++launch_counter();
        DMRG_CHECK_CUDA(cudaMemcpyAsync(nrm.data(), d_norm, sizeof(double) * 2 * nmat, cudaMemcpyDeviceToHost, st));
        DMRG_CHECK_CUDA(cudaStreamSynchronize(st));
        double worst = 0.0;
        for (int g = 0; g < nmat; ++g)
            if (nrm[2 * g + 1] > 0.0) worst = std::max(worst, nrm[2 * g] / nrm[2 * g + 1]);
        if (hist) hist->push_back(std::sqrt(worst));
        *final_worst = worst;
        if (worst <= tol * tol || sweeps >= max_sweeps) break;
        // a stalled sweep ends the stage only near the arithmetic's floor (early
        // sweeps of a dense matrix may also reduce off/|A| slowly)
        if (prev >= 0.0 && worst < stall_from * stall_from && worst > stall * stall * prev) break;
        prev = worst;
        for (int r = 0; r < ne_max - 1; ++r) {
            bj_solve<T><<<njob, NT, smem, st>>>(d_mats, d_off, nmat, r, Qall, max_inner);
            bool done = false;
            if constexpr (sizeof(T) == 8) {
                if (df) {
                    bj_rows_df<<<njob * ntile, NT, smem, st>>>(d_mats, d_off, nmat, r, Qall, ntile);
                    bj_cols_df<<<njob * ntile, NT, smem, st>>>(d_mats, d_off, nmat, r, Qall, ntile);
                    done = true;
                }
            }
            if (!done) {
                bj_rows<T><<<njob * ntile, NT, smem, st>>>(d_mats, d_off, nmat, r, Qall, ntile);
                bj_cols<T><<<njob * ntile, NT, smem, st>>>(d_mats, d_off, nmat, r, Qall, ntile);
            }
            launch_counter() += 3;
        }
        DMRG_CHECK_CUDA(cudaGetLastError());
        ++sweeps;
    }
    return sweeps;
}

// A <- (A + A^T) / 2 (the product V^T rho V is symmetric only up to rounding)
__global__ void __launch_bounds__(NT) bj_sym(const BJMat<double>* __restrict__ mats) {
    const BJMat<double> M = mats[blockIdx.y];
    const int64_t nn = (int64_t)M.n * M.n;
    for (int64_t e = blockIdx.x * (int64_t)NT + threadIdx.x; e < nn; e += (int64_t)gridDim.x * NT) {
        const int i = (int)(e / M.n), j = (int)(e % M.n);
        if (i < j) {
            const double x = 0.5 * (M.A[e] + M.A[(int64_t)j * M.n + i]);
            M.A[e] = x;
            M.A[(int64_t)j * M.n + i] = x;
        }
    }
}

}  // namespace

int block_jacobi_eigh(const std::vector<EigJob>& jobs, int max_sweeps, double tol, cudaStream_t st,
                      const std::function<double*(int64_t)>& alloc_f,
                      const std::function<void(double*, int64_t)>& free_f, std::vector<double>* hist,
                      int* sweeps32_out, double tol32, bool df_rot) {
    const int nmat = (int)jobs.size();
    if (hist) hist->clear();
    if (sweeps32_out) *sweeps32_out = 0;
    if (nmat == 0) return 0;
    std::vector<BJMat<double>> mats(nmat);
    std::vector<BJMat<float>> m32(nmat);
    std::vector<int> job_off(nmat + 1, 0);
    int64_t nn_tot = 0;
    int ntile = 1, ne_max = 2, nmax = 0;
    for (int g = 0; g < nmat; ++g) {
        DMRG_REQUIRE(jobs[g].n >= 0 && jobs[g].lda >= jobs[g].n, DMRG_EINVAL, "bad eigenproblem extent");
        // at least two blocks, so that every matrix has a live pair
        const int n = (int)std::max<int64_t>(round_up(std::max(jobs[g].n, 1), BB), 2 * BB);
        mats[g].n = m32[g].n = n;
        mats[g].nb = m32[g].nb = n / BB;
        nn_tot += (int64_t)n * n;
        const int ne = mats[g].nb + (mats[g].nb & 1);
        job_off[g + 1] = job_off[g] + ne / 2;
        ntile = std::max(ntile, (n + SB - 1) / SB);
        ne_max = std::max(ne_max, ne);
        nmax = std::max(nmax, n);
    }
    // large problems first sweep in FP32 (cheap), then are brought back to FP64
    const bool two_stage = nmax >= kTwoStageMin;
    const int njob = job_off[nmat];
    const int64_t n_tab = (int64_t)((sizeof(BJMat<double>) + sizeof(BJMat<float>) + sizeof(EigJob) +
                                     sizeof(GemmJob)) * nmat + sizeof(int) * (nmat + 1) + 7) / 8;
    // FP64: A, V (+ two work matrices); FP32: A32, V32 (one double's worth per element pair)
    const int64_t n_mat = (two_stage ? 5 : 2) * nn_tot;
    const int64_t n_buf = n_mat + (int64_t)njob * SB * SB + 2 * nmat + n_tab;
    double* buf = alloc_f(n_buf);
    double* Qall = buf + n_mat;
    double* d_norm = Qall + (int64_t)njob * SB * SB;
    char* tab = (char*)(d_norm + 2 * nmat);
    BJMat<double>* d_mats = (BJMat<double>*)tab;
    BJMat<float>* d_m32 = (BJMat<float>*)(tab + sizeof(BJMat<double>) * nmat);
    EigJob* d_jobs = (EigJob*)(tab + (sizeof(BJMat<double>) + sizeof(BJMat<float>)) * nmat);
    GemmJob* d_gj = (GemmJob*)(tab + (sizeof(BJMat<double>) + sizeof(BJMat<float>) + sizeof(EigJob)) * nmat);
    int* d_off = (int*)(tab + (sizeof(BJMat<double>) + sizeof(BJMat<float>) + sizeof(EigJob) + sizeof(GemmJob)) * nmat);
    std::vector<double*> W1(nmat), W2(nmat);
    int64_t off = 0;
    for (int g = 0; g < nmat; ++g) {
        const int64_t nn = (int64_t)mats[g].n * mats[g].n;
        mats[g].A = buf + off;
        mats[g].V = buf + off + nn;
        off += 2 * nn;
        if (two_stage) {
            W1[g] = buf + off;
            W2[g] = buf + off + nn;
            m32[g].A = (float*)(buf + off + 2 * nn);
            m32[g].V = m32[g].A + nn;
            off += 3 * nn;
        }
        mats[g].floor = m32[g].floor = 0.0;
        mats[g].tau = m32[g].tau = 0.0;
    }
    DMRG_CHECK_CUDA(cudaMemcpyAsync(d_mats, mats.data(), sizeof(BJMat<double>) * nmat, cudaMemcpyHostToDevice, st));
    DMRG_CHECK_CUDA(cudaMemcpyAsync(d_jobs, jobs.data(), sizeof(EigJob) * nmat, cudaMemcpyHostToDevice, st));
    DMRG_CHECK_CUDA(cudaMemcpyAsync(d_off, job_off.data(), sizeof(int) * (nmat + 1), cudaMemcpyHostToDevice, st));
    if (two_stage)
        DMRG_CHECK_CUDA(cudaMemcpyAsync(d_m32, m32.data(), sizeof(BJMat<float>) * nmat, cudaMemcpyHostToDevice, st));
    const int gx = (int)std::min<int64_t>(((int64_t)nmax * nmax + NT - 1) / NT, 1024);
    bj_load<<<dim3(gx, nmat), NT, 0, st>>>(d_mats, two_stage ? d_m32 : nullptr, d_jobs);
    bj_norms<double><<<nmat, NT, 0, st>>>(d_mats, d_norm);
    launch_counter() += 2;
    std::vector<double> nrm(2 * nmat);
    DMRG_CHECK_CUDA(cudaMemcpyAsync(nrm.data(), d_norm, sizeof(double) * 2 * nmat, cudaMemcpyDeviceToHost, st));
    DMRG_CHECK_CUDA(cudaStreamSynchronize(st));
    for (int g = 0; g < nmat; ++g) {
        mats[g].floor = 1e-17 * std::sqrt(nrm[2 * g + 1]) + 1e-300;
        m32[g].floor = 1e-9 * std::sqrt(nrm[2 * g + 1]) + 1e-300;
    }
    DMRG_CHECK_CUDA(cudaMemcpyAsync(d_mats, mats.data(), sizeof(BJMat<double>) * nmat, cudaMemcpyHostToDevice, st));
    double worst = 0.0;
    if (two_stage) {
        DMRG_CHECK_CUDA(cudaMemcpyAsync(d_m32, m32.data(), sizeof(BJMat<float>) * nmat, cudaMemcpyHostToDevice, st));
        // stage 1: FP32 sweeps down to the FP32 rounding level
        const int s32 = bj_sweeps<float>(d_m32, d_off, nmat, njob, ne_max, ntile, (float*)Qall, d_norm,
                                         kMaxSweeps32, tol32 > 0.0 ? tol32 : kTol32, kStall32, kStallFrom32,
                                         kInner32, st, hist, &worst);
        if (sweeps32_out) *sweeps32_out = s32;
        // stage 2 (FP64): V = V32 made orthonormal by two Newton-Schulz steps
        // V <- V (3 I - V^T V) / 2, then A = V^T rho V
        bj_widen<<<dim3(gx, nmat), NT, 0, st>>>(d_mats, d_m32);
        ++launch_counter();
        std::vector<GemmJob> gj(nmat);
        const int nt = (nmax + GT - 1) / GT;
        auto gemm = [&](auto make) {
            for (int g = 0; g < nmat; ++g) gj[g] = make(g);
            DMRG_CHECK_CUDA(cudaMemcpyAsync(d_gj, gj.data(), sizeof(GemmJob) * nmat, cudaMemcpyHostToDevice, st));
            bj_gemm<<<dim3(nt * nt, nmat), NT, 0, st>>>(d_gj);
            ++launch_counter();
            // the job table is rewritten by the next product: wait for this one
            DMRG_CHECK_CUDA(cudaStreamSynchronize(st));
        };
        for (int step = 0; step < 2; ++step) {
            gemm([&](int g) { return GemmJob{mats[g].V, mats[g].V, nullptr, W1[g], mats[g].n, 1, 1.0, 0.0}; });
            gemm([&](int g) { return GemmJob{mats[g].V, W1[g], mats[g].V, W2[g], mats[g].n, 0, -0.5, 1.5}; });
            for (int g = 0; g < nmat; ++g) std::swap(mats[g].V, W2[g]);
        }
        gemm([&](int g) { return GemmJob{mats[g].A, mats[g].V, nullptr, W1[g], mats[g].n, 0, 1.0, 0.0}; });
        gemm([&](int g) { return GemmJob{mats[g].V, W1[g], nullptr, W2[g], mats[g].n, 1, 1.0, 0.0}; });
        for (int g = 0; g < nmat; ++g) {
            std::swap(mats[g].A, W2[g]);
            mats[g].tau = kTau * std::sqrt(nrm[2 * g + 1]);
        }
        DMRG_CHECK_CUDA(cudaMemcpyAsync(d_mats, mats.data(), sizeof(BJMat<double>) * nmat, cudaMemcpyHostToDevice, st));
        bj_sym<<<dim3(gx, nmat), NT, 0, st>>>(d_mats);
        ++launch_counter();
    }
    // FP64 sweeps to the tolerance
    // after an FP32 stage the rotations of the FP64 sweeps run in double-float
    // arithmetic (~48 bits, the FP32 units' rate); small matrices stay FP64
    const int sweeps = bj_sweeps<double>(d_mats, d_off, nmat, njob, ne_max, ntile, Qall, d_norm, max_sweeps, tol,
                                         kStall64, kStallFrom64, kInner64, st, hist, &worst,
                                         two_stage && df_rot);
    bj_store<<<dim3(gx, nmat), NT, 0, st>>>(d_mats, d_jobs);
    ++launch_counter();
    DMRG_CHECK_CUDA(cudaGetLastError());
    DMRG_CHECK_CUDA(cudaStreamSynchronize(st));
    free_f(buf, n_buf);
    return sweeps;
}

}  // namespace dmrg

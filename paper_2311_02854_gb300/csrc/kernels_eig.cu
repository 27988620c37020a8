// Block Jacobi eigensolver for the reduced density matrices of the
// decimation step (Sec. 2.1).
//
// Each matrix is padded to a multiple of BB and cut into BB x BB blocks.  A
// sweep pairs the blocks round-robin; in every round each pair (I, J) has its
// 2BB x 2BB diagonal subproblem diagonalised approximately (one cyclic Jacobi
// sweep in shared memory, giving an orthogonal Q), after which A <- Q^T A Q
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

struct BJMat {
    double* A;  // n x n, padded copy
    double* V;  // n x n
    int n, nb;
    double floor;
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

struct PairRef {
    BJMat M;
    int I, J;
    bool live;
};

__device__ __forceinline__ PairRef pair_of(const BJMat* mats, const int* job_off, int nmat, int round, int job) {
    PairRef r;
    const int g = find_mat(job_off, nmat, job);
    r.M = mats[g];
    const int ne = r.M.nb + (r.M.nb & 1);
    rr_pair(round % (ne - 1), job - job_off[g], ne, r.I, r.J);
    r.live = r.J < r.M.nb;  // J == nb: the padding player of an odd block count
    return r;
}

// global index of row a (0 <= a < SB) of the pair's subproblem
__device__ __forceinline__ int sub_index(const PairRef& p, int a) { return a < BB ? p.I * BB + a : p.J * BB + a - BB; }

// Q of each job (SB x SB, row-major) from one cyclic Jacobi sweep over its subproblem
__global__ void __launch_bounds__(NT) bj_solve(const BJMat* __restrict__ mats, const int* __restrict__ job_off,
                                              int nmat, int round, double* __restrict__ Qall) {
    extern __shared__ double sm[];
    double* S = sm;             // SB x LD
    double* Qs = sm + SB * LD;  // SB x LD
    __shared__ double cs[BB], sn[BB];
    __shared__ int pp[BB], qq[BB];
    const PairRef pr = pair_of(mats, job_off, nmat, round, blockIdx.x);
    double* Q = Qall + (int64_t)blockIdx.x * SB * SB;
    const int tid = threadIdx.x;
    for (int e = tid; e < SB * SB; e += NT) {
        const int a = e / SB, b = e % SB;
        S[a * LD + b] = pr.live ? pr.M.A[(int64_t)sub_index(pr, a) * pr.M.n + sub_index(pr, b)] : 0.0;
        Qs[a * LD + b] = (a == b) ? 1.0 : 0.0;
    }
    __syncthreads();
    if (pr.live) {
        for (int r = 0; r < SB - 1; ++r) {
            if (tid < BB) {
                int p, q;
                rr_pair(r, tid, SB, p, q);
                double c = 1.0, s = 0.0;
                const double apq = S[p * LD + q], app = S[p * LD + p], aqq = S[q * LD + q];
                if (fabs(apq) > pr.M.floor && fabs(apq) > 1e-15 * sqrt(fabs(app * aqq))) {
                    const double tau = (aqq - app) / (2.0 * apq);
                    const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                    c = 1.0 / sqrt(1.0 + t * t);
                    s = t * c;
                }
                cs[tid] = c;
                sn[tid] = s;
                pp[tid] = p;
                qq[tid] = q;
            }
            __syncthreads();
            for (int e = tid; e < BB * SB; e += NT) {  // rows p, q of S
                const int u = e / SB, k = e % SB;
                const double s = sn[u];
                if (s == 0.0) continue;
                const int p = pp[u], q = qq[u];
                const double c = cs[u], x = S[p * LD + k], y = S[q * LD + k];
                S[p * LD + k] = c * x - s * y;
                S[q * LD + k] = s * x + c * y;
            }
            __syncthreads();
            for (int e = tid; e < BB * SB; e += NT) {  // columns p, q of S and Q
                const int u = e / SB, k = e % SB;
                const double s = sn[u];
                if (s == 0.0) continue;
                const int p = pp[u], q = qq[u];
                const double c = cs[u];
                double x = S[k * LD + p], y = S[k * LD + q];
                S[k * LD + p] = c * x - s * y;
                S[k * LD + q] = s * x + c * y;
                x = Qs[k * LD + p];
                y = Qs[k * LD + q];
                Qs[k * LD + p] = c * x - s * y;
                Qs[k * LD + q] = s * x + c * y;
            }
            __syncthreads();
        }
    }
    for (int e = tid; e < SB * SB; e += NT) Q[e] = Qs[(e / SB) * LD + e % SB];
}

// A[rows I u J, column tile] <- Q^T A[rows I u J, column tile]; one CTA per (job, tile)
__global__ void __launch_bounds__(NT) bj_rows(const BJMat* __restrict__ mats, const int* __restrict__ job_off,
                                             int nmat, int round, const double* __restrict__ Qall, int ntile) {
    extern __shared__ double sm[];
    double* Qs = sm;
    double* As = sm + SB * LD;
    const int job = blockIdx.x / ntile, tile = blockIdx.x % ntile;
    const PairRef pr = pair_of(mats, job_off, nmat, round, job);
    if (!pr.live || tile * SB >= pr.M.n) return;
    const double* Q = Qall + (int64_t)job * SB * SB;
    const int n = pr.M.n, tid = threadIdx.x;
    for (int e = tid; e < SB * SB; e += NT) {
        const int a = e / SB, b = e % SB, col = tile * SB + b;
        Qs[a * LD + b] = Q[e];
        As[a * LD + b] = (col < n) ? pr.M.A[(int64_t)sub_index(pr, a) * n + col] : 0.0;
    }
    __syncthreads();
    for (int e = tid; e < SB * SB; e += NT) {
        const int a = e / SB, b = e % SB, col = tile * SB + b;
        double acc = 0.0;
#pragma unroll 16
        for (int k = 0; k < SB; ++k) acc = fma(Qs[k * LD + a], As[k * LD + b], acc);
        if (col < n) pr.M.A[(int64_t)sub_index(pr, a) * n + col] = acc;
    }
}

// X[row tile, columns I u J] <- X[row tile, columns I u J] Q for X = A, then X = V
__global__ void __launch_bounds__(NT) bj_cols(const BJMat* __restrict__ mats, const int* __restrict__ job_off,
                                             int nmat, int round, const double* __restrict__ Qall, int ntile) {
    extern __shared__ double sm[];
    double* Qs = sm;
    double* As = sm + SB * LD;
    const int job = blockIdx.x / ntile, tile = blockIdx.x % ntile;
    const PairRef pr = pair_of(mats, job_off, nmat, round, job);
    if (!pr.live || tile * SB >= pr.M.n) return;
    const double* Q = Qall + (int64_t)job * SB * SB;
    const int n = pr.M.n, tid = threadIdx.x;
    for (int e = tid; e < SB * SB; e += NT) Qs[(e / SB) * LD + e % SB] = Q[e];
    for (int which = 0; which < 2; ++which) {
        double* X = which ? pr.M.V : pr.M.A;
        for (int e = tid; e < SB * SB; e += NT) {
            const int a = e / SB, b = e % SB, row = tile * SB + a;
            As[a * LD + b] = (row < n) ? X[(int64_t)row * n + sub_index(pr, b)] : 0.0;
        }
        __syncthreads();
        for (int e = tid; e < SB * SB; e += NT) {
            const int a = e / SB, b = e % SB, row = tile * SB + a;
            double acc = 0.0;
#pragma unroll 16
            for (int k = 0; k < SB; ++k) acc = fma(As[a * LD + k], Qs[k * LD + b], acc);
            if (row < n) X[(int64_t)row * n + sub_index(pr, b)] = acc;
        }
        __syncthreads();
    }
}

// out[2g] = |off(A_g)|_F^2, out[2g+1] = |A_g|_F^2
__global__ void __launch_bounds__(NT) bj_norms(const BJMat* __restrict__ mats, double* __restrict__ out) {
    const BJMat M = mats[blockIdx.x];
    __shared__ double s_off[NT], s_all[NT];
    double off = 0.0, all = 0.0;
    const int64_t nn = (int64_t)M.n * M.n;
    for (int64_t e = threadIdx.x; e < nn; e += NT) {
        const double x = M.A[e];
        all += x * x;
        if (e / M.n != e % M.n) off += x * x;
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

// padded copy of A_g, V_g <- identity
__global__ void __launch_bounds__(NT) bj_load(const BJMat* __restrict__ mats, const EigJob* __restrict__ jobs) {
    const BJMat M = mats[blockIdx.y];
    const EigJob J = jobs[blockIdx.y];
    const int64_t nn = (int64_t)M.n * M.n;
    for (int64_t e = blockIdx.x * (int64_t)NT + threadIdx.x; e < nn; e += (int64_t)gridDim.x * NT) {
        const int i = (int)(e / M.n), j = (int)(e % M.n);
        M.A[e] = (i < J.n && j < J.n) ? J.A[(int64_t)i * J.lda + j] : 0.0;
        M.V[e] = (i == j) ? 1.0 : 0.0;
    }
}

// eigenvectors (the leading n x n of V) and eigenvalues out
__global__ void __launch_bounds__(NT) bj_store(const BJMat* __restrict__ mats, const EigJob* __restrict__ jobs) {
    const BJMat M = mats[blockIdx.y];
    const EigJob J = jobs[blockIdx.y];
    const int64_t nn = (int64_t)J.n * J.n;
    for (int64_t e = blockIdx.x * (int64_t)NT + threadIdx.x; e < nn; e += (int64_t)gridDim.x * NT) {
        const int i = (int)(e / J.n), j = (int)(e % J.n);
        J.V[(int64_t)i * J.lda + j] = M.V[(int64_t)i * M.n + j];
        if (i == j) J.w[i] = M.A[(int64_t)i * M.n + i];
    }
}

}  // namespace

int block_jacobi_eigh(const std::vector<EigJob>& jobs, int max_sweeps, double tol, cudaStream_t st,
                      const std::function<double*(int64_t)>& alloc_f,
                      const std::function<void(double*, int64_t)>& free_f) {
    const int nmat = (int)jobs.size();
    if (nmat == 0) return 0;
    std::vector<BJMat> mats(nmat);
    std::vector<int> job_off(nmat + 1, 0);
    int64_t tot = 0;
    int ntile = 1, ne_max = 2, nmax = 0;
    for (int g = 0; g < nmat; ++g) {
        DMRG_REQUIRE(jobs[g].n >= 0 && jobs[g].lda >= jobs[g].n, DMRG_EINVAL, "bad eigenproblem extent");
        // at least two blocks, so that every matrix has a live pair
        const int n = (int)std::max<int64_t>(round_up(std::max(jobs[g].n, 1), BB), 2 * BB);
        mats[g].n = n;
        mats[g].nb = n / BB;
        tot += 2 * (int64_t)n * n;
        const int ne = mats[g].nb + (mats[g].nb & 1);
        job_off[g + 1] = job_off[g] + ne / 2;
        ntile = std::max(ntile, (n + SB - 1) / SB);
        ne_max = std::max(ne_max, ne);
        nmax = std::max(nmax, n);
    }
    const int njob = job_off[nmat];
    const int64_t n_tab = (int64_t)((sizeof(BJMat) + sizeof(EigJob)) * nmat + sizeof(int) * (nmat + 1) + 7) / 8;
    const int64_t n_buf = tot + (int64_t)njob * SB * SB + 2 * nmat + n_tab;
    double* buf = alloc_f(n_buf);
    double* Qall = buf + tot;
    double* d_norm = Qall + (int64_t)njob * SB * SB;
    char* tab = (char*)(d_norm + 2 * nmat);
    BJMat* d_mats = (BJMat*)tab;
    EigJob* d_jobs = (EigJob*)(tab + sizeof(BJMat) * nmat);
    int* d_off = (int*)(tab + (sizeof(BJMat) + sizeof(EigJob)) * nmat);
    int64_t off = 0;
    for (int g = 0; g < nmat; ++g) {
        mats[g].A = buf + off;
        off += (int64_t)mats[g].n * mats[g].n;
        mats[g].V = buf + off;
        off += (int64_t)mats[g].n * mats[g].n;
        mats[g].floor = 0.0;
    }
    DMRG_CHECK_CUDA(cudaMemcpyAsync(d_mats, mats.data(), sizeof(BJMat) * nmat, cudaMemcpyHostToDevice, st));
    DMRG_CHECK_CUDA(cudaMemcpyAsync(d_jobs, jobs.data(), sizeof(EigJob) * nmat, cudaMemcpyHostToDevice, st));
    DMRG_CHECK_CUDA(cudaMemcpyAsync(d_off, job_off.data(), sizeof(int) * (nmat + 1), cudaMemcpyHostToDevice, st));
    const size_t smem = 2 * SB * LD * sizeof(double);
    static bool attr = false;
    if (!attr) {
        DMRG_CHECK_CUDA(cudaFuncSetAttribute(bj_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        DMRG_CHECK_CUDA(cudaFuncSetAttribute(bj_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        DMRG_CHECK_CUDA(cudaFuncSetAttribute(bj_cols, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        attr = true;
    }
    const int gx = (int)std::min<int64_t>(((int64_t)nmax * nmax + NT - 1) / NT, 1024);
    bj_load<<<dim3(gx, nmat), NT, 0, st>>>(d_mats, d_jobs);
    bj_norms<<<nmat, NT, 0, st>>>(d_mats, d_norm);
    launch_counter() += 2;
    std::vector<double> nrm(2 * nmat);
    DMRG_CHECK_CUDA(cudaMemcpyAsync(nrm.data(), d_norm, sizeof(double) * 2 * nmat, cudaMemcpyDeviceToHost, st));
    DMRG_CHECK_CUDA(cudaStreamSynchronize(st));
    for (int g = 0; g < nmat; ++g) mats[g].floor = 1e-17 * std::sqrt(nrm[2 * g + 1]) + 1e-300;
    DMRG_CHECK_CUDA(cudaMemcpyAsync(d_mats, mats.data(), sizeof(BJMat) * nmat, cudaMemcpyHostToDevice, st));
    int sweeps = 0;
    for (int sw = 0; sw < max_sweeps; ++sw) {
        double worst = 0.0;
        for (int g = 0; g < nmat; ++g)
            if (nrm[2 * g + 1] > 0.0) worst = std::max(worst, nrm[2 * g] / nrm[2 * g + 1]);
        if (worst <= tol * tol) break;
        for (int r = 0; r < ne_max - 1; ++r) {
            bj_solve<<<njob, NT, smem, st>>>(d_mats, d_off, nmat, r, Qall);
            bj_rows<<<njob * ntile, NT, smem, st>>>(d_mats, d_off, nmat, r, Qall, ntile);
            bj_cols<<<njob * ntile, NT, smem, st>>>(d_mats, d_off, nmat, r, Qall, ntile);
            launch_counter() += 3;
        }
        DMRG_CHECK_CUDA(cudaGetLastError());
        bj_norms<<<nmat, NT, 0, st>>>(d_mats, d_norm);
        ++launch_counter();
        DMRG_CHECK_CUDA(cudaMemcpyAsync(nrm.data(), d_norm, sizeof(double) * 2 * nmat, cudaMemcpyDeviceToHost, st));
        DMRG_CHECK_CUDA(cudaStreamSynchronize(st));
        ++sweeps;
    }
    bj_store<<<dim3(gx, nmat), NT, 0, st>>>(d_mats, d_jobs);
    ++launch_counter();
    DMRG_CHECK_CUDA(cudaGetLastError());
    DMRG_CHECK_CUDA(cudaStreamSynchronize(st));
    free_f(buf, n_buf);
    return sweeps;
}

}  // namespace dmrg

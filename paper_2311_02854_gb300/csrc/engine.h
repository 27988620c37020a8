// Device engine of libdmrg: the segmented grouped GEMM that performs every
// block product of the method (Sec. 2.2, the "GEMM step" with the
// "reduction" fused into the accumulator), plus the small FP64 kernels of
// Davidson and decimation.
#pragma once

#include <cstdint>
#include <vector>

#include "common.h"

namespace dmrg {

// One K-segment: C_tile += alpha * op(A)[rows of tile, 0:k] * op(B)[0:k, cols of tile].
// A is m x k: element (i, j) at A[i*lda + j] (a_tr = 0) or A[j*lda + i] (a_tr = 1).
// B is k x n: element (i, j) at B[i*ldb + j] (b_tr = 0) or B[j*ldb + i] (b_tr = 1).
struct Seg {
    int64_t a_off, b_off;
    int32_t k, lda, ldb;
    uint8_t a_buf, b_buf, a_tr, b_tr;
    double alpha;
};

enum TileMode : uint8_t { TILE_STORE = 0, TILE_ATOMIC = 1 };

// One output tile (at most 64 x 64) of an output block C (m x n, leading dim ldc).
struct Tile {
    int64_t c_off;        // block origin in buffer c_buf
    int32_t ldc, m, n;    // block leading dim and extents
    int32_t m0, n0;       // tile origin inside the block
    int32_t seg_beg, seg_end;
    uint8_t c_buf, mode;
    uint16_t nst;         // tensor-core engine: 64-deep K stages of the tile (set by the TMA work list)
    float alpha;          // epilogue scale (tensor-core engine; the FP64 engine scales per segment)
    int32_t tn;           // TMA tensor-core engine: tile width (64 or 128 columns)
};
static_assert(sizeof(Tile) == 48, "Tile keeps its 48-byte record");

constexpr int kMaxBufs = 8;
// Base pointers of the buffers a work list refers to, with the per-vector
// stride (elements) used when several vectors run in one launch (grid.y).
struct BufTable {
    double* p[kMaxBufs];
    int64_t vstride[kMaxBufs];
    // buffers whose bit is set in pmask hold bf16 pieces: p[i] is the hi piece
    // (as raw bf16) and lo[i] the lo piece (may be null); they are read as hi + lo.
    const void* lo[kMaxBufs];
    int64_t pstride[kMaxBufs];  // three pieces: piece 2 at lo + pstride (0: none)
    uint32_t pmask;
};

// A work list in host memory plus its device copy.
struct WorkList {
    std::vector<Tile> tiles;
    std::vector<Seg> segs;
    Tile* d_tiles = nullptr;
    Seg* d_segs = nullptr;
    size_t cap_tiles = 0, cap_segs = 0;
    double flops = 0.0;
    bool rank1 = false;  // every segment has K = 1 (run by the rank-1 kernel)
    // tile shape of add_block when nonzero (rows, columns); 128 x 64 lists run on
    // the FP64-accurate tensor-core engine (launch_seg_gemm_f64 dispatches on it)
    int tile_m = 0, tile_n = 0;
    void clear() {
        tiles.clear();
        segs.clear();
        flops = 0.0;
    }
    // Add an output block with its segments, split into 64x64 tiles (and into
    // K-chunks of at most kchunk when the block is atomically accumulated).
    void add_block(int64_t c_off, int c_buf, int m, int n, int ldc, const std::vector<Seg>& s,
                   uint8_t mode, int64_t kchunk = 0, int tile = 64, float alpha = 1.0f);
    void upload(cudaStream_t st);
    void release();
};

void launch_seg_gemm_f64(const WorkList& w, const BufTable& bt, int nvec, cudaStream_t st);
// FP64-accurate products on the bf16 tensor cores (kernels_oz.cu): work lists
// lowered with oz_tile_rows() x oz_tile_cols() tiles over FP64 buffers
void launch_seg_gemm_oz(const WorkList& w, const BufTable& bt, int nvec, int* d_err, cudaStream_t st);
int oz_tile_rows();
int oz_tile_cols();
int oz_stage_depth();
// device error word of the FP64 tensor-core engine (set when a bounded wait
// gave up); oz_take_error reads and clears it (synchronises the stream)
int* oz_error_word();
bool oz_take_error(cudaStream_t st);
// FP64 grouped GEMM with the work list in a static device array (noalloc.cu);
// a, b, c as buffers 0, 1, 2 of the work list
void grouped_gemm_f64_noalloc(const WorkList& host_wl, const double* a, const double* b, double* c, cudaStream_t st);
int64_t noalloc_scratch_bytes();
// the same kernel on device tile / segment lists owned by the caller (one vector)
void launch_seg_gemm_f64_lists(const Tile* d_tiles, int64_t ntiles, const Seg* d_segs, const BufTable& bt,
                               cudaStream_t st);

// --- small FP64 kernels (Davidson / decimation) ---------------------------
// out[i] = sum_k X[i*ldx + k] * y[k], i < m   (deterministic two-pass)
void dev_dots(const double* X, int64_t ldx, int m, const double* y, int64_t n, double* out,
              double* work, cudaStream_t st);
// y[k] = sum_i c[i] * X[i*ldx + k]  (c on device)
void dev_combine(const double* X, int64_t ldx, int m, const double* c, int64_t n, double* y,
                 cudaStream_t st);
// y = a*x + b*y
void dev_axpby(double a, const double* x, double b, double* y, int64_t n, cudaStream_t st);
// t = -r / (d - theta), |d - theta| clamped to >= 1e-8 keeping its sign
void dev_jacobi_precond(const double* r, const double* d, double theta, double* t, int64_t n,
                        cudaStream_t st);
// symmetric eigensolver (cyclic Jacobi with round-robin ordering, one CTA per
// matrix): A (n x n, row-major, ld lda) is overwritten (its diagonal ends as
// the eigenvalues, also written to w[n]); V (n x n, ld lda) receives the
// eigenvectors as columns.  Jobs live in device memory.
struct EigJob {
    double* A;
    double* V;
    double* w;
    int n, lda;
};
void dev_jacobi_eigh_batched(const EigJob* d_jobs, int njobs, int max_sweeps, cudaStream_t st);
void dev_fill(double* x, double v, int64_t n, cudaStream_t st);
// x[i] += amp * (u(i, seed) - 1/2) with a 32-bit integer hash u in [0, 1)
void dev_perturb(double* x, int64_t n, uint32_t seed, double amp, cudaStream_t st);
void dev_identity(double* x, int n, cudaStream_t st);
int64_t& launch_counter();
// selftest.cu: one bounded mbarrier wait (arrived on or not); false if it gave up
bool wait_selftest(double seconds, bool arrive, cudaStream_t st);

}  // namespace dmrg
